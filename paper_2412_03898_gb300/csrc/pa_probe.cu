// Throughput probe of the units that bound the forward and adjoint sample
// loops: the FP32 FMA pipe (scalar FFMA and packed FP32x2 FMA) and the SFU
// base-2 exponential.  A measurement aid for the roofline denominators; the
// paper has no counterpart.
//
// Each probe kernel runs eight independent dependency chains per thread in a
// grid of exactly one full wave (every SM at its occupancy limit), so the
// unit, not latency, sets the rate.  Block 0 records its own elapsed SM
// cycles (clock64) and nanoseconds (%globaltimer), which give the SM clock
// during the kernel; the launch is timed with CUDA events.  The rate is
//     lane operations / (event seconds x SMs x SM clock)
// per SM per clock (an FMA counts as one operation, a packed FMA as two).
#include <algorithm>

#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

// Sink for the chains' results (written only when `write` is set, which the
// host never does; the compiler cannot know that) and block 0's timing.
__device__ float g_probe_sink[kProbeThreads];
__device__ unsigned long long g_probe_clk[2];

enum ProbeKind { kFfma = 0, kFfma2 = 1, kEx2 = 2 };

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_probe(long long iters, int write) {
  const unsigned long long c0 = clock64();
  const unsigned long long t0 = global_ns();
  float x[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) x[i] = 1e-3f * (float)(threadIdx.x + 1) + 0.125f * (float)i;
  if (KIND == kFfma) {
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < kProbeChains; ++i) x[i] = fmaf(x[i], 0.99993896484375f, 6.103515625e-05f);
    }
  } else if (KIND == kFfma2) {
    float2 y[kProbeChains / 2];
#pragma unroll
    for (int i = 0; i < kProbeChains / 2; ++i) y[i] = make_float2(x[2 * i], x[2 * i + 1]);
    const float2 m = make_float2(0.99993896484375f, 0.99993896484375f);
    const float2 c = make_float2(6.103515625e-05f, 6.103515625e-05f);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < kProbeChains / 2; ++i) y[i] = __ffma2_rn(y[i], m, c);
    }
#pragma unroll
    for (int i = 0; i < kProbeChains / 2; ++i) {
      x[2 * i] = y[i].x;
      x[2 * i + 1] = y[i].y;
    }
  } else {
    // x stays in (0, 1]: 2^(-x) maps (0, 1] into [0.5, 1)
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < kProbeChains; ++i) x[i] = ex2(-x[i]);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) s += x[i];
  if (write) g_probe_sink[threadIdx.x] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    g_probe_clk[0] = clock64() - c0;
    g_probe_clk[1] = global_ns() - t0;
  }
}

template <int KIND>
cudaError_t probe_once(long long iters, int sms, cudaStream_t st, double &rate, double &mhz) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_probe<KIND>, kProbeThreads, 0);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int grid = sms * occ;
  // warm-up: clocks up, code loaded
  k_probe<KIND><<<grid, kProbeThreads, 0, st>>>(std::max(1LL, iters / 16), 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cudaEvent_t ev[2];
  if ((e = cudaEventCreate(&ev[0])) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&ev[1])) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return e;
  }
  e = cudaEventRecord(ev[0], st);
  if (e == cudaSuccess) {
    k_probe<KIND><<<grid, kProbeThreads, 0, st>>>(iters, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  unsigned long long clk[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(clk, g_probe_clk, sizeof(clk));
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) return e;
  if (!(ms > 0.f) || clk[1] == 0) return cudaErrorUnknown;
  mhz = 1e3 * (double)clk[0] / (double)clk[1];
  const double lane_ops = (double)grid * kProbeThreads * (double)iters * kProbeChains;
  rate = lane_ops / (1e-3 * (double)ms * (double)sms * mhz * 1e6);
  return cudaSuccess;
}

}  // namespace

cudaError_t measure_unit_rates(int sms, cudaStream_t st, double out[4]) {
  // ~30 ms per FMA probe at 128 lanes per SM per clock and 2 GHz; the SFU
  // probe runs a quarter of the iterations
  const long long iters = 1LL << 19;
  double mhz = 0.0, mhz2 = 0.0, mhz3 = 0.0;
  cudaError_t e = probe_once<kFfma>(iters, sms, st, out[0], mhz);
  if (e == cudaSuccess) e = probe_once<kFfma2>(iters, sms, st, out[1], mhz2);
  if (e == cudaSuccess) e = probe_once<kEx2>(iters / 4, sms, st, out[2], mhz3);
  out[3] = mhz;
  return e;
}

}  // namespace pa
