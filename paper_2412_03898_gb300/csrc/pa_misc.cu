// Deformation (Eq. 1-2), the FP64 L2 loss / residual, and Adam.
#include <algorithm>

#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kFrameChunk = 8;

// Eq. 1-2: one thread per (channel, ball, chunk of up to kFrameChunk
// frames), so that even one frame gives 5 N threads.  The deformation
// parameters of a (channel, ball) are read once per chunk, coalesced across
// threads (ball index fastest), several basis functions' loads in flight.
__global__ void __launch_bounds__(256) k_deform(const float *__restrict__ canon, const float *__restrict__ omega,
                                                const float *__restrict__ theta, const float *__restrict__ sigma,
                                                long long n, long long stride, int nb,
                                                const float *__restrict__ t, int F, float *__restrict__ out,
                                                unsigned *err) {
  const float L2E_HALF = 0.72134752044448170368f;  // log2(e)/2
  const int nchunks = (F + kFrameChunk - 1) / kFrameChunk;
  const long long total = 5 * n * nchunks;
  bool dom = false;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
       it += (long long)gridDim.x * blockDim.x) {
    const long long b = it % n;
    const long long r = it / n;
    const int c = (int)(r % 5);
    const int f0 = (int)(r / 5) * kFrameChunk;
    const int fc = min(kFrameChunk, F - f0);
    float tf[kFrameChunk];
#pragma unroll
    for (int j = 0; j < kFrameChunk; ++j) tf[j] = j < fc ? __ldg(t + f0 + j) : 0.f;
    float H[kFrameChunk];
#pragma unroll
    for (int j = 0; j < kFrameChunk; ++j) H[j] = 0.f;
    const long long g0 = (long long)c * nb * stride + b;
#pragma unroll 4
    for (int k = 0; k < nb; ++k) {
      const long long gi = g0 + (long long)k * stride;
      const float om = __ldg(omega + gi), th = __ldg(theta + gi), sg = __ldg(sigma + gi);
      if (!(sg > 0.f)) {
        dom = true;
        continue;
      }
      const float is = 1.f / sg;
#pragma unroll
      for (int j = 0; j < kFrameChunk; ++j) {
        const float d = (tf[j] - th) * is;
        H[j] = fmaf(om, ex2(-d * d * L2E_HALF), H[j]);
      }
    }
    const float q0 = __ldg(canon + (long long)c * stride + b);
#pragma unroll
    for (int j = 0; j < kFrameChunk; ++j)
      if (j < fc) out[((long long)(f0 + j) * 5 + c) * stride + b] = q0 * (1.f + H[j]);
  }
  if (dom) set_error(err, PA_ERR_DOMAIN);
}

// Chain rule of Eq. 1-2 from per-frame state gradients g(f) = dL/dq(t_f) to
// the canonical cloud and the deformation parameters.  One thread per
// (channel, ball); basis functions in the outer loop, frames in the inner
// one, so every output is written once (no read-modify-write).  With
// d = (t_f - theta)/sigma and b = exp(-d^2/2):
//   dL/domega = q0 sum_f g b
//   dL/dtheta = q0 omega/sigma sum_f g b d
//   dL/dsigma = q0 omega/sigma sum_f g b d^2
//   dL/dq0    = sum_f g (1 + H(t_f)) = sum_f g + sum_n omega_n sum_f g b_n.
// g(f) of a thread is re-read per basis function from L1 (one 128-byte line
// per warp and frame).
__global__ void __launch_bounds__(256) k_deform_backward(const float *__restrict__ canon,
                                                         const float *__restrict__ omega,
                                                         const float *__restrict__ theta,
                                                         const float *__restrict__ sigma, long long n,
                                                         long long stride, int nb, const float *__restrict__ t,
                                                         int F, const float *__restrict__ gstate,
                                                         float *__restrict__ g_canon, float *__restrict__ g_omega,
                                                         float *__restrict__ g_theta, float *__restrict__ g_sigma,
                                                         bool acc, unsigned *err) {
  const float L2E_HALF = 0.72134752044448170368f;  // log2(e)/2
  bool dom = false;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < 5 * n;
       it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it / n);
    const long long b = it - (long long)c * n;
    const float q0 = __ldg(canon + (long long)c * stride + b);
    const float *gq = gstate + (long long)c * stride + b;  // frame f at gq[f * 5 * stride]
    float gsum = 0.f;
    for (int f = 0; f < F; ++f) gsum += __ldg(gq + (long long)f * 5 * stride);
    float gcan = gsum;
#pragma unroll 4
    for (int k = 0; k < nb; ++k) {
      const long long gi = ((long long)c * nb + k) * stride + b;
      const float om = __ldg(omega + gi), th = __ldg(theta + gi), sg = __ldg(sigma + gi);
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      float is = 0.f;
      if (sg > 0.f) {
        is = 1.f / sg;
        for (int f = 0; f < F; ++f) {
          const float g = __ldg(gq + (long long)f * 5 * stride);
          const float d = (__ldg(t + f) - th) * is;
          const float gb = g * ex2(-d * d * L2E_HALF);
          s0 += gb;
          s1 = fmaf(gb, d, s1);
          s2 = fmaf(gb * d, d, s2);
        }
      } else {
        dom = true;  // term skipped, as in the forward deformation
      }
      gcan = fmaf(om, s0, gcan);
      const float qo = q0 * om * is;
      float vo = q0 * s0, vt = qo * s1, vs = qo * s2;
      if (acc) {
        vo += g_omega[gi];
        vt += g_theta[gi];
        vs += g_sigma[gi];
      }
      g_omega[gi] = vo;
      g_theta[gi] = vt;
      g_sigma[gi] = vs;
    }
    float *dst = g_canon + (long long)c * stride + b;
    *dst = acc ? *dst + gcan : gcan;
  }
  if (dom) set_error(err, PA_ERR_DOMAIN);
}

// Self-test of the bounded mbarrier wait that guards every TMA stage: one
// thread waits for a phase of an mbarrier that nothing completes; the wait
// gives up after limit_ns and records PA_ERR_TIMEOUT, as the forward does
// when a copy never lands.  Nothing is in flight when the block exits.
__global__ void k_selftest_wait(unsigned long long limit_ns, unsigned *err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, limit_ns)) set_error(err, PA_ERR_TIMEOUT);
}

// Per-frame partial sums of squared residuals in FP64 (each float4 is summed
// in fp32 then promoted), optional residual 2 scale (pred - meas).
__global__ void __launch_bounds__(256) k_loss_partial(const float4 *__restrict__ pred, const float4 *__restrict__ meas,
                                                      long long per4, const float *__restrict__ scale,
                                                      float4 *__restrict__ resid, double *__restrict__ partials) {
  const int f = blockIdx.y;
  const float4 *p = pred + (long long)f * per4;
  const float4 *m = meas ? meas + (long long)f * per4 : nullptr;
  float4 *r = resid ? resid + (long long)f * per4 : nullptr;
  const float two_s = 2.f * (scale ? __ldg(scale + f) : 1.f);
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per4;
       i += (long long)gridDim.x * blockDim.x) {
    float4 d = __ldg(p + i);
    if (m) {
      const float4 q = __ldg(m + i);
      d.x -= q.x;
      d.y -= q.y;
      d.z -= q.z;
      d.w -= q.w;
    }
    acc += (double)fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, d.w * d.w)));
    if (r) r[i] = make_float4(two_s * d.x, two_s * d.y, two_s * d.z, two_s * d.w);
  }
  __shared__ double red[8];
  acc = warp_sum_d(acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    double v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    v = warp_sum_d(v);
    if (lane == 0) partials[(long long)f * gridDim.x + blockIdx.x] = v;
  }
}

// loss[f] = sum of the frame's partials, in a fixed order.
__global__ void k_loss_final(const double *__restrict__ partials, int bpf, double *__restrict__ loss) {
  const int f = blockIdx.x, lane = threadIdx.x;
  double v = 0.0;
  for (int i = lane; i < bpf; i += 32) v += partials[(long long)f * bpf + i];
  v = warp_sum_d(v);
  if (lane == 0) loss[f] = v;
}

__global__ void k_adam(float4 *__restrict__ x, const float4 *__restrict__ g, float4 *__restrict__ m,
                       float4 *__restrict__ v, long long n4, float lr, float b1, float b2, float omb1, float omb2,
                       float eps, float bc1, float bc2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    float4 xi = x[i], gi = __ldg(g + i), mi = m[i], vi = v[i];
    float *px = &xi.x, *pg = &gi.x, *pm = &mi.x, *pv = &vi.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pm[k] = fmaf(b1, pm[k], omb1 * pg[k]);
      pv[k] = fmaf(b2, pv[k], omb2 * pg[k] * pg[k]);
      const float mh = pm[k] / bc1;
      const float vh = pv[k] / bc2;
      px[k] -= lr * mh / (sqrtf(vh) + eps);
    }
    x[i] = xi;
    m[i] = mi;
    v[i] = vi;
  }
}

__global__ void k_adam_tail(float *x, const float *g, float *m, float *v, long long start, long long n, float lr,
                            float b1, float b2, float omb1, float omb2, float eps, float bc1, float bc2) {
  const long long i = start + threadIdx.x;
  if (i >= n) return;
  m[i] = fmaf(b1, m[i], omb1 * g[i]);
  v[i] = fmaf(b2, v[i], omb2 * g[i] * g[i]);
  x[i] -= lr * (m[i] / bc1) / (sqrtf(v[i] / bc2) + eps);
}

// Adam with t = *step from device memory (see pa_adam_step_scheduled).
__global__ void k_adam_sched(float *__restrict__ x, const float *__restrict__ g, float *__restrict__ m,
                             float *__restrict__ v, long long n, float lr0, float b1, float b2, float omb1, float omb2,
                             float eps, int step_size, float gamma, const int *__restrict__ step) {
  const int t = max(*step, 1);
  const float lr = lr0 * powf(gamma, (float)((t - 1) / step_size));
  const float bc1 = 1.f - powf(b1, (float)t);
  const float bc2 = 1.f - powf(b2, (float)t);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], omb1 * gi);
    const float vi = fmaf(b2, v[i], omb2 * gi * gi);
    m[i] = mi;
    v[i] = vi;
    x[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

__global__ void k_step_increment(int *step) { *step += 1; }

}  // namespace

cudaError_t launch_adam_sched(float *x, const float *g, float *m, float *v, long long n, float lr0, float b1,
                              float b2, float omb1, float omb2, float eps, int step_size, float gamma,
                              const int *step, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  k_adam_sched<<<(unsigned)blocks, 256, 0, st>>>(x, g, m, v, n, lr0, b1, b2, omb1, omb2, eps, step_size, gamma,
                                                 step);
  return cudaGetLastError();
}

cudaError_t launch_step_increment(int *step, cudaStream_t st) {
  k_step_increment<<<1, 1, 0, st>>>(step);
  return cudaGetLastError();
}

cudaError_t launch_deform(const float *canon, const float *omega, const float *theta, const float *sigma,
                          long long n, long long stride, int nb, const float *t, int F, float *out, unsigned *err,
                          cudaStream_t st) {
  const long long total = 5 * n * ((F + kFrameChunk - 1) / kFrameChunk);
  if (total == 0) return cudaSuccess;
  const long long blocks = std::min<long long>((total + 255) / 256, 152LL * 32);
  k_deform<<<(unsigned)blocks, 256, 0, st>>>(canon, omega, theta, sigma, n, stride, nb, t, F, out, err);
  return cudaGetLastError();
}

cudaError_t launch_deform_backward(const float *canon, const float *omega, const float *theta, const float *sigma,
                                   long long n, long long stride, int nb, const float *t, int F, const float *gstate,
                                   float *g_canon, float *g_omega, float *g_theta, float *g_sigma, bool acc,
                                   unsigned *err, cudaStream_t st) {
  const long long total = 5 * n;
  if (total == 0) return cudaSuccess;
  const long long blocks = std::min<long long>((total + 255) / 256, 152LL * 32);
  k_deform_backward<<<(unsigned)blocks, 256, 0, st>>>(canon, omega, theta, sigma, n, stride, nb, t, F, gstate,
                                                      g_canon, g_omega, g_theta, g_sigma, acc, err);
  return cudaGetLastError();
}

cudaError_t launch_selftest_wait(unsigned long long limit_ns, unsigned *err, cudaStream_t st) {
  k_selftest_wait<<<1, 32, 0, st>>>(limit_ns, err);
  return cudaGetLastError();
}

int loss_blocks_per_frame(long long per_frame) {
  const long long per4 = per_frame / 4;
  return (int)std::max(1LL, std::min(1024LL, (per4 + 8191) / 8192));
}

cudaError_t launch_loss(const float *pred, const float *meas, long long per_frame, int F, const float *scale,
                        double *loss, float *resid, double *partials, int bpf, cudaStream_t st) {
  if (F == 0) return cudaSuccess;
  dim3 grid(bpf, F);
  k_loss_partial<<<grid, 256, 0, st>>>(reinterpret_cast<const float4 *>(pred),
                                       reinterpret_cast<const float4 *>(meas), per_frame / 4, scale,
                                       reinterpret_cast<float4 *>(resid), partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || loss == nullptr) return e;
  k_loss_final<<<F, 32, 0, st>>>(partials, bpf, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float *x, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                        float omb1, float omb2, float eps, float bc1, float bc2, cudaStream_t st) {
  const long long n4 = n / 4;
  if (n4 > 0) {
    const long long blocks = std::min<long long>((n4 + 255) / 256, 152LL * 16);
    k_adam<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<float4 *>(x), reinterpret_cast<const float4 *>(g),
                                             reinterpret_cast<float4 *>(m), reinterpret_cast<float4 *>(v), n4, lr,
                                             b1, b2, omb1, omb2, eps, bc1, bc2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (n4 * 4 < n) {
    k_adam_tail<<<1, 4, 0, st>>>(x, g, m, v, n4 * 4, n, lr, b1, b2, omb1, omb2, eps, bc1, bc2);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace pa
