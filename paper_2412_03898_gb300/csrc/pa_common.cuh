// Device helpers shared by the library's kernels: error-free float
// transformations (double-float distance), the hardware base-2 exponential,
// TMA bulk copies with mbarrier completion, bounded waits and the device error
// word.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pa.h"

namespace pa {

constexpr unsigned FULL = 0xffffffffu;

// sqrt(log2(e)/2): with u = tau * K_S / a, exp(-tau^2/(2a^2)) = 2^(-u^2).
constexpr float K_S = 0.849321800288019f;
// 2 ln 2: 1 - tau^2/a^2 = 1 - 2 ln2 * u^2.
constexpr float K_2LN2 = 1.3862943611198906f;

// Bounded waits give up after this many nanoseconds of %globaltimer.
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;

// ---------------------------------------------------------------------------
// Error word: the first data-dependent error of a launch sequence wins.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_error(unsigned *err, unsigned code) {
  if (err != nullptr) atomicCAS(err, 0u, code);
}

// ---------------------------------------------------------------------------
// Error-free transformations (Knuth TwoSum, Dekker FastTwoSum, FMA TwoProd).
// The _rn intrinsics are never contracted into FMAs, which keeps the
// transformations exact.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// |b - s| as a double-float (hi, lo), relative error ~2^-44, from fp32
// coordinates.  The coordinate differences are exact (TwoSum), the squares
// exact to first order (TwoProd), the sum compensated, and the square root
// refined by one Newton step on the residual.  The step starts from
// x * rsqrt(x) (a few ulp): its error after the step is of order ulp^2, so a
// correctly rounded square root would buy nothing.  (hi, lo) is not
// normalised (|lo| can reach a few ulp of hi); callers renormalise.
__device__ __forceinline__ void distance_df(float bx, float by, float bz, float sx, float sy,
                                            float sz, float &rh, float &rl) {
  float dxh, dxl, dyh, dyl, dzh, dzl;
  two_sum(bx, -sx, dxh, dxl);
  two_sum(by, -sy, dyh, dyl);
  two_sum(bz, -sz, dzh, dzl);
  float pxh = __fmul_rn(dxh, dxh), pyh = __fmul_rn(dyh, dyh), pzh = __fmul_rn(dzh, dzh);
  float pxl = fmaf(2.f * dxh, dxl, fmaf(dxh, dxh, -pxh));
  float pyl = fmaf(2.f * dyh, dyl, fmaf(dyh, dyh, -pyh));
  float pzl = fmaf(2.f * dzh, dzl, fmaf(dzh, dzh, -pzh));
  float s1, e1, s2, e2;
  two_sum(pxh, pyh, s1, e1);
  two_sum(s1, pzh, s2, e2);
  float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(pxl, pyl), pzl));
  float sh, sl;
  fast_two_sum(s2, lo, sh, sl);
  const float y = rsqrtf(sh);
  const float r = __fmul_rn(sh, y);
  rh = r;
  rl = __fmul_rn(__fadd_rn(fmaf(-r, r, sh), sl), 0.5f * y);
}

// ---------------------------------------------------------------------------
// 2^x on the SFU (PTX ex2.approx.ftz.f32; relative error ~2^-22).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Eight consecutive floats from read-only global memory in one 256-bit load
// (PTX ld.global.nc.v8.f32, sm_100 and later); p must be 32-byte aligned.
__device__ __forceinline__ void ldg8(const float *p, float4 &lo, float4 &hi) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
               : "l"(p));
}

// ldg8 when `pred` holds, else lo and hi keep their values (predicated load,
// no branch).
__device__ __forceinline__ void ldg8_if(const float *p, bool pred, float4 &lo, float4 &hi) {
  asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %9, 0;\n\t"
      "@q ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t}"
      : "+f"(lo.x), "+f"(lo.y), "+f"(lo.z), "+f"(lo.w), "+f"(hi.x), "+f"(hi.y), "+f"(hi.z), "+f"(hi.w)
      : "l"(p), "r"((int)pred));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (TMA, non-tensor form).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Global -> shared bulk copy completing on `bar`.  dst, src 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of `bar` for at most WAIT_LIMIT_NS; false if it
// ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity,
                                                  unsigned long long limit_ns = WAIT_LIMIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long start = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - start > limit_ns) return false;
  }
}

// ---------------------------------------------------------------------------
// Warp reductions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Sorts distinct unsigned keys across the 32 lanes of a warp, ascending
// (bitonic network on shuffles).  Callers pack the lane index into the low
// bits, which makes the keys distinct and carries the payload.
__device__ __forceinline__ unsigned warp_sort(unsigned key, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const unsigned other = __shfl_xor_sync(FULL, key, j);
      const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
      key = keep_min ? min(key, other) : max(key, other);
    }
  }
  return key;
}

// ---------------------------------------------------------------------------
// Acquisition scalars prepared on the host in double precision and split
// into float pairs: delta = c/fs (distance per sample) and ct0 = c*t0.
// ---------------------------------------------------------------------------
struct Acq {
  const float *sensors;  // [3][sstride]
  int S, sstride, T;
  float kappa;
  float inv_delta;  // fs/c
  float dh, dl;     // c/fs = dh + dl
  float ct0h, ct0l; // c*t0 = ct0h + ct0l
};

// Parameters of one (ball, sensor) pair on a sample range [k_begin, k_end].
struct PairWin {
  float u0;   // scaled tau at k_lo: u = tau * K_S / a (tau / a for the uniform profile)
  float du;   // decrement of u per sample
  float amp;  // p / (2 R s): v = amp * u * 2^(-u^2)
  float R;    // distance (hi part)
  int klo;    // first sample of the window (clipped)
  int W;      // number of samples (0 = empty)
  bool domain_err;
};

// Window and phase of one pair, shared by pa_forward, pa_adjoint and
// pa_count_contributions so that all three sum exactly the same terms.
// The window is every k in [k_begin, k_end] with |R - c t_k| <= h, h = kappa a
// (h = a for the uniform profile).  tau at k_lo is assembled in double-float:
//   tau0 = (R - c t0) - k_lo * (c/fs)
// and rounded once to fp32, so its error is below ulp(h)/2 ~ kappa a 2^-24.
template <bool UNIFORM>
__device__ __forceinline__ PairWin pair_window(const Acq &q, float bx, float by, float bz, float a,
                                               float p, float sx, float sy, float sz, int k_begin,
                                               int k_end) {
  PairWin w;
  w.W = 0;
  w.domain_err = false;
  w.klo = 0;
  w.u0 = w.du = w.amp = w.R = 0.f;
  if (!(a > 0.f) || p == 0.f) return w;
  float rh, rl;
  distance_df(bx, by, bz, sx, sy, sz, rh, rl);
  w.R = rh;
  const float h = UNIFORM ? a : q.kappa * a;
  if (!(rh > h)) {
    w.domain_err = true;
    return w;
  }
  // R - c t0 as a double-float
  float ch, cl;
  two_sum(rh, -q.ct0h, ch, cl);
  cl = __fadd_rn(cl, __fsub_rn(rl, q.ct0l));
  float rch, rcl;
  fast_two_sum(ch, cl, rch, rcl);
  const float flo = ceilf(__fmul_rn(__fadd_rn(__fsub_rn(rch, h), rcl), q.inv_delta));
  const float fhi = floorf(__fmul_rn(__fadd_rn(__fadd_rn(rch, h), rcl), q.inv_delta));
  const float klo_f = fmaxf(flo, (float)k_begin);
  const float khi_f = fminf(fhi, (float)k_end);
  if (!(khi_f >= klo_f)) return w;
  // tau0 = (rch + rcl) - klo * (dh + dl)
  const float ph = __fmul_rn(klo_f, q.dh);
  const float pl = fmaf(klo_f, q.dh, -ph);
  const float t = __fsub_rn(rch, ph);
  const float tau0 = __fadd_rn(t, __fsub_rn(__fsub_rn(rcl, pl), __fmul_rn(klo_f, q.dl)));
  // u = tau s: the window is |u| <= kappa K_S (Gaussian) or |u| <= 1 (uniform)
  // (an approximate quotient only rescales u and amp consistently: v keeps
  // its amplitude and the Gaussian width changes by ~2^-22 relative)
  const float s = UNIFORM ? __fdividef(1.f, a) : __fdividef(K_S, a);
  w.u0 = tau0 * s;
  w.du = q.dh * s;
  w.amp = __fdividef(p, 2.f * rh * s);
  w.klo = (int)klo_f;
  w.W = (int)khi_f - w.klo + 1;
  return w;
}

}  // namespace pa
