// Adjoint of the forward projection: gradients of the L2 loss (Sec. 2.2,
// last paragraph) with respect to the per-frame ball states and, in 4D mode,
// through Eq. 1-2 to the canonical cloud and the deformation parameters
// (Sec. 2.2: baseline attributes and (theta, sigma, omega) are learnable).
//
// Design (GB300, sm_103a): ball-major, no atomics.
//  - One warp owns one ball (static mode: one (frame, ball) item) and loops
//    over all sensors.  The 32 lanes compute the windows and phases of 32
//    (ball, sensor) pairs in parallel and compact the valid ones to the
//    front lanes with register shuffles; then each lane walks one pair's window,
//    eight consecutive samples per step (one 256-bit residual load from L2
//    when the rows are 32-byte aligned, else two float4 loads;
//    packed FP32x2 arithmetic; the next step's load in flight, unpredicated
//    and double-buffered on the steps inside every lane's window),
//    accumulating
//        S1 = sum g E u,  S3 = sum g E u^3,  SR = sum g E (1 - tau^2/a^2)
//    and folding them with the pair's factors into its gradient
//    accumulators.
//  - A warp-shuffle reduction over lanes (i.e. over sensors and samples) at
//    the end of the ball gives dL/d(x, y, z, a, p); one lane writes it.
//  - 4D mode recomputes the deformed state of the ball per frame in registers
//    (never stored) and applies the chain rule of Eq. 1-2, accumulating the
//    (omega, theta, sigma) gradients in per-warp shared memory across frames.
//
// Derivatives used, for v = A tau E, A = p/(2R), E = exp(-tau^2/(2a^2)),
// tau = R - c t_k, u = tau s, s = K_S/a (so E = 2^(-u^2)):
//   dv/dp = tau E/(2R)                     -> gp += S1 * a/(2 R K_S)
//   dv/da = A tau^3 E / a^3                -> ga += S3 * A/K_S^3
//   dv/dR = -A tau E/R + A E (1 - tau^2/a^2) -> dR = S1 * (-A a/(R K_S)) + A SR
//   dR/dmu = (mu - x_s)/R.
#include <algorithm>
#include <type_traits>

#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kAdjWarps = 8;
// Static mode runs one block of 32 warps per SM: its shared memory is one
// copy of the sensor table per SM, which leaves the most L1 to the residual
// rows that neighbouring balls re-read (8-warp blocks, four per SM, hold four
// copies and measured 4% slower with 37% more L2 traffic).
constexpr int kAdjStaticWarps = 32;

// dL/d(x, y, z, a, p) of one ball at frame f, summed over all sensors and
// samples.  Returns the totals (identical in every lane).
// Sensor coordinates are read from sens[c * sstr + s] (shared memory, or the
// global sensor array of a batched scene).
// Bit position of the (i+1)-th set bit of m (0 <= i < popc(m)), by binary
// search over prefix counts.
__device__ __forceinline__ int nth_set_bit(unsigned m, int i) {
  int lo = 0;
#pragma unroll
  for (int w = 16; w > 0; w >>= 1)
    if (__popc(m & ((1u << (lo + w)) - 1u)) <= i) lo += w;
  return lo;
}

// Walk forms: eight samples per step from one 256-bit load (rows 32-byte
// aligned) or from two float4 loads; kWalkAuto picks per call.
enum WalkForm { kWalkFloat4 = 0, kWalkWide = 1, kWalkAuto = 2 };

template <int WALK>
__device__ __forceinline__ void ball_frame_grad(const Acq &q, const float *gframe, const float *sens, int sstr,
                                                int lane, float bx, float by, float bz, float a, float p,
                                                float out[5], bool &dom) {
  const int S = q.S, T = q.T;
  const float umax2 = (q.kappa * K_S) * (q.kappa * K_S);  // the forward's window test u^2 <= umax2
  // 256-bit residual loads need 32-byte aligned rows
  const bool wide = WALK == kWalkWide ||
                    (WALK == kWalkAuto && (T & 7) == 0 && (reinterpret_cast<uintptr_t>(gframe) & 31) == 0);
  float gx = 0.f, gy = 0.f, gz = 0.f, ga = 0.f, gp = 0.f;
  if (a > 0.f && p != 0.f) {
    for (int s0 = 0; s0 < S; s0 += 32) {
      int W = 0, klo = 0;
      float u0 = 0.f, du = 0.f, R = 0.f;
      if (s0 + lane < S) {
        const int s = s0 + lane;
        const float sx = sens[s], sy = sens[sstr + s], sz = sens[2 * sstr + s];
        const PairWin w = pair_window<false>(q, bx, by, bz, a, p, sx, sy, sz, 0, T - 1);
        dom |= w.domain_err;
        W = w.W;
        klo = w.klo;
        u0 = w.u0;
        du = w.du;
        R = w.R;
      }
      // compact the valid pairs to the front lanes: lane i takes the i-th
      // valid pair (register shuffles; no shared memory)
      const unsigned mask = __ballot_sync(FULL, W > 0);
      const int nv = __popc(mask);
      if (nv == 0) continue;
      const bool act = lane < nv;
      // An inactive lane takes a copy of the first valid pair (its walk
      // reads inside that pair's window and its sums are discarded).
      const int src = mask == FULL ? lane : nth_set_bit(mask, act ? lane : 0);
      if (mask != FULL) {
        W = __shfl_sync(FULL, W, src);
        klo = __shfl_sync(FULL, klo, src);
        u0 = __shfl_sync(FULL, u0, src);
        du = __shfl_sync(FULL, du, src);
        R = __shfl_sync(FULL, R, src);
      }
      const int sp = s0 + src;  // sensor of this lane's pair
      // Each lane walks its pair's whole window, eight (or four) consecutive
      // samples per step (one 256-bit or float4 residual load, issued one
      // step ahead; packed FP32x2 halves).  All pairs belong to one ball, so
      // their windows have nearly the same length and the lanes finish
      // together.  Samples of the aligned loads outside the window get
      // weight 0 from the window test (u^2 <= (kappa K_S)^2, the forward's
      // own test).
      const float2 one = make_float2(1.f, 1.f);
      const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
      {
        const int khi = act ? klo + W - 1 : -1;
        const float *rowf = gframe + (long long)sp * T;
        float2 S1 = make_float2(0.f, 0.f), S3 = S1, SR = S1;
        // nsq = -u^2 (the exponent of E = 2^(-u^2)) from one packed multiply
        // by -u; S3 accumulates -sum g E u^3 and is negated once per pair
        const float2 pk2 = make_float2(K_2LN2, K_2LN2);
        auto half = [&](const float2 u2, const float2 g2) {
          const float2 nsq = __fmul2_rn(u2, make_float2(-u2.x, -u2.y));             // -u^2
          // exp(-tau^2/(2a^2)) inside the window, 0 outside it (compare and
          // select on the ALU pipe, which has room; the FMA pipe has not)
          const float2 E = make_float2(nsq.x >= -umax2 ? ex2(nsq.x) : 0.f, nsq.y >= -umax2 ? ex2(nsq.y) : 0.f);
          const float2 ge = __fmul2_rn(g2, E);
          const float2 gu = __fmul2_rn(ge, u2);
          S1 = __fadd2_rn(S1, gu);                                                   // sum g E u
          S3 = __ffma2_rn(gu, nsq, S3);                                              // -sum g E u^3
          SR = __ffma2_rn(ge, __ffma2_rn(nsq, pk2, one), SR);                        // sum g E (1 - tau^2/a^2)
        };
        auto halfu = [&](const float2 u2, const float2 g2) {  // `half` inside the window (no test)
          const float2 nsq = __fmul2_rn(u2, make_float2(-u2.x, -u2.y));
          const float2 E = make_float2(ex2(nsq.x), ex2(nsq.y));
          const float2 ge = __fmul2_rn(g2, E);
          const float2 gu = __fmul2_rn(ge, u2);
          S1 = __fadd2_rn(S1, gu);
          S3 = __ffma2_rn(gu, nsq, S3);
          SR = __ffma2_rn(ge, __ffma2_rn(nsq, pk2, one), SR);
        };
        // The walk, eight samples per step.  WIDE: one 256-bit load per step
        // from a 32-byte aligned start (rows are 32-byte aligned when
        // T % 8 == 0; a load starting at k <= khi <= T - 1 with k % 8 == 0
        // ends at k + 7 <= T - 1).  Else two float4 loads from a 16-byte
        // aligned start (T % 4 == 0), the second one predicated on starting
        // inside the walk (a float4 starting at k <= khi with k % 4 == 0 ends
        // at k + 3 <= T - 1).
        auto walk = [&](auto W) {
          constexpr bool WIDE = decltype(W)::value;
          const int ka = WIDE ? (klo & ~7) : (klo & ~3);
          const int nit = act ? ((khi - ka) >> 3) + 1 : 0;
          const int nmax = __reduce_max_sync(FULL, nit);
          int k = ka;
          float2 ua, ub, uc, ud;  // u at k, k + 1 | k + 2, k + 3 | k + 4, k + 5 | k + 6, k + 7
          ua.x = fmaf((float)(k - klo), -du, u0);
          ua.y = ua.x - du;
          ub.x = fmaf(-2.f, du, ua.x);
          ub.y = fmaf(-3.f, du, ua.x);
          uc.x = fmaf(-4.f, du, ua.x);
          uc.y = fmaf(-5.f, du, ua.x);
          ud.x = fmaf(-6.f, du, ua.x);
          ud.y = fmaf(-7.f, du, ua.x);
          const float2 nd8 = make_float2(-8.f * du, -8.f * du);
          const float *pk = rowf + k;
          // the step starting at p = pk + off, k + off: predicated on lying in
          // the walk (x keeps its zeros past it) or, for the first half of a
          // step inside every lane's walk, unpredicated
          auto load = [&](int off, bool first_in_walk, float4 &x0, float4 &x1) {
            if constexpr (WIDE) {
              if (first_in_walk)
                ldg8(pk + off, x0, x1);
              else
                ldg8_if(pk + off, k + off <= khi, x0, x1);
            } else {
              if (first_in_walk || k + off <= khi) x0 = __ldg(reinterpret_cast<const float4 *>(pk + off));
              if (k + off + 4 <= khi) x1 = __ldg(reinterpret_cast<const float4 *>(pk + off + 4));
            }
          };
          auto eval = [&](auto masked, const float4 &x0, const float4 &x1) {
            if (decltype(masked)::value) {
              half(ua, make_float2(x0.x, x0.y));
              half(ub, make_float2(x0.z, x0.w));
              half(uc, make_float2(x1.x, x1.y));
              half(ud, make_float2(x1.z, x1.w));
            } else {
              halfu(ua, make_float2(x0.x, x0.y));
              halfu(ub, make_float2(x0.z, x0.w));
              halfu(uc, make_float2(x1.x, x1.y));
              halfu(ud, make_float2(x1.z, x1.w));
            }
            ua = __fadd2_rn(ua, nd8);
            ub = __fadd2_rn(ub, nd8);
            uc = __fadd2_rn(uc, nd8);
            ud = __fadd2_rn(ud, nd8);
            pk += 8;
            k += 8;
          };
          // A step with the window test, its successor's load predicated on
          // lying in the walk (zeros past it).
          auto edge_step = [&](float4 &c0, float4 &c1) {
            float4 n0 = zero4, n1 = zero4;
            load(8, false, n0, n1);
            eval(std::true_type{}, c0, c1);
            c0 = n0;
            c1 = n1;
          };
          // Only a walk's first and last step can hold samples outside its
          // window: steps 1 .. nit - 2 lie strictly inside it (the test is
          // exactly 1 there).  Steps 1 .. e1 - 1, inside every active lane's
          // walk, skip the test, and their successors' loads (steps up to
          // e1 <= mn - 1 <= nit - 1) lie inside every active lane's walk, so
          // they are issued unpredicated (an inactive lane reads pair 0's row
          // inside pair 0's walk and discards its sums).  The split is
          // warp-uniform.
          const int mn = __reduce_min_sync(FULL, act ? nit : 0x7fffffff);
          const int e1 = min(mn - 1, nmax);
          float4 c0 = zero4, c1 = zero4;
          load(0, false, c0, c1);
          int it = 0;
          if (nmax > 0) {
            edge_step(c0, c1);
            ++it;
          }
          for (; it + 1 < e1; it += 2) {  // two interior steps, loads double-buffered
            float4 n0 = zero4, n1 = zero4;
            load(8, true, n0, n1);
            eval(std::false_type{}, c0, c1);
            if constexpr (!WIDE) c1 = zero4;
            load(8, true, c0, c1);
            eval(std::false_type{}, n0, n1);
          }
          if (it < e1) {
            float4 n0 = zero4, n1 = zero4;
            load(8, true, n0, n1);
            eval(std::false_type{}, c0, c1);
            c0 = n0;
            c1 = n1;
            ++it;
          }
          for (; it < nmax; ++it) edge_step(c0, c1);
        };
        if constexpr (WALK == kWalkWide) {
          walk(std::true_type{});
        } else if constexpr (WALK == kWalkFloat4) {
          walk(std::false_type{});
        } else {
          if (wide)
            walk(std::true_type{});
          else
            walk(std::false_type{});
        }
        const float s1 = S1.x + S1.y, s3 = -(S3.x + S3.y), sr = SR.x + SR.y;
        if (act) {
          // the pair's gradient factors (see the derivatives above)
          const float sx = sens[sp], sy = sens[sstr + sp], sz = sens[2 * sstr + sp];
          const float invR = __fdividef(1.f, R);
          const float amp = 0.5f * p * invR;  // A = p/(2R)
          const float aK = a * (1.f / K_S);   // 1/s
          gp = fmaf(s1, 0.5f * invR * aK, gp);
          ga = fmaf(s3, amp * (1.f / (K_S * K_S * K_S)), ga);
          const float dR = fmaf(s1, -amp * invR * aK, amp * sr);
          gx = fmaf(dR, (bx - sx) * invR, gx);
          gy = fmaf(dR, (by - sy) * invR, gy);
          gz = fmaf(dR, (bz - sz) * invR, gz);
        }
      }
    }
  }
  out[0] = warp_sum(gx);
  out[1] = warp_sum(gy);
  out[2] = warp_sum(gz);
  out[3] = warp_sum(ga);
  out[4] = warp_sum(gp);
}

__device__ __forceinline__ void load_sensors(const AdjArgs &A, float *ssens) {
  const int S = A.q.S;
  for (int i = threadIdx.x; i < 3 * S; i += blockDim.x) {
    const int c = i / S, s = i - c * S;
    ssens[i] = A.q.sensors[c * A.q.sstride + s];
  }
}

// Static mode: item = (frame, ball).  QUEUE: persistent warps take items
// from the work-queue counter A.queue; else a grid-stride loop.  WIDE: the
// residual rows are 32-byte aligned (256-bit loads), else float4 loads.
// (One instantiation per combination, so that each holds only its own
// loop's and walk's state.)
template <bool QUEUE, bool WIDE>
__global__ void __launch_bounds__(32 * kAdjStaticWarps, 1) k_adjoint_static(const AdjArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *ssens = reinterpret_cast<float *>(smem_raw);
  load_sensors(A, ssens);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool dom = false;
  auto body = [&](long long item) {
    const int f = (int)(item / A.n);
    const long long b = item - (long long)f * A.n;
    const float *st = A.state + (long long)f * 5 * A.stride;
    float v[5];
    // lanes 0..4 fetch the five channels, then broadcast
    const float mine = lane < 5 ? st[lane * A.stride + b] : 0.f;
#pragma unroll
    for (int c = 0; c < 5; ++c) v[c] = __shfl_sync(FULL, mine, c);
    float g[5];
    ball_frame_grad<WIDE ? kWalkWide : kWalkFloat4>(A.q, A.g + (long long)f * A.q.S * A.q.T, ssens, A.q.S, lane,
                                                     v[0], v[1], v[2], v[3],
                       v[4], g, dom);
    const float sc = A.frame_scale ? __ldg(A.frame_scale + f) : 1.f;
    if (lane < 5) {
      float gv = g[0];
#pragma unroll
      for (int c = 1; c < 5; ++c)
        if (lane == c) gv = g[c];
      gv *= sc;
      float *dst = A.g_state + (long long)f * 5 * A.stride + lane * A.stride + b;
      *dst = (A.flags & PA_ACCUMULATE) ? *dst + gv : gv;
    }
  };
  if constexpr (QUEUE) {
    // Persistent warps take A.queue_chunk items at a time from the counter,
    // so a warp that drew cheap balls (small windows) takes more of them and
    // no block waits for its slowest warp.  Each item is still computed whole
    // by one warp: the results do not depend on the assignment.
    while (true) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(A.queue, (unsigned long long)A.queue_chunk);
      base = __shfl_sync(FULL, base, 0);
      if ((long long)base >= A.n_items) break;
      const long long end = min((long long)base + A.queue_chunk, A.n_items);
      for (long long item = (long long)base; item < end; ++item) body(item);
    }
  } else {
    for (long long item = (long long)blockIdx.x * kAdjStaticWarps + warp; item < A.n_items;
         item += (long long)gridDim.x * kAdjStaticWarps)
      body(item);
  }
  if (dom) set_error(A.err, PA_ERR_DOMAIN);
}

// 4D mode: item = ball; frames looped inside, in chunks of kAdj4dFrames.
// Pass 1 (per frame): H of Eq. 2 for the 5 channels (lanes over basis
// functions), the deformed state of Eq. 1, the state gradient of the ball at
// that frame, and its share of the canonical gradient; the scaled frame
// gradients g_c(f) q0_c go to a per-warp buffer.  Pass 2: lanes over the
// (channel, basis) slots sum the chain rule over the buffered frames and write
// each (omega, theta, sigma) gradient once per chunk.  The deformation
// parameters are read through L1/L2 rather than held in shared memory, which
// keeps the block at ~12 KB of shared memory (sensors and the frame buffers)
// and 4 blocks per SM.
constexpr int kAdj4dFrames = 32;

__global__ void __launch_bounds__(32 * kAdjWarps, 4) k_adjoint_4d(const AdjArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = A.nb;
  const int per = 5 * nb;
  float *ssens = reinterpret_cast<float *>(smem_raw);
  float *gbase = ssens + 3 * A.q.S;  // per warp: [kAdj4dFrames][5] scaled frame gradients
  load_sensors(A, ssens);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *gq = gbase + warp * (kAdj4dFrames * 5);
  const float L2E_HALF = 0.72134752044448170368f;  // log2(e)/2
  const bool acc = (A.flags & PA_ACCUMULATE) != 0;
  bool dom = false;
  for (long long b = (long long)blockIdx.x * kAdjWarps + warp; b < A.n_items;
       b += (long long)gridDim.x * kAdjWarps) {
    const float mine = lane < 5 ? A.canon[lane * A.stride + b] : 0.f;
    float q0[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) q0[c] = __shfl_sync(FULL, mine, c);
    float gcan[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int f0 = 0; f0 < A.F; f0 += kAdj4dFrames) {
      const int fc = min(kAdj4dFrames, A.F - f0);
      // pass 1
      for (int j = 0; j < fc; ++j) {
        const int f = f0 + j;
        const float t = __ldg(A.t_frames + f);
        float H[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          float h = 0.f;
          for (int n = lane; n < nb; n += 32) {
            const long long gi = (long long)(c * nb + n) * A.stride + b;
            const float sg = __ldg(A.sigma + gi);
            if (sg > 0.f) {
              const float d = (t - __ldg(A.theta + gi)) / sg;
              h = fmaf(__ldg(A.omega + gi), ex2(-d * d * L2E_HALF), h);
            } else {
              dom = true;  // term skipped, as in pa_deform_balls
            }
          }
          H[c] = warp_sum(h);
        }
        float g[5];
        ball_frame_grad<kWalkFloat4>(A.q, A.g + (long long)f * A.q.S * A.q.T, ssens, A.q.S, lane, q0[0] * (1.f + H[0]),
                        q0[1] * (1.f + H[1]), q0[2] * (1.f + H[2]), q0[3] * (1.f + H[3]), q0[4] * (1.f + H[4]), g,
                        dom);
        const float sc = A.frame_scale ? __ldg(A.frame_scale + f) : 1.f;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const float gc = g[c] * sc;
          gcan[c] = fmaf(gc, 1.f + H[c], gcan[c]);
          if (lane == c) gq[j * 5 + c] = gc * q0[c];
        }
      }
      __syncwarp();
      // pass 2: with d = (t_f - theta)/sigma, b = exp(-d^2/2) and w = g q0 b:
      // dL/domega += sum w, dL/dtheta += omega/sigma sum w d,
      // dL/dsigma += omega/sigma sum w d^2
      for (int i = lane; i < per; i += 32) {
        const int c = i / nb;
        const long long gi = (long long)i * A.stride + b;  // [ch][n] rows are contiguous in i
        const float om = __ldg(A.omega + gi), th = __ldg(A.theta + gi), sg = __ldg(A.sigma + gi);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, is = 0.f;
        if (sg > 0.f) {
          is = 1.f / sg;
          for (int j = 0; j < fc; ++j) {
            const float d = (__ldg(A.t_frames + f0 + j) - th) * is;
            const float w = gq[j * 5 + c] * ex2(-d * d * L2E_HALF);
            s0 += w;
            s1 = fmaf(w, d, s1);
            s2 = fmaf(w * d, d, s2);
          }
        }
        const float oi = om * is;
        float vo = s0, vt = oi * s1, vs = oi * s2;
        if (f0 > 0 || acc) {
          vo += A.g_omega[gi];
          vt += A.g_theta[gi];
          vs += A.g_sigma[gi];
        }
        A.g_omega[gi] = vo;
        A.g_theta[gi] = vt;
        A.g_sigma[gi] = vs;
      }
      __syncwarp();
    }
    if (lane < 5) {
      float gv = gcan[0];
#pragma unroll
      for (int c = 1; c < 5; ++c)
        if (lane == c) gv = gcan[c];
      float *dst = A.g_state + lane * A.stride + b;
      *dst = acc ? *dst + gv : gv;
    }
  }
  if (dom) set_error(A.err, PA_ERR_DOMAIN);
}

// Batched static mode: persistent warps take chunks of A.chunk (scene, frame,
// ball) items from a global counter; scenes are ordered heaviest first by the
// host.

__global__ void __launch_bounds__(32 * kAdjWarps) k_adjoint_batched(const BatchAdjArgs A) {
  const int lane = threadIdx.x & 31;
  bool dom = false;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(A.counter, (unsigned long long)A.chunk);
    base = __shfl_sync(FULL, base, 0);
    if ((long long)base >= A.total_items) break;
    const long long end = min((long long)base + A.chunk, A.total_items);
    for (long long item = (long long)base; item < end; ++item) {
      int sc = 0;
      while (sc + 1 < A.n_scenes && item >= A.sc[sc + 1].item_begin) ++sc;
      const SceneAdj &d = A.sc[sc];
      const long long local = item - d.item_begin;
      const int f = (int)(local / d.n);
      const long long b = local - (long long)f * d.n;
      const float *st = d.state + (long long)f * 5 * d.stride;
      const float mine = lane < 5 ? st[lane * d.stride + b] : 0.f;
      float v[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) v[c] = __shfl_sync(FULL, mine, c);
      float g[5];
      ball_frame_grad<kWalkAuto>(d.q, d.g + (long long)f * d.q.S * d.q.T, d.q.sensors, d.q.sstride, lane, v[0], v[1], v[2],
                      v[3], v[4], g, dom);
      if (lane < 5) {
        float gv = g[0];
#pragma unroll
        for (int c = 1; c < 5; ++c)
          if (lane == c) gv = g[c];
        float *dst = d.g_state + (long long)f * 5 * d.stride + lane * d.stride + b;
        *dst = (A.flags & PA_ACCUMULATE) ? *dst + gv : gv;
      }
    }
  }
  if (dom) set_error(A.err, PA_ERR_DOMAIN);
}


// Grid-stride launch of a kernel with `warps` warps per block and one item
// per warp and trip.
template <typename K>
cudaError_t launch_gridstride(K kern, int warps, const AdjArgs &a, size_t smem, int sms, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * warps, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const long long need = (a.n_items + warps - 1) / warps;
  const long long grid = std::max(1LL, std::min(need, (long long)sms * occ * 4));
  kern<<<(unsigned)grid, 32 * warps, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t adj_static_smem(int S) { return sizeof(float) * 3 * (size_t)S; }
size_t adj_4d_smem(int S) { return adj_static_smem(S) + sizeof(float) * (size_t)kAdjWarps * kAdj4dFrames * 5; }

template <bool WIDE>
cudaError_t launch_adjoint_static_form(const AdjArgs &a0, int sms, cudaStream_t st) {
  const size_t smem = adj_static_smem(a0.q.S);
  if (a0.queue == nullptr)
    return launch_gridstride(k_adjoint_static<false, WIDE>, kAdjStaticWarps, a0, smem, sms, st);
  // work queue: one wave of persistent blocks
  AdjArgs a = a0;
  cudaError_t e =
      cudaFuncSetAttribute(k_adjoint_static<true, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adjoint_static<true, WIDE>, 32 * kAdjStaticWarps, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const long long warps = (long long)sms * occ * kAdjStaticWarps;
  // Items per grab: one while a warp's share is small, so that the balls in
  // flight at any time are the fewest consecutive ones (neighbours in space,
  // whose residual windows overlap and are shared in L1: one item per grab
  // against two took L2 traffic from 6.6 to 4.9 GB on static-100k) and the
  // tail is short; up to 16 for very large calls, to bound the atomics.
  a.queue_chunk = (int)std::max(1LL, std::min(16LL, a.n_items / (warps * 32)));
  e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  k_adjoint_static<true, WIDE><<<(unsigned)(sms * occ), 32 * kAdjStaticWarps, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_static(const AdjArgs &a, int sms, cudaStream_t st) {
  if (a.n_items == 0) return cudaSuccess;
  // every frame's rows are 32-byte aligned when the base is and T % 8 == 0
  const bool wide = (a.q.T & 7) == 0 && (reinterpret_cast<uintptr_t>(a.g) & 31) == 0;
  return wide ? launch_adjoint_static_form<true>(a, sms, st) : launch_adjoint_static_form<false>(a, sms, st);
}

cudaError_t launch_adjoint_batched(const BatchAdjArgs &a, int sms, cudaStream_t st) {
  if (a.total_items == 0) return cudaSuccess;
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adjoint_batched, 32 * kAdjWarps, 0);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const long long need = (a.total_items + a.chunk - 1) / a.chunk;
  const long long grid = std::max(1LL, std::min((need + kAdjWarps - 1) / kAdjWarps, (long long)sms * occ));
  k_adjoint_batched<<<(unsigned)grid, 32 * kAdjWarps, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_4d(const AdjArgs &a, int sms, cudaStream_t st) {
  if (a.n_items == 0) return cudaSuccess;
  // Each warp takes its ball through every frame of a launch, so all of the
  // launch's residual frames are live in L2 at once.  Launch over chunks of
  // at most ~32 MB of [S][T] residuals (the 126 MB L2 then holds them), the
  // chunks after the first accumulating into the outputs.
  const long long frame_bytes = std::max(1LL, (long long)a.q.S * a.q.T * (long long)sizeof(float));
  const int fc = (int)std::max(1LL, std::min<long long>(a.F, (32LL << 20) / frame_bytes));
  for (int f0 = 0; f0 < a.F; f0 += fc) {
    AdjArgs c = a;
    c.F = std::min(fc, a.F - f0);
    c.t_frames = a.t_frames + f0;
    c.g = a.g + (long long)f0 * a.q.S * a.q.T;
    c.frame_scale = a.frame_scale ? a.frame_scale + f0 : nullptr;
    if (f0 > 0) c.flags |= PA_ACCUMULATE;
    cudaError_t e = launch_gridstride(k_adjoint_4d, kAdjWarps, c, adj_4d_smem(a.q.S), sms, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pa
