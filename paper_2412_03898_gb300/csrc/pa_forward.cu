// Forward projection kernel (the radiator of Sec. 2.2, last paragraph) and
// the contribution counter.
//
// Design (GB300, sm_103a):
//  - One CTA owns a tile of s_tile sensors x t_tile samples of one frame and a
//    range of balls.  Each warp owns one sensor: its trace tile lives in
//    shared memory and only that warp writes it, so accumulation is a plain
//    load-add-store with no atomics.
//  - Ball tiles (x, y, z, a, p rows of nb_tile balls) are streamed from HBM
//    into shared memory by TMA bulk copies (cp.async.bulk) completing on
//    mbarriers, double buffered, issued by one thread.
//  - Each landed ball tile is swept in radius-class order (a stable in-CTA
//    counting sort), so that grouped windows have similar lengths.
//  - Per 32-ball chunk, the 32 lanes compute the window and phase of 32
//    (ball, sensor) pairs in parallel (double-float distance, once per pair).
//    The warp sorts the pairs by first sample (bitonic network on shuffles);
//    lane i then holds the i-th pair, and each group of G consecutive sorted
//    pairs gets one shared-memory record with its first sample, its step
//    count and every member's phase at that sample.  The warp sweeps each
//    group over the union of its windows: each lane owns one sample of a
//    32-sample step and adds the G balls' pulses to it in one register, one
//    predicated FMA per ball,
//        u -= 32 du;  v = amp u 2^(-u^2)  if |u| <= kappa K_S
//    then does one compensated shared-memory update per sample and group.
//    Sorted groups overlap almost completely, so the sweep wastes few lanes;
//    two steps per loop trip give independent chains.  Trace rows carry 32
//    samples of padding, so a group's last step needs no bound test (lanes
//    past every window add an exact zero).
//  - Trace tiles are flushed with coalesced float4 stores.  With more than
//    one ball split, partial traces go to the workspace and a second kernel
//    sums them in split order (deterministic).
#include <algorithm>

#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kMaxThreads = 512;  // at most 16 sensors (warps) per CTA

constexpr int kRowPad = 32;   // samples of padding after every trace row
constexpr int kClasses = 17;  // 16 radius classes + 1 for slots past the tile's end

// Bytes of the per-tile ordering area: class counts [kClasses][nchunk] and
// the order [nchunk * 32], nchunk = 32-ball chunks per tile.
__host__ __device__ constexpr int order_bytes(int nb_tile) {
  return ((((nb_tile + 31) >> 5) * (kClasses * 4 + 32 * 2)) + 15) & ~15;
}

// Shared-memory layout of a forward CTA.
struct FwdSmem {
  uint64_t *bars;         // 2 mbarriers (TMA stages)
  float *sball;           // [2][5][nb_tile] ball tiles
  float *sgrp;            // [s_tile][128] group records of the current chunk
  int *scnt;              // [kClasses][nchunk] class counts, then their offsets
  unsigned short *sperm;  // [nchunk * 32] tile positions in sweep order
  float *str;             // [s_tile][t_tile + kRowPad] trace tiles (high part)
  float *strlo;           // [s_tile][t_tile + kRowPad] rounding errors of str (compensated sum)
};

__device__ __forceinline__ FwdSmem fwd_smem(unsigned char *raw, int s_tile, int t_tile, int nb_tile) {
  FwdSmem m;
  m.bars = reinterpret_cast<uint64_t *>(raw);
  m.sball = reinterpret_cast<float *>(raw + 128);
  m.sgrp = m.sball + 2 * 5 * nb_tile;
  m.scnt = reinterpret_cast<int *>(m.sgrp + s_tile * 128);
  m.sperm = reinterpret_cast<unsigned short *>(m.scnt + kClasses * ((nb_tile + 31) >> 5));
  m.str = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(m.scnt) + order_bytes(nb_tile));
  m.strlo = m.str + s_tile * (t_tile + kRowPad);
  return m;
}

// Radius class of a ball: half-octaves of a (the float's exponent and its
// leading mantissa bit), modulo 16.  Balls of one class have windows whose
// lengths differ by less than 41%; with the cloud in spatial order, classes
// twice as large as quarter-octaves keep each class's balls closer in space,
// which pays more than the closer lengths (static-100k: 1.97 against 2.02 ms
// in Morton order, 2.08 against 2.08 ms along the tubes).
__device__ __forceinline__ int radius_class(float a) { return (int)((__float_as_uint(a) >> 22) & 15u); }

// Sweep order of one ball tile: a stable counting sort of the tile's slots by
// radius class, slots past `cnt` last.  Sorted groups of pairs then have
// windows of nearly the same length, so the union sweep wastes fewer lanes.
// The order depends only on the tile's contents (deterministic).  Block-wide:
// every thread calls it.
__device__ __forceinline__ void order_tile(const float *ba, int nbt, int cnt, int *scnt, unsigned short *sperm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int nchunk = (nbt + 31) >> 5;
  for (int j = warp; j < nchunk; j += nw) {
    const int i = j * 32 + lane;
    const int c = i < cnt ? radius_class(ba[i]) : kClasses - 1;
#pragma unroll
    for (int cc = 0; cc < kClasses; ++cc) {
      const unsigned mk = __ballot_sync(FULL, c == cc);
      if (lane == cc) scnt[cc * nchunk + j] = __popc(mk);
    }
  }
  __syncthreads();
  if (warp == 0) {
    // exclusive scan over (class, chunk), class-major
    const int E = kClasses * nchunk, L = (E + 31) >> 5;
    const int e0 = min(lane * L, E), e1 = min(e0 + L, E);
    int sum = 0;
    for (int e = e0; e < e1; ++e) sum += scnt[e];
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    int run = incl - sum;
    for (int e = e0; e < e1; ++e) {
      const int v = scnt[e];
      scnt[e] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int j = warp; j < nchunk; j += nw) {
    const int i = j * 32 + lane;
    const int c = i < cnt ? radius_class(ba[i]) : kClasses - 1;
    const unsigned same = __match_any_sync(FULL, c);
    sperm[scnt[c * nchunk + j] + __popc(same & ((1u << lane) - 1u))] = (unsigned short)i;
  }
  __syncthreads();
}

// Group records in a warp's 128-float area (16-byte aligned).  G >= 2: per
// group, H = G/2 float4 (u_x, u_y, -32 du_x, -32 du_y) of ball pairs, H float2
// (amp_x, amp_y), then (first sample, step count) as ints; stride rounded up
// to 4 floats.  G = 1: one float4 (u, -du, amp, first | steps << 16) each.
template <int G>
__host__ __device__ constexpr int grp_stride() {
  return G == 1 ? 4 : ((6 * (G / 2) + 2) + 3) & ~3;
}
static_assert(32 / 2 * grp_stride<2>() <= 128 && 32 / 4 * grp_stride<4>() <= 128 &&
                  32 / 8 * grp_stride<8>() <= 128 && 32 / 16 * grp_stride<16>() <= 128 &&
                  32 * grp_stride<1>() <= 128,
              "group records exceed a warp's area");

// One work item: frame state `state_f`, sensors [st*s_tile, +s_tile), samples
// [k0, k0+klen), balls [b_begin, b_end); `cull` enables a cheap per-chunk
// window test (for arrival bands wider than one tile).  Writes (or adds) the
// trace tile to dst_f[s][k] (frame base of a [S][T] array).  `phase` holds the
// parity of each TMA stage's next completion and is carried across items of a
// persistent CTA.  Returns false after a bounded wait ran out.
template <bool UNIFORM, int G>
__device__ __forceinline__ bool forward_item(const Acq &q, const float *state_f, long long stride,
                                             long long b_begin, long long b_end, int s_tile, int t_tile, int nbt,
                                             int st, int k0, int klen, bool cull, float *dst_f, bool acc,
                                             const FwdSmem &m, unsigned &phase, unsigned *err) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = q.T;
  const int s = st * s_tile + warp;
  const bool s_ok = s < q.S;
  const int ntiles = b_end > b_begin ? (int)((b_end - b_begin + nbt - 1) / nbt) : 0;
  float *sball = m.sball;
  uint64_t *bars = m.bars;

  __syncthreads();  // the previous item (if any) is done with the trace tiles
  float4 *str4 = reinterpret_cast<float4 *>(m.str);
  const int nz = 2 * s_tile * (t_tile + kRowPad) / 4;  // high and low parts, padding included
  for (int i = tid; i < nz; i += blockDim.x) str4[i] = make_float4(0.f, 0.f, 0.f, 0.f);

  auto issue = [&](int t) {
    const int stage = t & 1;
    const long long b0 = b_begin + (long long)t * nbt;
    const int cnt = (int)min((long long)nbt, b_end - b0);
    const unsigned bytes = (unsigned)(((cnt + 3) & ~3) * 4);
    mbar_arrive_expect_tx(&bars[stage], 5u * bytes);
#pragma unroll
    for (int ch = 0; ch < 5; ++ch)
      bulk_copy_g2s(sball + (stage * 5 + ch) * nbt, state_f + ch * stride + b0, bytes, &bars[stage]);
  };
  if (tid == 0) {
    fence_proxy_async();
    if (ntiles > 0) issue(0);
    if (ntiles > 1) issue(1);
  }
  __syncthreads();  // trace tiles zeroed

  float sx = 0.f, sy = 0.f, sz = 0.f;
  if (s_ok) {
    sx = q.sensors[s];
    sy = q.sensors[q.sstride + s];
    sz = q.sensors[2 * q.sstride + s];
  }
  float *mytr = m.str + warp * (t_tile + kRowPad);
  float *mylo = m.strlo + warp * (t_tile + kRowPad);
  float *mygrp = m.sgrp + warp * 128;
  constexpr int H = (G + 1) / 2;  // ball pairs per group
  constexpr int GS = grp_stride<G>();
  bool dom = false;
  // window bound in scaled units: |u| <= kappa K_S (Gaussian), |u| <= 1 (uniform)
  const float umax2 = UNIFORM ? 1.f : (q.kappa * K_S) * (q.kappa * K_S);

  for (int t = 0; t < ntiles; ++t) {
    const int stage = t & 1;
    const unsigned par = (phase >> stage) & 1u;
    const bool ok = mbar_wait_bounded(&bars[stage], par);
    phase ^= 1u << stage;
    const int cnt = (int)min((long long)nbt, b_end - (b_begin + (long long)t * nbt));
    const float *bx = sball + stage * 5 * nbt;
    // (after a timed-out wait the order is built from stale data and unused)
    order_tile(bx + 3 * nbt, nbt, cnt, m.scnt, m.sperm);
    if (ok && s_ok) {
      for (int c0 = 0; c0 < cnt; c0 += 32) {
        // this lane's ball: position c0 + lane of the tile's sweep order
        const int bi = c0 + lane < cnt ? (int)m.sperm[c0 + lane] : nbt;
        if (cull) {
          // cheap FP32 estimate of the window: skip chunks with no pair in
          // this tile (only when the arrival band spans several sample
          // tiles; within one tile it costs more than it saves)
          bool maybe = false;
          if (bi < cnt) {
            const float dx = bx[bi] - sx, dy = bx[nbt + bi] - sy, dz = bx[2 * nbt + bi] - sz;
            const float a = bx[3 * nbt + bi];
            const float h = (UNIFORM ? 1.f : q.kappa) * a;
            const float rc = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) - q.ct0h;
            const float lo = (rc - h) * q.inv_delta, hi = (rc + h) * q.inv_delta;
            maybe = a > 0.f && bx[4 * nbt + bi] != 0.f && hi >= (float)(k0 - 2) && lo <= (float)(k0 + klen + 1);
          }
          if (__ballot_sync(FULL, maybe) == 0) continue;
        }
        PairWin w;
        w.W = 0;
        w.u0 = w.du = w.amp = 0.f;
        w.domain_err = false;
        if (bi < cnt)
          w = pair_window<UNIFORM>(q, bx[bi], bx[nbt + bi], bx[2 * nbt + bi], bx[3 * nbt + bi],
                                   bx[4 * nbt + bi], sx, sy, sz, k0, k0 + klen - 1);
        dom |= w.domain_err;
        const bool valid = w.W > 0;
        const int nv = __popc(__ballot_sync(FULL, valid));
        if (nv == 0) continue;
        if constexpr (G == 16) {
          // Two groups of 16 per chunk: a pivot at the mean first sample splits
          // the pairs (below it first, then the other valid pairs, then the
          // invalid ones as zero-amplitude pads).  The order inside a group
          // does not matter, since each group is swept over the union of its
          // windows, so this ballot partition replaces a full sort.
          const unsigned vmask = __ballot_sync(FULL, valid);
          const int key = valid ? w.klo - k0 : 0;  // first sample relative to k0
          const int sum = (int)__reduce_add_sync(FULL, (unsigned)key);
          const bool below = valid && key * nv < sum;
          const unsigned bmask = __ballot_sync(FULL, below);
          const unsigned lt = (1u << lane) - 1u;
          const int nb = __popc(bmask);
          const int pos = below ? __popc(bmask & lt)
                                : (valid ? nb + __popc(vmask & ~bmask & lt) : nv + __popc(~vmask & lt));
          const bool first = pos < 16;
          const int kend = valid ? key + w.W - 1 : -1;
          const int kmin0 = __reduce_min_sync(FULL, valid && first ? key : 0x7fffffff);
          const int kmin1 = __reduce_min_sync(FULL, valid && !first ? key : 0x7fffffff);
          const int kmax0 = __reduce_max_sync(FULL, first ? kend : -1);
          const int kmax1 = __reduce_max_sync(FULL, first ? -1 : kend);
          const int kmin = first ? kmin0 : kmin1;
          const int nsteps = (((first ? kmax0 : kmax1) - kmin) >> 5) + 1;
          // phase at the group's first sample (kmin - key is a small exact
          // integer); pads sit far outside every window with zero amplitude
          const float us = valid ? fmaf((float)(kmin - key), -w.du, w.u0) : 1e30f;
          const float nd = valid ? -w.du : 0.f;
          const float am = valid ? w.amp : 0.f;
          __syncwarp();  // the previous chunk's groups are done with the records
          const int j = pos & 15;
          float *r = mygrp + (pos >> 4) * GS;
          r[(j >> 1) * 4 + (j & 1)] = us;
          r[(j >> 1) * 4 + 2 + (j & 1)] = 32.f * nd;  // one 32-sample step
          r[4 * H + j] = am;
          if (j == 0) reinterpret_cast<int2 *>(r + 6 * H)[0] = make_int2(kmin, nsteps);
        } else {
          // sort by first sample; invalid pairs last; lane index in the low bits
          const unsigned key = warp_sort(((valid ? (unsigned)(w.klo - k0) : 0xffffu) << 5) | (unsigned)lane, lane);
          // lane i takes the i-th pair in that order (positions >= nv are pads)
          const int src = (int)(key & 31u);
          const float pu0 = __shfl_sync(FULL, w.u0, src);
          const float pdu = __shfl_sync(FULL, w.du, src);
          const float pamp = __shfl_sync(FULL, w.amp, src);
          const int pW = __shfl_sync(FULL, w.W, src);
          const bool real = lane < nv;
          const int kl = (int)(key >> 5);  // first sample relative to k0
          // the group's first sample (sorted: its first member's) and last sample
          const int kmin = __shfl_sync(FULL, kl, lane & ~(G - 1));
          int kmax = real ? kl + pW - 1 : -1;
#pragma unroll
          for (int o = 1; o < G; o <<= 1) kmax = max(kmax, __shfl_xor_sync(FULL, kmax, o));
          const int nsteps = ((kmax - kmin) >> 5) + 1;
          // phase at the group's first sample: kmin - kl is a small exact
          // integer; pads sit far outside every window with zero amplitude
          const float us = real ? fmaf((float)(kmin - kl), -pdu, pu0) : 1e30f;
          const float nd = real ? -pdu : 0.f;
          const float am = real ? pamp : 0.f;
          __syncwarp();  // the previous chunk's groups are done with the records
          if (G == 1) {
            reinterpret_cast<float4 *>(mygrp)[lane] = make_float4(us, nd, am, __int_as_float(kmin | (nsteps << 16)));
          } else {
            const int j = lane & (G - 1);
            float *r = mygrp + (lane / G) * GS;
            r[(j >> 1) * 4 + (j & 1)] = us;
            r[(j >> 1) * 4 + 2 + (j & 1)] = 32.f * nd;  // one 32-sample step
            r[4 * H + j] = am;
            if (j == 0) reinterpret_cast<int2 *>(r + 6 * H)[0] = make_int2(kmin, nsteps);
          }
        }
        __syncwarp();
        const float lf = (float)lane;
        const float lf32 = lf * 0.03125f;  // lane / 32, exact
        for (int g0 = 0; g0 < nv; g0 += G) {
          // balls in twos: u, its step and amp*u of two balls share one packed
          // FP32x2 instruction; u starts at this lane's first sample
          float2 u2[H], nd2[H], amp2[H];
          int kb, ns;
          if (G == 1) {
            const float4 r = reinterpret_cast<const float4 *>(mygrp)[g0];
            u2[0] = make_float2(fmaf(lf, r.y, r.x), 1e30f);
            nd2[0] = make_float2(32.f * r.y, 0.f);
            amp2[0] = make_float2(r.z, 0.f);
            kb = __float_as_int(r.w) & 0xffff;
            ns = __float_as_int(r.w) >> 16;
          } else {
            const float *r = mygrp + (g0 / G) * GS;
#pragma unroll
            for (int h = 0; h < H; ++h) {
              // the record holds 32 x (-du); (lane / 32) x that is exactly
              // lane x (-du), so u starts at this lane's sample exactly
              const float4 ud = reinterpret_cast<const float4 *>(r)[h];
              const float2 nd32 = make_float2(ud.z, ud.w);
              u2[h] = __ffma2_rn(make_float2(lf32, lf32), nd32, make_float2(ud.x, ud.y));
              nd2[h] = nd32;
              amp2[h] = reinterpret_cast<const float2 *>(r + 4 * H)[h];
            }
            const int2 kn = reinterpret_cast<const int2 *>(r + 6 * H)[0];
            kb = kn.x;
            ns = kn.y;
          }
          float *pt = mytr + kb + lane;
          float *pl = mylo + kb + lane;
          // two steps per trip: their loads, SFU work and stores interleave
#pragma unroll 2
          for (int it = 0; it < ns; ++it, pt += 32, pl += 32) {
            // the group's pulses at this sample, summed in one register: a
            // predicated FMA per ball inside its window (fewer instructions
            // than a select per ball and a tree of partial sums; the two
            // unrolled steps give the independent chains)
            float t = 0.f;
#pragma unroll
            for (int h = 0; h < H; ++h) {
              const float2 sq = __fmul2_rn(u2[h], u2[h]);
              const float2 w = __fmul2_rn(amp2[h], u2[h]);
              const float ex = UNIFORM ? 1.f : ex2(-sq.x);
              const float ey = UNIFORM ? 1.f : ex2(-sq.y);
              if (sq.x <= umax2) t = fmaf(w.x, ex, t);
              if (sq.y <= umax2) t = fmaf(w.y, ey, t);
            }
            // compensated accumulation: a sample collects the cancelling
            // pulses of thousands of balls, and a plain FP32 running sum
            // loses ~1e-5 relative by 1e5 balls.  Dekker's FastTwoSum is
            // exact when |running sum| >= |t|, which holds after the first
            // few groups; otherwise its error term loses about eps |t|.
            float hs, he;
            fast_two_sum(*pt, t, hs, he);
            *pt = hs;
            *pl += he;
#pragma unroll
            for (int h = 0; h < H; ++h) u2[h] = __fadd2_rn(u2[h], nd2[h]);
          }
          __syncwarp();  // the next group's lanes read what this one wrote
        }
      }
    }
    const int abort = __syncthreads_or(!ok);
    if (abort) {
      // A copy did not complete in time: record it and give the copy still in
      // flight a bounded chance to land before the shared memory is reused.
      // If that second wait also runs out the CTA returns with the copy
      // possibly still writing its shared memory, which is undefined: this
      // path is reached only after a real stall of the copy engine, and no
      // test makes a real copy stall (the self-test waits on an mbarrier with
      // no copy behind it).
      if (tid == 0) {
        set_error(err, PA_ERR_TIMEOUT);
        mbar_wait_bounded(&bars[stage], par);
        if (t + 1 < ntiles) mbar_wait_bounded(&bars[(t + 1) & 1], (phase >> ((t + 1) & 1)) & 1u);
      }
      __syncthreads();
      return false;
    }
    if (tid == 0 && t + 2 < ntiles) {
      fence_proxy_async();
      issue(t + 2);
    }
  }
  if (dom) set_error(err, PA_ERR_DOMAIN);

  if (s_ok) {
    float4 *d4 = reinterpret_cast<float4 *>(dst_f + (long long)s * T + k0);
    const float4 *s4 = reinterpret_cast<const float4 *>(mytr);
    const float4 *l4 = reinterpret_cast<const float4 *>(mylo);
    for (int i = lane; i < klen / 4; i += 32) {
      float4 v = s4[i];
      const float4 lo = l4[i];
      v.x += lo.x;
      v.y += lo.y;
      v.z += lo.z;
      v.w += lo.w;
      if (acc) {
        const float4 o = d4[i];
        v.x += o.x;
        v.y += o.y;
        v.z += o.z;
        v.w += o.w;
      }
      d4[i] = v;
    }
  }
  return true;
}

// First sample of sample tile `tt` when the CTA's tiles are laid over the band
// where the pulses of balls [b_begin, b_end) arrive at sensors
// [st*s_tile, st*s_tile + s_tile): the band runs from the nearest to the
// farthest point of the active balls' bounding box, widened by the largest
// window half-width and two samples.  Returns -1 when the tile holds no
// arrival (the caller has zeroed the output).  Block-wide: every thread calls
// it; `red` is shared scratch of at least 8 * (warps + 1) floats.  `whole`
// tells whether one tile holds the whole band.
template <bool UNIFORM>
__device__ int band_tile_start(const Acq &q, const float *state_f, long long stride, long long b_begin,
                               long long b_end, int s_tile, int st, int t_tile, int tt, float *red, bool &whole) {
  whole = true;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const float INF = __int_as_float(0x7f800000);
  float v[7] = {INF, INF, INF, -INF, -INF, -INF, 0.f};  // min xyz, max xyz, max a
  for (long long b = b_begin + tid; b < b_end; b += blockDim.x) {
    const float a = state_f[3 * stride + b], p = state_f[4 * stride + b];
    if (a > 0.f && p != 0.f) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float x = state_f[c * stride + b];
        v[c] = fminf(v[c], x);
        v[3 + c] = fmaxf(v[3 + c], x);
      }
      v[6] = fmaxf(v[6], a);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = fminf(v[c], __shfl_xor_sync(FULL, v[c], o));
#pragma unroll
    for (int c = 3; c < 7; ++c) v[c] = fmaxf(v[c], __shfl_xor_sync(FULL, v[c], o));
  }
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < 7; ++c) red[warp * 8 + c] = v[c];
  __syncthreads();
  if (tid < 7) {
    float r = red[tid];
    for (int w = 1; w < nw; ++w) r = tid < 3 ? fminf(r, red[w * 8 + tid]) : fmaxf(r, red[w * 8 + tid]);
    red[nw * 8 + tid] = r;
  }
  __syncthreads();
  float box[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) box[c] = red[nw * 8 + c];
  __syncthreads();  // red is reused below
  // per warp: distances from its sensor to the box
  const int s = st * s_tile + warp;
  float dmin = INF, dmax = -INF;
  if (s < q.S && box[6] > 0.f) {
    float n2 = 0.f, f2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float sc = q.sensors[c * q.sstride + s];
      const float dn = fmaxf(fmaxf(box[c] - sc, sc - box[3 + c]), 0.f);
      const float df = fmaxf(fabsf(sc - box[c]), fabsf(sc - box[3 + c]));
      n2 = fmaf(dn, dn, n2);
      f2 = fmaf(df, df, f2);
    }
    dmin = sqrtf(n2);
    dmax = sqrtf(f2);
  }
  if (lane == 0) {
    red[warp * 2] = dmin;
    red[warp * 2 + 1] = dmax;
  }
  __syncthreads();
  float rmin = INF, rmax = -INF;
  for (int w = 0; w < nw; ++w) {
    rmin = fminf(rmin, red[w * 2]);
    rmax = fmaxf(rmax, red[w * 2 + 1]);
  }
  __syncthreads();
  if (!(rmax >= rmin)) return -1;  // no active ball or no sensor
  const float h = (UNIFORM ? 1.f : q.kappa) * box[6];
  const float lo = floorf((rmin - h - q.ct0h) * q.inv_delta) - 2.f;
  const float hi = ceilf((rmax + h - q.ct0h) * q.inv_delta) + 2.f;
  const int T = q.T;
  if (!(hi >= 0.f) || !(lo <= (float)(T - 1))) return -1;
  const int kb_lo = ((int)fmaxf(lo, 0.f)) & ~3;
  const int kb_hi = (int)fminf(hi, (float)(T - 1));
  const long long start = (long long)kb_lo + (long long)tt * t_tile;
  if (start > kb_hi || start >= T) return -1;
  whole = kb_lo + (long long)t_tile > kb_hi;
  return (int)start;
}

__device__ __forceinline__ void init_bars(uint64_t *bars) {
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
}

// One CTA per (frame, sensor tile, sample tile, ball split).
template <bool UNIFORM, int G>
__global__ void __launch_bounds__(kMaxThreads, 1) k_forward(const FwdArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const FwdSmem m = fwd_smem(smem_raw, A.s_tile, A.t_tile, A.nb_tile);
  init_bars(m.bars);
  int item = blockIdx.x;
  const int split = item % A.n_splits;
  item /= A.n_splits;
  const int tt = item % A.n_ttiles;
  item /= A.n_ttiles;
  const int st = item % A.n_stiles;
  const int f = item / A.n_stiles;
  const int T = A.q.T;
  const long long b_begin = (long long)split * A.balls_per_split;
  const long long b_end = min(A.n, b_begin + A.balls_per_split);
  const float *state_f0 = A.state + (long long)f * 5 * A.stride;
  bool whole;
  const int k0 = band_tile_start<UNIFORM>(A.q, state_f0, A.stride, b_begin, b_end, A.s_tile, st, A.t_tile, tt,
                                          m.sgrp, whole);
  if (k0 < 0) return;  // no arrival in this tile; the output was zeroed
  const int klen = min(A.t_tile, T - k0);
  const bool single = A.n_splits == 1;
  float *dst_f = single ? A.out + (long long)f * A.q.S * T
                        : A.partial + ((long long)split * A.F + f) * A.q.S * T;
  unsigned phase = 0;
  forward_item<UNIFORM, G>(A.q, A.state + (long long)f * 5 * A.stride, A.stride, b_begin, b_end, A.s_tile, A.t_tile,
                           A.nb_tile, st, k0, klen, !whole, dst_f, single && (A.flags & PA_ACCUMULATE), m, phase,
                           A.err);
}

// Persistent CTAs over the work items of several scenes: an item is
// (scene, frame, sensor tile, sample tile, ball split), taken from a global
// counter in the order of the scene table (the host orders scenes by item
// cost, heaviest first).  A scene with several ball splits writes partial
// traces that the host sums afterwards (k_reduce_splits, split order).
template <int G>
__global__ void __launch_bounds__(kMaxThreads, 1) k_forward_batched(const BatchFwdArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const FwdSmem m = fwd_smem(smem_raw, A.s_tile, A.t_tile, A.nb_tile);
  __shared__ long long s_item;
  init_bars(m.bars);
  unsigned phase = 0;
  while (true) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(A.counter, 1ull);
    __syncthreads();
    const long long item = s_item;
    if (item >= A.total_items) break;
    int sc = 0;
    while (sc + 1 < A.n_scenes && item >= A.sc[sc + 1].item_begin) ++sc;
    const SceneFwd &d = A.sc[sc];
    long long local = item - d.item_begin;
    const int split = (int)(local % d.n_splits);
    local /= d.n_splits;
    const int tt = (int)(local % d.n_ttiles);
    local /= d.n_ttiles;
    const int st = (int)(local % d.n_stiles);
    const int f = (int)(local / d.n_stiles);
    const long long b_begin = (long long)split * d.balls_per_split;
    const long long b_end = min(d.n, b_begin + d.balls_per_split);
    const float *state_f = d.state + (long long)f * 5 * d.stride;
    bool whole;
    const int k0 = band_tile_start<false>(d.q, state_f, d.stride, b_begin, b_end, A.s_tile, st, A.t_tile, tt,
                                          m.sgrp, whole);
    if (k0 < 0) continue;  // no arrival in this tile; the outputs were zeroed
    const int klen = min(A.t_tile, d.q.T - k0);
    const long long frame = (long long)d.q.S * d.q.T;
    const bool single = d.n_splits == 1;
    float *dst = single ? d.out + f * frame : d.partial + ((long long)split * d.F + f) * frame;
    const bool ok = forward_item<false, G>(d.q, state_f, d.stride, b_begin, b_end, A.s_tile, A.t_tile, A.nb_tile,
                                           st, k0, klen, !whole, dst, single && (A.flags & PA_ACCUMULATE) != 0, m,
                                           phase, A.err);
    if (!ok) break;
  }
}

// out[i] (+)= sum over splits of partial[split][i], splits in order, with
// compensated (TwoSum) accumulation: partials of different ball ranges can
// cancel each other.
__global__ void k_reduce_splits(const float4 *__restrict__ partial, float4 *__restrict__ out,
                                long long n4, int n_splits, bool accumulate) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    float4 v = accumulate ? out[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int sp = 0; sp < n_splits; ++sp) {
      const float4 p = __ldg(&partial[sp * n4 + i]);
      float r;
      two_sum(v.x, p.x, v.x, r);
      e.x += r;
      two_sum(v.y, p.y, v.y, r);
      e.y += r;
      two_sum(v.z, p.z, v.z, r);
      e.z += r;
      two_sum(v.w, p.w, v.w, r);
      e.w += r;
    }
    out[i] = make_float4(v.x + e.x, v.y + e.y, v.z + e.z, v.w + e.w);
  }
}

__global__ void k_count(const Acq q, const float *state, long long n, long long stride, int F,
                        unsigned long long *out) {
  const long long total = (long long)F * q.S * n;
  unsigned long long mine = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i % n;
    const long long fs = i / n;
    const int s = (int)(fs % q.S);
    const int f = (int)(fs / q.S);
    const float *st = state + (long long)f * 5 * stride;
    const PairWin w = pair_window<false>(q, st[b], st[stride + b], st[2 * stride + b], st[3 * stride + b],
                                         st[4 * stride + b], q.sensors[s], q.sensors[q.sstride + s],
                                         q.sensors[2 * q.sstride + s], 0, q.T - 1);
    mine += (unsigned long long)w.W;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(FULL, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(out, mine);
}

}  // namespace

size_t forward_smem_bytes(int s_tile, int t_tile, int nb_tile) {
  return 128 + sizeof(float) * (size_t)(2 * 5 * nb_tile) + sizeof(float) * (size_t)(s_tile * 128) +
         (size_t)order_bytes(nb_tile) + 2 * sizeof(float) * (size_t)s_tile * (t_tile + kRowPad);
}

namespace {
using FwdKernel = void (*)(const FwdArgs);
FwdKernel forward_kernel(bool uniform, int group) {
  if (uniform) return k_forward<true, 4>;
  switch (group) {
    case 1: return k_forward<false, 1>;
    case 2: return k_forward<false, 2>;
    case 4: return k_forward<false, 4>;
    case 16: return k_forward<false, 16>;
    default: return k_forward<false, 8>;
  }
}
}  // namespace

int forward_blocks_per_sm(const FwdPlan &p, bool uniform) {
  int nb = 0;
  auto fn = forward_kernel(uniform, p.group);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 32 * p.s_tile, p.smem) != cudaSuccess) {
    // a plan larger than shared memory: the caller rejects it; leave no
    // pending error for the next launch's cudaGetLastError
    (void)cudaGetLastError();
    return 0;
  }
  return nb;
}

int forward_default_s_tile(int t_tile, int nb_tile) {
  const long long budget = 232448 - 128 - (long long)sizeof(float) * 2 * 5 * nb_tile - order_bytes(nb_tile);
  const long long per_sensor = 2LL * (long long)sizeof(float) * (t_tile + kRowPad) + (long long)sizeof(float) * 128;
  return (int)std::max(1LL, std::min(16LL, budget / per_sensor));
}

FwdPlan forward_plan(int S, int T, long long n, int F, int sms, int s_tile_o, int t_tile_o,
                     int nb_tile_o, int splits_o, int group_o) {
  FwdPlan p{};
  // 16 pairs per sweep by default: 2-5% faster than 8 on 1e5-1e6 balls
  p.group = (group_o == 1 || group_o == 2 || group_o == 4 || group_o == 8) ? group_o : 16;
  // Default: up to kDefaultTTile samples per CTA, 512-ball TMA stages, and as
  // many sensors (warps) as fit in 227 KB of shared memory with the
  // compensated (high, low) trace tiles, at most 16: 16 x 1536.  More sensors
  // per CTA share each ball's load and cull; with arrival-band tiles the
  // shorter tiles cost little.
  int tt = t_tile_o > 0 ? t_tile_o : std::min(T, kDefaultTTile);
  tt = std::min(std::min(tt, T), 16384);
  tt = (tt + 3) & ~3;
  p.t_tile = tt;
  p.nb_tile = nb_tile_o > 0 ? nb_tile_o : 512;
  p.s_tile = s_tile_o > 0 ? s_tile_o : forward_default_s_tile(tt, p.nb_tile);
  p.n_stiles = (S + p.s_tile - 1) / p.s_tile;
  p.n_ttiles = (T + p.t_tile - 1) / p.t_tile;
  p.smem = forward_smem_bytes(p.s_tile, p.t_tile, p.nb_tile);
  const long long base_ctas = std::max(1LL, (long long)F * p.n_stiles * p.n_ttiles);
  const long long max_splits = std::max(1LL, (n + p.nb_tile - 1) / p.nb_tile);
  long long splits = 1;
  if (splits_o > 0) {
    splits = splits_o;
  } else {
    // Smallest number of ball splits whose CTA count fills whole waves to at
    // least 90% (the per-CTA work is uniform across tiles).
    const long long slots = (long long)sms * std::max(1, forward_blocks_per_sm(p, false));
    for (long long waves = 1; waves <= 16; ++waves) {
      const long long sp = std::max(1LL, (waves * slots + base_ctas / 2) / base_ctas);
      const long long ctas = base_ctas * sp;
      const long long used = (ctas + slots - 1) / slots * slots;
      splits = sp;
      if (ctas >= slots && (double)ctas / (double)used >= 0.9) break;
      if (sp >= max_splits) break;
    }
  }
  // Smaller ball ranges have tighter bounding boxes, hence narrower arrival
  // bands and fewer culled chunks per CTA: at least one split per
  // kMaxBallsPerSplit balls (on 1e6 balls x 50 frames x 1024 sensors with
  // earlier kernels: 1 split 4.01 s, 2 splits 3.48 s, 8 splits 3.20 s).
  if (splits_o <= 0) splits = std::max(splits, (n + kMaxBallsPerSplit - 1) / kMaxBallsPerSplit);
  splits = std::max(1LL, std::min(splits, max_splits));
  // balls per split: multiple of 4 so every TMA source stays 16-byte aligned
  long long bps = (n + splits - 1) / splits;
  bps = (bps + 3) & ~3LL;
  if (bps <= 0) bps = 4;
  p.balls_per_split = bps;
  p.n_splits = (int)std::max(1LL, (n + bps - 1) / bps);
  p.ws_bytes = p.n_splits > 1 ? sizeof(float) * (size_t)p.n_splits * F * S * T : 0;
  return p;
}

cudaError_t launch_forward(const FwdArgs &a, const FwdPlan &p, bool uniform, cudaStream_t st) {
  auto fn = forward_kernel(uniform, p.group);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  if (e != cudaSuccess) return e;
  // CTAs write only the sample band their balls reach: zero the rest first
  const size_t frame_bytes = sizeof(float) * (size_t)a.F * a.q.S * a.q.T;
  if (p.n_splits > 1) {
    e = cudaMemsetAsync(a.partial, 0, frame_bytes * p.n_splits, st);
  } else if (!(a.flags & PA_ACCUMULATE)) {
    e = cudaMemsetAsync(a.out, 0, frame_bytes, st);
  }
  if (e != cudaSuccess) return e;
  const long long grid = (long long)a.F * p.n_stiles * p.n_ttiles * p.n_splits;
  fn<<<(unsigned)grid, 32 * p.s_tile, p.smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess || p.n_splits == 1) return e;
  const long long n4 = (long long)a.F * a.q.S * a.q.T / 4;
  const long long blocks = std::min<long long>((n4 + 255) / 256, 152LL * 16);
  k_reduce_splits<<<(unsigned)std::max(1LL, blocks), 256, 0, st>>>(
      reinterpret_cast<const float4 *>(a.partial), reinterpret_cast<float4 *>(a.out), n4, p.n_splits,
      (a.flags & PA_ACCUMULATE) != 0);
  return cudaGetLastError();
}

cudaError_t launch_forward_batched(const BatchFwdArgs &a, int group, size_t smem, int sms, cudaStream_t st) {
  void (*fn)(const BatchFwdArgs) = k_forward_batched<8>;
  switch (group) {
    case 1: fn = k_forward_batched<1>; break;
    case 2: fn = k_forward_batched<2>; break;
    case 4: fn = k_forward_batched<4>; break;
    case 16: fn = k_forward_batched<16>; break;
    default: break;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * a.s_tile, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  // CTAs write only the sample band a split's balls reach: zero the partials
  for (int j = 0; j < a.n_scenes && e == cudaSuccess; ++j) {
    const SceneFwd &d = a.sc[j];
    if (d.n_splits > 1)
      e = cudaMemsetAsync(d.partial, 0, sizeof(float) * (size_t)d.n_splits * d.F * d.q.S * d.q.T, st);
  }
  if (e != cudaSuccess) return e;
  const long long grid = std::max(1LL, std::min(a.total_items, (long long)sms * occ));
  fn<<<(unsigned)grid, 32 * a.s_tile, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int j = 0; j < a.n_scenes; ++j) {
    const SceneFwd &d = a.sc[j];
    if (d.n_splits <= 1) continue;
    const long long n4 = (long long)d.F * d.q.S * d.q.T / 4;
    const long long blocks = std::min<long long>((n4 + 255) / 256, 152LL * 16);
    k_reduce_splits<<<(unsigned)std::max(1LL, blocks), 256, 0, st>>>(
        reinterpret_cast<const float4 *>(d.partial), reinterpret_cast<float4 *>(d.out), n4, d.n_splits,
        (a.flags & PA_ACCUMULATE) != 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_count(const Acq &q, const float *state, long long n, long long stride, int F,
                         unsigned long long *out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const long long total = (long long)F * q.S * n;
  if (total == 0) return cudaSuccess;
  const long long blocks = std::min<long long>((total + 255) / 256, 152LL * 32);
  k_count<<<(unsigned)blocks, 256, 0, st>>>(q, state, n, stride, F, out);
  return cudaGetLastError();
}

}  // namespace pa
