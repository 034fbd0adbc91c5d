// Spatial order of a ball cloud and the gather that applies it.  A layout
// tool, not part of the method: the paper's sums over balls do not depend on
// the order in which the balls are stored, but the forward kernel sweeps
// tiles of consecutive balls, and the narrower a tile's bounding box, the
// narrower its arrival band at every sensor and the tighter its groups of
// windows.  Storing a cloud in Morton (Z-curve) order of its centres makes
// consecutive balls neighbours in space.
//
// Order: bounding box of the centres (min/max on the order-preserving
// unsigned image of the floats, deterministic), a 30-bit Morton code per
// ball from 10-bit indices of cubic cells (edge: the power of two nearest to
// the mean radius, at least the largest extent / 1024), then a stable LSD
// radix sort of (code, index) pairs with 8-bit digits (four passes: per-tile
// digit histograms, one exclusive scan over (digit, tile), a stable
// scatter).  The permutation is deterministic: equal codes keep their index
// order.
#include <algorithm>

#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;                              // items per thread per tile
constexpr int kSortTile = kSortThreads * kSortItems;       // 2048
constexpr int kRadixBins = 256;
constexpr int kMaxBboxBlocks = 2048;                        // partial sums of the radius

// Order-preserving map of a float to an unsigned integer (and back).
__device__ __forceinline__ unsigned f2ord(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// bbox[0..2] = ordered minima of x, y, z; bbox[3..5] = ordered maxima.
__global__ void k_bbox_init(unsigned *bbox) {
  if (threadIdx.x < 3) bbox[threadIdx.x] = 0xffffffffu;
  else if (threadIdx.x < 6) bbox[threadIdx.x] = 0u;
}

__global__ void __launch_bounds__(kSortThreads) k_bbox(const float *state, long long stride, long long n,
                                                       unsigned *bbox, double2 *partial) {
  __shared__ double2 ws[kSortThreads / 32];
  unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  double sa = 0.0, na = 0.0;  // sum and count of the positive radii
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const unsigned u = f2ord(state[c * stride + i]);
      lo[c] = min(lo[c], u);
      hi[c] = max(hi[c], u);
    }
    const float a = state[3 * stride + i];
    if (a > 0.f) {
      sa += (double)a;
      na += 1.0;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    lo[c] = __reduce_min_sync(FULL, lo[c]);
    hi[c] = __reduce_max_sync(FULL, hi[c]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(FULL, sa, o);
    na += __shfl_xor_sync(FULL, na, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicMin(&bbox[c], lo[c]);
      atomicMax(&bbox[3 + c], hi[c]);
    }
    ws[warp] = make_double2(sa, na);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = ws[0];
    for (int w = 1; w < kSortThreads / 32; ++w) {
      t.x += ws[w].x;
      t.y += ws[w].y;
    }
    partial[blockIdx.x] = t;  // fixed order: the mean below is deterministic
  }
}

// Cell edge: the power of two nearest to the mean positive radius (balls
// closer than about their own size keep their index order), at least the
// largest extent / 1024 (so that 1024 cells per axis cover the box).
// Writes 1 / edge (a power of two, exact) to *scale.
__global__ void k_cell(const unsigned *bbox, const double2 *partial, int nparts, float *scale) {
  if (threadIdx.x != 0) return;
  double sa = 0.0, na = 0.0;
  for (int i = 0; i < nparts; ++i) {
    sa += partial[i].x;
    na += partial[i].y;
  }
  float ext = 0.f;
  for (int c = 0; c < 3; ++c) ext = fmaxf(ext, __fsub_rn(ord2f(bbox[3 + c]), ord2f(bbox[c])));
  int k = na > 0.0 ? (int)rint(log2(sa / na)) : -126;
  k = max(-126, min(k, 100));
  while (k < 100 && ldexp(1.0, k) * 1024.0 < (double)ext) ++k;
  *scale = (float)ldexp(1.0, -k);
}

// Spread the low 10 bits of v to every third bit.
__device__ __forceinline__ unsigned spread3(unsigned v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Cell index of coordinate x: floor((x - lo) * scale), clamped to [0, 1023];
// the subtraction is one rounded float operation and the scale a power of
// two, so that a host replay in float32 gives the same cells.
__device__ __forceinline__ unsigned cell10(float x, float lo, float scale) {
  const float t = __fmul_rn(__fsub_rn(x, lo), scale);
  const int q = (int)floorf(t);
  return (unsigned)min(1023, max(0, q));
}

__global__ void __launch_bounds__(kSortThreads) k_morton(const float *state, long long stride, long long n,
                                                         const unsigned *bbox, const float *pscale, unsigned *code,
                                                         int *idx) {
  // cubic cells: one scale for the three axes
  float lo[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) lo[c] = ord2f(bbox[c]);
  const float scale = *pscale;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned cx = cell10(state[i], lo[0], scale);
    const unsigned cy = cell10(state[stride + i], lo[1], scale);
    const unsigned cz = cell10(state[2 * stride + i], lo[2], scale);
    code[i] = spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2);
    idx[i] = (int)i;
  }
}

// Digit histogram of each tile: hist[d * ntiles + tile].
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const unsigned *key, long long n, int shift,
                                                             unsigned *hist, int ntiles) {
  __shared__ unsigned h[kRadixBins];
  h[threadIdx.x] = 0u;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const long long i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(key[i] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of hist[0 .. m) in place (one block of 1024 threads, each
// over a contiguous segment).
__global__ void __launch_bounds__(1024) k_radix_scan(unsigned *hist, long long m) {
  __shared__ unsigned wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long seg = (m + 1023) / 1024;
  const long long e0 = min((long long)tid * seg, m), e1 = min(e0 + seg, m);
  unsigned sum = 0u;
  for (long long e = e0; e < e1; ++e) sum += hist[e];
  unsigned incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned w = wsum[lane], wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(FULL, wi, o);
      if (lane >= o) wi += v;
    }
    wsum[lane] = wi - w;  // exclusive over warps
  }
  __syncthreads();
  unsigned run = wsum[warp] + incl - sum;
  for (long long e = e0; e < e1; ++e) {
    const unsigned v = hist[e];
    hist[e] = run;
    run += v;
  }
}

// Stable scatter of one tile: items in index order, 256 per round; an item's
// place among the round's items of its digit is its rank within its warp
// (match_any) plus the counts of the lower warps.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const unsigned *key_in, const int *idx_in,
                                                                unsigned *key_out, int *idx_out, long long n,
                                                                int shift, const unsigned *offs, int ntiles) {
  constexpr int W = kSortThreads / 32;
  __shared__ unsigned base[kRadixBins];
  __shared__ unsigned cnt[W][kRadixBins];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offs[(long long)tid * ntiles + blockIdx.x];
#pragma unroll
  for (int w = 0; w < W; ++w) cnt[w][tid] = 0u;
  __syncthreads();
  const long long tile0 = (long long)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    const long long i = tile0 + r * kSortThreads + tid;
    const bool ok = i < n;
    unsigned k = 0u;
    int v = 0;
    if (ok) {
      k = key_in[i];
      v = idx_in[i];
    }
    const unsigned d = ok ? ((k >> shift) & 0xffu) : kRadixBins;  // past the end: its own class
    const unsigned peers = __match_any_sync(FULL, d);
    const unsigned rank = __popc(peers & ((1u << lane) - 1u));
    if (ok && rank == 0) cnt[warp][d] = __popc(peers);
    __syncthreads();
    if (ok) {
      unsigned before = 0u;
      for (int w = 0; w < warp; ++w) before += cnt[w][d];
      const unsigned pos = base[d] + before + rank;
      key_out[pos] = k;
      idx_out[pos] = v;
    }
    __syncthreads();
    unsigned tot = 0u;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      tot += cnt[w][tid];
      cnt[w][tid] = 0u;
    }
    base[tid] += tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSortThreads) k_gather_rows(const float *in, float *out, long long n,
                                                              long long stride, int rows, const int *perm) {
  const long long total = (long long)rows * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n, i = e - r * n;
    out[r * stride + i] = in[r * stride + perm[i]];
  }
}

inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

inline long long sort_tiles(long long n) { return (n + kSortTile - 1) / kSortTile; }

}  // namespace

size_t spatial_order_workspace(long long n) {
  if (n <= 0) return 0;
  return round256(64) + round256(sizeof(double2) * kMaxBboxBlocks) + 3 * round256(sizeof(unsigned) * (size_t)n) + round256(sizeof(int) * (size_t)n) +
         round256(sizeof(unsigned) * (size_t)kRadixBins * (size_t)sort_tiles(n));
}

cudaError_t launch_spatial_order(const float *state, long long stride, long long n, int *perm, void *ws,
                                 int sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  char *p = static_cast<char *>(ws);
  unsigned *bbox = reinterpret_cast<unsigned *>(p);
  float *scale = reinterpret_cast<float *>(p + 32);
  p += round256(64);
  double2 *partial = reinterpret_cast<double2 *>(p);
  p += round256(sizeof(double2) * kMaxBboxBlocks);
  unsigned *key0 = reinterpret_cast<unsigned *>(p);
  p += round256(sizeof(unsigned) * (size_t)n);
  unsigned *key1 = reinterpret_cast<unsigned *>(p);
  p += round256(sizeof(unsigned) * (size_t)n);
  int *idx0 = reinterpret_cast<int *>(p);
  p += round256(sizeof(unsigned) * (size_t)n);
  int *idx1 = reinterpret_cast<int *>(p);
  p += round256(sizeof(int) * (size_t)n);
  unsigned *hist = reinterpret_cast<unsigned *>(p);
  const long long ntiles = sort_tiles(n);
  const unsigned grid = (unsigned)std::max(
      1LL, std::min({(n + kSortThreads - 1) / kSortThreads, 8LL * sms, (long long)kMaxBboxBlocks}));
  k_bbox_init<<<1, 32, 0, st>>>(bbox);
  k_bbox<<<grid, kSortThreads, 0, st>>>(state, stride, n, bbox, partial);
  k_cell<<<1, 32, 0, st>>>(bbox, partial, (int)grid, scale);
  k_morton<<<grid, kSortThreads, 0, st>>>(state, stride, n, bbox, scale, key0, idx0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // four 8-bit passes over the 30-bit codes; the last one writes the
  // permutation straight into `perm` (idx ping-pongs idx0 -> idx1 -> idx0 ->
  // idx1 -> perm)
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 8 * pass;
    const unsigned *kin = pass & 1 ? key1 : key0;
    unsigned *kout = pass & 1 ? key0 : key1;
    const int *iin = pass == 0 ? idx0 : (pass & 1 ? idx1 : idx0);
    int *iout = pass == 3 ? perm : (pass & 1 ? idx0 : idx1);
    k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, st>>>(kin, n, shift, hist, (int)ntiles);
    k_radix_scan<<<1, 1024, 0, st>>>(hist, (long long)kRadixBins * ntiles);
    k_radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, st>>>(kin, iin, kout, iout, n, shift, hist, (int)ntiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_gather_rows(const float *in, float *out, long long n, long long stride, int rows,
                               const int *perm, int sms, cudaStream_t st) {
  const long long total = (long long)rows * n;
  if (total <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::max(1LL, std::min((total + kSortThreads - 1) / kSortThreads, 8LL * sms));
  k_gather_rows<<<grid, kSortThreads, 0, st>>>(in, out, n, stride, rows, perm);
  return cudaGetLastError();
}

}  // namespace pa
