// Imaging side of 4D SlingBAG (Sec. 3.1-3.2, Tab. 1): the universal
// back-projection (UBP) the paper compares against, the conversion of a ball
// cloud into a voxel grid, maximum amplitude projections (MAPs) and the SSIM
// of two MAPs.  The paper names these methods without printing them; each
// kernel computes the textbook definition:
//  - UBP (Xu and Wang): b(t) = 2 p(t) - 2 t dp/dt per trace, then
//    p0(r) = sum_s w_s b_s(|r - r_s| / c) / sum_s w_s with the solid-angle
//    weight w_s = cos(theta_s) / |r - r_s|^2 of sensor s (inward normal
//    towards the array centre; sensors facing away are left out) and linear
//    interpolation between samples;
//  - voxels: v(r) = sum_b p_b exp(-|r - mu_b|^2 / (2 a_b^2)) on the closed
//    support |r - mu_b| <= kappa a_b;
//  - MAP: the maximum of the volume along one axis;
//  - SSIM (Wang, Bovik, Sheikh, Simoncelli): 11 x 11 Gaussian window,
//    sigma 1.5, C1 = (0.01 L)^2, C2 = (0.03 L)^2, mean over the positions
//    where the window fits.
// Voxel grids are [nz][ny][nx], voxel (ix, iy, iz) centred at
// origin + h (ix, iy, iz).
#include <algorithm>
#include <cmath>

#include "pa_internal.h"

namespace pa {

namespace {

// ---------------------------------------------------------------------------
// UBP filter: one thread per sample (HBM-bound elementwise pass).
__global__ void __launch_bounds__(256) k_ubp_filter(const float *__restrict__ p, long long n_traces, int T,
                                                    float fs, float t0, float *__restrict__ b) {
  const long long total = n_traces * T;
  const float half_fs = 0.5f * fs;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i % T);
    const float pk = p[i];
    float dpdt;
    if (k == 0)
      dpdt = (p[i + 1] - pk) * fs;
    else if (k == T - 1)
      dpdt = (pk - p[i - 1]) * fs;
    else
      dpdt = (p[i + 1] - p[i - 1]) * half_fs;
    const float t = t0 + (float)k / fs;
    b[i] = 2.f * pk - 2.f * t * dpdt;
  }
}

// ---------------------------------------------------------------------------
// UBP back-projection.  CTA = an 8 x 8 x 8 brick (x fastest), 256 threads;
// thread (tx, ty, tz) owns voxels (tx, ty, tz) and (tx, ty, tz + 4), which
// share the sensor loads, dx, dy and the in-plane partial sums, the rest of
// the arithmetic running on both as packed FP32x2.  The 32 voxels of a warp
// are close together, so each sensor's filtered trace is read from one or two
// L1 lines.  Sensor positions and unit inward normals are staged in shared
// memory, kUbpChunk sensors at a time.
constexpr int kUbpChunk = 1024;

__device__ __forceinline__ float ubp_interp(const float *brow, float f, float hi_f) {
  const float fl = floorf(f);
  float val = 0.f;
  if (fl >= 0.f && fl <= hi_f) {  // false for NaN
    const int i = (int)fl;
    const float v0 = __ldg(brow + i), v1 = __ldg(brow + i + 1);
    val = fmaf(f - fl, v1 - v0, v0);
  }
  return val;
}

__global__ void __launch_bounds__(256) k_ubp(const UbpArgs A) {
  __shared__ float4 s_pos[kUbpChunk];
  __shared__ float4 s_nrm[kUbpChunk];
  const int tid = threadIdx.x;
  const int ix = blockIdx.x * 8 + (tid & 7);
  const int iy = blockIdx.y * 8 + ((tid >> 3) & 7);
  const int iz = blockIdx.z * 8 + (tid >> 6);  // and iz + 4
  const bool okxy = ix < A.nx && iy < A.ny;
  const float rx = fmaf((float)ix, A.h, A.ox), ry = fmaf((float)iy, A.h, A.oy);
  const float2 rz = make_float2(fmaf((float)iz, A.h, A.oz), fmaf((float)(iz + 4), A.h, A.oz));
  const float hi_f = (float)(A.T - 2);
  const float2 fsc2 = make_float2(A.fs_c, A.fs_c), mt2 = make_float2(-A.t0_fs, -A.t0_fs);
  float2 num = make_float2(0.f, 0.f), den = num;
  for (int s0 = 0; s0 < A.S; s0 += kUbpChunk) {
    const int cnt = min(kUbpChunk, A.S - s0);
    __syncthreads();  // the previous chunk is consumed
    for (int j = tid; j < cnt; j += blockDim.x) {
      const float sx = A.sensors[s0 + j], sy = A.sensors[A.sstride + s0 + j], sz = A.sensors[2 * A.sstride + s0 + j];
      const float nx = A.cx - sx, ny = A.cy - sy, nz = A.cz - sz;
      const float nn = sqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
      const float inv = nn > 0.f ? 1.f / nn : 0.f;
      s_pos[j] = make_float4(sx, sy, sz, 0.f);
      s_nrm[j] = make_float4(nx * inv, ny * inv, nz * inv, 0.f);
    }
    __syncthreads();
    if (okxy) {
      const float *brow = A.b + (long long)s0 * A.T;
      for (int j = 0; j < cnt; ++j, brow += A.T) {
        const float4 sp = s_pos[j], sn = s_nrm[j];
        const float dx = rx - sp.x, dy = ry - sp.y;
        const float dxy = fmaf(dx, dx, dy * dy);
        const float nxy = fmaf(sn.x, dx, sn.y * dy);
        const float2 dz = __fadd2_rn(rz, make_float2(-sp.z, -sp.z));
        const float2 d2 = __ffma2_rn(dz, dz, make_float2(dxy, dxy));
        const float2 dot = __ffma2_rn(make_float2(sn.z, sn.z), dz, make_float2(nxy, nxy));
        const float2 ir = make_float2(rsqrtf(d2.x), rsqrtf(d2.y));
        const float2 d = __fmul2_rn(d2, ir);
        float2 w = __fmul2_rn(__fmul2_rn(dot, ir), __fmul2_rn(ir, ir));  // cos(theta) / d^2
        w.x = dot.x > 0.f ? w.x : 0.f;  // sensors facing away are left out
        w.y = dot.y > 0.f ? w.y : 0.f;
        const float2 f = __ffma2_rn(d, fsc2, mt2);
        const float2 val = make_float2(ubp_interp(brow, f.x, hi_f), ubp_interp(brow, f.y, hi_f));
        num = __ffma2_rn(w, val, num);
        den = __fadd2_rn(den, w);
      }
    }
  }
  if (okxy) {
    if (iz < A.nz) A.vol[((long long)iz * A.ny + iy) * A.nx + ix] = den.x > 0.f ? num.x / den.x : 0.f;
    if (iz + 4 < A.nz) A.vol[((long long)(iz + 4) * A.ny + iy) * A.nx + ix] = den.y > 0.f ? num.y / den.y : 0.f;
  }
}

// ---------------------------------------------------------------------------
// Ball cloud -> voxels.  One CTA per 16 x 16 x 16 brick, 512 threads; thread
// (tx, ty, tz) owns voxels (tx, ty, tz + 2j), j = 0..7.  The CTA walks all
// balls in index order, keeps (by a block-wide compaction that preserves the
// order) those whose support box meets the brick, and every thread adds the
// kept balls to its 8 voxels in registers.  No atomics; deterministic.
constexpr int kSplatBrick = 16;
constexpr int kSplatThreads = 512;
constexpr int kSplatList = 2 * kSplatThreads;

__global__ void __launch_bounds__(kSplatThreads) k_splat(const SplatArgs A) {
  __shared__ float4 s_b[kSplatList];   // x, y, z, -log2(e) / (2 a^2)
  __shared__ float2 s_b2[kSplatList];  // p, (kappa a)^2
  __shared__ int s_warp[kSplatThreads / 32];
  __shared__ int s_count;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tid & 15, ty = (tid >> 4) & 15, tz = tid >> 8;  // tz in {0, 1}
  const int ix = blockIdx.x * kSplatBrick + tx, iy = blockIdx.y * kSplatBrick + ty;
  const int iz0 = blockIdx.z * kSplatBrick + tz;
  const float rx = fmaf((float)ix, A.h, A.ox), ry = fmaf((float)iy, A.h, A.oy);
  float rz[8], acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    rz[j] = fmaf((float)(iz0 + 2 * j), A.h, A.oz);
    acc[j] = 0.f;
  }
  // brick bounds (voxel centres)
  const float bx0 = fmaf((float)(blockIdx.x * kSplatBrick), A.h, A.ox), bx1 = bx0 + (kSplatBrick - 1) * A.h;
  const float by0 = fmaf((float)(blockIdx.y * kSplatBrick), A.h, A.oy), by1 = by0 + (kSplatBrick - 1) * A.h;
  const float bz0 = fmaf((float)(blockIdx.z * kSplatBrick), A.h, A.oz), bz1 = bz0 + (kSplatBrick - 1) * A.h;
  const float L2E = 1.4426950408889634f;
  if (tid == 0) s_count = 0;
  __syncthreads();
  auto consume = [&](int cnt) {
    for (int i = 0; i < cnt; ++i) {
      const float4 q = s_b[i];
      const float2 q2 = s_b2[i];
      const float dx = rx - q.x, dy = ry - q.y;
      const float dxy = fmaf(dx, dx, dy * dy);
      if (dxy > q2.y) continue;  // this thread's column misses the ball
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float dz = rz[j] - q.z;
        const float r2 = fmaf(dz, dz, dxy);
        if (r2 <= q2.y) acc[j] = fmaf(q2.x, ex2(r2 * q.w), acc[j]);
      }
    }
  };
  for (long long b0 = 0; b0 < A.n; b0 += kSplatThreads) {
    const long long b = b0 + tid;
    bool keep = false;
    float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 rec2 = make_float2(0.f, 0.f);
    if (b < A.n) {
      const float x = A.state[b], y = A.state[A.stride + b], z = A.state[2 * A.stride + b];
      const float a = A.state[3 * A.stride + b], p = A.state[4 * A.stride + b];
      if (a > 0.f && p != 0.f) {
        const float R = A.kappa * a;
        keep = x + R >= bx0 && x - R <= bx1 && y + R >= by0 && y - R <= by1 && z + R >= bz0 && z - R <= bz1;
        rec = make_float4(x, y, z, -L2E / (2.f * a * a));
        rec2 = make_float2(p, R * R);
      }
    }
    // order-preserving compaction: warp ballots, warp offsets, lane ranks
    const unsigned m = __ballot_sync(FULL, keep);
    if (lane == 0) s_warp[warp] = __popc(m);
    __syncthreads();
    int off = s_count;
    for (int w = 0; w < warp; ++w) off += s_warp[w];
    int total = s_count;
    for (int w = 0; w < kSplatThreads / 32; ++w) total += s_warp[w];
    if (keep) {
      const int pos = off + __popc(m & ((1u << lane) - 1u));
      s_b[pos] = rec;
      s_b2[pos] = rec2;
    }
    __syncthreads();
    if (total > kSplatList - kSplatThreads) {  // room for one more pass? else drain
      consume(total);
      __syncthreads();
      total = 0;
    }
    if (tid == 0) s_count = total;
    __syncthreads();
  }
  consume(s_count);
  if (ix < A.nx && iy < A.ny) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int iz = iz0 + 2 * j;
      if (iz < A.nz) A.vol[((long long)iz * A.ny + iy) * A.nx + ix] = acc[j];
    }
  }
}

// ---------------------------------------------------------------------------
// Maximum amplitude projections.
__global__ void __launch_bounds__(256) k_map_z(const float *__restrict__ v, int nx, int ny, int nz,
                                               float *__restrict__ xy) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // iy * nx + ix
  if (i >= (long long)nx * ny) return;
  float m = v[i];
  for (int z = 1; z < nz; ++z) m = fmaxf(m, v[(long long)z * nx * ny + i]);
  xy[i] = m;
}

__global__ void __launch_bounds__(256) k_map_y(const float *__restrict__ v, int nx, int ny, int nz,
                                               float *__restrict__ xz) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // iz * nx + ix
  if (i >= (long long)nx * nz) return;
  const long long z = i / nx, x = i - z * nx;
  const float *col = v + z * (long long)nx * ny + x;
  float m = col[0];
  for (int y = 1; y < ny; ++y) m = fmaxf(m, col[(long long)y * nx]);
  xz[i] = m;
}

// one warp per (iy, iz) row, lanes over x
__global__ void __launch_bounds__(256) k_map_x(const float *__restrict__ v, int nx, int ny, int nz,
                                               float *__restrict__ yz) {
  const long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;  // iz * ny + iy
  const int lane = threadIdx.x & 31;
  if (row >= (long long)ny * nz) return;  // warp-uniform
  const float *r = v + row * nx;
  float m = -INFINITY;
  for (int x = lane; x < nx; x += 32) m = fmaxf(m, r[x]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
  if (lane == 0) yz[row] = m;
}

// ---------------------------------------------------------------------------
// Per-image minimum and maximum (for the [0, 1] normalisation before SSIM):
// fixed grid, per-block partials, one final warp; deterministic.
constexpr int kMinMaxBlocks = 128;

__global__ void __launch_bounds__(256) k_minmax2(const float *__restrict__ x, const float *__restrict__ y,
                                                 long long n, float4 *__restrict__ partials) {
  __shared__ float4 s_w[8];
  float4 m = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);  // xmin, xmax, ymin, ymax
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float a = x[i], b = y[i];
    m.x = fminf(m.x, a);
    m.y = fmaxf(m.y, a);
    m.z = fminf(m.z, b);
    m.w = fmaxf(m.w, b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m.x = fminf(m.x, __shfl_xor_sync(FULL, m.x, o));
    m.y = fmaxf(m.y, __shfl_xor_sync(FULL, m.y, o));
    m.z = fminf(m.z, __shfl_xor_sync(FULL, m.z, o));
    m.w = fmaxf(m.w, __shfl_xor_sync(FULL, m.w, o));
  }
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float4 t = s_w[0];
    for (int w = 1; w < 8; ++w) {
      t.x = fminf(t.x, s_w[w].x);
      t.y = fmaxf(t.y, s_w[w].y);
      t.z = fminf(t.z, s_w[w].z);
      t.w = fmaxf(t.w, s_w[w].w);
    }
    partials[blockIdx.x] = t;
  }
}

// Reduces the partials to (x offset, x scale, y offset, y scale) with
// v' = (v - offset) * scale in [0, 1]; a constant image maps to 0.
__global__ void k_minmax_final(const float4 *partials, int nb, float4 *out) {
  float4 m = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
  for (int i = threadIdx.x; i < nb; i += 32) {
    const float4 t = partials[i];
    m.x = fminf(m.x, t.x);
    m.y = fmaxf(m.y, t.y);
    m.z = fminf(m.z, t.z);
    m.w = fmaxf(m.w, t.w);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m.x = fminf(m.x, __shfl_xor_sync(FULL, m.x, o));
    m.y = fmaxf(m.y, __shfl_xor_sync(FULL, m.y, o));
    m.z = fminf(m.z, __shfl_xor_sync(FULL, m.z, o));
    m.w = fmaxf(m.w, __shfl_xor_sync(FULL, m.w, o));
  }
  if (threadIdx.x == 0) {
    const float rx = m.y - m.x, ry = m.w - m.z;
    *out = make_float4(m.x, rx > 0.f ? 1.f / rx : 0.f, m.z, ry > 0.f ? 1.f / ry : 0.f);
  }
}

// ---------------------------------------------------------------------------
// SSIM: one output pixel per thread, 16 x 16 output tile per CTA with its
// 26 x 26 input window of both images in shared memory; per-CTA FP64 partial
// sums reduced in a fixed order by k_ssim_final.
constexpr int kSsimTile = 16;
constexpr int kSsimIn = kSsimTile + 10;

__global__ void __launch_bounds__(256) k_ssim(const SsimArgs A) {
  __shared__ float sx[kSsimIn][kSsimIn + 1];
  __shared__ float sy[kSsimIn][kSsimIn + 1];
  __shared__ double s_part[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int oh = A.H - 10, ow = A.W - 10;
  const int r0 = blockIdx.y * kSsimTile, q0 = blockIdx.x * kSsimTile;
  float4 nrm = make_float4(0.f, 1.f, 0.f, 1.f);  // identity: (v - 0) * 1
  if (A.norm) nrm = *A.norm;
  for (int i = tid; i < kSsimIn * kSsimIn; i += blockDim.x) {
    const int rr = i / kSsimIn, qq = i - rr * kSsimIn;
    const int r = r0 + rr, q = q0 + qq;
    const bool in = r < A.H && q < A.W;
    sx[rr][qq] = in ? (A.x[(long long)r * A.W + q] - nrm.x) * nrm.y : 0.f;
    sy[rr][qq] = in ? (A.y[(long long)r * A.W + q] - nrm.z) * nrm.w : 0.f;
  }
  __syncthreads();
  const int tr = tid >> 4, tq = tid & 15;
  const int r = r0 + tr, q = q0 + tq;
  double mine = 0.0;
  if (r < oh && q < ow) {
    float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
    for (int i = 0; i < 11; ++i) {
      float rx = 0.f, ry = 0.f, rxx = 0.f, ryy = 0.f, rxy = 0.f;
#pragma unroll
      for (int j = 0; j < 11; ++j) {
        const float a = sx[tr + i][tq + j], b = sy[tr + i][tq + j], g = A.g[j];
        const float ga = g * a, gb = g * b;
        rx += ga;
        ry += gb;
        rxx = fmaf(ga, a, rxx);
        ryy = fmaf(gb, b, ryy);
        rxy = fmaf(ga, b, rxy);
      }
      const float g = A.g[i];
      mx = fmaf(g, rx, mx);
      my = fmaf(g, ry, my);
      xx = fmaf(g, rxx, xx);
      yy = fmaf(g, ryy, yy);
      xy = fmaf(g, rxy, xy);
    }
    const float vx = xx - mx * mx, vy = yy - my * my, cxy = xy - mx * my;
    const float s = ((2.f * mx * my + A.C1) * (2.f * cxy + A.C2)) /
                    ((mx * mx + my * my + A.C1) * (vx + vy + A.C2));
    if (A.map) A.map[(long long)r * ow + q] = s;
    mine = (double)s;
  }
  mine = warp_sum_d(mine);
  if (lane == 0) s_part[warp] = mine;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s_part[w];
    A.partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_ssim_final(const double *partials, int n, double inv_count, double *out) {
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) t += partials[i];
  t = warp_sum_d(t);
  if (threadIdx.x == 0) *out = t * inv_count;
}

}  // namespace

cudaError_t launch_ubp_filter(const float *p, long long n_traces, int T, float fs, float t0, float *b,
                              cudaStream_t st) {
  const long long total = n_traces * T;
  if (total == 0) return cudaSuccess;
  const long long blocks = std::min<long long>((total + 255) / 256, 152LL * 16);
  k_ubp_filter<<<(unsigned)blocks, 256, 0, st>>>(p, n_traces, T, fs, t0, b);
  return cudaGetLastError();
}

cudaError_t launch_ubp(const UbpArgs &a, cudaStream_t st) {
  if ((long long)a.nx * a.ny * a.nz == 0) return cudaSuccess;
  dim3 grid((a.nx + 7) / 8, (a.ny + 7) / 8, (a.nz + 7) / 8);
  k_ubp<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_splat(const SplatArgs &a, cudaStream_t st) {
  if ((long long)a.nx * a.ny * a.nz == 0) return cudaSuccess;
  dim3 grid((a.nx + kSplatBrick - 1) / kSplatBrick, (a.ny + kSplatBrick - 1) / kSplatBrick,
            (a.nz + kSplatBrick - 1) / kSplatBrick);
  k_splat<<<grid, kSplatThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_map(const float *v, int nx, int ny, int nz, float *xy, float *yz, float *xz, cudaStream_t st) {
  if ((long long)nx * ny * nz == 0) return cudaSuccess;
  if (xy) {
    const long long n = (long long)nx * ny;
    k_map_z<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, nx, ny, nz, xy);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (xz) {
    const long long n = (long long)nx * nz;
    k_map_y<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, nx, ny, nz, xz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (yz) {
    const long long rows = (long long)ny * nz;
    k_map_x<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(v, nx, ny, nz, yz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int ssim_blocks(int H, int W) {
  return ((W - 10 + kSsimTile - 1) / kSsimTile) * ((H - 10 + kSsimTile - 1) / kSsimTile);
}

int minmax_partials() { return kMinMaxBlocks; }

cudaError_t launch_ssim(const SsimArgs &a, double *out, float4 *minmax_ws, cudaStream_t st) {
  if (a.norm) {
    const long long n = (long long)a.H * a.W;
    k_minmax2<<<kMinMaxBlocks, 256, 0, st>>>(a.x, a.y, n, minmax_ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_minmax_final<<<1, 32, 0, st>>>(minmax_ws, kMinMaxBlocks, const_cast<float4 *>(a.norm));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  dim3 grid((a.W - 10 + kSsimTile - 1) / kSsimTile, (a.H - 10 + kSsimTile - 1) / kSsimTile);
  k_ssim<<<grid, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n = (int)(grid.x * grid.y);
  k_ssim_final<<<1, 32, 0, st>>>(a.partials, n, 1.0 / ((double)(a.H - 10) * (double)(a.W - 10)), out);
  return cudaGetLastError();
}

}  // namespace pa
