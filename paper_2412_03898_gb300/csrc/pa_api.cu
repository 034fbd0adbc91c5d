// C ABI of the library (declared in include/pa.h): host-side validation,
// tile plans, the per-device error word, and kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>

#include "pa_internal.h"

// Launch plan of the forward and batched calls (opaque to C callers).
struct pa_plan {
  int32_t tiles[5];          // sensors per CTA, samples per CTA, balls per stage, ball splits, pairs per sweep
  int32_t frames_per_chunk;  // frames per launch of pa_forward_4d / pa_adjoint_4d (0 = from the L2 size)
  int32_t adj_chunk;         // (scene, frame, ball) items per queue grab of pa_adjoint_batched
  int32_t tuned;             // 1 when chosen by timing candidates
  float fwd_ms;              // best forward time measured while tuning (0 if not tuned)
  float adj_ms;              // best batched-adjoint time measured while tuning (0 if not tuned)
  int32_t candidates;        // plans timed
};

namespace {

// One error word per device: kernels record the first data-dependent error.
__device__ unsigned g_pa_error_word;

constexpr int kMaxDevices = 64;

struct DevInfo {
  unsigned *err = nullptr;
  int sms = 0;
  int max_smem = 0;
  bool ready = false;
};
DevInfo g_dev[kMaxDevices];
std::mutex g_dev_mu;

const DevInfo *dev_info() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DevInfo &d = g_dev[dev];
  if (!d.ready) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pa_error_word) != cudaSuccess) return nullptr;
    d.err = static_cast<unsigned *>(p);
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return nullptr;
    if (cudaDeviceGetAttribute(&d.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return nullptr;
    d.ready = true;
  }
  return &d;
}

inline bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }
inline bool finite_pos(float v) { return std::isfinite(v) && v > 0.f; }

// Explicit tile plan {sensors per CTA, samples per CTA, balls per stage,
// ball splits, pairs per sweep}: NULL, or every entry in range.
bool tiles_ok(const int32_t *t) {
  if (t == nullptr) return true;
  return t[0] >= 0 && t[0] <= 16 && t[1] >= 0 && (t[1] & 3) == 0 && t[2] >= 0 && t[2] <= 8192 &&
         (t[2] & 3) == 0 && t[3] >= 0 && t[4] >= 0 && t[4] <= 16;
}

int check_geom(const pa_geom *g) {
  if (g == nullptr || g->sensors == nullptr) return PA_ERR_INVALID_ARG;
  if (g->n_sensors < 1 || g->sensor_stride < g->n_sensors) return PA_ERR_INVALID_ARG;
  if (!finite_pos(g->c) || !finite_pos(g->fs)) return PA_ERR_INVALID_ARG;
  if (!std::isfinite(g->t0) || g->t0 < 0.f) return PA_ERR_INVALID_ARG;
  if (g->n_samples < 4 || (g->n_samples & 3) != 0) return PA_ERR_INVALID_ARG;
  if (!(g->kappa >= 1.f && g->kappa <= 8.f)) return PA_ERR_INVALID_ARG;
  return PA_OK;
}

int check_balls(const pa_balls *b) {
  if (b == nullptr || b->n < 0 || b->stride < b->n || (b->stride & 3) != 0) return PA_ERR_INVALID_ARG;
  if (b->n > 0 && (b->state == nullptr || !aligned(b->state, 16))) return PA_ERR_INVALID_ARG;
  return PA_OK;
}

int check_canon(const pa_canon *c) {
  if (c == nullptr || c->n < 0 || c->stride < c->n || (c->stride & 3) != 0) return PA_ERR_INVALID_ARG;
  if (c->n_basis < 1 || c->n_basis > 128) return PA_ERR_INVALID_ARG;
  if (c->n > 0 && (!c->canon || !c->omega || !c->theta || !c->sigma)) return PA_ERR_INVALID_ARG;
  return PA_OK;
}

int check_grid(const pa_grid *g) {
  if (g == nullptr || !(g->h > 0.f) || g->nx < 1 || g->ny < 1 || g->nz < 1) return PA_ERR_INVALID_ARG;
  if (!std::isfinite(g->origin[0]) || !std::isfinite(g->origin[1]) || !std::isfinite(g->origin[2]))
    return PA_ERR_INVALID_ARG;
  return PA_OK;
}

pa::Acq make_acq(const pa_geom *g) {
  pa::Acq q;
  q.sensors = g->sensors;
  q.S = g->n_sensors;
  q.sstride = g->sensor_stride;
  q.T = g->n_samples;
  q.kappa = g->kappa;
  const double delta = (double)g->c / (double)g->fs;
  q.dh = (float)delta;
  q.dl = (float)(delta - (double)q.dh);
  const double ct0 = (double)g->c * (double)g->t0;
  q.ct0h = (float)ct0;
  q.ct0l = (float)(ct0 - (double)q.ct0h);
  q.inv_delta = (float)((double)g->fs / (double)g->c);
  return q;
}

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? PA_OK : PA_ERR_CUDA; }

// The forward's split partials ([splits][frames][S][T] floats) are kept
// within kMaxPartialBytes by launching frames in chunks: the chunk is halved
// from all frames until its plan's partials fit.
constexpr size_t kMaxPartialBytes = 1ull << 30;

struct FwdChunking {
  int frames;  // frames per launch
  size_t ws;   // workspace bytes of the largest chunk
};

pa::FwdPlan plan_for(const DevInfo *d, const pa_geom *g, long long n, int F, const int32_t *tiles) {
  return pa::forward_plan(g->n_sensors, g->n_samples, n, F, d->sms, tiles ? tiles[0] : 0, tiles ? tiles[1] : 0,
                          tiles ? tiles[2] : 0, tiles ? tiles[3] : 0, tiles ? tiles[4] : 0);
}

FwdChunking forward_chunking(const DevInfo *d, const pa_geom *g, long long n, int F, const int32_t *tiles) {
  FwdChunking c{std::max(F, 1), 0};
  c.ws = plan_for(d, g, n, c.frames, tiles).ws_bytes;
  while (c.ws > kMaxPartialBytes && c.frames > 1) {
    c.frames = std::max(1, c.frames / 2);
    c.ws = plan_for(d, g, n, c.frames, tiles).ws_bytes;
  }
  if (F > c.frames && F % c.frames != 0) c.ws = std::max(c.ws, plan_for(d, g, n, F % c.frames, tiles).ws_bytes);
  return c;
}

// Launches the forward over F frames of states [F][5][stride] (in frame
// chunks that keep the split partials within kMaxPartialBytes); arguments
// already checked.
int forward_launch(const DevInfo *d, const pa_geom *geom, const float *state, long long n, long long stride,
                   int32_t F, float *traces, uint32_t flags, const int32_t *tiles, void *ws, size_t ws_bytes,
                   cudaStream_t st) {
  const FwdChunking ch = forward_chunking(d, geom, n, F, tiles);
  if (ch.ws > 0 && (ws == nullptr || ws_bytes < ch.ws || !aligned(ws, 256))) return PA_ERR_WORKSPACE;
  const size_t per_frame = (size_t)geom->n_sensors * geom->n_samples;
  for (int f0 = 0; f0 < F; f0 += ch.frames) {
    const int k = std::min(ch.frames, F - f0);
    const pa::FwdPlan p = plan_for(d, geom, n, k, tiles);
    if (p.smem > (size_t)d->max_smem) return PA_ERR_INVALID_ARG;
    pa::FwdArgs a;
    a.q = make_acq(geom);
    a.state = state + (size_t)f0 * 5 * stride;
    a.n = n;
    a.stride = stride;
    a.F = k;
    a.out = traces + per_frame * f0;
    a.partial = static_cast<float *>(ws);
    a.s_tile = p.s_tile;
    a.t_tile = p.t_tile;
    a.nb_tile = p.nb_tile;
    a.n_splits = p.n_splits;
    a.n_stiles = p.n_stiles;
    a.n_ttiles = p.n_ttiles;
    a.balls_per_split = p.balls_per_split;
    a.flags = flags;
    a.err = d->err;
    const int rc = cuda_status(pa::launch_forward(a, p, (flags & PA_PROFILE_UNIFORM) != 0, st));
    if (rc) return rc;
  }
  return PA_OK;
}

int forward_impl(const pa_geom *geom, const pa_balls *balls, int32_t F, float *traces, uint32_t flags,
                 const int32_t *tiles, void *ws, size_t ws_bytes, void *stream) {
  int rc = check_geom(geom);
  if (rc) return rc;
  if ((rc = check_balls(balls))) return rc;
  if (F < 0 || (flags & ~(PA_ACCUMULATE | PA_PROFILE_UNIFORM)) != 0) return PA_ERR_INVALID_ARG;
  if (F == 0) return PA_OK;
  if (traces == nullptr || !aligned(traces, 16)) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (balls->n == 0) {
    if (flags & PA_ACCUMULATE) return PA_OK;
    return cuda_status(
        cudaMemsetAsync(traces, 0, sizeof(float) * (size_t)F * geom->n_sensors * geom->n_samples, st));
  }
  if (!tiles_ok(tiles)) return PA_ERR_INVALID_ARG;
  return forward_launch(d, geom, balls->state, balls->n, balls->stride, F, traces, flags, tiles, ws, ws_bytes, st);
}

// Frames per launch of the 4D calls: as many as keep one chunk's states and
// state gradients ([K][5][stride] floats each, 40 B per ball and frame)
// within an eighth of the deformation parameters' own memory ((omega, theta,
// sigma) [5][Nb][stride], 60 Nb B per ball), i.e. K = floor(3 Nb / 16), at
// least 1 and at most F; a plan may fix the number.  The transient memory of
// the 4D calls is then a fixed fraction of the model's, whatever the number
// of frames.
int frames_per_chunk(const pa_plan *plan, int n_basis, int F) {
  if (F <= 0) return 1;
  if (plan && plan->frames_per_chunk > 0) return std::min(plan->frames_per_chunk, F);
  return std::max(1, std::min(3 * n_basis / 16, F));
}

inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of one chunk's per-frame buffer [K][5][stride] (256-byte multiple).
inline size_t chunk_state_bytes(const pa_canon *c, int K) {
  return round256(sizeof(float) * 5 * (size_t)c->stride * (size_t)K);
}

// Forward split partials of the largest chunk of a 4D forward.
size_t forward_4d_partials(const DevInfo *d, const pa_geom *g, const pa_canon *c, int32_t F, int K,
                           const int32_t *tiles) {
  size_t ws = 0;
  for (int k : {K, F % K})
    if (k > 0) ws = std::max(ws, forward_chunking(d, g, c->n, k, tiles).ws);
  return ws;
}

// One event-timed run of fn() (returning a PA status) on `st`.
template <typename Fn>
int time_once(Fn fn, cudaStream_t st, float &ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PA_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PA_ERR_CUDA;
  }
  int rc = cudaEventRecord(e0, st) == cudaSuccess ? PA_OK : PA_ERR_CUDA;
  if (rc == PA_OK) rc = fn();
  if (rc == PA_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    rc = PA_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// Best of `reps` event-timed runs of fn() (returning a PA status) on `st`
// after one untimed run.
template <typename Fn>
int time_best(Fn fn, cudaStream_t st, int reps, float &best_ms) {
  int rc = fn();
  if (rc) return rc;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PA_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PA_ERR_CUDA;
  }
  best_ms = 3.4e38f;
  for (int r = 0; r < reps && rc == PA_OK; ++r) {
    float ms = 0.f;
    if (cudaEventRecord(e0, st) != cudaSuccess) rc = PA_ERR_CUDA;
    if (rc == PA_OK) rc = fn();
    if (rc == PA_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = PA_ERR_CUDA;
    if (rc == PA_OK) best_ms = std::min(best_ms, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// Candidate forward tile plans the tuner times: {sensors per CTA, samples per
// CTA, balls per stage, ball splits (0 = the planner's), pairs per sweep}.
constexpr int32_t kTileCandidates[][5] = {
    {16, 1536, 512, 0, 16}, {16, 1536, 512, 0, 8}, {12, 2048, 512, 0, 16}, {12, 2048, 512, 0, 8},
    {16, 1536, 256, 0, 16}, {16, 1024, 512, 0, 16}, {8, 2048, 512, 0, 16}, {16, 1536, 512, 0, 4},
};
constexpr int kNumTileCandidates = sizeof(kTileCandidates) / sizeof(kTileCandidates[0]);
constexpr int32_t kAdjChunkCandidates[] = {1, 2, 4, 8, 16};

// Bytes at the start of a batched or pa_adjoint_4d workspace: its work-queue
// counter.
constexpr size_t kQueueBytes = 256;
static_assert(kQueueBytes == PA_ADJOINT_WORKSPACE_BYTES, "one queue slot layout");

// Ball splits of one scene in a batched forward: the plan's split count, else
// one split per kMaxBallsPerBatchedSplit balls (narrower arrival bands per split), at
// most one per TMA stage of balls; balls per split a multiple of 4.
void batched_splits(long long n, const int32_t *tiles, int nb_tile, int &n_splits, long long &bps) {
  long long sp = tiles && tiles[3] > 0 ? tiles[3] : (n + pa::kMaxBallsPerBatchedSplit - 1) / pa::kMaxBallsPerBatchedSplit;
  sp = std::max(1LL, std::min(sp, (n + nb_tile - 1) / nb_tile));
  bps = (((n + sp - 1) / sp) + 3) & ~3LL;
  if (bps <= 0) bps = 4;
  n_splits = (int)std::max(1LL, (n + bps - 1) / bps);
}

int batched_nb_tile(const int32_t *tiles) { return tiles && tiles[2] > 0 ? tiles[2] : 512; }

// Split partials [splits][F][S][T] of one scene of a batched forward.
size_t batched_partial_bytes(const pa_scene &sc, const int32_t *tiles) {
  if (sc.n_frames <= 0 || sc.balls.n <= 0) return 0;
  int sp;
  long long bps;
  batched_splits(sc.balls.n, tiles, batched_nb_tile(tiles), sp, bps);
  if (sp <= 1) return 0;
  return round256(sizeof(float) * (size_t)sp * sc.n_frames * sc.geom.n_sensors * sc.geom.n_samples);
}

// Tile shape of a batched forward over these scenes: samples per CTA capped by
// the longest trace, then the sensors per CTA that fit.
struct BatchedTiles {
  int s_tile, t_tile, nb_tile, group;
  size_t smem;
};
BatchedTiles batched_tiles(const pa_scene *scenes, int32_t n_scenes, const int32_t *tiles) {
  int maxT = 4;
  for (int i = 0; i < n_scenes; ++i) maxT = std::max(maxT, scenes[i].geom.n_samples);
  BatchedTiles b;
  b.t_tile = tiles && tiles[1] > 0 ? tiles[1] : pa::kDefaultTTile;
  b.t_tile = std::min(std::min(b.t_tile, maxT), 16384);
  b.nb_tile = tiles && tiles[2] > 0 ? tiles[2] : 512;
  b.s_tile = tiles && tiles[0] > 0 ? tiles[0] : pa::forward_default_s_tile(b.t_tile, b.nb_tile);
  b.group = tiles && (tiles[4] == 1 || tiles[4] == 2 || tiles[4] == 4 || tiles[4] == 8) ? tiles[4] : 16;
  b.smem = pa::forward_smem_bytes(b.s_tile, b.t_tile, b.nb_tile);
  return b;
}

int check_scenes(const pa_scene *scenes, int32_t n_scenes) {
  if (n_scenes < 1 || n_scenes > PA_MAX_SCENES || scenes == nullptr) return PA_ERR_INVALID_ARG;
  for (int i = 0; i < n_scenes; ++i) {
    int rc = check_geom(&scenes[i].geom);
    if (rc) return rc;
    if ((rc = check_balls(&scenes[i].balls))) return rc;
    if (scenes[i].n_frames < 0) return PA_ERR_INVALID_ARG;
  }
  return PA_OK;
}

}  // namespace

extern "C" {

const char *pa_status_string(int32_t status) {
  switch (status) {
    case PA_OK: return "PA_OK";
    case PA_ERR_INVALID_ARG: return "PA_ERR_INVALID_ARG: invalid argument";
    case PA_ERR_DOMAIN: return "PA_ERR_DOMAIN: sensor inside a ball support or non-positive basis width";
    case PA_ERR_CUDA: return "PA_ERR_CUDA: CUDA runtime error";
    case PA_ERR_TIMEOUT: return "PA_ERR_TIMEOUT: bounded wait ran out inside a kernel";
    case PA_ERR_WORKSPACE: return "PA_ERR_WORKSPACE: workspace missing, misaligned or too small";
    default: return "unknown status";
  }
}

int32_t pa_version(void) { return 202; }

int32_t pa_device_error(void *stream, int32_t *out) {
  if (out == nullptr) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, d->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d->err, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return PA_ERR_CUDA;
  *out = (int32_t)v;
  return PA_OK;
}

int32_t pa_deform_balls(const pa_canon *canon, const float *t_frames, int32_t n_frames, float *state_out,
                        void *stream) {
  int rc = check_canon(canon);
  if (rc) return rc;
  if (n_frames < 0) return PA_ERR_INVALID_ARG;
  if (n_frames == 0 || canon->n == 0) return PA_OK;
  if (t_frames == nullptr || state_out == nullptr) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  return cuda_status(pa::launch_deform(canon->canon, canon->omega, canon->theta, canon->sigma, canon->n,
                                       canon->stride, canon->n_basis, t_frames, n_frames, state_out, d->err,
                                       static_cast<cudaStream_t>(stream)));
}

int32_t pa_deform_backward(const pa_canon *canon, const float *t_frames, int32_t n_frames, const float *g_state,
                           pa_grads *grads, uint32_t flags, void *stream) {
  int rc = check_canon(canon);
  if (rc) return rc;
  if (n_frames < 0 || (flags & ~PA_ACCUMULATE) != 0 || grads == nullptr) return PA_ERR_INVALID_ARG;
  if (canon->n == 0) return PA_OK;
  if (!grads->state || !grads->omega || !grads->theta || !grads->sigma) return PA_ERR_INVALID_ARG;
  if (n_frames > 0 && (t_frames == nullptr || g_state == nullptr)) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  return cuda_status(pa::launch_deform_backward(canon->canon, canon->omega, canon->theta, canon->sigma, canon->n,
                                                canon->stride, canon->n_basis, t_frames, n_frames, g_state,
                                                grads->state, grads->omega, grads->theta, grads->sigma,
                                                (flags & PA_ACCUMULATE) != 0, d->err,
                                                static_cast<cudaStream_t>(stream)));
}

size_t pa_forward_workspace_size_ex(const pa_geom *geom, const pa_balls *balls, int32_t n_frames,
                                    const int32_t *tiles) {
  if (!tiles_ok(tiles) || check_geom(geom) || check_balls(balls) || n_frames <= 0 || balls->n == 0) return 0;
  const DevInfo *d = dev_info();
  if (!d) return 0;
  return forward_chunking(d, geom, balls->n, n_frames, tiles).ws;
}

size_t pa_forward_workspace_size(const pa_geom *geom, const pa_balls *balls, int32_t n_frames) {
  return pa_forward_workspace_size_ex(geom, balls, n_frames, nullptr);
}

int32_t pa_forward(const pa_geom *geom, const pa_balls *balls, int32_t n_frames, float *traces, uint32_t flags,
                   void *workspace, size_t workspace_bytes, void *stream) {
  return forward_impl(geom, balls, n_frames, traces, flags, nullptr, workspace, workspace_bytes, stream);
}

int32_t pa_forward_ex(const pa_geom *geom, const pa_balls *balls, int32_t n_frames, float *traces, uint32_t flags,
                      const int32_t *tiles, void *workspace, size_t workspace_bytes, void *stream) {
  return forward_impl(geom, balls, n_frames, traces, flags, tiles, workspace, workspace_bytes, stream);
}

int32_t pa_forward_plan_info(const pa_geom *geom, const pa_balls *balls, int32_t n_frames, const int32_t *tiles,
                             int32_t *out7) {
  if (out7 == nullptr) return PA_ERR_INVALID_ARG;
  if (!tiles_ok(tiles)) return PA_ERR_INVALID_ARG;
  int rc = check_geom(geom);
  if (rc) return rc;
  if ((rc = check_balls(balls))) return rc;
  if (n_frames <= 0) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  const pa::FwdPlan p = pa::forward_plan(geom->n_sensors, geom->n_samples, balls->n, n_frames, d->sms,
                                         tiles ? tiles[0] : 0, tiles ? tiles[1] : 0, tiles ? tiles[2] : 0,
                                         tiles ? tiles[3] : 0, tiles ? tiles[4] : 0);
  out7[0] = p.s_tile;
  out7[1] = p.t_tile;
  out7[2] = p.nb_tile;
  out7[3] = p.n_splits;
  out7[4] = p.group;
  out7[5] = (int32_t)((long long)n_frames * p.n_stiles * p.n_ttiles * p.n_splits);
  out7[6] = (int32_t)p.smem;
  return PA_OK;
}

int32_t pa_adjoint(const pa_geom *geom, const pa_balls *balls, const pa_canon *canon, const float *t_frames,
                   int32_t n_frames, const float *trace_grad, const float *frame_scale, pa_grads *grads,
                   uint32_t flags, void *workspace, size_t workspace_bytes, void *stream) {
  int rc = check_geom(geom);
  if (rc) return rc;
  if (n_frames < 0 || grads == nullptr || (flags & ~PA_ACCUMULATE) != 0) return PA_ERR_INVALID_ARG;
  if (workspace != nullptr && (workspace_bytes < PA_ADJOINT_WORKSPACE_BYTES || !aligned(workspace, 256)))
    return PA_ERR_WORKSPACE;
  const bool four_d = canon != nullptr;
  if ((balls != nullptr) == four_d) return PA_ERR_INVALID_ARG;  // exactly one mode
  if (four_d) {
    if ((rc = check_canon(canon))) return rc;
    if (canon->n > 0 && (!grads->state || !grads->omega || !grads->theta || !grads->sigma))
      return PA_ERR_INVALID_ARG;
    if (n_frames > 0 && t_frames == nullptr) return PA_ERR_INVALID_ARG;
  } else {
    if ((rc = check_balls(balls))) return rc;
    if (balls->n > 0 && grads->state == nullptr) return PA_ERR_INVALID_ARG;
  }
  const long long n = four_d ? canon->n : balls->n;
  if (n == 0) return PA_OK;
  if (n_frames > 0 && (trace_grad == nullptr || !aligned(trace_grad, 16))) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pa::AdjArgs a;
  std::memset(&a, 0, sizeof(a));
  a.q = make_acq(geom);
  a.F = n_frames;
  a.g = trace_grad;
  a.frame_scale = frame_scale;
  a.g_state = grads->state;
  a.flags = flags;
  a.err = d->err;
  a.n = n;
  if (four_d) {
    a.canon = canon->canon;
    a.omega = canon->omega;
    a.theta = canon->theta;
    a.sigma = canon->sigma;
    a.nb = canon->n_basis;
    a.stride = canon->stride;
    a.t_frames = t_frames;
    a.g_omega = grads->omega;
    a.g_theta = grads->theta;
    a.g_sigma = grads->sigma;
    a.n_items = n;
    const size_t smem = pa::adj_4d_smem(geom->n_sensors);
    if ((long long)smem > d->max_smem) return PA_ERR_INVALID_ARG;
    if (n_frames == 0) {
      // no frame contributes: gradients are zero
      if (flags & PA_ACCUMULATE) return PA_OK;
      const size_t rows = sizeof(float) * (size_t)canon->stride;
      cudaError_t e = cudaMemsetAsync(grads->state, 0, rows * 5, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(grads->omega, 0, rows * 5 * canon->n_basis, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(grads->theta, 0, rows * 5 * canon->n_basis, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(grads->sigma, 0, rows * 5 * canon->n_basis, st);
      return cuda_status(e);
    }
    return cuda_status(pa::launch_adjoint_4d(a, d->sms, st));
  }
  a.state = balls->state;
  a.stride = balls->stride;
  a.n_items = (long long)n_frames * n;
  a.queue = static_cast<unsigned long long *>(workspace);
  const size_t smem = pa::adj_static_smem(geom->n_sensors);
  if ((long long)smem > d->max_smem) return PA_ERR_INVALID_ARG;
  return cuda_status(pa::launch_adjoint_static(a, d->sms, st));
}

size_t pa_batched_workspace_size(const pa_scene *scenes, int32_t n_scenes, const pa_plan *plan) {
  size_t ws = kQueueBytes;
  if (n_scenes <= 0 || scenes == nullptr || n_scenes > PA_MAX_SCENES) return ws;
  const int32_t *tiles = plan ? plan->tiles : nullptr;
  for (int i = 0; i < n_scenes; ++i) ws += batched_partial_bytes(scenes[i], tiles);
  return ws;
}

int32_t pa_forward_batched(const pa_scene *scenes, int32_t n_scenes, uint32_t flags, const pa_plan *plan,
                           void *workspace, size_t workspace_bytes, void *stream) {
  const int32_t *tiles = plan ? plan->tiles : nullptr;
  if (n_scenes < 0 || n_scenes > PA_MAX_SCENES || (n_scenes > 0 && scenes == nullptr)) return PA_ERR_INVALID_ARG;
  if ((flags & ~PA_ACCUMULATE) != 0) return PA_ERR_INVALID_ARG;
  if (!tiles_ok(tiles)) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n_scenes; ++i) {
    const pa_scene &sc = scenes[i];
    int rc = check_geom(&sc.geom);
    if (rc) return rc;
    if ((rc = check_balls(&sc.balls))) return rc;
    if (sc.n_frames < 0) return PA_ERR_INVALID_ARG;
    if (sc.n_frames > 0 && (sc.traces == nullptr || !aligned(sc.traces, 16))) return PA_ERR_INVALID_ARG;
  }
  const BatchedTiles bt = batched_tiles(scenes, n_scenes, tiles);
  const int t_tile = bt.t_tile, nb_tile = bt.nb_tile, s_tile = bt.s_tile, group = bt.group;
  const size_t smem = bt.smem;
  if ((long long)smem > d->max_smem) return PA_ERR_INVALID_ARG;
  if (workspace == nullptr || workspace_bytes < pa_batched_workspace_size(scenes, n_scenes, plan) ||
      !aligned(workspace, 256))
    return PA_ERR_WORKSPACE;
  // scenes with balls, heaviest items (most balls per split) first
  int order[PA_MAX_SCENES];
  int m = 0;
  for (int i = 0; i < n_scenes; ++i) {
    const pa_scene &sc = scenes[i];
    if (sc.n_frames == 0) continue;
    if (sc.balls.n == 0) {
      if (!(flags & PA_ACCUMULATE)) {
        cudaError_t e = cudaMemsetAsync(
            sc.traces, 0, sizeof(float) * (size_t)sc.n_frames * sc.geom.n_sensors * sc.geom.n_samples, st);
        if (e != cudaSuccess) return PA_ERR_CUDA;
      }
      continue;
    }
    order[m++] = i;
  }
  auto item_balls = [&](int i) {
    int sp;
    long long bps;
    batched_splits(scenes[i].balls.n, tiles, nb_tile, sp, bps);
    return std::min<long long>(bps, scenes[i].balls.n);
  };
  std::sort(order, order + m, [&](int x, int y) { return item_balls(x) > item_balls(y); });
  pa::BatchFwdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_scenes = m;
  a.s_tile = s_tile;
  a.t_tile = t_tile;
  a.nb_tile = nb_tile;
  a.counter = static_cast<unsigned long long *>(workspace);
  a.flags = flags;
  a.err = d->err;
  long long items = 0;
  char *partials = static_cast<char *>(workspace) + kQueueBytes;
  for (int j = 0; j < m; ++j) {
    const pa_scene &sc = scenes[order[j]];
    pa::SceneFwd &o = a.sc[j];
    o.q = make_acq(&sc.geom);
    o.state = sc.balls.state;
    o.n = sc.balls.n;
    o.stride = sc.balls.stride;
    o.F = sc.n_frames;
    o.out = sc.traces;
    o.n_stiles = (sc.geom.n_sensors + s_tile - 1) / s_tile;
    o.n_ttiles = (sc.geom.n_samples + t_tile - 1) / t_tile;
    batched_splits(sc.balls.n, tiles, nb_tile, o.n_splits, o.balls_per_split);
    o.partial = nullptr;
    if (o.n_splits > 1) {
      o.partial = reinterpret_cast<float *>(partials);
      partials += batched_partial_bytes(sc, tiles);
    }
    o.item_begin = items;
    items += (long long)sc.n_frames * o.n_stiles * o.n_ttiles * o.n_splits;
  }
  a.total_items = items;
  if (items == 0) return PA_OK;
  // CTAs write only the sample band a scene's balls reach: zero the rest
  // first (scenes with ball splits are written whole by the split reduction)
  if (!(flags & PA_ACCUMULATE)) {
    for (int j = 0; j < m; ++j) {
      if (a.sc[j].n_splits > 1) continue;
      const pa_scene &sc = scenes[order[j]];
      cudaError_t e = cudaMemsetAsync(
          sc.traces, 0, sizeof(float) * (size_t)sc.n_frames * sc.geom.n_sensors * sc.geom.n_samples, st);
      if (e != cudaSuccess) return PA_ERR_CUDA;
    }
  }
  return cuda_status(pa::launch_forward_batched(a, group, smem, d->sms, st));
}

int32_t pa_adjoint_batched(const pa_scene *scenes, int32_t n_scenes, uint32_t flags, const pa_plan *plan,
                           void *workspace, size_t workspace_bytes, void *stream) {
  if (n_scenes < 0 || n_scenes > PA_MAX_SCENES || (n_scenes > 0 && scenes == nullptr)) return PA_ERR_INVALID_ARG;
  if ((flags & ~PA_ACCUMULATE) != 0) return PA_ERR_INVALID_ARG;
  if (workspace == nullptr || workspace_bytes < kQueueBytes || !aligned(workspace, 16)) return PA_ERR_WORKSPACE;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  int order[PA_MAX_SCENES];
  int m = 0;
  for (int i = 0; i < n_scenes; ++i) {
    const pa_scene &sc = scenes[i];
    int rc = check_geom(&sc.geom);
    if (rc) return rc;
    if ((rc = check_balls(&sc.balls))) return rc;
    if (sc.n_frames < 0) return PA_ERR_INVALID_ARG;
    if (sc.n_frames == 0 || sc.balls.n == 0) continue;
    if (sc.trace_grad == nullptr || sc.grad_state == nullptr || !aligned(sc.trace_grad, 16)) return PA_ERR_INVALID_ARG;
    order[m++] = i;
  }
  std::sort(order, order + m,
            [&](int x, int y) { return scenes[x].geom.n_sensors > scenes[y].geom.n_sensors; });
  pa::BatchAdjArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_scenes = m;
  a.chunk = plan && plan->adj_chunk > 0 ? plan->adj_chunk : 1;
  a.counter = static_cast<unsigned long long *>(workspace);
  a.flags = flags;
  a.err = d->err;
  long long items = 0;
  for (int j = 0; j < m; ++j) {
    const pa_scene &sc = scenes[order[j]];
    pa::SceneAdj &o = a.sc[j];
    o.q = make_acq(&sc.geom);
    o.state = sc.balls.state;
    o.n = sc.balls.n;
    o.stride = sc.balls.stride;
    o.F = sc.n_frames;
    o.g = sc.trace_grad;
    o.g_state = sc.grad_state;
    o.item_begin = items;
    items += (long long)sc.n_frames * sc.balls.n;
  }
  a.total_items = items;
  if (items == 0) return PA_OK;
  return cuda_status(pa::launch_adjoint_batched(a, d->sms, static_cast<cudaStream_t>(stream)));
}

size_t pa_spatial_order_workspace_size(int64_t n) {
  if (n <= 0 || n > INT32_MAX) return 0;
  return pa::spatial_order_workspace(n);
}

int32_t pa_spatial_order(const pa_balls *balls, int32_t *perm, void *workspace, size_t workspace_bytes,
                         void *stream) {
  int rc = check_balls(balls);
  if (rc) return rc;
  if (balls->n > INT32_MAX) return PA_ERR_INVALID_ARG;
  if (balls->n == 0) return PA_OK;
  if (perm == nullptr || !aligned(perm, 4)) return PA_ERR_INVALID_ARG;
  if (workspace == nullptr || workspace_bytes < pa::spatial_order_workspace(balls->n) || !aligned(workspace, 256))
    return PA_ERR_WORKSPACE;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  return cuda_status(pa::launch_spatial_order(balls->state, balls->stride, balls->n, perm, workspace, d->sms,
                                              static_cast<cudaStream_t>(stream)));
}

int32_t pa_gather_rows(const float *in, float *out, int64_t n, int64_t stride, int32_t rows, const int32_t *perm,
                       void *stream) {
  if (n < 0 || stride < n || rows < 0 || n > INT32_MAX) return PA_ERR_INVALID_ARG;
  if (n == 0 || rows == 0) return PA_OK;
  if (in == nullptr || out == nullptr || perm == nullptr || in == out) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  return cuda_status(pa::launch_gather_rows(in, out, n, stride, rows, perm, d->sms, static_cast<cudaStream_t>(stream)));
}

size_t pa_loss_workspace_size(int64_t per_frame, int32_t n_frames) {
  if (per_frame <= 0 || n_frames <= 0) return 0;
  return sizeof(double) * (size_t)n_frames * pa::loss_blocks_per_frame(per_frame);
}

int32_t pa_residual_loss(const float *pred, const float *meas, int64_t per_frame, int32_t n_frames,
                         const float *frame_scale, double *loss, float *resid, void *workspace,
                         size_t workspace_bytes, void *stream) {
  if (per_frame < 4 || (per_frame & 3) != 0 || n_frames < 0) return PA_ERR_INVALID_ARG;
  if (n_frames == 0) return PA_OK;
  if (!pred || !meas || !aligned(pred, 16) || !aligned(meas, 16)) return PA_ERR_INVALID_ARG;
  if (resid && !aligned(resid, 16)) return PA_ERR_INVALID_ARG;
  if (!loss && !resid) return PA_ERR_INVALID_ARG;
  const size_t need = pa_loss_workspace_size(per_frame, n_frames);
  if (workspace == nullptr || workspace_bytes < need || !aligned(workspace, 16)) return PA_ERR_WORKSPACE;
  return cuda_status(pa::launch_loss(pred, meas, per_frame, n_frames, frame_scale, loss, resid,
                                     static_cast<double *>(workspace), pa::loss_blocks_per_frame(per_frame),
                                     static_cast<cudaStream_t>(stream)));
}

int32_t pa_sumsq(const float *x, int64_t n, double *out, void *workspace, size_t workspace_bytes, void *stream) {
  if (n < 4 || (n & 3) != 0 || !x || !out || !aligned(x, 16)) return PA_ERR_INVALID_ARG;
  const size_t need = pa_loss_workspace_size(n, 1);
  if (workspace == nullptr || workspace_bytes < need || !aligned(workspace, 16)) return PA_ERR_WORKSPACE;
  return cuda_status(pa::launch_loss(x, nullptr, n, 1, nullptr, out, nullptr, static_cast<double *>(workspace),
                                     pa::loss_blocks_per_frame(n), static_cast<cudaStream_t>(stream)));
}

int32_t pa_count_contributions(const pa_geom *geom, const pa_balls *balls, int32_t n_frames,
                               unsigned long long *out, void *stream) {
  int rc = check_geom(geom);
  if (rc) return rc;
  if ((rc = check_balls(balls))) return rc;
  if (n_frames < 0 || out == nullptr) return PA_ERR_INVALID_ARG;
  return cuda_status(pa::launch_count(make_acq(geom), balls->state, balls->n, balls->stride, n_frames, out,
                                      static_cast<cudaStream_t>(stream)));
}

int32_t pa_adam_step(float *x, const float *g, float *m, float *v, int64_t n, double lr, double beta1, double beta2,
                     double eps, int32_t step, void *stream) {
  if (n < 0 || step < 1 || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return PA_ERR_INVALID_ARG;
  if (n == 0) return PA_OK;
  if (!x || !g || !m || !v || !aligned(x, 16) || !aligned(g, 16) || !aligned(m, 16) || !aligned(v, 16))
    return PA_ERR_INVALID_ARG;
  const float bc1 = (float)(1.0 - std::pow(beta1, (double)step));
  const float bc2 = (float)(1.0 - std::pow(beta2, (double)step));
  return cuda_status(pa::launch_adam(x, g, m, v, n, (float)lr, (float)beta1, (float)beta2, (float)(1.0 - beta1),
                                     (float)(1.0 - beta2), (float)eps, bc1, bc2, static_cast<cudaStream_t>(stream)));
}

int32_t pa_adam_step_scheduled(float *x, const float *g, float *m, float *v, int64_t n, double lr0, double beta1,
                               double beta2, double eps, int32_t step_size, double gamma, const int32_t *step,
                               void *stream) {
  if (n < 0 || step_size < 1 || step == nullptr || !(beta1 >= 0.0 && beta1 < 1.0) ||
      !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) || !(gamma > 0.0))
    return PA_ERR_INVALID_ARG;
  if (n == 0) return PA_OK;
  if (!x || !g || !m || !v) return PA_ERR_INVALID_ARG;
  return cuda_status(pa::launch_adam_sched(x, g, m, v, n, (float)lr0, (float)beta1, (float)beta2,
                                           (float)(1.0 - beta1), (float)(1.0 - beta2), (float)eps, step_size,
                                           (float)gamma, step, static_cast<cudaStream_t>(stream)));
}

int32_t pa_step_increment(int32_t *step, void *stream) {
  if (step == nullptr) return PA_ERR_INVALID_ARG;
  return cuda_status(pa::launch_step_increment(step, static_cast<cudaStream_t>(stream)));
}


// ---------------------------------------------------------------------------
// Imaging.

int32_t pa_ubp_filter(const float *traces, int64_t n_traces, int32_t n_samples, float fs, float t0, float *b,
                      void *stream) {
  if (n_traces < 0 || n_samples < 2 || !(fs > 0.f) || !std::isfinite(t0)) return PA_ERR_INVALID_ARG;
  if (n_traces == 0) return PA_OK;
  if (traces == nullptr || b == nullptr || traces == b) return PA_ERR_INVALID_ARG;
  if (!dev_info()) return PA_ERR_CUDA;
  return cuda_status(pa::launch_ubp_filter(traces, n_traces, n_samples, fs, t0, b, static_cast<cudaStream_t>(stream)));
}

int32_t pa_ubp(const pa_geom *geom, const float *center, const float *b, const pa_grid *grid, float *vol,
               void *stream) {
  int rc = check_geom(geom);
  if (rc) return rc;
  if ((rc = check_grid(grid))) return rc;
  if (center == nullptr || b == nullptr || vol == nullptr) return PA_ERR_INVALID_ARG;
  if (!dev_info()) return PA_ERR_CUDA;
  pa::UbpArgs a;
  a.b = b;
  a.sensors = geom->sensors;
  a.S = geom->n_sensors;
  a.sstride = geom->sensor_stride;
  a.T = geom->n_samples;
  a.cx = center[0];
  a.cy = center[1];
  a.cz = center[2];
  a.fs_c = (float)((double)geom->fs / (double)geom->c);
  a.t0_fs = (float)((double)geom->t0 * (double)geom->fs);
  a.ox = grid->origin[0];
  a.oy = grid->origin[1];
  a.oz = grid->origin[2];
  a.h = grid->h;
  a.nx = grid->nx;
  a.ny = grid->ny;
  a.nz = grid->nz;
  a.vol = vol;
  return cuda_status(pa::launch_ubp(a, static_cast<cudaStream_t>(stream)));
}

int32_t pa_splat(const pa_balls *balls, float kappa, const pa_grid *grid, float *vol, void *stream) {
  int rc = check_balls(balls);
  if (rc) return rc;
  if ((rc = check_grid(grid))) return rc;
  if (!(kappa > 0.f) || vol == nullptr) return PA_ERR_INVALID_ARG;
  if (!dev_info()) return PA_ERR_CUDA;
  pa::SplatArgs a;
  a.state = balls->state;
  a.n = balls->n;
  a.stride = balls->stride;
  a.kappa = kappa;
  a.ox = grid->origin[0];
  a.oy = grid->origin[1];
  a.oz = grid->origin[2];
  a.h = grid->h;
  a.nx = grid->nx;
  a.ny = grid->ny;
  a.nz = grid->nz;
  a.vol = vol;
  return cuda_status(pa::launch_splat(a, static_cast<cudaStream_t>(stream)));
}

int32_t pa_map(const float *vol, const pa_grid *grid, float *xy, float *yz, float *xz, void *stream) {
  int rc = check_grid(grid);
  if (rc) return rc;
  if (vol == nullptr) return PA_ERR_INVALID_ARG;
  if (!dev_info()) return PA_ERR_CUDA;
  return cuda_status(pa::launch_map(vol, grid->nx, grid->ny, grid->nz, xy, yz, xz, static_cast<cudaStream_t>(stream)));
}

size_t pa_ssim_workspace_size(int32_t H, int32_t W) {
  if (H < 11 || W < 11) return 0;
  // normalisation (16 B) + min/max partials + FP64 SSIM partials
  return 16 + sizeof(float4) * (size_t)pa::minmax_partials() + sizeof(double) * (size_t)pa::ssim_blocks(H, W);
}

int32_t pa_ssim(const float *x, const float *y, int32_t H, int32_t W, float L, uint32_t flags, float *map,
                double *mean, void *workspace, size_t workspace_bytes, void *stream) {
  if ((flags & ~PA_SSIM_MINMAX) != 0) return PA_ERR_INVALID_ARG;
  if (flags & PA_SSIM_MINMAX) L = 1.f;
  if (H < 11 || W < 11 || !(L > 0.f) || x == nullptr || y == nullptr || mean == nullptr) return PA_ERR_INVALID_ARG;
  if (workspace == nullptr || workspace_bytes < pa_ssim_workspace_size(H, W) || !aligned(workspace, 16))
    return PA_ERR_WORKSPACE;
  if (!dev_info()) return PA_ERR_CUDA;
  pa::SsimArgs a;
  a.x = x;
  a.y = y;
  a.H = H;
  a.W = W;
  a.C1 = (float)((0.01 * (double)L) * (0.01 * (double)L));
  a.C2 = (float)((0.03 * (double)L) * (0.03 * (double)L));
  double g[11], gs = 0.0;
  for (int i = 0; i < 11; ++i) {
    g[i] = std::exp(-((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
    gs += g[i];
  }
  for (int i = 0; i < 11; ++i) a.g[i] = (float)(g[i] / gs);
  a.map = map;
  char *ws = static_cast<char *>(workspace);
  float4 *norm = reinterpret_cast<float4 *>(ws);
  float4 *mm = reinterpret_cast<float4 *>(ws + 16);
  a.partials = reinterpret_cast<double *>(ws + 16 + sizeof(float4) * (size_t)pa::minmax_partials());
  a.norm = (flags & PA_SSIM_MINMAX) ? norm : nullptr;
  return cuda_status(pa::launch_ssim(a, mean, mm, static_cast<cudaStream_t>(stream)));
}


int32_t pa_selftest_bounded_wait(uint64_t limit_ns, void *stream) {
  if (limit_ns < 1000ull || limit_ns > 1000000000ull) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  return cuda_status(pa::launch_selftest_wait(limit_ns, d->err, static_cast<cudaStream_t>(stream)));
}

int32_t pa_measure_unit_rates(void *stream, double *out4) {
  if (out4 == nullptr) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  return cuda_status(pa::measure_unit_rates(d->sms, static_cast<cudaStream_t>(stream), out4));
}

// ---------------------------------------------------------------------------
// Launch plans.

size_t pa_plan_workspace_size(const pa_scene *scenes, int32_t n_scenes) {
  if (check_scenes(scenes, n_scenes)) return 0;
  size_t ws = kQueueBytes;
  if (n_scenes > 1) {
    for (int c = -1; c < kNumTileCandidates; ++c) {
      pa_plan p;
      std::memset(&p, 0, sizeof(p));
      if (c >= 0) std::memcpy(p.tiles, kTileCandidates[c], sizeof(p.tiles));
      ws = std::max(ws, pa_batched_workspace_size(scenes, n_scenes, &p));
    }
    return ws;
  }
  const DevInfo *d = dev_info();
  if (!d) return 0;
  const pa_scene &sc = scenes[0];
  if (sc.n_frames <= 0 || sc.balls.n == 0) return ws;
  for (int c = -1; c < kNumTileCandidates; ++c) {
    const int32_t *t = c < 0 ? nullptr : kTileCandidates[c];
    const pa::FwdPlan p = plan_for(d, &sc.geom, sc.balls.n, 1, t);
    if (p.smem <= (size_t)d->max_smem) ws = std::max(ws, forward_chunking(d, &sc.geom, sc.balls.n, sc.n_frames, t).ws);
  }
  return ws;
}

int32_t pa_plan_from_values(const int32_t *values7, pa_plan **out) {
  if (out == nullptr) return PA_ERR_INVALID_ARG;
  *out = nullptr;
  if (values7 != nullptr) {
    if (!tiles_ok(values7) || values7[5] < 0 || values7[6] < 0 || values7[6] > 1024) return PA_ERR_INVALID_ARG;
  }
  pa_plan *p = new (std::nothrow) pa_plan;
  if (p == nullptr) return PA_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  if (values7 != nullptr) {
    std::memcpy(p->tiles, values7, sizeof(p->tiles));
    p->frames_per_chunk = values7[5];
    p->adj_chunk = values7[6];
  }
  *out = p;
  return PA_OK;
}

int32_t pa_plan_create(const pa_scene *scenes, int32_t n_scenes, uint32_t flags, void *workspace,
                       size_t workspace_bytes, void *stream, pa_plan **out) {
  if (out == nullptr) return PA_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = check_scenes(scenes, n_scenes);
  if (rc) return rc;
  if ((flags & ~PA_PLAN_TUNE) != 0) return PA_ERR_INVALID_ARG;
  pa_plan *plan = nullptr;
  if ((rc = pa_plan_from_values(nullptr, &plan))) return rc;
  if (!(flags & PA_PLAN_TUNE)) {
    *out = plan;
    return PA_OK;
  }
  const DevInfo *d = dev_info();
  if (!d) {
    delete plan;
    return PA_ERR_CUDA;
  }
  const size_t need = pa_plan_workspace_size(scenes, n_scenes);
  if (workspace == nullptr || workspace_bytes < need || !aligned(workspace, 256)) {
    delete plan;
    return PA_ERR_WORKSPACE;
  }
  for (int i = 0; i < n_scenes; ++i) {
    const pa_scene &sc = scenes[i];
    if (sc.n_frames > 0 && (sc.traces == nullptr || !aligned(sc.traces, 16))) {
      delete plan;
      return PA_ERR_INVALID_ARG;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Forward tiles: a single scene is timed through pa_forward_ex (ball
  // splits by the planner), several through one persistent batched launch.
  // Candidate -1 is the built-in heuristic.  Every candidate runs once
  // untimed, then all are timed in kTuneRounds interleaved rounds (so that a
  // drift of the clock touches them alike) and each keeps its best time; a
  // candidate replaces the heuristic only when it is faster by more than
  // kTuneMargin, so timing noise cannot select a worse plan.
  constexpr int kTuneRounds = 3;
  constexpr float kTuneMargin = 0.01f;
  float cand_ms[kNumTileCandidates + 1];
  bool cand_ok[kNumTileCandidates + 1];
  for (int c = -1; c < kNumTileCandidates; ++c) {
    const int32_t *t = c < 0 ? nullptr : kTileCandidates[c];
    const size_t smem = n_scenes == 1
                            ? plan_for(d, &scenes[0].geom, std::max<long long>(scenes[0].balls.n, 1), 1, t).smem
                            : batched_tiles(scenes, n_scenes, t).smem;
    cand_ok[c + 1] = smem <= (size_t)d->max_smem;
    cand_ms[c + 1] = 3.4e38f;
  }
  auto run_candidate = [&](int c) {
    const int32_t *t = c < 0 ? nullptr : kTileCandidates[c];
    pa_plan trial = *plan;
    std::memset(trial.tiles, 0, sizeof(trial.tiles));
    if (t) std::memcpy(trial.tiles, t, sizeof(trial.tiles));
    if (n_scenes == 1) {
      const pa_scene &sc = scenes[0];
      return forward_impl(&sc.geom, &sc.balls, sc.n_frames, sc.traces, 0, t, workspace, workspace_bytes, stream);
    }
    return pa_forward_batched(scenes, n_scenes, 0, &trial, workspace, workspace_bytes, stream);
  };
  for (int c = -1; c < kNumTileCandidates && rc == PA_OK; ++c)
    if (cand_ok[c + 1]) rc = run_candidate(c);  // untimed first run
  for (int round = 0; round < kTuneRounds && rc == PA_OK; ++round) {
    for (int c = -1; c < kNumTileCandidates && rc == PA_OK; ++c) {
      if (!cand_ok[c + 1]) continue;
      float ms = 0.f;
      rc = time_once([&] { return run_candidate(c); }, st, ms);
      if (rc == PA_OK) cand_ms[c + 1] = std::min(cand_ms[c + 1], ms);
    }
  }
  if (rc) {
    delete plan;
    return rc;
  }
  int best_c = -1;
  float best = cand_ms[0];
  for (int c = 0; c < kNumTileCandidates; ++c) {
    if (!cand_ok[c + 1]) continue;
    ++plan->candidates;
    if (cand_ms[c + 1] < best * (1.f - kTuneMargin) && cand_ms[c + 1] < (best_c < 0 ? best : cand_ms[best_c + 1])) {
      best_c = c;
    }
  }
  if (best_c >= 0) {
    std::memcpy(plan->tiles, kTileCandidates[best_c], sizeof(plan->tiles));
    best = cand_ms[best_c + 1];
  }
  plan->fwd_ms = best;
  // items per queue grab of the batched adjoint, when every scene with work
  // carries its residual and gradient buffers
  bool adj = n_scenes > 1;
  for (int i = 0; i < n_scenes && adj; ++i) {
    const pa_scene &sc = scenes[i];
    if (sc.n_frames > 0 && sc.balls.n > 0 && (sc.trace_grad == nullptr || sc.grad_state == nullptr)) adj = false;
  }
  if (adj) {
    float best_a = 3.4e38f;
    for (int32_t ch : kAdjChunkCandidates) {
      pa_plan trial = *plan;
      trial.adj_chunk = ch;
      float ms = 0.f;
      rc = time_best([&] { return pa_adjoint_batched(scenes, n_scenes, 0, &trial, workspace, workspace_bytes,
                                                     stream); },
                     st, 2, ms);
      if (rc) {
        delete plan;
        return rc;
      }
      ++plan->candidates;
      if (ms < best_a) {
        best_a = ms;
        plan->adj_chunk = ch;
        plan->adj_ms = ms;
      }
    }
  }
  plan->tuned = 1;
  *out = plan;
  return PA_OK;
}

int32_t pa_plan_get(const pa_plan *plan, int32_t *values7, float *timings2) {
  if (plan == nullptr || values7 == nullptr) return PA_ERR_INVALID_ARG;
  std::memcpy(values7, plan->tiles, sizeof(plan->tiles));
  values7[5] = plan->frames_per_chunk;
  values7[6] = plan->adj_chunk;
  if (timings2 != nullptr) {
    timings2[0] = plan->tuned ? plan->fwd_ms : 0.f;
    timings2[1] = plan->tuned ? plan->adj_ms : 0.f;
  }
  return PA_OK;
}

void pa_plan_destroy(pa_plan *plan) { delete plan; }

// ---------------------------------------------------------------------------
// 4D calls that recompute the deformed states per frame chunk.

size_t pa_forward_4d_workspace_size(const pa_geom *geom, const pa_canon *canon, int32_t n_frames,
                                    const pa_plan *plan) {
  if (check_geom(geom) || check_canon(canon) || n_frames <= 0 || canon->n == 0) return 0;
  const int32_t *tiles = plan ? plan->tiles : nullptr;
  if (!tiles_ok(tiles)) return 0;
  const DevInfo *d = dev_info();
  if (!d) return 0;
  const int K = frames_per_chunk(plan, canon->n_basis, n_frames);
  return chunk_state_bytes(canon, K) + forward_4d_partials(d, geom, canon, n_frames, K, tiles);
}

int32_t pa_forward_4d(const pa_geom *geom, const pa_canon *canon, const float *t_frames, int32_t n_frames,
                      float *traces, uint32_t flags, const pa_plan *plan, void *workspace, size_t workspace_bytes,
                      void *stream) {
  int rc = check_geom(geom);
  if (rc) return rc;
  if ((rc = check_canon(canon))) return rc;
  if (n_frames < 0 || (flags & ~PA_ACCUMULATE) != 0) return PA_ERR_INVALID_ARG;
  const int32_t *tiles = plan ? plan->tiles : nullptr;
  if (!tiles_ok(tiles)) return PA_ERR_INVALID_ARG;
  if (n_frames == 0) return PA_OK;
  if (traces == nullptr || !aligned(traces, 16) || t_frames == nullptr) return PA_ERR_INVALID_ARG;
  if (canon->n > 0 && !aligned(canon->canon, 16)) return PA_ERR_INVALID_ARG;
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t per_frame = (size_t)geom->n_sensors * geom->n_samples;
  if (canon->n == 0) {
    if (flags & PA_ACCUMULATE) return PA_OK;
    return cuda_status(cudaMemsetAsync(traces, 0, sizeof(float) * per_frame * n_frames, st));
  }
  const int K = frames_per_chunk(plan, canon->n_basis, n_frames);
  const size_t sbytes = chunk_state_bytes(canon, K);
  const size_t need = sbytes + forward_4d_partials(d, geom, canon, n_frames, K, tiles);
  if (workspace == nullptr || workspace_bytes < need || !aligned(workspace, 256)) return PA_ERR_WORKSPACE;
  float *states = static_cast<float *>(workspace);
  char *partials = static_cast<char *>(workspace) + sbytes;
  for (int f0 = 0; f0 < n_frames; f0 += K) {
    const int k = std::min(K, n_frames - f0);
    rc = cuda_status(pa::launch_deform(canon->canon, canon->omega, canon->theta, canon->sigma, canon->n,
                                       canon->stride, canon->n_basis, t_frames + f0, k, states, d->err, st));
    if (rc) return rc;
    rc = forward_launch(d, geom, states, canon->n, canon->stride, k, traces + per_frame * f0, flags, tiles,
                        partials, workspace_bytes - sbytes, st);
    if (rc) return rc;
  }
  return PA_OK;
}

size_t pa_adjoint_4d_workspace_size(const pa_geom *geom, const pa_canon *canon, int32_t n_frames,
                                    const pa_plan *plan) {
  if (check_geom(geom) || check_canon(canon) || n_frames <= 0 || canon->n == 0) return 0;
  const int K = frames_per_chunk(plan, canon->n_basis, n_frames);
  return kQueueBytes + 2 * chunk_state_bytes(canon, K);
}

int32_t pa_adjoint_4d(const pa_geom *geom, const pa_canon *canon, const float *t_frames, int32_t n_frames,
                      const float *trace_grad, const float *frame_scale, pa_grads *grads, uint32_t flags,
                      const pa_plan *plan, void *workspace, size_t workspace_bytes, void *stream) {
  int rc = check_geom(geom);
  if (rc) return rc;
  if ((rc = check_canon(canon))) return rc;
  if (n_frames < 0 || grads == nullptr || (flags & ~PA_ACCUMULATE) != 0) return PA_ERR_INVALID_ARG;
  if (canon->n == 0) return PA_OK;
  if (!grads->state || !grads->omega || !grads->theta || !grads->sigma) return PA_ERR_INVALID_ARG;
  if (n_frames > 0 && (t_frames == nullptr || trace_grad == nullptr || !aligned(trace_grad, 16)))
    return PA_ERR_INVALID_ARG;
  const size_t smem = pa::adj_static_smem(geom->n_sensors);
  const DevInfo *d = dev_info();
  if (!d) return PA_ERR_CUDA;
  if ((long long)smem > d->max_smem) return PA_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n_frames == 0) {
    if (flags & PA_ACCUMULATE) return PA_OK;
    const size_t rows = sizeof(float) * (size_t)canon->stride;
    cudaError_t e = cudaMemsetAsync(grads->state, 0, rows * 5, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(grads->omega, 0, rows * 5 * canon->n_basis, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(grads->theta, 0, rows * 5 * canon->n_basis, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(grads->sigma, 0, rows * 5 * canon->n_basis, st);
    return cuda_status(e);
  }
  const int K = frames_per_chunk(plan, canon->n_basis, n_frames);
  const size_t sbytes = chunk_state_bytes(canon, K);
  if (workspace == nullptr || workspace_bytes < kQueueBytes + 2 * sbytes || !aligned(workspace, 256))
    return PA_ERR_WORKSPACE;
  auto *queue = static_cast<unsigned long long *>(workspace);
  float *states = reinterpret_cast<float *>(static_cast<char *>(workspace) + kQueueBytes);
  float *gstates = reinterpret_cast<float *>(static_cast<char *>(workspace) + kQueueBytes + sbytes);
  const size_t per_frame = (size_t)geom->n_sensors * geom->n_samples;
  for (int f0 = 0; f0 < n_frames; f0 += K) {
    const int k = std::min(K, n_frames - f0);
    rc = cuda_status(pa::launch_deform(canon->canon, canon->omega, canon->theta, canon->sigma, canon->n,
                                       canon->stride, canon->n_basis, t_frames + f0, k, states, d->err, st));
    if (rc) return rc;
    pa::AdjArgs a;
    std::memset(&a, 0, sizeof(a));
    a.q = make_acq(geom);
    a.state = states;
    a.stride = canon->stride;
    a.n = canon->n;
    a.F = k;
    a.g = trace_grad + per_frame * f0;
    a.frame_scale = frame_scale ? frame_scale + f0 : nullptr;
    a.g_state = gstates;
    a.flags = 0;
    a.err = d->err;
    a.n_items = (long long)k * canon->n;
    a.queue = queue;
    rc = cuda_status(pa::launch_adjoint_static(a, d->sms, st));
    if (rc) return rc;
    rc = cuda_status(pa::launch_deform_backward(canon->canon, canon->omega, canon->theta, canon->sigma, canon->n,
                                                canon->stride, canon->n_basis, t_frames + f0, k, gstates,
                                                grads->state, grads->omega, grads->theta, grads->sigma,
                                                f0 > 0 || (flags & PA_ACCUMULATE) != 0, d->err, st));
    if (rc) return rc;
  }
  return PA_OK;
}

}  // extern "C"
