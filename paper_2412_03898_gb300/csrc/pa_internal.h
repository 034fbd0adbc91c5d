// Internal (host-side) interface between the C-ABI layer (pa_api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include "pa_common.cuh"

namespace pa {

// Tile plan of one pa_forward call.
struct FwdPlan {
  int s_tile;      // sensors per CTA (one warp each)
  int t_tile;      // samples per CTA
  int nb_tile;     // balls per TMA stage
  int n_splits;    // ball-range splits (partial traces summed by a second kernel)
  int group;       // pairs swept together per warp (1, 2, 4 or 8)
  int n_stiles, n_ttiles;
  long long balls_per_split;
  size_t smem;     // dynamic shared memory per CTA
  size_t ws_bytes; // workspace for split partials
};

struct FwdArgs {
  Acq q;
  const float *state;
  long long n, stride;
  int F;
  float *out;
  float *partial;
  int s_tile, t_tile, nb_tile, n_splits, n_stiles, n_ttiles;
  long long balls_per_split;
  unsigned flags;
  unsigned *err;
};

// Default plans split larger ball sets: a smaller ball range has a tighter
// bounding box, hence a narrower arrival band at every sensor.  Single-scene
// plans take at least one split per kMaxBallsPerSplit balls (one frame of 1e6
// balls in a 60 mm phantom at 1024 sensors: 8 splits 41.8 ms, 16 splits
// 38.3 ms, 32 splits 36.3 ms; 1e5 balls: unchanged at 4 or 16 splits); the
// batched forward, whose partials of all scenes share one workspace, one per
// kMaxBallsPerBatchedSplit (finer batched splits gave nothing on 16 uneven
// scenes: 310 against 309 ms).
constexpr long long kMaxBallsPerSplit = 32768;
constexpr long long kMaxBallsPerBatchedSplit = 131072;

// Batched (several scenes, one persistent launch).
constexpr int kMaxScenes = 64;

struct SceneFwd {
  Acq q;
  const float *state;
  long long n, stride;
  int F;
  float *out;
  float *partial;              // [n_splits][F][S][T] when n_splits > 1
  int n_stiles, n_ttiles, n_splits;
  long long balls_per_split;
  long long item_begin;  // first work item of this scene
};

struct BatchFwdArgs {
  int n_scenes;
  int s_tile, t_tile, nb_tile;
  long long total_items;
  unsigned long long *counter;  // work-queue counter, zero at launch
  unsigned flags;
  unsigned *err;
  SceneFwd sc[kMaxScenes];
};

struct SceneAdj {
  Acq q;
  const float *state;
  long long n, stride;
  int F;
  const float *g;
  float *g_state;
  long long item_begin;  // first (frame, ball) item of this scene
};

struct BatchAdjArgs {
  int n_scenes;
  int chunk;  // (scene, frame, ball) items per queue grab, >= 1
  long long total_items;
  unsigned long long *counter;
  unsigned flags;
  unsigned *err;
  SceneAdj sc[kMaxScenes];
};

struct AdjArgs {
  Acq q;
  // static mode
  const float *state;
  // 4D mode
  const float *canon, *omega, *theta, *sigma;
  int nb;
  const float *t_frames;
  long long n, stride;
  int F;
  const float *g;
  const float *frame_scale;
  float *g_state, *g_omega, *g_theta, *g_sigma;
  unsigned flags;
  unsigned *err;
  long long n_items;
  unsigned long long *queue;  // static mode: work-queue counter in a workspace, or nullptr (grid-stride loop)
  int queue_chunk;            // items per grab (set by the launcher)
};

// Plan selection (tile sizes, splits); `override` entries > 0 replace the
// heuristic (used by the autotuner).
FwdPlan forward_plan(int S, int T, long long n, int F, int sms, int s_tile_override,
                     int t_tile_override, int nb_tile_override, int splits_override, int group_override);
size_t forward_smem_bytes(int s_tile, int t_tile, int nb_tile);
// Most sensors per CTA (<= 16) whose compensated trace tiles fit in 227 KB.
// default samples per forward CTA (16 sensors x 1536 samples fill 227 KB)
constexpr int kDefaultTTile = 1536;
int forward_default_s_tile(int t_tile, int nb_tile);
int forward_blocks_per_sm(const FwdPlan &p, bool uniform);

cudaError_t launch_forward(const FwdArgs &a, const FwdPlan &p, bool uniform, cudaStream_t st);
cudaError_t launch_forward_batched(const BatchFwdArgs &a, int group, size_t smem, int sms, cudaStream_t st);
cudaError_t launch_adjoint_batched(const BatchAdjArgs &a, int sms, cudaStream_t st);
cudaError_t launch_count(const Acq &q, const float *state, long long n, long long stride, int F,
                         unsigned long long *out, cudaStream_t st);
// Dynamic shared memory of the static and 4D adjoint kernels (sensor
// coordinates; 4D adds per-warp frame-gradient buffers).
size_t adj_static_smem(int S);
size_t adj_4d_smem(int S);
cudaError_t launch_adjoint_static(const AdjArgs &a, int sms, cudaStream_t st);
// Spatial (Morton) order of a cloud and the row gather that applies it.
size_t spatial_order_workspace(long long n);
cudaError_t launch_spatial_order(const float *state, long long stride, long long n, int *perm, void *ws, int sms,
                                 cudaStream_t st);
cudaError_t launch_gather_rows(const float *in, float *out, long long n, long long stride, int rows,
                               const int *perm, int sms, cudaStream_t st);
cudaError_t launch_adjoint_4d(const AdjArgs &a, int sms, cudaStream_t st);
// Imaging kernels (pa_image.cu).
struct UbpArgs {
  const float *b;        // filtered traces [S][T]
  const float *sensors;  // [3][sstride]
  int S, sstride, T;
  float cx, cy, cz;      // array centre (the sensors' inward normals point at it)
  float fs_c;            // fs / c: samples per mm
  float t0_fs;           // t0 * fs
  float ox, oy, oz, h;   // grid origin and spacing
  int nx, ny, nz;
  float *vol;            // [nz][ny][nx]
};

struct SplatArgs {
  const float *state;  // [5][stride]
  long long n, stride;
  float kappa;
  float ox, oy, oz, h;
  int nx, ny, nz;
  float *vol;
};

struct SsimArgs {
  const float *x, *y;  // [H][W]
  int H, W;
  float C1, C2;
  float g[11];         // normalised 1D Gaussian window (sigma 1.5)
  float *map;          // [(H-10)][(W-10)] or nullptr
  double *partials;    // one per CTA
  const float4 *norm;  // (x offset, x scale, y offset, y scale) applied on load, or nullptr
};

cudaError_t launch_ubp_filter(const float *p, long long n_traces, int T, float fs, float t0, float *b,
                              cudaStream_t st);
cudaError_t launch_ubp(const UbpArgs &a, cudaStream_t st);
cudaError_t launch_splat(const SplatArgs &a, cudaStream_t st);
cudaError_t launch_map(const float *v, int nx, int ny, int nz, float *xy, float *yz, float *xz, cudaStream_t st);
int ssim_blocks(int H, int W);
int minmax_partials();
cudaError_t launch_ssim(const SsimArgs &a, double *out, float4 *minmax_ws, cudaStream_t st);

cudaError_t launch_selftest_wait(unsigned long long limit_ns, unsigned *err, cudaStream_t st);
// Unit-throughput probe (pa_probe.cu): out = {FFMA, FFMA2 lane ops, ex2} per SM
// per clock and the SM clock in MHz; synchronises st.
cudaError_t measure_unit_rates(int sms, cudaStream_t st, double out[4]);
cudaError_t launch_deform_backward(const float *canon, const float *omega, const float *theta, const float *sigma,
                                   long long n, long long stride, int nb, const float *t, int F, const float *gstate,
                                   float *g_canon, float *g_omega, float *g_theta, float *g_sigma, bool acc,
                                   unsigned *err, cudaStream_t st);
cudaError_t launch_deform(const float *canon, const float *omega, const float *theta,
                          const float *sigma, long long n, long long stride, int nb,
                          const float *t, int F, float *out, unsigned *err, cudaStream_t st);
cudaError_t launch_loss(const float *pred, const float *meas, long long per_frame, int F,
                        const float *scale, double *loss, float *resid, double *partials,
                        int blocks_per_frame, cudaStream_t st);
int loss_blocks_per_frame(long long per_frame);
cudaError_t launch_adam_sched(float *x, const float *g, float *m, float *v, long long n, float lr0, float b1,
                              float b2, float omb1, float omb2, float eps, int step_size, float gamma,
                              const int *step, cudaStream_t st);
cudaError_t launch_step_increment(int *step, cudaStream_t st);
cudaError_t launch_adam(float *x, const float *g, float *m, float *v, long long n, float lr, float b1,
                        float b2, float omb1, float omb2, float eps, float bc1, float bc2, cudaStream_t st);

}  // namespace pa
