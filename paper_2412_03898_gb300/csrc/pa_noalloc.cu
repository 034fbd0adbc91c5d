// pa_residual_loss_noalloc: the per-frame FP64 loss / residual without a
// caller-provided workspace.
//
// Some callers of this library cannot allocate device memory at the point of
// the call: a plugin inside a host application that owns every device
// allocation (a fixed memory pool handed out by the host), or a C caller with
// no allocator at hand that must not call cudaMalloc, which can implicitly
// synchronise the device and stall work already queued on other streams.
// pa_residual_loss needs scratch for its per-block FP64 partial sums; this
// entry point keeps that scratch in a fixed device array of this library
// instead, so such callers only pass their inputs and outputs.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its 128 KiB until the process exits.  Host code cannot pass
// the array's name to a kernel (on the host it is only a stand-in symbol), so
// the first call on each device looks up the array's device address with
// cudaGetSymbolAddress, with that device current, and caches it per device
// index for the life of the process.  That first call on a device should
// therefore come before any stream capture.  The cached address belongs to
// the device's primary context: after cudaDeviceReset, or from another
// (non-primary) context on the same device, it is stale, and such callers
// must not use this entry point.
//
// Every call shares the one array and reuses it without clearing it: each
// call's first kernel writes every partial its second kernel reads, so
// nothing needs to start at zero.  Calls that overlap on the GPU (on two
// streams, or from two threads) race on the array and must be serialised by
// the caller.
#include <mutex>

#include "pa_internal.h"

namespace {

// Capacity of the fixed scratch: one double per (frame, block) partial.
constexpr int kNoAllocPartials = 16384;

static __device__ __align__(256) double g_loss_partials[kNoAllocPartials];

constexpr int kMaxDevices = 64;
double *g_partials_ptr[kMaxDevices] = {};
std::mutex g_partials_mu;

// Device address of g_loss_partials on the current device (NULL on failure).
double *partials_on_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_partials_mu);
  if (g_partials_ptr[dev] == nullptr) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_loss_partials) != cudaSuccess) return nullptr;
    g_partials_ptr[dev] = static_cast<double *>(p);
  }
  return g_partials_ptr[dev];
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

extern "C" {

int32_t pa_residual_loss_noalloc(const float *pred, const float *meas, int64_t per_frame, int32_t n_frames,
                                 const float *frame_scale, double *loss, float *resid, void *stream) {
  if (per_frame < 4 || (per_frame & 3) != 0 || n_frames < 0) return PA_ERR_INVALID_ARG;
  if (n_frames == 0) return PA_OK;
  if (!pred || !meas || !aligned16(pred) || !aligned16(meas)) return PA_ERR_INVALID_ARG;
  if (resid && !aligned16(resid)) return PA_ERR_INVALID_ARG;
  if (!loss && !resid) return PA_ERR_INVALID_ARG;
  const int bpf = pa::loss_blocks_per_frame(per_frame);
  if ((long long)n_frames * bpf > kNoAllocPartials) return PA_ERR_WORKSPACE;
  double *partials = partials_on_current_device();
  if (partials == nullptr) return PA_ERR_CUDA;
  const cudaError_t e = pa::launch_loss(pred, meas, per_frame, n_frames, frame_scale, loss, resid, partials, bpf,
                                        static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

}  // extern "C"
