// fv_noalloc.cu -- exact decoding for callers that cannot allocate device
// memory.
//
// Some callers of this library cannot call cudaMalloc (or any allocating
// routine) at decode time: code running inside a strict memory budget that
// was fixed at start-up, plug-in hosts that own the device allocator and
// forbid their plug-ins from using it, or real-time paths where an
// allocation may block on a device-wide synchronisation.  fv_decode_noalloc
// serves them: it runs the same exact decoder as fv_decode, but its scratch
// memory (job table, longest-first order, backpointer table) lives in a
// file-scope device array of FV_NOALLOC_SCRATCH_BYTES that the CUDA runtime
// creates when the library's module is loaded on a device.  Nothing is
// allocated per call; the caller still provides inputs and outputs.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fv.h"

namespace {

constexpr size_t kScratchBytes = FV_NOALLOC_SCRATCH_BYTES;

// The scratch itself.  Every GPU that loads libfv holds these bytes until
// the process exits.  In host code `g_scratch` is only a host-side stand-in
// for the symbol, never a device address: the address is obtained with
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_scratch on the current device, looked up once per
// device (with that device current) and cached.  The cache is keyed by the
// device ordinal, so it belongs to the device's primary context (the one the
// CUDA runtime uses) and does not survive cudaDeviceReset.
fv_status scratch_on_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FV_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return FV_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return FV_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FV_OK;
}

}  // namespace

extern "C" fv_status fv_decode_noalloc(const fv_model* models, int32_t n_models, const fv_batch* batch,
                                       int32_t* paths_out, float* scores_out, fv_stream_t stream) {
  // Host lengths are required so the size check happens here, before
  // anything is enqueued.
  if (!batch || !batch->T_host || !models || n_models < 1) return FV_EINVAL;
  // Dense transitions only: a CSR model would be decoded by the full-width
  // beam, whose scratch this entry point does not promise to cover.
  for (int32_t m = 0; m < n_models; ++m)
    if (models[m].trans != FV_TRANS_DENSE) return FV_EUNSUPPORTED;
  fv_params p;
  p.mode = FV_VANILLA;
  p.P = 1;
  p.B = 0;
  p.mem_budget_bytes = 0;
  p.flags = 0;
  const size_t need = fv_workspace_size(models, n_models, batch, &p);
  if (need == 0) return FV_EINVAL;
  if (need > kScratchBytes) return FV_ENOMEM;  // request larger than the static scratch
  void* ws = nullptr;
  const fv_status s = scratch_on_current_device(&ws);
  if (s != FV_OK) return s;
  // The decoder resets every scratch field it reads (status word, work
  // counters, job table) in its first kernel, so the previous call's
  // contents need no clearing here.
  return fv_decode(models, n_models, batch, &p, ws, kScratchBytes, paths_out, scores_out, stream);
}

extern "C" fv_status fv_decode_noalloc_status(fv_stream_t stream) {
  // The status word sits at the start of the scratch (the workspace header),
  // so the ordinary reader applies once the scratch's address is known.
  void* ws = nullptr;
  const fv_status s = scratch_on_current_device(&ws);
  if (s != FV_OK) return s;
  return fv_last_device_status(ws, stream);
}
