// gs_render_fwd_static: the forward render for callers that cannot allocate
// device memory.  The workspace lives in a file-scope device array instead of
// a caller-provided buffer; everything else is the ordinary
// gs_preprocess -> gs_bin -> gs_render_fwd sequence.
#include <mutex>

#include "gs_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)GS_STATIC_SCRATCH_BYTES;

// Held by every GPU that loads the library, until the process exits.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device ordinal, looked up once per device.
constexpr int kMaxDevices = 64;
void* g_addr[kMaxDevices] = {};
std::mutex g_addr_mutex;

gs_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    return gs::set_error(GS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  if (dev < 0 || dev >= kMaxDevices) {
    return gs::set_error(GS_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
  }
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);   // with device `dev` current
    if (e != cudaSuccess || !p) {
      return gs::set_error(GS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s",
                           cudaGetErrorString(e));
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return GS_OK;
}

}  // namespace

extern "C" gs_status gs_render_fwd_static(const gs_frame* frame, const gs_maps* maps, gs_stats* stats,
                                          void* stream) {
  if (!frame || !maps) {
    return gs::set_error(GS_ERR_INVALID_ARG, "frame and maps must not be NULL");
  }
  gs_frame f = *frame;
  f.workspace = nullptr;
  f.workspace_bytes = 0;
  const size_t need = gs_workspace_size(&f);
  if (need == 0) return GS_ERR_INVALID_ARG;   // the error string says why
  if (need > kScratchBytes) {
    return gs::set_error(GS_ERR_INVALID_ARG,
                         "frame needs %zu bytes of workspace; the static scratch holds %zu (use "
                         "gs_preprocess with a caller-provided workspace, or fewer Gaussians, pixels "
                         "or pairs)",
                         need, kScratchBytes);
  }
  void* ws = nullptr;
  gs_status st = scratch_address(&ws);
  if (st != GS_OK) return st;
  f.workspace = ws;
  f.workspace_bytes = kScratchBytes;
  // gs_preprocess re-initialises the counters and status word; binning clears
  // the tile ranges; nothing else is read before it is written in this call.
  if ((st = gs_preprocess(&f, stream)) != GS_OK) return st;
  if ((st = gs_bin(&f, stream)) != GS_OK) return st;
  if ((st = gs_render_fwd(&f, maps, stream)) != GS_OK) return st;
  if (stats) return gs_check(&f, stats, stream);
  return GS_OK;
}
