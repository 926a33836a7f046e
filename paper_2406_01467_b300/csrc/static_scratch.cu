// gs_render_fwd_static: the forward render for callers that cannot allocate
// device memory.  The workspace lives in a file-scope device array instead of
// a caller-provided buffer; everything else is the ordinary
// gs_preprocess -> gs_bin -> gs_render_fwd sequence.
#include <cuda.h>   // driver types only (CUcontext, CUresult)

#include <mutex>

#include "gs_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)GS_STATIC_SCRATCH_BYTES;

// Held by every GPU that loads the library, until the process exits.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device ordinal, looked up with that device
// current the first time a call runs on it, and again whenever the device's
// context has changed since (a cudaDeviceReset, or a primary context released
// and re-created, reloads the module and may move the array).  The context is
// identified by the driver's context id, queried through entry points the
// runtime hands out (no link-time dependency on the driver library).
constexpr int kMaxDevices = 64;
struct ScratchAddr {
  void* ptr;
  unsigned long long ctx_id;
};
ScratchAddr g_addr[kMaxDevices] = {};
std::mutex g_addr_mutex;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Id of the calling thread's current context (0 if it cannot be read, which
// makes every call look the address up again).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(fn);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

gs_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    return gs::set_error(GS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  if (dev < 0 || dev >= kMaxDevices) {
    return gs::set_error(GS_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
  }
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev].ptr || ctx == 0 || g_addr[dev].ctx_id != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);   // with device `dev` current
    if (e != cudaSuccess || !p) {
      return gs::set_error(GS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s",
                           cudaGetErrorString(e));
    }
    g_addr[dev] = ScratchAddr{p, ctx};
  }
  *out = g_addr[dev].ptr;
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
  size_t need = 0;
  gs_status st = gs::frame_workspace_size(&f, &need);
  if (st != GS_OK) return st;   // the error string says why
  if (need > kScratchBytes) {
    return gs::set_error(GS_ERR_INVALID_ARG,
                         "frame needs %zu bytes of workspace; the static scratch holds %zu (use "
                         "gs_preprocess with a caller-provided workspace, or fewer Gaussians, pixels "
                         "or pairs)",
                         need, kScratchBytes);
  }
  void* ws = nullptr;
  st = scratch_address(&ws);
  if (st != GS_OK) return st;
  f.workspace = ws;
  f.workspace_bytes = kScratchBytes;
  // gs_preprocess re-initialises the counters and status word; binning clears
  // the tile ranges; nothing else is read before it is written in this call.
  if ((st = gs_preprocess(&f, stream)) != GS_OK) return st;
  if ((st = gs_bin(&f, stream)) != GS_OK) return st;
  if ((st = gs_render_fwd(&f, maps, stream)) != GS_OK) return st;
  if (stats) {
    st = gs_check(&f, stats, stream);
    stats->n_evals_bwd = 0;   // this call runs no backward
    return st;
  }
  return GS_OK;
}
