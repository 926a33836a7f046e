// extern "C" entry points of libgs: argument validation, workspace layout and
// the launch sequence of each stage.  See include/gs.h for the contract.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>

#include "gs_internal.cuh"
#include <cstddef>
#include <nvtx3/nvToolsExt.h>

namespace gs {

static thread_local char g_err[512] = "no error";

static gs_status fail(gs_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

gs_status set_error(gs_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

static gs_status cuda_fail(cudaError_t e, const char* where) {
  return fail(GS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

static int log2_exact(int x) {
  int s = 0;
  while ((1 << s) < x) ++s;
  return (1 << s) == x ? s : -1;
}

static size_t round_up(size_t x) { return (x + 255) & ~size_t(255); }

// Validates the frame and fills the device descriptor and the layout.
static gs_status prepare(const gs_frame* f, FrameDev& fd, Layout& L) {
  if (!f) return fail(GS_ERR_INVALID_ARG, "frame is NULL");
  if (!f->scenes || f->n_scenes < 1 || f->n_scenes > GS_MAX_SCENES)
    return fail(GS_ERR_INVALID_ARG, "n_scenes must be in [1, %d] with a scene array", GS_MAX_SCENES);
  if (!f->views || f->n_views < 1 || f->n_views > GS_MAX_VIEWS)
    return fail(GS_ERR_INVALID_ARG, "n_views must be in [1, %d] with a view array", GS_MAX_VIEWS);
  const gs_params& p = f->params;
  const int sx = log2_exact(p.tile_w), sy = log2_exact(p.tile_h);
  const int block = p.tile_w * p.tile_h;
  if (sx < 0 || sy < 0 || p.tile_w < 8 || p.tile_h < 4 || !(block == 64 || block == 128 || block == 256))
    return fail(GS_ERR_INVALID_ARG,
                "tile %dx%d: sides must be powers of two, width >= 8, height >= 4, 64, 128 or 256 pixels",
                p.tile_w, p.tile_h);
  if (!(p.lowpass >= 0.f) || !std::isfinite(p.lowpass))
    return fail(GS_ERR_INVALID_ARG, "lowpass must be finite and >= 0");
  if (!(p.alpha_min > 0.f && p.alpha_min < 1.f))
    return fail(GS_ERR_INVALID_ARG, "alpha_min must be in (0, 1)");
  if (!(p.alpha_max >= p.alpha_min && p.alpha_max < 1.f))
    return fail(GS_ERR_INVALID_ARG, "alpha_max must be in [alpha_min, 1)");
  if (!(p.T_min >= 0.f && p.T_min < 1.f)) return fail(GS_ERR_INVALID_ARG, "T_min must be in [0, 1)");
  if (!(p.median_T > 0.f && p.median_T < 1.f))
    return fail(GS_ERR_INVALID_ARG, "median_T must be in (0, 1)");
  if (!(p.clamp_margin >= 0.f) || !std::isfinite(p.clamp_margin))
    return fail(GS_ERR_INVALID_ARG, "clamp_margin must be finite and >= 0");
  if (p.losses != 0 && p.losses != 1) return fail(GS_ERR_INVALID_ARG, "losses must be 0 or 1");
  if (p.geometry_only != 0 && p.geometry_only != 1)
    return fail(GS_ERR_INVALID_ARG, "geometry_only must be 0 or 1");
  if (p.geometry_only && p.losses)
    return fail(GS_ERR_INVALID_ARG, "geometry_only excludes losses (no backward state)");
  if (p.batch != 0 && p.batch != 32 && p.batch != 64)
    return fail(GS_ERR_INVALID_ARG, "batch must be 0 (32), 32 or 64");
  if (f->pair_capacity < 1 || f->pair_capacity > (int64_t(1) << 31) - 1)
    return fail(GS_ERR_INVALID_ARG, "pair_capacity must be in [1, 2^31 - 1]");

  memset(&fd, 0, sizeof(fd));
  fd.n_views = f->n_views;
  fd.n_scenes = f->n_scenes;
  for (int i = 0; i < f->n_scenes; ++i) {
    const gs_scene& s = f->scenes[i];
    if (s.n < 0) return fail(GS_ERR_INVALID_ARG, "scene %d: n < 0", i);
    if (s.sh_degree < 0 || s.sh_degree > 3) return fail(GS_ERR_INVALID_ARG, "scene %d: sh_degree not in 0..3", i);
    if (s.dtype != GS_F32 && s.dtype != GS_BF16) return fail(GS_ERR_INVALID_ARG, "scene %d: bad dtype", i);
    if (s.n > 0 && (!s.means || !s.scales || !s.quats || !s.opacities || !s.sh))
      return fail(GS_ERR_INVALID_ARG, "scene %d: NULL parameter array", i);
    SceneDev& d = fd.scenes[i];
    d.means = s.means; d.scales = s.scales; d.quats = s.quats; d.opacities = s.opacities; d.sh = s.sh;
    d.filter_var = static_cast<const float*>(s.filter_var);
    d.n = s.n; d.sh_degree = s.sh_degree; d.dtype = s.dtype;
  }
  int64_t E = 0, NPIX = 0;
  int64_t T = 0, NCH = 0;
  for (int v = 0; v < f->n_views; ++v) {
    const gs_view& cv = f->views[v];
    if (cv.scene < 0 || cv.scene >= f->n_scenes) return fail(GS_ERR_INVALID_ARG, "view %d: bad scene index", v);
    if (cv.width < 1 || cv.height < 1 || cv.width > 16384 || cv.height > 16384)
      return fail(GS_ERR_INVALID_ARG, "view %d: image size must be in [1, 16384]", v);
    if (!(cv.fx > 0.f) || !(cv.fy > 0.f) || !std::isfinite(cv.fx) || !std::isfinite(cv.fy) ||
        !std::isfinite(cv.cx) || !std::isfinite(cv.cy))
      return fail(GS_ERR_INVALID_ARG, "view %d: intrinsics must be finite with fx, fy > 0", v);
    if (!(cv.near_plane > 0.f) || !std::isfinite(cv.near_plane))
      return fail(GS_ERR_INVALID_ARG, "view %d: near_plane must be finite and > 0", v);
    for (int k = 0; k < 16; ++k)
      if (!std::isfinite(cv.viewmat[k])) return fail(GS_ERR_INVALID_ARG, "view %d: non-finite viewmat", v);
    ViewDev& V = fd.views[v];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) V.R[3 * r + c] = cv.viewmat[4 * r + c];
      V.t[r] = cv.viewmat[4 * r + 3];
    }
    V.fx = cv.fx; V.fy = cv.fy; V.cx = cv.cx; V.cy = cv.cy;
    // bounds of x/z and y/z inside J: the image widened by clamp_margin on each side
    const double fx = cv.fx, fy = cv.fy, cx = cv.cx, cy = cv.cy, m = p.clamp_margin;
    const double mw = m * cv.width, mh = m * cv.height;
    V.lim[0] = (float)(-(cx + mw) / fx);
    V.lim[1] = (float)((cv.width + mw - cx) / fx);
    V.lim[2] = (float)(-(cy + mh) / fy);
    V.lim[3] = (float)((cv.height + mh - cy) / fy);
    for (int k = 0; k < 3; ++k)
      V.campos[k] = (float)(-((double)V.R[k] * V.t[0] + (double)V.R[3 + k] * V.t[1] + (double)V.R[6 + k] * V.t[2]));
    V.near_plane = cv.near_plane;
    V.width = cv.width; V.height = cv.height;
    V.tiles_x = (cv.width + p.tile_w - 1) / p.tile_w;
    V.tiles_y = (cv.height + p.tile_h - 1) / p.tile_h;
    V.scene = cv.scene;
    fd.scenes[cv.scene].n_views += 1;
    fd.entry_off[v] = E;
    fd.pix_off[v] = NPIX;
    fd.tile_off[v] = (int32_t)T;
    fd.chunk_off[v] = (int32_t)NCH;
    NCH += (f->scenes[cv.scene].n + 127) / 128;
    E += f->scenes[cv.scene].n;
    NPIX += (int64_t)cv.width * cv.height;
    T += (int64_t)V.tiles_x * V.tiles_y;
  }
  fd.entry_off[f->n_views] = E;
  fd.pix_off[f->n_views] = NPIX;
  fd.tile_off[f->n_views] = (int32_t)T;
  fd.chunk_off[f->n_views] = (int32_t)NCH;
  fd.n_chunks = (int32_t)NCH;
  if (E >= (int64_t(1) << 31)) return fail(GS_ERR_INVALID_ARG, "too many (view, Gaussian) entries: %lld", (long long)E);
  if (T >= (int64_t(1) << 31)) return fail(GS_ERR_INVALID_ARG, "too many tiles");
  fd.n_entries = E;
  fd.n_pixels = NPIX;
  fd.n_tiles = (int32_t)T;
  fd.pair_capacity = f->pair_capacity;
  fd.tile_w = p.tile_w; fd.tile_h = p.tile_h;
  fd.tile_shift_x = sx; fd.tile_shift_y = sy;
  fd.lowpass = p.lowpass; fd.alpha_min = p.alpha_min; fd.alpha_max = p.alpha_max;
  fd.T_min = p.T_min; fd.median_T = p.median_T;
  fd.ext_c = (float)(2.0 * std::log(1.0 / (double)p.alpha_min));
  fd.losses = p.losses;
  fd.geometry_only = p.geometry_only;
  fd.batch = p.batch == 0 ? 32 : p.batch;

  // ---- workspace layout ----
  memset(&L, 0, sizeof(L));
  L.E = E; L.T = T; L.NPIX = NPIX; L.Pcap = f->pair_capacity;
  L.nb_E = (int32_t)std::max<int64_t>(1, (E + kSortTile - 1) / kSortTile);
  L.nb_P = (int32_t)std::max<int64_t>(1, (L.Pcap + kSortTile - 1) / kSortTile);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += round_up(bytes); return o; };
  L.hdr = take(sizeof(Header));
  L.frame = take(sizeof(FrameDev));
  L.rec = take(64 * (size_t)E);
  L.rect = take(8 * (size_t)E);
  L.key = take(4 * (size_t)E);
  L.touched = take(4 * (size_t)E);
  for (int i = 0; i < 2; ++i) { L.vkey[i] = take(4 * (size_t)E); L.vval[i] = take(4 * (size_t)E); }
  L.pair_off = take(4 * (size_t)E);
  L.chunk_first = take(4 * (size_t)((L.Pcap + kEmitChunk - 1) / kEmitChunk + 1));
  for (int i = 0; i < 2; ++i) { L.ptile[i] = take(4 * (size_t)L.Pcap); L.pval[i] = take(4 * (size_t)L.Pcap); }
  const int passes = (tile_sort_bits(T) + kRadixBits - 1) / kRadixBits;
  L.ptile_final = L.ptile[passes & 1];
  L.pval_final = L.pval[passes & 1];
  // histograms + tickets, then the look-back words of the 4 depth passes or of the tile passes
  L.sortaux_bytes[0] = 8192 + (size_t)4 * L.nb_E * kRadix * 8;
  L.sortaux_bytes[1] = 8192 + (size_t)passes * L.nb_P * kRadix * 8;
  L.sortaux[0] = take(L.sortaux_bytes[0]);   // these four regions are contiguous:
  L.sortaux[1] = take(L.sortaux_bytes[1]);   // binning clears them with one memset
  L.scanaux = take(64 + 2 * 8 * (size_t)L.nb_E);
  L.ranges = take(8 * (size_t)T);
  L.tile_order = take(4 * (size_t)T);
  const bool bwd_state = !p.geometry_only;   // per-pixel replay state and 2D gradients
  L.px_T = take(bwd_state ? 4 * (size_t)NPIX : 0);
  L.px_last = take(bwd_state ? 4 * (size_t)NPIX : 0);
  L.px_med = take(bwd_state ? 4 * (size_t)NPIX : 0);
  L.bwdcnt = take(bwd_state ? 256 : 0);
  L.grad2d = take(bwd_state ? 64 * (size_t)E : 0);
  L.px_loss = take(p.losses ? 4 * (size_t)kLossPlanes * NPIX : 0);
  // chunk k of tile t's list, 8x4 block b: word b * cmask_words + (start_t >> 5) + t + k;
  // distinct for all (t, k) because floor(a/32) + floor(l/32) <= floor((a+l)/32)
  L.cmask_words = (L.Pcap >> 5) + T + 2;
  L.cmask = take(bwd_state ? 4 * (size_t)(p.tile_w * p.tile_h / 32) * (size_t)L.cmask_words : 0);
  L.total = off;
  return GS_OK;
}

static gs_status prepare_ws(const gs_frame* f, FrameDev& fd, Layout& L) {
  gs_status st = prepare(f, fd, L);
  if (st != GS_OK) return st;
  if (!f->workspace) return fail(GS_ERR_INVALID_ARG, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(f->workspace) % 256 != 0)
    return fail(GS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (f->workspace_bytes < L.total)
    return fail(GS_ERR_INVALID_ARG, "workspace has %zu bytes, %zu needed", f->workspace_bytes, L.total);
  return GS_OK;
}

// Copies the used part of the frame description (the first n_views views and
// n_scenes scenes, the first n_views + 1 offsets of each table, the scalars):
// the parameter words are read from the constant bank, where the lanes' distinct
// addresses serialise, so the unused view and scene slots (most of the 11 KB)
// are left out; no kernel reads them.
__global__ void k_setup(FrameDev fd, FrameDev* dst, Header* hdr, BwdCounters* bc) {
  pdl_wait();
  pdl_trigger();
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&fd);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  const int nv = fd.n_views, ns = fd.n_scenes;
  auto copy = [&](size_t off, size_t bytes) {
    const int w0 = (int)(off / 4), nw = (int)(bytes / 4);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) d[w0 + i] = src[w0 + i];
  };
  copy(offsetof(FrameDev, views), nv * sizeof(ViewDev));
  copy(offsetof(FrameDev, scenes), ns * sizeof(SceneDev));
  copy(offsetof(FrameDev, entry_off), (nv + 1) * sizeof(int64_t));
  copy(offsetof(FrameDev, pix_off), (nv + 1) * sizeof(int64_t));
  copy(offsetof(FrameDev, tile_off), (nv + 1) * sizeof(int32_t));
  copy(offsetof(FrameDev, chunk_off), (nv + 1) * sizeof(int32_t));
  copy(offsetof(FrameDev, n_views), sizeof(FrameDev) - offsetof(FrameDev, n_views));
  uint32_t* h = reinterpret_cast<uint32_t*>(hdr);
  for (int i = threadIdx.x; i < (int)(sizeof(Header) / 4); i += blockDim.x) h[i] = 0u;
  // the backward's counters too, so a frame rendered without a backward reports
  // no backward evaluations (the backward re-clears them before it runs)
  if (bc && threadIdx.x == 0) *bc = BwdCounters{0, 0, 0};
}

static_assert(sizeof(FrameDev) % 4 == 0, "FrameDev must be a whole number of words");
static_assert(sizeof(ViewDev) % 4 == 0 && sizeof(SceneDev) % 4 == 0 && offsetof(FrameDev, views) % 4 == 0 &&
                  offsetof(FrameDev, scenes) % 4 == 0 && offsetof(FrameDev, tile_off) % 4 == 0 &&
                  offsetof(FrameDev, chunk_off) % 4 == 0 && offsetof(FrameDev, n_views) % 4 == 0,
              "the frame description's tables are whole words");
static_assert(sizeof(Header) == 256, "Header is one 256-byte block");

cudaError_t launch_setup(const FrameDev& fd, void* ws, const Layout& L, cudaStream_t s) {
  launch_pdl(k_setup, 1, 256, 0, s, fd, at<FrameDev>(ws, L.frame), at<Header>(ws, L.hdr),
             fd.geometry_only ? nullptr : at<BwdCounters>(ws, L.bwdcnt));
  return cudaGetLastError();
}

__global__ void k_debug_rect(const short4* rect, int64_t E, int4* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E; i += (int64_t)gridDim.x * blockDim.x) {
    short4 r = rect[i];
    out[i] = make_int4(r.x, r.y, r.z, r.w);
  }
}

// The backward clears only the visible entries' 2D-gradient rows: a culled
// entry's row may hold an earlier frame's values, which the copy shows as 0.
__global__ void k_debug_grad2d(const float4* src, const uint32_t* key, int64_t E, float4* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 4 * E;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = key[i >> 2] == kInvalidKey ? make_float4(0.f, 0.f, 0.f, 0.f) : src[i];
}

gs_status frame_workspace_size(const gs_frame* frame, size_t* bytes) {
  FrameDev fd;
  Layout L;
  *bytes = 0;
  const gs_status st = prepare(frame, fd, L);
  if (st == GS_OK) *bytes = L.total;
  return st;
}

}  // namespace gs

using namespace gs;

// An NVTX range around each stage's entry point, named after it, so that a
// profiler's timeline (and ncu's --nvtx filters) can pick out the library's
// stages; it costs nothing when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

extern "C" {

size_t gs_workspace_size(const gs_frame* frame) {
  size_t bytes = 0;
  return frame_workspace_size(frame, &bytes) == GS_OK ? bytes : 0;
}

gs_status gs_preprocess(const gs_frame* frame, void* stream) {
  NvtxRange nvtx_range("gs_preprocess");
  FrameDev fd;
  Layout L;
  gs_status st = prepare_ws(frame, fd, L);
  if (st != GS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_setup(fd, frame->workspace, L, s);
  if (e != cudaSuccess) return cuda_fail(e, "setup");
  e = launch_preprocess(frame->workspace, L, fd, s);
  if (e != cudaSuccess) return cuda_fail(e, "preprocess");
  return GS_OK;
}

gs_status gs_bin(const gs_frame* frame, void* stream) {
  NvtxRange nvtx_range("gs_bin");
  FrameDev fd;
  Layout L;
  gs_status st = prepare_ws(frame, fd, L);
  if (st != GS_OK) return st;
  cudaError_t e = launch_bin(frame->workspace, L, fd, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "bin");
  return GS_OK;
}

gs_status gs_render_fwd(const gs_frame* frame, const gs_maps* maps, void* stream) {
  NvtxRange nvtx_range("gs_render_fwd");
  FrameDev fd;
  Layout L;
  gs_status st = prepare_ws(frame, fd, L);
  if (st != GS_OK) return st;
  if (!maps) return fail(GS_ERR_INVALID_ARG, "maps is NULL");
  if (!fd.losses && (maps->dist || maps->nloss))
    return fail(GS_ERR_INVALID_ARG, "the dist and nloss maps need params.losses = 1");
  if (fd.geometry_only && maps->color)
    return fail(GS_ERR_INVALID_ARG, "geometry_only renders no colour: maps->color must be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_render_fwd(frame->workspace, L, fd, *maps, s);
  if (e != cudaSuccess) return cuda_fail(e, "render_fwd");
  if (maps->nloss) {
    e = launch_nloss_fwd(frame->workspace, L, fd, maps->nloss, s);
    if (e != cudaSuccess) return cuda_fail(e, "nloss_fwd");
  }
  return GS_OK;
}

gs_status gs_composite_bwd(const gs_frame* frame, const gs_map_grads* dmaps, void* stream) {
  NvtxRange nvtx_range("gs_composite_bwd");
  FrameDev fd;
  Layout L;
  gs_status st = prepare_ws(frame, fd, L);
  if (st != GS_OK) return st;
  if (!dmaps) return fail(GS_ERR_INVALID_ARG, "dmaps must not be NULL");
  if (fd.geometry_only) return fail(GS_ERR_INVALID_ARG, "geometry_only frames have no backward");
  if (!fd.losses && (dmaps->ddist || dmaps->dnloss))
    return fail(GS_ERR_INVALID_ARG, "ddist and dnloss need params.losses = 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (dmaps->dnloss) {
    e = launch_nloss_bwd(frame->workspace, L, fd, dmaps->dnloss, s);
    if (e != cudaSuccess) return cuda_fail(e, "nloss_bwd");
  }
  e = launch_render_bwd(frame->workspace, L, fd, *dmaps, s);
  if (e != cudaSuccess) return cuda_fail(e, "composite_bwd");
  return GS_OK;
}

gs_status gs_preprocess_bwd(const gs_frame* frame, const gs_scene_grads* grads, void* stream) {
  NvtxRange nvtx_range("gs_preprocess_bwd");
  FrameDev fd;
  Layout L;
  gs_status st = prepare_ws(frame, fd, L);
  if (st != GS_OK) return st;
  if (!grads) return fail(GS_ERR_INVALID_ARG, "grads must not be NULL");
  if (fd.geometry_only) return fail(GS_ERR_INVALID_ARG, "geometry_only frames have no backward");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GradPtrs gp;
  memset(&gp, 0, sizeof(gp));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < frame->n_scenes; ++i) {
    gp.g[i] = grads[i];
    const gs_scene& sc = frame->scenes[i];
    if (fd.scenes[i].n_views > 1 && sc.n > 0) {  // several views add into the same buffers
      const size_t n = (size_t)sc.n;
      const size_t K = (size_t)(sc.sh_degree + 1) * (sc.sh_degree + 1);
      if (e == cudaSuccess && grads[i].dmeans) e = cudaMemsetAsync(grads[i].dmeans, 0, 12 * n, s);
      if (e == cudaSuccess && grads[i].dscales) e = cudaMemsetAsync(grads[i].dscales, 0, 12 * n, s);
      if (e == cudaSuccess && grads[i].dquats) e = cudaMemsetAsync(grads[i].dquats, 0, 16 * n, s);
      if (e == cudaSuccess && grads[i].dopacities) e = cudaMemsetAsync(grads[i].dopacities, 0, 4 * n, s);
      if (e == cudaSuccess && grads[i].dsh) e = cudaMemsetAsync(grads[i].dsh, 0, 12 * K * n, s);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "zeroing gradients");
  e = launch_preprocess_bwd(frame->workspace, L, fd, gp, s);
  if (e != cudaSuccess) return cuda_fail(e, "preprocess_bwd");
  return GS_OK;
}

gs_status gs_render_bwd(const gs_frame* frame, const gs_map_grads* dmaps, const gs_scene_grads* grads,
                        void* stream) {
  if (!dmaps || !grads) return fail(GS_ERR_INVALID_ARG, "dmaps and grads must not be NULL");
  gs_status st = gs_composite_bwd(frame, dmaps, stream);
  if (st != GS_OK) return st;
  return gs_preprocess_bwd(frame, grads, stream);
}

gs_status gs_filter3d(const gs_frame* frame, int32_t scene, float scale, float* filter_var, void* stream) {
  NvtxRange nvtx_range("gs_filter3d");
  FrameDev fd;
  Layout L;
  gs_status st = prepare_ws(frame, fd, L);
  if (st != GS_OK) return st;
  if (scene < 0 || scene >= frame->n_scenes) return fail(GS_ERR_INVALID_ARG, "scene index %d out of range", scene);
  if (!(scale >= 0.f) || !std::isfinite(scale)) return fail(GS_ERR_INVALID_ARG, "scale must be finite and >= 0");
  if (frame->scenes[scene].n > 0 && !filter_var) return fail(GS_ERR_INVALID_ARG, "filter_var is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_setup(fd, frame->workspace, L, s);
  if (e == cudaSuccess) e = launch_filter3d(frame->workspace, L, fd, scene, scale, filter_var, s);
  if (e != cudaSuccess) return cuda_fail(e, "filter3d");
  return GS_OK;
}

gs_status gs_debug_copy(const gs_frame* frame, float* rec, int32_t* rect, int32_t* pair_tile,
                        int32_t* pair_entry, int32_t* ranges, float* grad2d, void* stream) {
  FrameDev fd;
  Layout L;
  gs_status st = prepare_ws(frame, fd, L);
  if (st != GS_OK) return st;
  if (fd.geometry_only && grad2d)
    return fail(GS_ERR_INVALID_ARG, "geometry_only frames keep no 2D gradients");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* ws = frame->workspace;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, size_t off, size_t bytes) {
    if (dst && bytes && e == cudaSuccess)
      e = cudaMemcpyAsync(dst, at<char>(ws, off), bytes, cudaMemcpyDeviceToDevice, s);
  };
  cp(rec, L.rec, 64 * (size_t)L.E);
  cp(pair_tile, L.ptile_final, 4 * (size_t)L.Pcap);
  cp(pair_entry, L.pval_final, 4 * (size_t)L.Pcap);
  cp(ranges, L.ranges, 8 * (size_t)L.T);
  if (e == cudaSuccess && grad2d && L.E > 0) {
    int g = (int)std::min<int64_t>((4 * L.E + 255) / 256, 4096);
    k_debug_grad2d<<<g, 256, 0, s>>>(at<float4>(ws, L.grad2d), at<uint32_t>(ws, L.key), L.E,
                                     reinterpret_cast<float4*>(grad2d));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && rect && L.E > 0) {
    int g = (int)std::min<int64_t>((L.E + 255) / 256, 4096);
    k_debug_rect<<<g, 256, 0, s>>>(at<short4>(ws, L.rect), L.E, reinterpret_cast<int4*>(rect));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(e, "debug_copy");
  return GS_OK;
}

gs_status gs_debug_wait_timeout(const gs_frame* frame, int32_t spin_limit, void* stream) {
  FrameDev fd;
  Layout L;
  gs_status st = prepare_ws(frame, fd, L);
  if (st != GS_OK) return st;
  if (spin_limit < 1 || spin_limit > (1 << 22))
    return fail(GS_ERR_INVALID_ARG, "spin_limit %d outside [1, 4194304]", spin_limit);
  cudaError_t e = launch_wait_timeout(frame->workspace, L, spin_limit, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "wait_timeout");
  return GS_OK;
}

gs_status gs_check(const gs_frame* frame, gs_stats* out, void* stream) {
  FrameDev fd;
  Layout L;
  gs_status st = prepare_ws(frame, fd, L);
  if (st != GS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  Header h;
  e = cudaMemcpy(&h, at<Header>(frame->workspace, L.hdr), sizeof(Header), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading the workspace header");
  if (out) {
    out->n_entries = L.E;
    out->n_visible = (int64_t)h.n_vis;
    out->n_pairs = (int64_t)h.n_pairs;
    out->n_nonfinite = (int64_t)h.n_nonfinite;
    out->n_evals_fwd = (int64_t)h.n_evals_fwd;
    BwdCounters bc = {0, 0, 0};
    if (!fd.geometry_only) {
      e = cudaMemcpy(&bc, at<BwdCounters>(frame->workspace, L.bwdcnt), sizeof(bc), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "reading the backward counters");
    }
    out->n_evals_bwd = (int64_t)bc.n_evals_bwd;
    out->n_blended = (int64_t)h.n_blend;
    out->status = h.status;
  }
  if (h.status == GS_ERR_CAPACITY)
    return fail(GS_ERR_CAPACITY, "%llu pairs needed, capacity %lld", h.n_pairs, (long long)L.Pcap);
  if (h.status == GS_ERR_NUMERIC)
    return fail(GS_ERR_NUMERIC, "%llu entries had non-finite inputs and were culled", h.n_nonfinite);
  if (h.status == GS_ERR_BOUNDS) {
    static const char* const kSites[] = {"?", "compositing forward: tile-list entry",
                                         "compositing backward: tile-list entry", "tile ranges: pair tile",
                                         "radix sort: scatter destination", "emission: pair tile",
                                         "emission: pair entry"};
    const int site = (int)((h.debug_word >> 48) & 0x7FFF);
    const long long index = (long long)(h.debug_word & 0xFFFFFFFFFFFFull);
    return fail(GS_ERR_BOUNDS, "index out of range at %s (site %d): %lld",
                site >= 1 && site <= 6 ? kSites[site] : kSites[0], site, index);
  }
  if (h.status != 0) return fail((gs_status)h.status, "device status %d", h.status);
  return GS_OK;
}

const char* gs_last_error_string(void) { return g_err; }

int32_t gs_debug_checks(void) {
#ifdef GS_DEBUG
  return 1;
#else
  return 0;
#endif
}

}  // extern "C"
