// Internal definitions shared by the libgs kernels: the device copy of a frame
// descriptor, the workspace layout and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <utility>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

constexpr int kRecFloats = 16;            // per-entry record / 2D-gradient slots
constexpr uint32_t kInvalidKey = 0xFFFFFFFFu;
constexpr int kSortThreads = 256;         // radix sort / scan block size
constexpr int kSortItems = 16;            // items per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 items per block
constexpr int kRadixBits = 8;
constexpr int kEmitChunk = 2048;          // pairs per emission slice
constexpr int kRadix = 1 << kRadixBits;
// Per-entry word written by the preprocess: the number of tiles the entry's
// pixel rectangle touches (0: culled) in the low 29 bits (a view of at most
// 32767 x 32767 pixels has fewer tiles), and in bit 29 + k whether colour
// channel k was above 0 (not clamped by max(SH + 1/2, 0)), which the
// preprocess backward needs.
constexpr int kTouchedBits = 29;
constexpr uint32_t kTouchedMask = (1u << kTouchedBits) - 1u;

// The record of a (view, Gaussian) entry: four float4s
//   #0 (u, v, a', b')             #1 (c', opacity, n_y, n_z)
//   #2 (p0, p1, z_c, 0)           #3 (r, g, b, n_x)
// with (a', b', c') = log2(e) (a / 2, b, c / 2) for the conic (a, b, c), so
// that sigma log2(e) = a' dx^2 + b' dx dy + c' dy^2.
// #0 and #1 hold everything the alpha test needs; #2 only the planar depth.
// Slots of the per-entry 2D-gradient row the compositing backward accumulates
// (gs = dL/dsigma, sd = dL/dd per pixel; the preprocess backward turns the
// first ten into record gradients with the entry's conic, p and opacity):
enum GradSlot {
  G_U = 0, G_V = 1, G_CA = 2, G_CB = 3,      // S gs dx, S gs dy, S gs dx^2, S gs dx dy
  G_CC = 4, G_O = 5, G_UNUSED = 6, G_Z = 7,  // S gs dy^2, S gs, -, S sd
  G_P0 = 8, G_P1 = 9, G_N1 = 10, G_N2 = 11,  // S sd dx, S sd dy, dL/dn_y, dL/dn_z
  G_R = 12, G_G = 13, G_B = 14, G_N0 = 15    // dL/d(r, g, b), dL/dn_x
};

struct ViewDev {
  float R[9];         // world->camera rotation, row-major
  float t[3];
  float fx, fy, cx, cy;
  float lim[4];       // clamp bounds of x/z (lo, hi) and y/z (lo, hi) inside J
  float campos[3];    // camera centre in world space
  float near_plane;
  int32_t width, height;
  int32_t tiles_x, tiles_y;
  int32_t scene;
  int32_t pad_;
};

struct SceneDev {
  const void* means;
  const void* scales;
  const void* quats;
  const void* opacities;
  const void* sh;
  int64_t n;
  int32_t sh_degree;
  int32_t dtype;
  int32_t n_views;    // views rendering this scene (1 => gradients are stored, else added)
  int32_t pad_;
  const float* filter_var;  // [n] Mip-Splatting 3D filter variances, or NULL
};

// Mip-Splatting 3D filter, the exactly rounded FP32 chain shared by the forward
// (where it feeds the binning decisions) and the backward:
// s~ = sqrt(s^2 + v), o' = ((o * (s0/s~0)) * (s1/s~1)) * (s2/s~2).
__device__ inline void filter3d_apply(float v, float (&s)[3], float& o) {
  float r[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float st = __fsqrt_rn(__fadd_rn(__fmul_rn(s[k], s[k]), v));
    r[k] = __fdiv_rn(s[k], st);
    s[k] = st;
  }
  o = __fmul_rn(__fmul_rn(__fmul_rn(o, r[0]), r[1]), r[2]);
}

struct FrameDev {
  ViewDev views[GS_MAX_VIEWS];
  SceneDev scenes[GS_MAX_SCENES];
  int64_t entry_off[GS_MAX_VIEWS + 1];  // entries of view v: [entry_off[v], entry_off[v+1])
  int64_t pix_off[GS_MAX_VIEWS + 1];    // pixels of view v in the concatenated maps
  int32_t tile_off[GS_MAX_VIEWS + 1];   // global tile ids of view v
  int32_t chunk_off[GS_MAX_VIEWS + 1];  // per-Gaussian kernels: 128-entry chunks before view v
  int32_t n_views, n_scenes;
  int64_t n_entries, n_pixels, pair_capacity;
  int32_t n_tiles, n_chunks;
  int32_t tile_w, tile_h, tile_shift_x, tile_shift_y;
  float lowpass, alpha_min, alpha_max, T_min, median_T;
  float ext_c;        // float32(2 ln(1/alpha_min))
  int32_t losses;     // per-pixel state of the Eq. 23-24 losses is kept
  int32_t geometry_only;  // forward-only alpha / depth / normal, no backward state
  int32_t batch;      // records a compositing warp stages per round: 32 or 64
};

// Per-pixel planes of the loss state (each [n_pixels] floats, global pixel
// index), present when FrameDev::losses is set.
enum LossPlane {
  LP_MEAN = 0,             // sum w d / sum w: weighted mean planar depth (Eq. 23 backward)
  LP_DEPTH = 1,            // copy of the median depth map
  LP_N0 = 2,               // copy of the normal map, 3 planes
  LP_DD = 5,               // d L_n / d depth (Eq. 24 backward)
  LP_DN0 = 6,              // d L_n / d normal map, 3 planes
  LP_DA = 9,               // d L_n / d alpha map
  kLossPlanes = 10
};

// Parameter-gradient outputs, passed by value to the backward kernel.
struct GradPtrs {
  gs_scene_grads g[GS_MAX_SCENES];
};

// A device-side count, clamped to the capacity it was computed against.
__device__ inline int64_t clamp_count(const unsigned long long* p, int64_t cap) {
  unsigned long long c = *p;
  return (int64_t)(c < (unsigned long long)cap ? c : (unsigned long long)cap);
}

struct Header {
  unsigned long long n_vis;
  unsigned long long n_pairs;
  unsigned long long n_nonfinite;
  // reset together (one 24-byte memset) before every forward render
  unsigned long long n_evals_fwd;
  unsigned long long n_blend;   // (pixel, splat) pairs blended by the last forward
  int32_t work_fwd;             // work-queue counter of the persistent forward
  int32_t pad0_;
  int32_t status;
  uint32_t filter_max;          // bits of the largest 3D-filter variance of seen Gaussians
  unsigned long long debug_word;   // GS_DEBUG builds: the frame's first index out of range
  int32_t pad_[48];
};

// Counters of the compositing backward; they sit right before the 2D-gradient
// buffer so that one memset clears both.
struct BwdCounters {
  unsigned long long n_evals_bwd;
  int32_t work_bwd;             // work-queue counter of the persistent backward
  int32_t pad_;
};

// Byte offsets of every buffer inside the caller's workspace.
struct Layout {
  int64_t E, T, NPIX, Pcap;
  int32_t nb_E, nb_P;       // radix blocks over entries / pairs
  size_t hdr, frame, rec, rect, key, touched;
  size_t vkey[2], vval[2];  // depth sort ping-pong
  size_t pair_off;          // exclusive scan of tiles_touched in depth order
  size_t chunk_first;       // [Pcap / kEmitChunk + 1] entry holding each emission chunk's first pair
  size_t scanaux;           // the two scans: tickets (64 B), then nb_E look-back words each
  size_t ptile[2], pval[2]; // pair sort ping-pong
  size_t ptile_final, pval_final;  // where the sorted pairs end up
  size_t sortaux[2];        // depth and tile radix sorts: digit histograms, tickets, look-back
  size_t sortaux_bytes[2];  // words; they, the scan words and the tile ranges are cleared by one memset
  size_t ranges;            // [T] int2
  size_t tile_order;        // [T] int: compositing work order (heaviest tiles first)
  size_t px_T, px_last, px_med;
  size_t bwdcnt;            // BwdCounters (one 256-byte block right before grad2d)
  size_t grad2d;            // [E][16] float
  size_t px_loss;           // [kLossPlanes][NPIX] float when losses, else 0 bytes
  size_t cmask;             // [subs][cmask_words] uint: records each 8x4 block blended, per chunk
  int64_t cmask_words;
  size_t total;
};

template <typename T> __host__ __device__ inline T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

// Programmatic dependent launch.  A kernel launched by launch_pdl may be
// scheduled, and its blocks may start, while the kernel before it in the
// stream is still finishing; pdl_wait() returns once that kernel has completed
// and its writes are visible.  Every such kernel calls pdl_wait() before any
// access to memory, then pdl_trigger(), which lets the next kernel be
// scheduled in turn: only launch latency overlaps, never the work itself.
__device__ inline void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ inline void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

__device__ inline void set_status(Header* h, int code) {
  atomicCAS(&h->status, 0, code);
}

// Bounds checks of a GS_DEBUG build.  GS_IN_BOUNDS(h, ok, site, index) is
// `ok`, and when `ok` is false it records (site, index) as the frame's first
// violation (bit 63 set, the site in bits 48-62, the index in bits 0-47) and
// sets the status to GS_ERR_BOUNDS; the caller skips the access.  In an
// ordinary build it is the constant true, and the code is that of no check.
enum BoundsSite : int {
  BS_FWD_ENTRY = 1,   // compositing forward: a tile list's entry
  BS_BWD_ENTRY = 2,   // compositing backward: a tile list's entry
  BS_RANGE_TILE = 3,  // tile ranges: a pair's tile
  BS_SORT_DST = 4,    // radix sort: a scatter destination
  BS_EMIT_TILE = 5,   // emission: a pair's tile
  BS_EMIT_ENTRY = 6,  // emission: a pair's entry
};
#ifdef GS_DEBUG
__device__ inline bool gs_in_bounds(Header* h, bool ok, int site, int64_t index) {
  if (!ok) {
    const unsigned long long w =
        (1ull << 63) | ((unsigned long long)site << 48) | ((unsigned long long)index & 0xFFFFFFFFFFFFull);
    if (atomicCAS(&h->debug_word, 0ull, w) == 0ull) set_status(h, GS_ERR_BOUNDS);
  }
  return ok;
}
#define GS_IN_BOUNDS(h, ok, site, index) gs_in_bounds((h), (ok), (site), (int64_t)(index))
#else
#define GS_IN_BOUNDS(h, ok, site, index) true
#endif

__device__ inline int find_view(const int64_t* off, int n_views, int64_t e) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ inline int find_view_tile(const int32_t* off, int n_views, int32_t t) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T> __device__ inline float ldf(const T* p, int64_t i);
template <> __device__ inline float ldf<float>(const float* p, int64_t i) { return __ldg(p + i); }
template <> __device__ inline float ldf<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

int tile_sort_bits(int64_t n_tiles);

// Sets the calling thread's error string (printf-style) and returns `s`.
gs_status set_error(gs_status s, const char* fmt, ...);
// gs_workspace_size with the validation status (the error string says why).
gs_status frame_workspace_size(const gs_frame* frame, size_t* bytes);

// ---- launchers (each .cu file owns its kernels) ---------------------------
cudaError_t launch_setup(const FrameDev& fd, void* ws, const Layout& L, cudaStream_t s);
cudaError_t launch_preprocess(void* ws, const Layout& L, const FrameDev& host_fd, cudaStream_t s);
cudaError_t launch_wait_timeout(void* ws, const Layout& L, int spin_limit, cudaStream_t s);
cudaError_t launch_bin(void* ws, const Layout& L, const FrameDev& host_fd, cudaStream_t s);
cudaError_t launch_tile_order(void* ws, const Layout& L, const uint32_t* cost, int* order, cudaStream_t s);
cudaError_t launch_render_fwd(void* ws, const Layout& L, const FrameDev& host_fd,
                              const gs_maps& maps, cudaStream_t s);
cudaError_t launch_render_bwd(void* ws, const Layout& L, const FrameDev& host_fd,
                              const gs_map_grads& g, cudaStream_t s);
cudaError_t launch_preprocess_bwd(void* ws, const Layout& L, const FrameDev& host_fd,
                                  const GradPtrs& gp, cudaStream_t s);
cudaError_t launch_filter3d(void* ws, const Layout& L, const FrameDev& host_fd, int scene, float scale,
                            float* out, cudaStream_t s);
cudaError_t launch_nloss_fwd(void* ws, const Layout& L, const FrameDev& host_fd, float* nloss,
                             cudaStream_t s);
cudaError_t launch_nloss_bwd(void* ws, const Layout& L, const FrameDev& host_fd, const float* dnloss,
                             cudaStream_t s);

}  // namespace gs
