/*
 * gs.h -- C ABI of the B300 depth/normal Gaussian-splat rasterizer (libgs.so).
 *
 * The library renders, for one or more views of one or more sets of 3D
 * Gaussians, the colour map (alpha blending, Eq. 3 of RaDe-GS, arxiv
 * 2406.01467), the alpha map, the rasterized planar depth map (Eq. 4 with the
 * plane coefficients of Eq. 13-17 and the median rule of Sec. 1) and the normal
 * map (Eq. 18-22), and the gradients of a loss on those maps with respect to
 * the Gaussian parameters.  Optionally it also renders the two per-pixel
 * geometric regularisers of Sec. 3.4 -- the depth distortion L_d (Eq. 23) and
 * the normal consistency L_n (Eq. 24) -- and their gradients.
 *
 * Conventions
 *   - camera frame: +x right, +y down, +z forward; viewmat is the row-major 4x4
 *     world->camera matrix [R | t; 0 0 0 1] (W of Eq. 2 is R);
 *   - pinhole u = fx x/z + cx, v = fy y/z + cy; pixel (i, j) is sampled at
 *     (i + 0.5, j + 0.5);
 *   - quaternions (w, x, y, z), normalised inside; scales > 0 and opacities in
 *     (0, 1] are already activated (Eq. 1: Sigma = R S S^T R^T);
 *   - SH coefficients [n][(deg+1)^2][3], real basis with Condon-Shortley phase,
 *     colour = max(SH(dir) + 0.5, 0), dir = normalize(mean - camera centre);
 *   - output maps are FP32, planar: colour and normal [3][H][W], alpha and depth
 *     [H][W]; the views' maps are concatenated in view order.
 *
 * Ownership: every pointer is caller-owned device memory except the gs_* structs
 * themselves, which are read on the host during the call and may be freed
 * afterwards.  The library allocates nothing, keeps no state between calls
 * apart from a thread-local error string, and never synchronises the stream:
 * a gs_preprocess / gs_bin / gs_render_fwd / gs_render_bwd sequence can be
 * captured in a CUDA graph.  Device-side problems (pair capacity exceeded,
 * non-finite inputs) set a sticky word inside the workspace that gs_check reads.
 * The kernels are launched with programmatic dependent launch: each waits for
 * the work before it in the stream to complete before it touches memory, and
 * lets the next kernel be scheduled early.  A caller's kernel that follows them
 * with that launch attribute must itself wait (cudaGridDependencySynchronize)
 * before it reads their outputs; ordinary launches need nothing.
 *
 * Errors: argument errors are detected on the host and returned at once
 * (GS_ERR_INVALID_ARG, nothing is enqueued); a failed launch returns
 * GS_ERR_CUDA.  gs_last_error_string() describes the last non-OK status of the
 * calling thread.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is out of range */
  GS_ERR_CAPACITY = 2,    /* more (tile, Gaussian) pairs than pair_capacity */
  GS_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
  GS_ERR_TIMEOUT = 4,     /* a bounded device wait ran out (scan / radix-sort look-back) */
  GS_ERR_NUMERIC = 5,     /* non-finite inputs; those Gaussians were culled */
  GS_ERR_BOUNDS = 6       /* only in a library built with -DGS_DEBUG (gs_debug_checks):
                             an index into a workspace buffer was out of range, a
                             library fault; the access was skipped and gs_check names
                             the site and the index */
} gs_status;

typedef enum { GS_F32 = 0, GS_BF16 = 1 } gs_dtype;

enum { GS_MAX_VIEWS = 64, GS_MAX_SCENES = 16 };

/* Size of the device array behind gs_render_fwd_static (32 MiB). */
#define GS_STATIC_SCRATCH_BYTES (32u << 20)

/* One set of Gaussians (Sec. 3.1).  All arrays are device pointers of the
 * element type `dtype`, contiguous, row-major. */
typedef struct {
  const void* means;     /* [n][3] world-space centres x_c */
  const void* scales;    /* [n][3] activated scales (diagonal of S) */
  const void* quats;     /* [n][4] rotation quaternions (w, x, y, z) */
  const void* opacities; /* [n]    activated opacities */
  const void* sh;        /* [n][(sh_degree+1)^2][3] SH coefficients */
  int64_t n;             /* number of Gaussians, >= 0 */
  int32_t sh_degree;     /* 0..3 */
  int32_t dtype;         /* gs_dtype of every array above */
  const float* filter_var; /* [n] FP32 (whatever dtype is) Mip-Splatting 3D filter
                              variances v >= 0, or NULL for no filter (Sec. 4.1.1):
                              the covariance becomes Sigma + v I, i.e. every scale
                              s -> sqrt(s^2 + v), and the opacity is multiplied by
                              prod s / sqrt(s^2 + v) (the integral of o G is kept).
                              Gradients flow to the unfiltered scales and opacity. */
} gs_scene;

/* One camera (Sec. 3.1: W is the world->camera rotation). */
typedef struct {
  float viewmat[16];  /* row-major world->camera */
  float fx, fy, cx, cy;
  int32_t width, height; /* 1..16384 */
  float near_plane;      /* Gaussians with camera z <= near_plane are culled */
  int32_t scene;         /* index of the gs_scene this view renders */
} gs_view;

/* Render parameters; the paper keeps the 3D GS defaults (Sec. 4.1.1). */
typedef struct {
  int32_t tile_w, tile_h; /* tile size: powers of two, tile_w >= 8, tile_h >= 4,
                             tile_w * tile_h in {64, 128, 256} */
  float lowpass;          /* px^2 added to the 2x2 screen covariance, >= 0 */
  float alpha_min;        /* in (0, 1): splats below it are skipped at a pixel */
  float alpha_max;        /* in [alpha_min, 1): alpha clamp */
  float T_min;            /* in [0, 1): stop before T would fall below it */
  float median_T;         /* in (0, 1): median depth threshold on T */
  float clamp_margin;     /* x/z, y/z inside J clamped to the image widened by this */
  int32_t losses;         /* 0 or 1.  1 keeps, per pixel, the state that the loss maps
                             of Eq. 23-24 and their backward need (10 floats per pixel
                             of workspace); with 0, gs_maps.dist / nloss and
                             gs_map_grads.ddist / dnloss must be NULL */
  int32_t geometry_only;  /* 0 or 1.  1 renders alpha, depth and normal only, for
                             fusing many views into a volume: the SH coefficients are
                             not read (so non-finite SH do not cull), no colour is
                             blended (gs_maps.color must be NULL), and no per-pixel
                             backward state or 2D-gradient buffer is kept, so the
                             workspace shrinks by 12 B per pixel and 64 B per entry and
                             the backward calls return GS_ERR_INVALID_ARG.  Excludes
                             losses = 1. */
  int32_t batch;          /* Gaussians a compositing warp stages in shared memory per round
                             (the batch of records it tests against its pixels and blends):
                             32 or 64; 0 means 32.  A performance knob only: the maps and
                             gradients do not depend on it. */
} gs_params;

/* Everything a call needs to know about one frame (a batch of views). */
typedef struct {
  const gs_scene* scenes; /* host array [n_scenes] */
  int32_t n_scenes;       /* 1..GS_MAX_SCENES */
  const gs_view* views;   /* host array [n_views] */
  int32_t n_views;        /* 1..GS_MAX_VIEWS */
  gs_params params;
  int64_t pair_capacity;  /* maximum (tile, Gaussian) pairs, >= 1 */
  void* workspace;        /* device, 256-byte aligned, gs_workspace_size() bytes */
  size_t workspace_bytes;
} gs_frame;

/* Output maps (device, FP32), all views concatenated.  Any pointer may be NULL
 * (that map is not written).
 *
 * dist (Eq. 23): sum over ordered pairs (i, j) of the splats blended at the
 *   pixel of w_i w_j (d_i - d_j)^2, with w the blending weights alpha_i T_i and
 *   d_i the planar depth of splat i at the pixel (Eq. 4).
 * nloss (Eq. 24): sum_i w_i (1 - n_i . n~) = alpha - normal . n~, where n~ is
 *   the unit normal of the depth map back-projected to camera space,
 *   P(i, j) = depth(i, j) ((i + 1/2 - cx)/fx, (j + 1/2 - cy)/fy, 1),
 *   n~ = normalize((P(i, j+1) - P(i, j-1)) x (P(i+1, j) - P(i-1, j))).  It is
 *   defined at pixels not on the image border whose alpha and whose four
 *   neighbours' alphas are > 0 (and where that cross product is not zero);
 *   elsewhere nloss is 0.  Both need params.losses = 1. */
typedef struct {
  float* color;  /* [sum_v 3 H_v W_v] */
  float* alpha;  /* [sum_v H_v W_v]   1 - final transmittance */
  float* depth;  /* [sum_v H_v W_v]   median planar depth, 0 where nothing blends */
  float* normal; /* [sum_v 3 H_v W_v] blended camera-space unit normals */
  float* dist;   /* [sum_v H_v W_v]   depth distortion L_d (Eq. 23) */
  float* nloss;  /* [sum_v H_v W_v]   normal consistency L_n (Eq. 24) */
} gs_maps;

/* Upstream gradients dL/d(maps), same layouts as gs_maps; any may be NULL (zero).
 * The weights w of Eq. 23 are treated as constants (Sec. 4.1.1), so ddist
 * reaches the parameters through the splats' planar depths only; dnloss
 * reaches them through w, the splat normals n_i and, by the finite
 * differences, the median depths of the pixel and its four neighbours.
 * ddist and dnloss need params.losses = 1 and a gs_render_fwd of the same
 * frame with it. */
typedef struct {
  const float* dcolor;
  const float* dalpha;
  const float* ddepth;
  const float* dnormal;
  const float* ddist;
  const float* dnloss;
} gs_map_grads;

/* Parameter gradients of one scene (device, FP32, same shapes as gs_scene's
 * arrays).  They are overwritten, not accumulated.  Any pointer may be NULL. */
typedef struct {
  float* dmeans;
  float* dscales;
  float* dquats;
  float* dopacities;
  float* dsh;
} gs_scene_grads;

/* Counters read back by gs_check. */
typedef struct {
  int64_t n_entries;    /* (view, Gaussian) entries processed */
  int64_t n_visible;    /* entries that touch at least one pixel */
  int64_t n_pairs;      /* (tile, Gaussian) pairs needed */
  int64_t n_nonfinite;  /* entries culled for non-finite inputs */
  int64_t n_evals_fwd;  /* (pixel, splat) pairs tested by the last gs_render_fwd: the splats
                           that pass the pixel's 8x4 block test, in every 32-splat chunk of
                           the tile list that the pixel enters unfinished */
  int64_t n_evals_bwd;  /* (pixel, splat) evaluations of the last gs_composite_bwd */
  int64_t n_blended;    /* (pixel, splat) pairs blended (Eq. 3) by the last gs_render_fwd */
  int32_t status;       /* sticky gs_status of the device work */
} gs_stats;

/* Bytes of workspace the frame needs (its workspace fields are ignored).
 * Returns 0 and sets the error string on invalid arguments. */
size_t gs_workspace_size(const gs_frame* frame);

/* Per-Gaussian stage (Eq. 1-2, 8-22): projection, EWA covariance and conic,
 * SH colour, depth-plane coefficients p (Eq. 15-17) and normal (Eq. 22) for
 * every (view, Gaussian) entry; culling; pixel and tile rectangles; depth keys.
 * Resets the workspace's counters and sticky status.  `stream` is a
 * cudaStream_t (NULL = legacy default stream). */
gs_status gs_preprocess(const gs_frame* frame, void* stream);

/* Binning (inherited from 3D GS, Sec. 4.1.1): orders visible entries by depth
 * (own LSD radix sort), emits one pair per overlapped tile, sorts the pairs by
 * tile (stable, so each tile's list stays in depth order, ties by Gaussian
 * index) and finds each tile's [start, end).  Sets GS_ERR_CAPACITY on the
 * device if the pairs exceed pair_capacity; later stages then do nothing. */
gs_status gs_bin(const gs_frame* frame, void* stream);

/* Front-to-back compositing (Eq. 3, Eq. 4, Sec. 1, Eq. 22) of every view into
 * `maps`; stores the per-pixel state the backward pass replays.  With
 * params.losses = 1 the same pass accumulates sum w, sum w d and sum w d^2 per
 * pixel for Eq. 23, and a second kernel evaluates Eq. 24 when maps->nloss is
 * set.  GS_ERR_INVALID_ARG if dist or nloss is set with params.losses = 0. */
gs_status gs_render_fwd(const gs_frame* frame, const gs_maps* maps, void* stream);

/* Backward of gs_render_fwd and of gs_preprocess: replays each pixel back to
 * front and writes dL/d(means, scales, quats, opacities, sh) for every scene
 * (`grads` is a host array [n_scenes]).  Equivalent to gs_composite_bwd
 * followed by gs_preprocess_bwd. */
gs_status gs_render_bwd(const gs_frame* frame, const gs_map_grads* dmaps,
                        const gs_scene_grads* grads, void* stream);

/* First half of gs_render_bwd: the compositing backward (back-to-front replay
 * of Eq. 3, Eq. 4 and the normal blend) into per-entry gradients of the
 * projected quantities (kept in the workspace). */
gs_status gs_composite_bwd(const gs_frame* frame, const gs_map_grads* dmaps, void* stream);

/* Second half of gs_render_bwd: chain rule of the per-Gaussian stage (Eq. 1-2,
 * 8-22 and the SH colour) from the workspace's per-entry gradients to the
 * parameters.  Buffers of scenes seen by several views are zeroed, then summed. */
gs_status gs_preprocess_bwd(const gs_frame* frame, const gs_scene_grads* grads, void* stream);

/* Mip-Splatting 3D filter variances of scene `scene` from the frame's views of
 * it (Sec. 4.1.1): v = scale * min_n (z_n / fx_n)^2 over the views n in which
 * the Gaussian's centre has camera z > near_plane and projects inside the image
 * widened by 15 % of its size on each side; a Gaussian seen by no view gets the
 * largest v of the seen ones (0 if none is seen).  `filter_var` is device FP32
 * [n]; Mip-Splatting's scale is 0.2.  Runs on `stream` and resets the
 * workspace's counters and status like gs_preprocess. */
gs_status gs_filter3d(const gs_frame* frame, int32_t scene, float scale, float* filter_var, void* stream);

/* ---- Decoupled per-view appearance (Sec. 4.1.1, after VastGaussian) -------
 * The paper trains with a learned per-view colour correction so that exposure
 * and white-balance changes between photographs are not baked into the
 * Gaussians.  Here each training view owns an embedding e (embed_dim floats);
 * a two-layer perceptron h = relu(W1 e + b1), a = W2 h + b2 (12 outputs) gives
 * the affine c' = (I + A) c + t of the rendered colour, A = a[0..8] row-major,
 * t = a[9..11].  The loss of a view is the mean over its pixels and channels of
 * |c' - target|.  With W2 = b2 = 0 the correction is the identity.
 *
 * params / grads: device FP32 [gs_appearance_param_count()], flat layout
 *   embed [n_embeddings][embed_dim], W1 [hidden][embed_dim], b1 [hidden],
 *   W2 [12][hidden], b2 [12]. */
typedef struct {
  int32_t n_embeddings; /* >= 1: one per training view */
  int32_t embed_dim;    /* 1..256 */
  int32_t hidden;       /* 1..256 */
  int32_t pad_;
  float* params;
  float* grads;         /* gs_appearance_fwd_bwd adds to it */
} gs_appearance;

/* Floats of device scratch gs_appearance_fwd_bwd needs per view. */
#define GS_APPEARANCE_STATE_FLOATS 32

/* Parameters of an appearance model; 0 (and the error string) on bad sizes. */
size_t gs_appearance_param_count(int32_t n_embeddings, int32_t embed_dim, int32_t hidden);

/* For every view of `frame` (only its views' sizes are used): the affine from
 * embedding row embed_index[v] (host array [n_views]), the corrected colour
 * (written to `corrected` if not NULL), the loss (device [n_views], if not
 * NULL), dL/dc into `dcolor` (if not NULL; overwritten, the colour gradient
 * for gs_render_bwd), and dL/d(params) added to app->grads.  color, target,
 * corrected and dcolor are device FP32 maps in the gs_maps colour layout;
 * state is device scratch of GS_APPEARANCE_STATE_FLOATS * n_views floats. */
gs_status gs_appearance_fwd_bwd(const gs_frame* frame, const gs_appearance* app, const int32_t* embed_index,
                                const float* color, const float* target, float* corrected, float* dcolor,
                                float* loss, float* state, void* stream);

/* One Adam step (Kingma and Ba) on n FP32 parameters, `step` >= 1 counting
 * from 1: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps); then g = 0 if
 * zero_grads.  All buffers device FP32 [n]. */
gs_status gs_adam_step(float* params, float* grads, float* m, float* v, int64_t n, float lr, float beta1,
                       float beta2, float eps, int32_t step, int32_t zero_grads, void* stream);

/* Intermediate results for tests and tools, copied to caller device buffers on
 * `stream`; any pointer may be NULL.  rec: [n_entries][16] FP32 per-entry
 * records (u, v, a' b' c', opacity, n1 n2, p0 p1, z, 0, r g b, n0), where
 * (a', b', c') = log2(e) (a / 2, b, c / 2) for the conic (a, b, c);
 * rect: [n_entries][4] int32 pixel rectangle (i0, i1, j0, j1), (0,-1,0,-1)
 * when culled; pair_tile/pair_entry: [pair_capacity] int32 sorted pairs;
 * ranges: [total tiles][2] int32.  grad2d: [n_entries][16] FP32 per-entry sums
 * of the compositing backward, valid after gs_render_bwd: with gs = dL/dsigma
 * and sd = dL/dd per pixel, (S gs dx, S gs dy, S gs dx^2, S gs dx dy,
 * S gs dy^2, S gs, 0, S sd, S sd dx, S sd dy) and dL/d(n1, n2, r, g, b, n0);
 * dL/d(record) follows with the entry's conic, p and opacity. */
gs_status gs_debug_copy(const gs_frame* frame, float* rec, int32_t* rect,
                        int32_t* pair_tile, int32_t* pair_entry, int32_t* ranges,
                        float* grad2d, void* stream);

/* Forward render (gs_preprocess, gs_bin, gs_render_fwd) that allocates nothing.
 *
 * The paper has no counterpart; this is a convenience of the library.  Some
 * callers cannot allocate device memory: code that runs inside a host
 * application which owns the device allocator (a plugin), real-time loops that
 * forbid allocation once they run, and processes that must not grow their
 * memory footprint after start-up.  Such callers cannot provide the workspace
 * the staged calls above need.  Here the workspace is a file-scope device array
 * of GS_STATIC_SCRATCH_BYTES; every GPU that loads the library holds it until
 * the process exits.  frame->workspace and frame->workspace_bytes are ignored;
 * everything else, including pair_capacity, is used as given, and the caller
 * still provides the scene arrays and the output maps.  A frame whose
 * workspace would not fit (gs_workspace_size) is rejected with
 * GS_ERR_INVALID_ARG and a message giving both sizes.
 *
 * The first call on a device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  The address is kept per device together with the id of
 * the device's CUDA context, and looked up again when a call finds another
 * context current (after cudaDeviceReset, or a primary context released and
 * re-created); the first call after such a reset should also precede any
 * capture.  No call runs cudaMalloc, cudaFree or an allocating library
 * routine.  All calls share the one array and each call re-initialises what
 * must start at zero (counters, status word, tile ranges), so consecutive calls
 * are independent; calls whose work overlaps on the GPU (other streams or
 * threads) race on the array and must be serialised by the caller.  If `stats`
 * is not NULL the call synchronises `stream` and returns the device status as
 * gs_check does (a pair overflow leaves the maps unwritten). */
gs_status gs_render_fwd_static(const gs_frame* frame, const gs_maps* maps, gs_stats* stats,
                               void* stream);

/* Synchronises `stream`, then reads the counters and sticky status. */
gs_status gs_check(const gs_frame* frame, gs_stats* out, void* stream);

/* Test hook for the device's bounded waits (the decoupled look-back of the
 * scans and radix sorts, which poll other blocks' words): one block polls a
 * word that nothing publishes, gives up after `spin_limit` polls (1 ..
 * 4194304, the limit the real waits use), sets the sticky status to
 * GS_ERR_TIMEOUT and returns, so the context stays usable.  gs_check then
 * reports GS_ERR_TIMEOUT; the next gs_preprocess clears the status.  Uses the
 * frame's workspace (its binning words, which the next gs_bin clears); the
 * frame must have been prepared as for gs_preprocess. */
gs_status gs_debug_wait_timeout(const gs_frame* frame, int32_t spin_limit, void* stream);

/* 1 if this library was built with -DGS_DEBUG, else 0.  Such a build checks
 * the data-dependent indices of the device code (the entries named by the
 * tile lists, the tiles named by the pairs, the radix sort's scatter
 * destinations) before it uses them; an index out of range skips the access,
 * is recorded in the workspace (the first one of a frame) and sets the sticky
 * status to GS_ERR_BOUNDS.  Its results are otherwise those of the ordinary
 * build.  A stand-in for a memory checker: a test harness, not the product. */
int32_t gs_debug_checks(void);

/* ---- Throughput probes (measurement support; the paper has no counterpart) --
 * The compositing kernels are bound by instruction issue, the FP32 and MUFU
 * pipes and shared memory rather than by HBM; these probes measure those
 * units' peak rates on the GPU at hand so that a benchmark can state the
 * kernels' fractions of them.  Each call enqueues on `stream` (a cudaStream_t)
 * one resident wave of blocks (every SM, as many blocks as fit) that runs
 * long chains of one operation, and stores in *work (host) how many of them
 * the launch performs: FMAs (GS_PEAK_FFMA: scalar fma.rn.f32; GS_PEAK_FFMA2:
 * packed fma.rn.f32x2, two FMAs per instruction), base-2 exponentials
 * (GS_PEAK_EX2: ex2.approx.ftz.f32) or bytes read from shared memory
 * (GS_PEAK_LDS128: 16-byte loads, consecutive per lane, no bank conflicts).
 * The caller times the launch.  `iters` (1 .. 2^24) sets its length: each
 * thread runs 16 * iters steps of 8 independent chains.  `sink` is a device
 * float the probe never actually writes.  GS_ERR_INVALID_ARG for a bad kind,
 * count or pointer; GS_ERR_CUDA if the launch fails. */
enum { GS_PEAK_FFMA = 0, GS_PEAK_FFMA2 = 1, GS_PEAK_EX2 = 2, GS_PEAK_LDS128 = 3 };
gs_status gs_peak_probe(int32_t kind, int32_t iters, float* sink, int64_t* work, void* stream);

/* Human-readable description of the calling thread's last error. */
const char* gs_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* GS_H_ */
