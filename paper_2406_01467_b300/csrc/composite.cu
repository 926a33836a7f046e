// Per-tile compositing: front-to-back forward and back-to-front backward.
//
// Forward, per pixel (one thread), over its tile's depth-ordered list, staged
// through shared memory one batch of records at a time:
//   Delta = (u_c - u, v_c - v); sigma = 1/2 Delta^T conic Delta;
//   alpha = min(alpha_max, o exp(-sigma)), skipped below alpha_min;
//   (the record holds the conic times log2(e), its diagonal halved, so that
//   s = sigma log2(e) takes two multiplies and two fused multiply-adds and
//   exp(-sigma) = 2^-s one ex2)
//   stop before T (1 - alpha) < T_min;  w = alpha T;
//   colour += w rgb (Eq. 3); normal += w n (Eq. 22);
//   depth = z_c + p Delta (Eq. 4) of the first splat with T' <= median_T
//   (the median depth of Sec. 1), else of the last contributor;
//   alpha map = 1 - T_final.
//
// Each warp owns an 8x4 block of the tile's pixels and walks the tile's list on
// its own.  A record is evaluated only if the splat can reach the block: the
// minimum of sigma over the block's rectangle of pixel centres (exact, over the
// two edges facing the splat's centre) is at most sigma_cut = ln(o / alpha_min)
// plus a small margin.  A
// splat skipped this way is one every pixel of the block would have skipped by
// the alpha test, so the maps are the same as without the culling.
//
// With the loss state on (LOSS), the forward also accumulates, per pixel, the
// shifted moments S1 = sum w (d - d0), S2 = sum w (d - d0)^2 of the splats'
// planar depths d (d0 = the first contributor's depth), which give the depth
// distortion of Eq. 23 as 2 (W S2 - S1^2), W = sum w, in one pass: the double
// sum over pairs expands to that, and the shift leaves it unchanged while
// keeping the FP32 cancellation small.
//
// Backward replays each pixel from its last contributor toward the front,
// recovering T by division (alpha <= alpha_max < 1) and the colour / normal
// "behind" sums recursively; nothing per (pixel, splat) is stored.  It replays
// only the records the forward marked as blended by some pixel of the warp's
// block, two per round.  Each warp reduces the per-splat sums of its 32
// pixels (one shuffle fold, then a transpose through shared memory) and issues
// one atomic per sum; the sums are linear in the splat's conic, p and opacity,
// which the preprocess backward applies once per entry.  Without Eq. 23 only a
// pixel's median splat gets a depth gradient, so the three depth sums leave the
// reduction (12 values instead of 16) and the lanes whose median is the
// record add them with atomics of their own.
// Eq. 23 with constant weights adds dL/dd_k = 4 w_k W (d_k - mean) to each
// contributor's planar depth; Eq. 24 enters through the map gradients of
// alpha, normal and depth that the normal-consistency backward stored.
#include "gs_internal.cuh"

namespace gs {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kSubW = 8, kSubH = 4;  // pixels of one warp's block

// Adds the warp's evaluation count to a header counter (one atomic per warp).
__device__ inline void count_evals(uint32_t n, unsigned long long* counter) {
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(kFull, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(counter, (unsigned long long)n);
}

struct TileCtx {
  int view, px, py, W, H;
  int x0, y0;          // first pixel of the tile
  bool inside;
  int64_t pix;         // global pixel index (concatenated views)
  int64_t pix_local;   // index inside the view
  int64_t pix_base;    // first pixel of the view
};

__device__ inline TileCtx tile_ctx(const FrameDev* fd, int tile, int sub) {
  TileCtx c;
  c.view = find_view_tile(fd->tile_off, fd->n_views, tile);
  const ViewDev& V = fd->views[c.view];
  const int local = tile - fd->tile_off[c.view];
  const int tx = local % V.tiles_x, ty = local / V.tiles_x;
  const int warp = sub, lane = threadIdx.x & 31;
  const int sub_per_row = fd->tile_w / kSubW;
  c.x0 = tx * fd->tile_w;
  c.y0 = ty * fd->tile_h;
  c.px = c.x0 + (warp % sub_per_row) * kSubW + (lane % kSubW);
  c.py = c.y0 + (warp / sub_per_row) * kSubH + (lane / kSubW);
  c.W = V.width;
  c.H = V.height;
  c.inside = c.px < c.W && c.py < c.H;
  c.pix_base = fd->pix_off[c.view];
  c.pix_local = (int64_t)c.py * c.W + c.px;
  c.pix = c.pix_base + c.pix_local;
  return c;
}

// s = sigma log2(e) at offset (dx, dy) from the centre, from the record's
// scaled conic (a, b, c) = log2(e) (conic_00 / 2, conic_01, conic_11 / 2).
__device__ inline float quad(float a, float b, float c, float dx, float dy) {
  return a * dx * dx + c * dy * dy + b * dx * dy;
}

// The same with a fixed rounding sequence: the forward and the backward both
// evaluate alpha through it, so they take identical alpha >= alpha_min decisions.
// d = (dx, dy), d2 = (dx^2, dy^2) (each product rounded once).
__device__ inline float splat_s(float a, float b, float c, float2 d, float2 d2) {
  return __fmaf_rn(b, __fmul_rn(d.x, d.y), __fmaf_rn(a, d2.x, __fmul_rn(c, d2.y)));
}

// 2^x (PTX ex2.approx: relative error near 2^-22): exp(-sigma) = 2^-s.
__device__ inline float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Minimum of sigma over the rectangle [X0, X1] x [Y0, Y1] (pixel-centre
// coordinates).  It lies on an edge facing the centre, if the centre is
// outside: sigma grows along the segment from the centre to any point of the
// rectangle (it scales with the square of the distance along it), and that
// segment enters the rectangle through an edge whose outside holds the centre.
// So two candidates suffice, each a 1D convex quadratic minimised along a
// line and clamped to the rectangle: x = u clamped to [X0, X1] (the facing
// vertical edge, or the centre's own column), and y = v clamped likewise.
// Both are points of the rectangle, and with the centre inside the first is
// the centre itself (sigma 0).
__device__ inline float rect_min_sigma(float u, float v, float a, float b, float c, float ia,
                                       float ic, float X0, float X1, float Y0, float Y1) {
  // x fixed: dy minimises 2 c dy + b dx = 0 (ic = 1 / 2c)
  const float dx = u - fminf(fmaxf(u, X0), X1);
  const float y = fminf(fmaxf(v + b * dx * ic, Y0), Y1);
  // y fixed
  const float dy = v - fminf(fmaxf(v, Y0), Y1);
  const float x = fminf(fmaxf(u + b * dy * ia, X0), X1);
  return fminf(quad(a, b, c, dx, v - y), quad(a, b, c, u - x, dy));
}

// Rectangle of warp w's pixel centres inside the tile starting at (x0, y0).
struct SubRect {
  float X0, X1, Y0, Y1;
};

__device__ inline SubRect sub_rect(int x0, int y0, int sub_per_row, int sub) {
  const int w = sub;
  SubRect r;
  r.X0 = (float)(x0 + (w % sub_per_row) * kSubW) + 0.5f;
  r.Y0 = (float)(y0 + (w / sub_per_row) * kSubH) + 0.5f;
  r.X1 = r.X0 + (kSubW - 1);
  r.Y1 = r.Y0 + (kSubH - 1);
  return r;
}

// Can the splat (first two record float4s) reach any pixel of the rectangle?
// s_cut = log2(o) - log2(alpha_min) (lg_amin): beyond it alpha < alpha_min, with a margin
// (1e-4 relative, 1.5e-4 absolute) far above the error of the FP32 operations
// and of __log2f, so the test only ever skips splats the alpha test rejects at
// every pixel.
__device__ inline bool reaches(const float4& f0, const float4& f1, const SubRect& R, float lg_amin) {
  const float ia = __fdividef(0.5f, f0.z), ic = __fdividef(0.5f, f1.x);
  const float cut = (__log2f(f1.y) - lg_amin) * 1.0001f + 1.5e-4f;
  return rect_min_sigma(f0.x, f0.y, f0.z, f0.w, f1.x, ia, ic, R.X0, R.X1, R.Y0, R.Y1) <= cut;
}

// Asynchronous global->shared copies (cp.async): each lane stages whole
// 64-byte records, so the next chunk's gathers are in flight while the warp
// evaluates the current one.
// L1: keep the lines in L1 (.ca, the forward, whose staging is double
// buffered), else L2 only (.cg, the backward, which is bound by the L1 data
// pipe: 0.639 -> 0.624 ms; the forward is 0.004 ms slower with .cg).
template <bool L1>
__device__ inline void cp_async16(uint32_t dst, const void* src) {
  if (L1)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ inline void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// A chunk buffer is slot-major ([slots][32] float4): lane l's 16-byte pieces
// sit 512 bytes apart, so per-lane accesses are free of bank conflicts.  The
// depth plane (piece 2) is staged only when every contributor's depth is
// needed (PLANE); then the slots are pieces 0-3, else pieces 0, 1 and 3.
template <bool PLANE> constexpr int kSlots = PLANE ? 4 : 3;
template <bool PLANE> constexpr int kColourSlot = PLANE ? 3 : 2;   // piece 3: (r, g, b, n0)

template <bool PLANE, bool L1 = true>
__device__ inline void stage_record(float4 (*chunk)[32], int lane, const float4* r) {
  const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(&chunk[0][lane]));
  cp_async16<L1>(dst, r);
  cp_async16<L1>(dst + 512, r + 1);
  if (PLANE) cp_async16<L1>(dst + 1024, r + 2);
  cp_async16<L1>(dst + 512 * kColourSlot<PLANE>, r + 3);
}

// One work item: warp-sized block `sub` of tile `tile`.  The warp walks the
// tile's list on its own, CH records at a time (the batch: 32 or 64, one or two
// per lane), through two shared buffers: while it evaluates chunk k (every
// lane tests its records against the warp's rectangle, then the records that
// pass are evaluated by all 32 lanes in list order), the records of chunk k+1
// are being copied in, and the entry indices of chunk k+2 are being loaded.
// The walk ends as soon as the block's own pixels are done (after the copies
// in flight have landed).  buf[b][s] is sub-chunk s (32 records) of buffer b.
template <bool LOSS, bool GEO, int CH>
__device__ inline void fwd_item(const FrameDev* __restrict__ fd, void* __restrict__ ws, const Layout& L,
                                const gs_maps& maps, int tile, int sub, float4 (*buf)[CH / 32][kSlots<LOSS>][32],
                                uint32_t& evals, uint32_t& blended) {
  constexpr int NS = CH / 32;   // 32-record sub-chunks per chunk
  const TileCtx c = tile_ctx(fd, tile, sub);
  const int2 range = at<int2>(ws, L.ranges)[tile];
  const uint32_t* pval = at<uint32_t>(ws, L.pval_final);
  const float4* rec = at<float4>(ws, L.rec);
  Header* hdr = at<Header>(ws, L.hdr);   // (bounds checks of a GS_DEBUG build)
  const float amin = fd->alpha_min, amax = fd->alpha_max, tmin = fd->T_min, tmed = fd->median_T;
  const float lg_amin = __log2f(amin);
  const float fpx = c.px + 0.5f, fpy = c.py + 0.5f;
  const float2 nfp = make_float2(-fpx, -fpy);
  const int lane = threadIdx.x & 31;
  const SubRect R = sub_rect(c.x0, c.y0, fd->tile_w / kSubW, sub);

  // per-chunk masks of blended records of this 8x4 block (word k: chunk k of the list)
  uint32_t* cmask = at<uint32_t>(ws, L.cmask) + (int64_t)sub * L.cmask_words + (range.x >> 5) + tile;
  float T = 1.f, depth = 0.f;
  // blended (r, g), (b, n0), (n1, n2): the record's aligned pairs
  float2 Crg = make_float2(0.f, 0.f), Cbn = make_float2(0.f, 0.f), N12 = make_float2(0.f, 0.f);
  float Ws = 0.f, S1 = 0.f, S2 = 0.f, d0 = 0.f;   // Eq. 23 moments (LOSS only)
  int last = -1, med = -1;
  uint32_t nblend = 0;
  bool done = !c.inside;
  int cur = 0;
  uint32_t e_next[NS];   // entries of this lane's records in the chunk after the one in flight
#pragma unroll
  for (int q = 0; q < NS; ++q) e_next[q] = 0;
  if (range.x < range.y) {
#pragma unroll
    for (int q = 0; q < NS; ++q)
      if (range.x + 32 * q + lane < range.y) {
        const uint32_t e = __ldg(pval + range.x + 32 * q + lane);
        if (GS_IN_BOUNDS(hdr, e < L.E, BS_FWD_ENTRY, e)) stage_record<LOSS>(buf[0][q], lane, rec + 4 * (int64_t)e);
      }
    cp_async_commit();
#pragma unroll
    for (int q = 0; q < NS; ++q)
      if (range.x + CH + 32 * q + lane < range.y) e_next[q] = __ldg(pval + range.x + CH + 32 * q + lane);
  }
  for (int c00 = range.x; c00 < range.y; c00 += CH) {
    if (__all_sync(kFull, done)) break;
#pragma unroll
    for (int q = 0; q < NS; ++q)
      if (c00 + CH + 32 * q + lane < range.y && GS_IN_BOUNDS(hdr, e_next[q] < L.E, BS_FWD_ENTRY, e_next[q]))
        stage_record<LOSS>(buf[cur ^ 1][q], lane, rec + 4 * (int64_t)e_next[q]);
    cp_async_commit();
#pragma unroll
    for (int q = 0; q < NS; ++q)
      if (c00 + 2 * CH + 32 * q + lane < range.y) e_next[q] = __ldg(pval + c00 + 2 * CH + 32 * q + lane);
    cp_async_wait<1>();     // this lane's copies of chunk c00 have landed
    __syncwarp();           // ... and every lane's are visible
#pragma unroll
    for (int q = 0; q < NS; ++q) {
    const int c0 = c00 + 32 * q;
    if (c0 >= range.y) break;   // past the list: no records and no mask word of this tile
    float4 (*my)[32] = buf[cur][q];
    const bool rel = c0 + lane < range.y && reaches(my[0][lane], my[1][lane], R, lg_amin);
    unsigned m = __ballot_sync(kFull, rel);
    uint32_t cm = 0;        // records of the chunk this lane blends
    // Two records per round, the odd one alone: both alphas are computed
    // before the blends (the chain through T is the only serial part).
    // Branch-free: a lane that is done, whose alpha misses the cut, or whose
    // transmittance would fall below T_min blends with alpha 0, which leaves
    // every sum and T exactly as they were (w = 0 adds +/-0).
    auto blend_one = [&](int j, float al0, float4 b, float2 d) {
      const float Tn = T * (1.f - al0);
      const bool hit = !done && al0 >= amin;
      const bool bl = hit && Tn >= tmin;
      done = done || (hit && !bl);
      cm |= static_cast<uint32_t>(bl) << j;
      const float w = bl ? al0 * T : 0.f;
      const float4 e3 = my[kColourSlot<LOSS>][j];
      const float2 w2 = make_float2(w, w);
      if (!GEO) Crg = __ffma2_rn(w2, make_float2(e3.x, e3.y), Crg);
      Cbn = __ffma2_rn(w2, make_float2(e3.z, e3.w), Cbn);   // (b, n0); b is 0 in GEO records
      N12 = __ffma2_rn(w2, make_float2(b.z, b.w), N12);
      // the splat's planar depth here (Eq. 4): for Eq. 23 at every contributor;
      // otherwise only the median's, after the walk
      float dk = 0.f;
      if (LOSS) {
        const float4 e2 = my[2][j];
        dk = e2.z + e2.x * d.x + e2.y * d.y;
        if (bl && last < 0) d0 = dk;
        const float sd = dk - d0;
        Ws += w;
        S1 += w * sd;
        S2 += w * sd * sd;
      }
      if (bl && med < 0 && Tn <= tmed) {
        med = c0 + j;
        if (LOSS) depth = dk;
      }
      if (bl) {
        last = c0 + j;
        T = Tn;
      }
    };
    // tested pairs: the records that pass the block test, for a pixel still
    // unfinished at the chunk's start
    if (!done) evals += __popc(m);
    auto alpha_of = [&](int j, float4& b, float2& d) {
      const float4 a = my[0][j];
      b = my[1][j];
      d = __fadd2_rn(make_float2(a.x, a.y), nfp);   // (dx, dy)
      return fminf(amax, __fmul_rn(b.y, ex2(-splat_s(a.z, a.w, b.x, d, __fmul2_rn(d, d)))));
    };
    while (m & (m - 1)) {   // two or more records left
      const int jA = __ffs(m) - 1;
      m &= m - 1;
      const int jB = __ffs(m) - 1;
      m &= m - 1;
      float4 bA, bB;
      float2 dA, dB;
      const float alA = alpha_of(jA, bA, dA), alB = alpha_of(jB, bB, dB);
      blend_one(jA, alA, bA, dA);
      blend_one(jB, alB, bB, dB);
    }
    if (m) {
      const int j = __ffs(m) - 1;
      float4 b;
      float2 d;
      const float al = alpha_of(j, b, d);
      blend_one(j, al, b, d);
    }
    nblend += __popc(cm);
    if (!GEO) {             // the backward replays only records some lane blended
      const uint32_t wm = __reduce_or_sync(kFull, cm);
      if (lane == 0) cmask[(c0 - range.x) >> 5] = wm;
    }
    }
    __syncwarp();           // buf[cur] is refilled two chunks later
    cur ^= 1;
  }
  cp_async_wait<0>();       // no copy may land in the buffers after the item
  __syncwarp();
  blended += nblend;
  if (!c.inside) return;
  // the median's depth (Eq. 4), unless the walk computed it (LOSS); median
  // never reached: the last contributor's
  const bool have = LOSS && med >= 0;
  if (med < 0) med = last;
  if (!have && med >= 0 && GS_IN_BOUNDS(hdr, pval[med] < L.E, BS_FWD_ENTRY, pval[med])) {
    const float4* r = rec + 4 * (int64_t)pval[med];
    const float4 a = r[0], e2 = r[2];
    depth = e2.z + e2.x * (a.x - fpx) + e2.y * (a.y - fpy);
  }
  const int64_t HW = (int64_t)c.W * c.H;
  const int64_t p = c.pix_local;
  if (!GEO && maps.color) {
    float* col = maps.color + 3 * c.pix_base;
    col[p] = Crg.x; col[HW + p] = Crg.y; col[2 * HW + p] = Cbn.x;
  }
  if (maps.normal) {
    float* nrm = maps.normal + 3 * c.pix_base;
    nrm[p] = Cbn.y; nrm[HW + p] = N12.x; nrm[2 * HW + p] = N12.y;
  }
  if (maps.alpha) maps.alpha[c.pix] = 1.f - T;
  if (maps.depth) maps.depth[c.pix] = depth;
  if (GEO) return;   // forward-only geometry: no backward state
  at<float>(ws, L.px_T)[c.pix] = T;
  at<int>(ws, L.px_last)[c.pix] = last;
  at<int>(ws, L.px_med)[c.pix] = med;
  if (LOSS) {
    if (maps.dist) maps.dist[c.pix] = 2.f * (Ws * S2 - S1 * S1);
    float* P = at<float>(ws, L.px_loss);
    const int64_t NP = L.NPIX;
    P[LP_MEAN * NP + c.pix] = Ws > 0.f ? d0 + S1 / Ws : 0.f;
    P[LP_DEPTH * NP + c.pix] = depth;
    P[LP_N0 * NP + c.pix] = Cbn.y;
    P[(LP_N0 + 1) * NP + c.pix] = N12.x;
    P[(LP_N0 + 2) * NP + c.pix] = N12.y;
  }
}

// Warp reduction of the gradient slots of one or two records.  First lanes l
// and l^16 fold their values with shuffles: in each of NP pairs of float2
// slots the lower lane keeps one (P_k) and the upper lane the other (Q_k),
// each summed over both lanes; every lane computes the half it keeps and the
// half it sends, choosing them by its half of the warp as cheaply as the
// slot's form allows.  The 2 NP kept values then go to the warp's shared
// scratch as rows red[row][lane] (rows 0 .. 2NP-1: record A, 2NP .. 4NP-1:
// record B; stride kRedStride = 36 floats keeps the row stores and the 16-byte
// loads free of bank conflicts), and lane l adds the half row holding value
// s = l & 15 of record l >> 4 with four 16-byte loads: P_k for s < 2 NP, Q_k
// for 2 NP <= s < 4 NP.  The shuffle fold halves the shared-memory traffic of
// a transpose through shared memory.
//
// NP = 4 (16 values) carries the splat's planar-depth sums S sd, S sd dx,
// S sd dy; it serves Eq. 23, whose gradient reaches the depth of every
// contributor.  Without it only the median splat of a pixel receives a depth
// gradient (one splat per pixel), so NP = 3 (12 values) leaves those three
// sums out of the reduction and the few lanes whose median is the record add
// them with atomics of their own.
constexpr int kRedStride = 36;

template <int NP>
__device__ inline void fold_store(const float2 (&keep)[NP], const float2 (&send)[NP], float* __restrict__ rows) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float2 recv = make_float2(__shfl_xor_sync(kFull, send[k].x, 16), __shfl_xor_sync(kFull, send[k].y, 16));
    const float2 h = __fadd2_rn(keep[k], recv);
    rows[(2 * k) * kRedStride + lane] = h.x;
    rows[(2 * k + 1) * kRedStride + lane] = h.y;
  }
}

// The record slot that reduced value s = lane & 15 adds to (4 bits per value).
// NP = 4: P0 = gs d -> (U, V); P1 = w (dC0, dC1) -> (R, G); P2 = (gs dy^2, gs)
// -> (CC, O); P3 = sd d -> (P0, P1); Q0 = gs dx d -> (CA, CB); Q1 = w (dC2, dN0)
// -> (B, N0); Q2 = (0, sd) -> (CUT, Z); Q3 = w (dN1, dN2) -> (N1, N2).
// NP = 3: P0, P1, P2, Q0, Q1 as above; Q2 = w (dN1, dN2) -> (N1, N2); values
// 12-15 are unused.  Value s is read from row (s & 3) of half s >> 2 for s < 8
// and from row 4 + (s & 1) of half (s >> 1) & 1 for 8 <= s < 12, so that each
// group of 8 lanes reads 8 distinct 16-byte bank groups (row r of half q
// starts at bank group (9 r + 4 q) mod 8).
constexpr unsigned long long kFoldSlots4 = 0xba76fe329854dc10ull;
constexpr unsigned long long kFoldSlots3 = 0x6666ba54fe32dc10ull;

template <int NP>
__device__ inline float reduce_rows(const float* __restrict__ red) {
  const int lane = threadIdx.x & 31, s = lane & 15;
  if (s >= 4 * NP) return 0.f;
  int q, row;   // the half (P or Q) and the row of value s
  if (NP == 4) {
    q = s >> 3;
    row = s & 7;
  } else {
    q = s < 8 ? s >> 2 : (s >> 1) & 1;
    row = s < 8 ? s & 3 : 4 + (s & 1);
  }
  const float4* r =
      reinterpret_cast<const float4*>(red + ((lane >> 4) * 2 * NP + row) * kRedStride + q * 16);
  float2 h[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 a = r[i];
    h[i] = __fadd2_rn(make_float2(a.x, a.y), make_float2(a.z, a.w));
  }
  const float2 t = __fadd2_rn(__fadd2_rn(h[0], h[1]), __fadd2_rn(h[2], h[3]));
  return t.x + t.y;
}
// A staged 16-byte record piece read by every lane of the warp (one address),
// as two 8-byte shared loads: in the backward's visit that takes fewer
// shared-memory cycles than one 16-byte load (0.5627 -> 0.5557 ms; the
// forward's evaluation loop is no faster that way).  The backward also takes
// a replayed record's entry index from the lane that staged it by a shuffle
// instead of from shared memory (0.5557 -> 0.5506 ms).
__device__ inline float4 lds_bcast2(const float4* q) {
  float4 r;
  const uint32_t ad = (uint32_t)__cvta_generic_to_shared(q);
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(ad));
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+8];" : "=f"(r.z), "=f"(r.w) : "r"(ad));
  return r;
}

// One backward work item (same decomposition as fwd_item): the warp replays
// its pixels from their last contributors toward the front of the list.
template <bool LOSS>
__device__ inline void bwd_item(const FrameDev* __restrict__ fd, void* __restrict__ ws, const Layout& L,
                                const gs_map_grads& g, int tile, int sub, float4 (*my)[32],
                                float* my_red,
                                uint32_t& evals) {
  const TileCtx c = tile_ctx(fd, tile, sub);
  const int2 range = at<int2>(ws, L.ranges)[tile];
  const uint32_t* pval = at<uint32_t>(ws, L.pval_final);
  const float4* rec = at<float4>(ws, L.rec);
  float* grad = at<float>(ws, L.grad2d);
  Header* hdr = at<Header>(ws, L.hdr);   // (bounds checks of a GS_DEBUG build)
  const float amin = fd->alpha_min, amax = fd->alpha_max;
  const float fpx = c.px + 0.5f, fpy = c.py + 0.5f;
  const int lane = threadIdx.x & 31;
  const SubRect R = sub_rect(c.x0, c.y0, fd->tile_w / kSubW, sub);

  float Tf = 1.f;
  int last = -1, med = -1;
  float dC[3] = {0.f, 0.f, 0.f}, dN[3] = {0.f, 0.f, 0.f}, dA = 0.f, dD = 0.f;
  float c4 = 0.f, dmean = 0.f;   // Eq. 23 (LOSS only)
  if (c.inside) {
    Tf = at<float>(ws, L.px_T)[c.pix];
    last = at<int>(ws, L.px_last)[c.pix];
    med = at<int>(ws, L.px_med)[c.pix];
    const int64_t HW = (int64_t)c.W * c.H, p = c.pix_local;
    if (g.dcolor) {
      const float* d = g.dcolor + 3 * c.pix_base;
      dC[0] = d[p]; dC[1] = d[HW + p]; dC[2] = d[2 * HW + p];
    }
    if (g.dnormal) {
      const float* d = g.dnormal + 3 * c.pix_base;
      dN[0] = d[p]; dN[1] = d[HW + p]; dN[2] = d[2 * HW + p];
    }
    if (g.dalpha) dA = g.dalpha[c.pix];
    if (g.ddepth) dD = g.ddepth[c.pix];
    if (LOSS) {
      const float* P = at<float>(ws, L.px_loss);
      const int64_t NP = L.NPIX;
      if (g.dnloss) {   // Eq. 24 through the alpha, depth and normal maps
        dA += P[LP_DA * NP + c.pix];
        dD += P[LP_DD * NP + c.pix];
#pragma unroll
        for (int k = 0; k < 3; ++k) dN[k] += P[(LP_DN0 + k) * NP + c.pix];
      }
      if (g.ddist) {    // Eq. 23, weights constant: dL/dd_k = 4 w_k W (d_k - mean)
        c4 = 4.f * g.ddist[c.pix] * (1.f - Tf);
        dmean = P[LP_MEAN * NP + c.pix];
      }
    }
  }
  const int wmax = __reduce_max_sync(kFull, last);
  constexpr int NP = LOSS ? 4 : 3;   // float2 pairs per lane in the fold
  if (!LOSS && med >= 0 && dD != 0.f) {
    // Without Eq. 23 the depth map's gradient reaches the pixel's median splat
    // only (a contributor by definition): d = z_c + p . Delta there, so its
    // depth sums gain dD (1, dx, dy), added here once per pixel instead of in
    // every visit's reduction
    const uint32_t e = pval[med];
    if (GS_IN_BOUNDS(hdr, e < L.E, BS_BWD_ENTRY, e)) {
      const float4 a = rec[4 * (int64_t)e];
      float* row = grad + (int64_t)e * kRecFloats;
      atomicAdd(row + G_Z, dD);
      atomicAdd(row + G_P0, dD * (a.x - fpx));
      atomicAdd(row + G_P1, dD * (a.y - fpy));
    }
  }

  float T = Tf;
  const float dATf = dA * Tf;
  // running "behind" sums of (r, g, b, n0, n1, n2) and the upstream of the same six, as pairs
  float2 S01 = make_float2(0.f, 0.f), S23 = make_float2(0.f, 0.f), S45 = make_float2(0.f, 0.f);
  const float2 U01 = make_float2(dC[0], dC[1]), U23 = make_float2(dC[2], dN[0]), U45 = make_float2(dN[1], dN[2]);
  // the fold's pairs: lanes 0-15 keep P_k, lanes 16-31 Q_k (kFoldSlots4 / kFoldSlots3)
  const bool hi = lane & 16;
  const float2 Ukeep = hi ? U23 : U01, Usend = hi ? U01 : U23;
  const int slot = (int)(((LOSS ? kFoldSlots4 : kFoldSlots3) >> (4 * (lane & 15))) & 15u);
  const float2 nfp = make_float2(-fpx, -fpy);
  // the forward's per-chunk masks name the records some lane of this block
  // blended; the others have zero gradient here and are not replayed
  const uint32_t* cmask = at<uint32_t>(ws, L.cmask) + (int64_t)sub * L.cmask_words + (range.x >> 5) + tile;
  // the mask word and this lane's entry of the next chunk are loaded one chunk
  // ahead, so a chunk's staging waits for one round trip to L2, not three
  const int k_first = wmax >= range.x ? (wmax - range.x) >> 5 : -1;
  uint32_t wm_next = 0, e_next = 0;
  if (k_first >= 0) {
    wm_next = cmask[k_first];
    const int c = range.x + 32 * k_first + lane;
    e_next = c < range.y ? pval[c] : 0u;
  }
  for (int k = k_first; k >= 0; --k) {
    const uint32_t wm = wm_next, e_cur = e_next;
    if (k > 0) {
      wm_next = cmask[k - 1];
      e_next = pval[range.x + 32 * (k - 1) + lane];   // a full chunk: every chunk but the last is
    }
    if (wm == 0) continue;
    const int c0 = range.x + 32 * k;
    if ((wm >> lane) & 1u) {   // copies straight to shared memory, no registers
      if (GS_IN_BOUNDS(hdr, e_cur < L.E, BS_BWD_ENTRY, e_cur))
        stage_record<LOSS, false>(my, lane, rec + 4 * (int64_t)e_cur);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    // One visit: the splat's gradient at this lane's pixel, stored as 16 rows
    // of the reduction scratch.  Branch-free: every lane evaluates the splat;
    // lanes that do not blend it (behind their last contributor, or alpha below
    // alpha_min) take alpha = 0, which leaves T and the running sums unchanged
    // and zeroes every gradient.
    auto visit = [&](int j, float* rows) {
      const int idx = c0 + j;
      // slots as pairs: (U,V) (CA,CB) (CC,O) (CUT,Z) (P0,P1) (N1,N2) (R,G) (B,N0); the
      // first seven hold sums that are linear in the splat's conic, p and o:
      // (S gs dx, S gs dy) (S gs dx^2, S gs dx dy) (S gs dy^2, S gs) (0, S sd)
      // (S sd dx, S sd dy), with gs = dL/dsigma and sd = dL/dd; the preprocess
      // backward applies the constants once per entry.  They are folded in the
      // pairs (P_k, Q_k) of kFoldSlots4 / kFoldSlots3: this lane keeps one half,
      // sends the other
      float2 keep[NP], send[NP];
      const bool live = idx <= last;
      // the depth plane (p, z) only for Eq. 23
      const float4 a = lds_bcast2(&my[0][j]), b = lds_bcast2(&my[1][j]), e3 = lds_bcast2(&my[kColourSlot<LOSS>][j]);
      const float4 e2 = LOSS ? my[2][j] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float2 d = __fadd2_rn(make_float2(a.x, a.y), nfp);     // (dx, dy)
      const float dx = d.x, dy = d.y;
      const float2 d2 = __fmul2_rn(d, d);                           // (dx^2, dy^2)
      const float sl = splat_s(a.z, a.w, b.x, d, d2);
      const float G = ex2(-sl);
      const float raw = __fmul_rn(b.y, G);
      const float al0 = fminf(amax, raw);
      const bool contrib = live && al0 >= amin;
      const float al = contrib ? al0 : 0.f;
      const float ia = __fdividef(1.f, 1.f - al);
      T *= ia;                           // transmittance in front of this splat
      const float w = al * T;
      const float2 w2 = make_float2(w, w);
      // colour and normal: (rgb, n) and the upstream (dC, dN) as three pairs
      const float2 x0 = make_float2(e3.x, e3.y), x1 = make_float2(e3.z, e3.w), x2 = make_float2(b.z, b.w);
      keep[1] = __fmul2_rn(w2, Ukeep);   // w (dC0, dC1) | w (dC2, dN0)
      send[1] = __fmul2_rn(w2, Usend);
      // (x - S) enters both dL/dalpha and the update S += alpha (x - S)
      const float2 q0 = __fadd2_rn(x0, make_float2(-S01.x, -S01.y));
      const float2 q1 = __fadd2_rn(x1, make_float2(-S23.x, -S23.y));
      const float2 q2 = __fadd2_rn(x2, make_float2(-S45.x, -S45.y));
      float2 acc = __fmul2_rn(q0, U01);
      acc = __ffma2_rn(q1, U23, acc);
      acc = __ffma2_rn(q2, U45, acc);
      const float2 al2 = make_float2(al, al);
      S01 = __ffma2_rn(al2, q0, S01);
      S23 = __ffma2_rn(al2, q1, S23);
      S45 = __ffma2_rn(al2, q2, S45);
      const float dal = contrib ? T * (acc.x + acc.y) + dATf * ia : 0.f;
      // d = z_c + p . Delta (Eq. 4): the median splat, and Eq. 23 with the weights constant
      const float2 qn = __fmul2_rn(w2, U45);   // w (dN1, dN2)
      // alpha = o G below the clamp: dL/dsigma = -dL/dalpha alpha
      const float gs = raw <= amax ? -dal * al : 0.f;
      const float gsx = gs * dx;
      const float sk = hi ? gsx : gs, ss = hi ? gs : gsx;
      keep[0] = __fmul2_rn(make_float2(sk, sk), d);   // gs d | gs dx d
      send[0] = __fmul2_rn(make_float2(ss, ss), d);
      const float gy2 = gs * d2.y;
      if constexpr (LOSS) {
        const float sd = ((contrib && idx == med) ? dD : 0.f) + c4 * w * ((e2.z + e2.x * dx + e2.y * dy) - dmean);
        const float2 p3 = __fmul2_rn(make_float2(sd, sd), d);
        keep[3] = hi ? qn : p3;            // sd d | w (dN1, dN2)
        send[3] = hi ? p3 : qn;
        keep[2] = make_float2(hi ? 0.f : gy2, hi ? sd : gs);   // (gs dy^2, gs) | (0, sd)
        send[2] = make_float2(hi ? gy2 : 0.f, hi ? gs : sd);
      } else {
        const float2 p2 = make_float2(gy2, gs);
        keep[NP - 1] = hi ? qn : p2;       // (gs dy^2, gs) | w (dN1, dN2)
        send[NP - 1] = hi ? p2 : qn;
      }
      fold_store<NP>(keep, send, rows);
    };
    // some lane blends every replayed record (the forward's mask), so every
    // visit reduces.  Records go back to front, two per round where possible:
    // their evaluations overlap and one reduction and one atomic instruction
    // serve both.
    {   // evaluations of this lane: replayed records at or before its last contributor
      const int lj = last - c0;
      evals += lj < 0 ? 0u : __popc(lj >= 31 ? wm : wm & ((2u << lj) - 1u));
    }
    unsigned m = wm;
    while (m) {
      const int jA = 31 - __clz(m);
      m &= ~(1u << jA);
      const int jB = m ? 31 - __clz(m) : -1;
      visit(jA, my_red);
      if (jB >= 0) {
        m &= ~(1u << jB);
        visit(jB, my_red + 2 * NP * kRedStride);
      }
      __syncwarp();
      const float s = reduce_rows<NP>(my_red);   // lanes 16-31 read stale rows without jB
      __syncwarp();   // the scratch is rewritten by the next round
      const int j = lane < 16 ? jA : jB;
      const uint32_t ej = __shfl_sync(kFull, e_cur, j & 31);   // record j's entry, held by lane j
      if (j >= 0 && slot != G_UNUSED && s != 0.f && GS_IN_BOUNDS(hdr, ej < L.E, BS_BWD_ENTRY, ej))
        atomicAdd(grad + (int64_t)ej * kRecFloats + slot, s);
    }
    __syncwarp();
  }
}

// Persistent kernels: every warp pulls work items (tile, 8x4 block) from an
// atomic counter until the frame is done, so no warp waits for another.  Items
// come in the binning's work order (tiles with the longest lists first), so the
// last items handed out are short and the tail is small.  The result does not depend on which warp takes
// which item (each pixel is computed by exactly one warp).
constexpr int kRenderThreads = 256;
constexpr int kRenderBlocksPerSm = 3;

// The forward's staging buffers: per warp two buffers of CH records in
// kSlots<LOSS> 16-byte slots (dynamic shared memory, fwd_smem_bytes).
template <bool LOSS, int CH>
constexpr size_t fwd_smem_bytes() {
  return size_t(kRenderThreads / 32) * 2 * CH * kSlots<LOSS> * sizeof(float4);
}

template <bool LOSS, bool GEO, int CH>
__global__ void __launch_bounds__(kRenderThreads, kRenderBlocksPerSm)
k_render_fwd(const FrameDev* __restrict__ fd, void* __restrict__ ws, Layout L, gs_maps maps, int subs,
             int n_items) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) float4 s_dyn[];
  Header* hdr = at<Header>(ws, L.hdr);
  if (hdr->status == GS_ERR_CAPACITY) return;
  using Buf = float4[CH / 32][kSlots<LOSS>][32];
  Buf* buf = reinterpret_cast<Buf*>(s_dyn) + 2 * (threadIdx.x >> 5);
  const int* order = at<int>(ws, L.tile_order);
  const int lane = threadIdx.x & 31;
  uint32_t evals = 0, blended = 0;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&hdr->work_fwd, 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= n_items) break;
    fwd_item<LOSS, GEO, CH>(fd, ws, L, maps, order[item / subs], item % subs, buf, evals, blended);
    __syncwarp();
  }
  count_evals(evals, &hdr->n_evals_fwd);
  count_evals(blended, &hdr->n_blend);
}

template <bool LOSS>
__global__ void __launch_bounds__(kRenderThreads, kRenderBlocksPerSm)
k_render_bwd(const FrameDev* __restrict__ fd, void* __restrict__ ws, Layout L, gs_map_grads g, int subs,
             int n_items) {
  pdl_wait();
  pdl_trigger();
  __shared__ float4 s_rec[kRenderThreads / 32][kSlots<LOSS>][32];
  __shared__ __align__(16) float s_red[kRenderThreads / 32][4 * (LOSS ? 4 : 3) * kRedStride];
  Header* hdr = at<Header>(ws, L.hdr);
  BwdCounters* bc = at<BwdCounters>(ws, L.bwdcnt);
  if (hdr->status == GS_ERR_CAPACITY) return;
  float4 (*my)[32] = s_rec[threadIdx.x >> 5];
  const int* order = at<int>(ws, L.tile_order);
  const int lane = threadIdx.x & 31;
  uint32_t evals = 0;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(&bc->work_bwd, 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= n_items) break;
    bwd_item<LOSS>(fd, ws, L, g, order[item / subs], item % subs, my, s_red[threadIdx.x >> 5], evals);
    __syncwarp();
  }
  count_evals(evals, &bc->n_evals_bwd);
}

// A resident wave of blocks for a persistent kernel.
template <typename K>
static int persistent_grid(K kernel, int n_items, size_t smem = 0) {
  int dev = 0, sms = 148, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRenderThreads, smem);
  const int need = (n_items + kRenderThreads / 32 - 1) / (kRenderThreads / 32);
  // three resident blocks (24 warps) per SM measured fastest for both kernels:
  // a fourth adds issue contention and takes L1 capacity from the record reads
  const int blocks = per_sm < 1 ? 1 : (per_sm < kRenderBlocksPerSm ? per_sm : kRenderBlocksPerSm);
  int g = sms * blocks;
  return g < need ? g : (need < 1 ? 1 : need);
}

template <bool LOSS, bool GEO, int CH>
static cudaError_t launch_fwd_variant(const FrameDev* fd, void* ws, const Layout& L, const gs_maps& maps, int subs,
                                      int n_items, cudaStream_t s) {
  constexpr size_t smem = fwd_smem_bytes<LOSS, CH>();
  if (smem > 48 * 1024) {   // above the default dynamic limit: opt in (a host-side attribute)
    const cudaError_t e =
        cudaFuncSetAttribute(k_render_fwd<LOSS, GEO, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  launch_pdl(k_render_fwd<LOSS, GEO, CH>, persistent_grid(k_render_fwd<LOSS, GEO, CH>, n_items, smem),
             kRenderThreads, smem, s, fd, ws, L, maps, subs, n_items);
  return cudaGetLastError();
}

cudaError_t launch_render_fwd(void* ws, const Layout& L, const FrameDev& hf, const gs_maps& maps,
                              cudaStream_t s) {
  const FrameDev* fd = at<FrameDev>(ws, L.frame);
  Header* hdr = at<Header>(ws, L.hdr);
  cudaError_t err = cudaMemsetAsync(&hdr->n_evals_fwd, 0, 24, s);   // n_evals_fwd, n_blend, work_fwd
  if (err != cudaSuccess) return err;
  if (L.T == 0) return cudaSuccess;
  const int subs = hf.tile_w * hf.tile_h / 32;
  const int n_items = (int)L.T * subs;
  const bool big = hf.batch == 64;
  if (hf.geometry_only)
    return big ? launch_fwd_variant<false, true, 64>(fd, ws, L, maps, subs, n_items, s)
               : launch_fwd_variant<false, true, 32>(fd, ws, L, maps, subs, n_items, s);
  if (hf.losses)
    return big ? launch_fwd_variant<true, false, 64>(fd, ws, L, maps, subs, n_items, s)
               : launch_fwd_variant<true, false, 32>(fd, ws, L, maps, subs, n_items, s);
  return big ? launch_fwd_variant<false, false, 64>(fd, ws, L, maps, subs, n_items, s)
             : launch_fwd_variant<false, false, 32>(fd, ws, L, maps, subs, n_items, s);
}

__global__ void __launch_bounds__(256)
k_bwd_clear(const uint32_t* __restrict__ vis, const unsigned long long* n_vis_ptr, int64_t E,
            float4* __restrict__ grad2d, BwdCounters* bc) {
  pdl_wait();
  pdl_trigger();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    bc->n_evals_bwd = 0;
    bc->work_bwd = 0;
  }
  const int64_t n = clamp_count(n_vis_ptr, E);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 4 * n; i += (int64_t)gridDim.x * blockDim.x)
    grad2d[4 * (int64_t)vis[i >> 2] + (i & 3)] = make_float4(0.f, 0.f, 0.f, 0.f);
}

cudaError_t launch_render_bwd(void* ws, const Layout& L, const FrameDev& hf, const gs_map_grads& g,
                              cudaStream_t s) {
  const FrameDev* fd = at<FrameDev>(ws, L.frame);
  Header* hdr = at<Header>(ws, L.hdr);
  // zero the backward counters and the 2D-gradient rows of the visible entries
  // (the only rows the compositing accumulates into and the preprocess
  // backward reads), 4 threads per 64-byte row
  {
    const int g = (int)std::min<int64_t>(std::max<int64_t>((4 * L.E + 255) / 256, 1), 148 * 16);
    launch_pdl(k_bwd_clear, g, 256, 0, s, at<uint32_t>(ws, L.vval[0]), &hdr->n_vis, L.E, at<float4>(ws, L.grad2d),
               at<BwdCounters>(ws, L.bwdcnt));
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (L.T == 0) return cudaSuccess;
  const int subs = hf.tile_w * hf.tile_h / 32;
  const int n_items = (int)L.T * subs;
  if (hf.losses && (g.ddist || g.dnloss))
    launch_pdl(k_render_bwd<true>, persistent_grid(k_render_bwd<true>, n_items), kRenderThreads, 0, s, fd, ws, L, g,
               subs, n_items);
  else
    launch_pdl(k_render_bwd<false>, persistent_grid(k_render_bwd<false>, n_items), kRenderThreads, 0, s, fd, ws, L,
               g, subs, n_items);
  return cudaGetLastError();
}

}  // namespace gs
