// Normal consistency (Eq. 24): forward map and backward to the rendered maps.
//
// The depth map is back-projected to camera space, P(x, y) = D(x, y) r(x, y)
// with r = ((x + 1/2 - cx)/fx, (y + 1/2 - cy)/fy, 1), and its normal is taken
// from central differences: a = P(x+1, y) - P(x-1, y), b = P(x, y+1) - P(x, y-1),
// c = b x a (pointing toward the camera), n~ = c / |c|.  n~ is defined where
// the pixel is not on its view's border, the alpha of the pixel and of its four
// neighbours is > 0, and |c| > 0.  Since sum_i w_i = alpha and sum_i w_i n_i is
// the normal map N,
//     L_n = sum_i w_i (1 - n_i . n~) = alpha - N . n~.
//
// Backward, with g = dL/dL_n at a centre where n~ is defined:
//     dL/dalpha = g,  dL/dN = -g n~,
//     dL/dc = (I - n~ n~^T)(-g N) / |c|,  dL/da = dL/dc x b,  dL/db = a x dL/dc,
// and dL/dD(q) = r(q) . (da(q - e_x) - da(q + e_x) + db(q - e_y) - db(q + e_y)),
// gathered from the four centres whose stencils touch q.  One 32x8 block
// computes the (da, db) of its 34x10 centres (its pixels plus a one-pixel ring)
// in shared memory from a 36x12 window of depths and transmittances, then each
// thread gathers its pixel.  The results are stored as per-pixel map
// gradients that the compositing backward adds to the caller's.
#include "gs_internal.cuh"

namespace gs {

constexpr int kLX = 32, kLY = 8;                      // pixels per block
constexpr int kCX = kLX + 2, kCY = kLY + 2;           // centres (with the ring)
constexpr int kDX = kLX + 4, kDY = kLY + 4;           // depth window

// Blocks of every view, prefix-summed (host-filled, passed by value).
struct LossGrid {
  int32_t blk_off[GS_MAX_VIEWS + 1];
  int32_t bx[GS_MAX_VIEWS];   // blocks per row of view v
};

struct Stencil {
  float a[3], b[3], n[3], inv;   // differences, unit normal, 1/|c|
  bool ok;
};

// n~ at a centre from the depths of its four neighbours (left, right, up, down)
// and the ray components at x-1, x, x+1 and y-1, y, y+1.
__device__ inline Stencil stencil(float Dl, float Dr, float Du, float Dd, float rxm, float rx0, float rxp,
                                  float rym, float ry0, float ryp, bool alive) {
  Stencil s;
  s.a[0] = Dr * rxp - Dl * rxm;
  s.a[1] = (Dr - Dl) * ry0;
  s.a[2] = Dr - Dl;
  s.b[0] = (Dd - Du) * rx0;
  s.b[1] = Dd * ryp - Du * rym;
  s.b[2] = Dd - Du;
  const float c0 = s.b[1] * s.a[2] - s.b[2] * s.a[1];
  const float c1 = s.b[2] * s.a[0] - s.b[0] * s.a[2];
  const float c2 = s.b[0] * s.a[1] - s.b[1] * s.a[0];
  const float nn = c0 * c0 + c1 * c1 + c2 * c2;
  s.ok = alive && nn > 0.f;
  s.inv = s.ok ? rsqrtf(nn) : 0.f;
  s.n[0] = c0 * s.inv;
  s.n[1] = c1 * s.inv;
  s.n[2] = c2 * s.inv;
  return s;
}

__device__ inline float ray_x(const ViewDev& V, int x) { return ((float)x + 0.5f - V.cx) / V.fx; }
__device__ inline float ray_y(const ViewDev& V, int y) { return ((float)y + 0.5f - V.cy) / V.fy; }

__device__ inline int block_view(const LossGrid& G, int n_views, int b) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (G.blk_off[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Forward: one thread per pixel, neighbours read through the cache.
__global__ void __launch_bounds__(kLX * kLY)
k_nloss_fwd(const FrameDev* __restrict__ fd, void* __restrict__ ws, Layout L, LossGrid G, float* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  if (at<Header>(ws, L.hdr)->status == GS_ERR_CAPACITY) return;   // nothing was rendered
  const int v = block_view(G, fd->n_views, blockIdx.x);
  const ViewDev& V = fd->views[v];
  const int b = blockIdx.x - G.blk_off[v];
  const int x = (b % G.bx[v]) * kLX + (threadIdx.x & (kLX - 1));
  const int y = (b / G.bx[v]) * kLY + (threadIdx.x / kLX);
  const int W = V.width, H = V.height;
  if (x >= W || y >= H) return;
  const int64_t base = fd->pix_off[v];
  const int64_t p = base + (int64_t)y * W + x;
  const float* Tm = at<float>(ws, L.px_T);
  const float* P = at<float>(ws, L.px_loss);
  const int64_t NP = L.NPIX;
  float Ln = 0.f;
  if (x > 0 && y > 0 && x < W - 1 && y < H - 1) {
    const bool alive = __ldg(Tm + p) < 1.f && __ldg(Tm + p - 1) < 1.f && __ldg(Tm + p + 1) < 1.f &&
                       __ldg(Tm + p - W) < 1.f && __ldg(Tm + p + W) < 1.f;
    const float* D = P + LP_DEPTH * NP;
    const Stencil s = stencil(__ldg(D + p - 1), __ldg(D + p + 1), __ldg(D + p - W), __ldg(D + p + W),
                              ray_x(V, x - 1), ray_x(V, x), ray_x(V, x + 1), ray_y(V, y - 1), ray_y(V, y),
                              ray_y(V, y + 1), alive);
    if (s.ok) {
      const float Nd = P[LP_N0 * NP + p] * s.n[0] + P[(LP_N0 + 1) * NP + p] * s.n[1] +
                       P[(LP_N0 + 2) * NP + p] * s.n[2];
      Ln = (1.f - Tm[p]) - Nd;
    }
  }
  out[p] = Ln;
}

// Backward: stores dL/dD, dL/dN and dL/dalpha of every pixel in the loss planes.
__global__ void __launch_bounds__(kLX * kLY)
k_nloss_bwd(const FrameDev* __restrict__ fd, void* __restrict__ ws, Layout L, LossGrid G,
            const float* __restrict__ gin) {
  pdl_wait();
  pdl_trigger();
  __shared__ float sD[kDY][kDX];
  __shared__ unsigned char sA[kDY][kDX];
  __shared__ float sG[kCY][kCX][6];   // da, db of each centre (0 where n~ is undefined)
  if (at<Header>(ws, L.hdr)->status == GS_ERR_CAPACITY) return;   // nothing was rendered
  const int v = block_view(G, fd->n_views, blockIdx.x);
  const ViewDev& V = fd->views[v];
  const int b = blockIdx.x - G.blk_off[v];
  const int X0 = (b % G.bx[v]) * kLX, Y0 = (b / G.bx[v]) * kLY;
  const int W = V.width, H = V.height;
  const int64_t base = fd->pix_off[v];
  const float* Tm = at<float>(ws, L.px_T);
  float* P = at<float>(ws, L.px_loss);
  const int64_t NP = L.NPIX;
  const float* D = P + LP_DEPTH * NP;

  // depth window [X0-2, X0+kLX+1] x [Y0-2, Y0+kLY+1]; outside the view: dead
  for (int i = threadIdx.x; i < kDX * kDY; i += blockDim.x) {
    const int wx = i % kDX, wy = i / kDX;
    const int x = X0 - 2 + wx, y = Y0 - 2 + wy;
    float d = 0.f;
    unsigned char al = 0;
    if (x >= 0 && y >= 0 && x < W && y < H) {
      const int64_t p = base + (int64_t)y * W + x;
      d = __ldg(D + p);
      al = __ldg(Tm + p) < 1.f;
    }
    sD[wy][wx] = d;
    sA[wy][wx] = al;
  }
  __syncthreads();

  // centres [X0-1, X0+kLX] x [Y0-1, Y0+kLY]
  for (int i = threadIdx.x; i < kCX * kCY; i += blockDim.x) {
    const int cx = i % kCX, cy = i / kCX;
    const int x = X0 - 1 + cx, y = Y0 - 1 + cy;
    const int wx = cx + 1, wy = cy + 1;   // window coordinates of the centre
    float* o = sG[cy][cx];
    o[0] = o[1] = o[2] = o[3] = o[4] = o[5] = 0.f;
    const bool own = cx >= 1 && cx <= kLX && cy >= 1 && cy <= kLY && x < W && y < H;
    const bool interior = x > 0 && y > 0 && x < W - 1 && y < H - 1;
    float gdA = 0.f, gdN[3] = {0.f, 0.f, 0.f};
    if (interior) {
      const bool alive = sA[wy][wx] && sA[wy][wx - 1] && sA[wy][wx + 1] && sA[wy - 1][wx] && sA[wy + 1][wx];
      const Stencil s = stencil(sD[wy][wx - 1], sD[wy][wx + 1], sD[wy - 1][wx], sD[wy + 1][wx],
                                ray_x(V, x - 1), ray_x(V, x), ray_x(V, x + 1), ray_y(V, y - 1), ray_y(V, y),
                                ray_y(V, y + 1), alive);
      if (s.ok) {
        const int64_t p = base + (int64_t)y * W + x;
        const float g = __ldg(gin + p);
        const float N[3] = {P[LP_N0 * NP + p], P[(LP_N0 + 1) * NP + p], P[(LP_N0 + 2) * NP + p]};
        // dL/dn~ = -g N, projected onto the tangent plane of n~ and scaled by 1/|c|
        const float dn[3] = {-g * N[0], -g * N[1], -g * N[2]};
        const float pr = dn[0] * s.n[0] + dn[1] * s.n[1] + dn[2] * s.n[2];
        const float dc[3] = {(dn[0] - pr * s.n[0]) * s.inv, (dn[1] - pr * s.n[1]) * s.inv,
                             (dn[2] - pr * s.n[2]) * s.inv};
        // c = b x a:  dL/da = dc x b,  dL/db = a x dc
        o[0] = dc[1] * s.b[2] - dc[2] * s.b[1];
        o[1] = dc[2] * s.b[0] - dc[0] * s.b[2];
        o[2] = dc[0] * s.b[1] - dc[1] * s.b[0];
        o[3] = s.a[1] * dc[2] - s.a[2] * dc[1];
        o[4] = s.a[2] * dc[0] - s.a[0] * dc[2];
        o[5] = s.a[0] * dc[1] - s.a[1] * dc[0];
        gdA = g;
        gdN[0] = -g * s.n[0];
        gdN[1] = -g * s.n[1];
        gdN[2] = -g * s.n[2];
      }
    }
    if (own) {
      const int64_t p = base + (int64_t)y * W + x;
      P[LP_DA * NP + p] = gdA;
      P[LP_DN0 * NP + p] = gdN[0];
      P[(LP_DN0 + 1) * NP + p] = gdN[1];
      P[(LP_DN0 + 2) * NP + p] = gdN[2];
    }
  }
  __syncthreads();

  const int lx = threadIdx.x & (kLX - 1), ly = threadIdx.x / kLX;
  const int x = X0 + lx, y = Y0 + ly;
  if (x >= W || y >= H) return;
  const int cx = lx + 1, cy = ly + 1;   // centre coordinates of this pixel
  float s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    s[k] = sG[cy][cx - 1][k] - sG[cy][cx + 1][k] + sG[cy - 1][cx][3 + k] - sG[cy + 1][cx][3 + k];
  const float dD = s[0] * ray_x(V, x) + s[1] * ray_y(V, y) + s[2];
  P[LP_DD * NP + base + (int64_t)y * W + x] = dD;
}

static LossGrid loss_grid(const FrameDev& hf, int& n_blocks) {
  LossGrid G;
  int acc = 0;
  for (int v = 0; v < hf.n_views; ++v) {
    const ViewDev& V = hf.views[v];
    G.blk_off[v] = acc;
    G.bx[v] = (V.width + kLX - 1) / kLX;
    acc += G.bx[v] * ((V.height + kLY - 1) / kLY);
  }
  G.blk_off[hf.n_views] = acc;
  n_blocks = acc;
  return G;
}

cudaError_t launch_nloss_fwd(void* ws, const Layout& L, const FrameDev& hf, float* nloss, cudaStream_t s) {
  int nb = 0;
  const LossGrid G = loss_grid(hf, nb);
  if (nb == 0) return cudaSuccess;
  launch_pdl(k_nloss_fwd, nb, kLX * kLY, 0, s, at<FrameDev>(ws, L.frame), ws, L, G, nloss);
  return cudaGetLastError();
}

cudaError_t launch_nloss_bwd(void* ws, const Layout& L, const FrameDev& hf, const float* dnloss,
                             cudaStream_t s) {
  int nb = 0;
  const LossGrid G = loss_grid(hf, nb);
  if (nb == 0) return cudaSuccess;
  launch_pdl(k_nloss_bwd, nb, kLX * kLY, 0, s, at<FrameDev>(ws, L.frame), ws, L, G, dnloss);
  return cudaGetLastError();
}

}  // namespace gs
