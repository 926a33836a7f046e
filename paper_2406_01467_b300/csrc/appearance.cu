// Decoupled per-view appearance (Sec. 4.1.1, after VastGaussian) and Adam.
//
// Each training view owns an embedding e; a two-layer perceptron
//     h = relu(W1 e + b1),  a = W2 h + b2  (12 outputs)
// gives the colour affine c' = (I + A) c + t with A = a[0..8] row-major and
// t = a[9..11].  The loss of a view is the mean over its pixels and channels of
// |c' - target|.  Three kernels per call:
//   k_app_mlp_fwd   one block per view: a (12 floats) into the state buffer;
//   k_app_pixels    32x8 pixels per block: corrected colour, dL/dc (to the
//                   rasterizer's colour gradient), and the block's sums of
//                   dL/da and of the loss folded into the view's state with one
//                   atomic per value;
//   k_app_mlp_bwd   one block per view: back through the perceptron into the
//                   parameter gradients (atomics: views share the weights).
// k_adam is the textbook Adam update (Kingma and Ba) on a flat buffer.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gs_internal.cuh"

namespace gs {

constexpr int kAppThreads = 256;
constexpr int kAX = 32, kAY = 8;   // pixels per block of k_app_pixels

// Everything the kernels need, passed by value (under 2 KB).
struct AppDev {
  int32_t n_emb, E, H, n_views;
  int32_t idx[GS_MAX_VIEWS];          // embedding row of each view
  int32_t blk_off[GS_MAX_VIEWS + 1];  // k_app_pixels blocks before view v
  int32_t bx[GS_MAX_VIEWS];           // blocks per row of view v
  int32_t width[GS_MAX_VIEWS], height[GS_MAX_VIEWS];
  int64_t pix_off[GS_MAX_VIEWS + 1];  // pixels before view v in the concatenated maps
};

// Offsets of the parameter blocks in the flat buffer.
struct AppLayout {
  int64_t emb, W1, b1, W2, b2, total;
};

__host__ __device__ inline AppLayout app_layout(int n_emb, int E, int H) {
  AppLayout l;
  l.emb = 0;
  l.W1 = l.emb + (int64_t)n_emb * E;
  l.b1 = l.W1 + (int64_t)H * E;
  l.W2 = l.b1 + H;
  l.b2 = l.W2 + 12 * (int64_t)H;
  l.total = l.b2 + 12;
  return l;
}

// Pre-activations z = W1 e + b1 of view `view` into shared memory (threads < H).
__device__ inline void mlp_hidden(const float* __restrict__ P, const AppDev& A, const AppLayout& l, int view,
                                  float* s_e, float* s_z) {
  const float* e = P + l.emb + (int64_t)A.idx[view] * A.E;
  for (int k = threadIdx.x; k < A.E; k += blockDim.x) s_e[k] = e[k];
  __syncthreads();
  for (int j = threadIdx.x; j < A.H; j += blockDim.x) {
    const float* w = P + l.W1 + (int64_t)j * A.E;
    float acc = P[l.b1 + j];
    for (int k = 0; k < A.E; ++k) acc += w[k] * s_e[k];
    s_z[j] = acc;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kAppThreads) k_app_mlp_fwd(const float* __restrict__ P, AppDev A,
                                                             float* __restrict__ state) {
  __shared__ float s_e[256], s_z[256];
  const int v = blockIdx.x;
  const AppLayout l = app_layout(A.n_emb, A.E, A.H);
  mlp_hidden(P, A, l, v, s_e, s_z);
  float* st = state + (int64_t)GS_APPEARANCE_STATE_FLOATS * v;
  if (threadIdx.x < 12) {
    const int i = threadIdx.x;
    const float* w = P + l.W2 + (int64_t)i * A.H;
    float acc = P[l.b2 + i];
    for (int j = 0; j < A.H; ++j) acc += w[j] * fmaxf(s_z[j], 0.f);
    st[i] = acc;          // a
    st[12 + i] = 0.f;     // dL/da, summed by k_app_pixels
  }
  if (threadIdx.x == 0) st[24] = 0.f;   // loss
}

__device__ inline int app_view(const AppDev& A, int b) {
  int lo = 0, hi = A.n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.blk_off[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kAX * kAY)
k_app_pixels(AppDev A, const float* __restrict__ color, const float* __restrict__ target,
             float* __restrict__ corrected, float* __restrict__ dcolor, float* __restrict__ state) {
  __shared__ float s_red[kAX * kAY / 32][13];
  const int v = app_view(A, blockIdx.x);
  const int b = blockIdx.x - A.blk_off[v];
  const int x = (b % A.bx[v]) * kAX + (threadIdx.x & (kAX - 1));
  const int y = (b / A.bx[v]) * kAY + (threadIdx.x / kAX);
  const int W = A.width[v], H = A.height[v];
  float* st = state + (int64_t)GS_APPEARANCE_STATE_FLOATS * v;
  float a[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) a[i] = st[i];
  float part[13];
#pragma unroll
  for (int i = 0; i < 13; ++i) part[i] = 0.f;
  if (x < W && y < H) {
    const int64_t HW = (int64_t)W * H, p = (int64_t)y * W + x, base = 3 * A.pix_off[v];
    const float inv = 1.f / (3.f * (float)HW);
    float c[3], g[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = color[base + k * HW + p];
    float loss = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float cc = c[i] + a[3 * i] * c[0] + a[3 * i + 1] * c[1] + a[3 * i + 2] * c[2] + a[9 + i];
      if (corrected) corrected[base + i * HW + p] = cc;
      const float r = cc - target[base + i * HW + p];
      loss += fabsf(r);
      g[i] = (float)((r > 0.f) - (r < 0.f)) * inv;
    }
    if (dcolor) {
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dcolor[base + j * HW + p] = g[j] + a[j] * g[0] + a[3 + j] * g[1] + a[6 + j] * g[2];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int j = 0; j < 3; ++j) part[3 * i + j] = g[i] * c[j];
      part[9 + i] = g[i];
    }
    part[12] = loss * inv;
  }
  // block sums: warp shuffles, then one atomic per value and block
#pragma unroll
  for (int i = 0; i < 13; ++i)
    for (int o = 16; o > 0; o >>= 1) part[i] += __shfl_xor_sync(0xFFFFFFFFu, part[i], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 13; ++i) s_red[warp][i] = part[i];
  __syncthreads();
  if (threadIdx.x < 13) {
    float s = 0.f;
    for (int w = 0; w < kAX * kAY / 32; ++w) s += s_red[w][threadIdx.x];
    if (s != 0.f) atomicAdd(st + 12 + threadIdx.x, s);
  }
}

__global__ void __launch_bounds__(kAppThreads) k_app_mlp_bwd(const float* __restrict__ P, float* __restrict__ G,
                                                             AppDev A, const float* __restrict__ state,
                                                             float* __restrict__ loss) {
  __shared__ float s_e[256], s_z[256], s_dh[256], s_da[12];
  const int v = blockIdx.x;
  const AppLayout l = app_layout(A.n_emb, A.E, A.H);
  mlp_hidden(P, A, l, v, s_e, s_z);
  const float* st = state + (int64_t)GS_APPEARANCE_STATE_FLOATS * v;
  if (threadIdx.x < 12) s_da[threadIdx.x] = st[12 + threadIdx.x];
  if (threadIdx.x == 0 && loss) loss[v] = st[24];
  __syncthreads();
  // output layer: dW2[i][j] += da_i h_j, db2 += da; hidden: dh_j = relu'(z_j) sum_i W2[i][j] da_i
  for (int t = threadIdx.x; t < 12 * A.H; t += blockDim.x) {
    const int i = t / A.H, j = t % A.H;
    const float h = fmaxf(s_z[j], 0.f);
    if (s_da[i] != 0.f && h != 0.f) atomicAdd(G + l.W2 + t, s_da[i] * h);
  }
  if (threadIdx.x < 12 && s_da[threadIdx.x] != 0.f) atomicAdd(G + l.b2 + threadIdx.x, s_da[threadIdx.x]);
  for (int j = threadIdx.x; j < A.H; j += blockDim.x) {
    float acc = 0.f;
    if (s_z[j] > 0.f)
      for (int i = 0; i < 12; ++i) acc += P[l.W2 + (int64_t)i * A.H + j] * s_da[i];
    s_dh[j] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < A.H * A.E; t += blockDim.x) {
    const int j = t / A.E, k = t % A.E;
    const float d = s_dh[j] * s_e[k];
    if (d != 0.f) atomicAdd(G + l.W1 + t, d);
  }
  for (int j = threadIdx.x; j < A.H; j += blockDim.x)
    if (s_dh[j] != 0.f) atomicAdd(G + l.b1 + j, s_dh[j]);
  // embedding: de_k = sum_j W1[j][k] dh_j
  for (int k = threadIdx.x; k < A.E; k += blockDim.x) {
    float acc = 0.f;
    for (int j = 0; j < A.H; ++j) acc += P[l.W1 + (int64_t)j * A.E + k] * s_dh[j];
    if (acc != 0.f) atomicAdd(G + l.emb + (int64_t)A.idx[v] * A.E + k, acc);
  }
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float bc1, float bc2, int zero) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    if (zero) g[i] = 0.f;
  }
}

}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_appearance_param_count(int32_t n_embeddings, int32_t embed_dim, int32_t hidden) {
  if (n_embeddings < 1 || embed_dim < 1 || embed_dim > 256 || hidden < 1 || hidden > 256) {
    set_error(GS_ERR_INVALID_ARG, "appearance sizes: n_embeddings >= 1, embed_dim and hidden in [1, 256]");
    return 0;
  }
  return (size_t)app_layout(n_embeddings, embed_dim, hidden).total;
}

gs_status gs_appearance_fwd_bwd(const gs_frame* frame, const gs_appearance* app, const int32_t* embed_index,
                                const float* color, const float* target, float* corrected, float* dcolor,
                                float* loss, float* state, void* stream) {
  if (!frame || !app || !embed_index || !color || !target || !state)
    return set_error(GS_ERR_INVALID_ARG, "frame, app, embed_index, color, target and state must not be NULL");
  if (gs_appearance_param_count(app->n_embeddings, app->embed_dim, app->hidden) == 0) return GS_ERR_INVALID_ARG;
  if (!app->params || !app->grads) return set_error(GS_ERR_INVALID_ARG, "app->params and app->grads must be set");
  if (frame->n_views < 1 || frame->n_views > GS_MAX_VIEWS || !frame->views)
    return set_error(GS_ERR_INVALID_ARG, "n_views must be in [1, %d] with a view array", GS_MAX_VIEWS);
  AppDev A;
  memset(&A, 0, sizeof(A));
  A.n_emb = app->n_embeddings; A.E = app->embed_dim; A.H = app->hidden; A.n_views = frame->n_views;
  int64_t blocks = 0, pix = 0;
  for (int v = 0; v < frame->n_views; ++v) {
    const gs_view& cv = frame->views[v];
    if (cv.width < 1 || cv.height < 1 || cv.width > 16384 || cv.height > 16384)
      return set_error(GS_ERR_INVALID_ARG, "view %d: image size must be in [1, 16384]", v);
    if (embed_index[v] < 0 || embed_index[v] >= app->n_embeddings)
      return set_error(GS_ERR_INVALID_ARG, "view %d: embedding index %d out of range", v, embed_index[v]);
    A.idx[v] = embed_index[v];
    A.blk_off[v] = (int32_t)blocks;
    A.bx[v] = (cv.width + kAX - 1) / kAX;
    blocks += (int64_t)A.bx[v] * ((cv.height + kAY - 1) / kAY);
    A.width[v] = cv.width;
    A.height[v] = cv.height;
    A.pix_off[v] = pix;
    pix += (int64_t)cv.width * cv.height;
  }
  if (blocks >= (int64_t(1) << 31)) return set_error(GS_ERR_INVALID_ARG, "too many pixels");
  A.blk_off[frame->n_views] = (int32_t)blocks;
  A.pix_off[frame->n_views] = pix;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_app_mlp_fwd<<<frame->n_views, kAppThreads, 0, s>>>(app->params, A, state);
  k_app_pixels<<<(unsigned)blocks, kAX * kAY, 0, s>>>(A, color, target, corrected, dcolor, state);
  k_app_mlp_bwd<<<frame->n_views, kAppThreads, 0, s>>>(app->params, app->grads, A, state, loss);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GS_ERR_CUDA, "appearance: %s", cudaGetErrorString(e));
  return GS_OK;
}

gs_status gs_adam_step(float* params, float* grads, float* m, float* v, int64_t n, float lr, float beta1,
                       float beta2, float eps, int32_t step, int32_t zero_grads, void* stream) {
  if (n < 0 || (n > 0 && (!params || !grads || !m || !v)))
    return set_error(GS_ERR_INVALID_ARG, "adam: NULL buffer or n < 0");
  if (step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) ||
      !std::isfinite(lr))
    return set_error(GS_ERR_INVALID_ARG, "adam: step >= 1, betas in [0, 1), eps > 0, finite lr");
  if (n == 0) return GS_OK;
  const float bc1 = (float)(1.0 - std::pow((double)beta1, step));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, step));
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
  k_adam<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grads, m, v, n, lr, beta1, beta2, eps, bc1,
                                                               bc2, zero_grads ? 1 : 0);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GS_ERR_CUDA, "adam: %s", cudaGetErrorString(e));
  return GS_OK;
}

}  // extern "C"
