// Per-Gaussian stage of the rasterizer and its backward pass.
//
// Forward (one thread per (view, Gaussian) entry):
//   x_c = W m + t, u = fx x/z + cx (Sec. 3.1);
//   Sigma = R S S^T R^T (Eq. 1); Sigma' = J W Sigma W^T J^T (Eq. 2), with the
//   third row of J the derivative of t = |x| (ray space, Eq. 8);
//   A = Sigma'[0:2,0:2] + lowpass I, conic = A^-1;
//   q = -b^T A^-1 with b = Sigma'[0:2,2]: the first two entries of
//   q_hat = v'^T Sigma'^-1 / (v'^T Sigma'^-1 v') (Eq. 13) by the Schur complement;
//   p = (z_c/t_c) q (Eq. 15-17); n = normalize(J^T n'), n' = -(q, 1) (Eq. 21-22);
//   colour from real SH of degree <= 3 (Sec. 3.1).
// The chain that decides visibility, the pixel rectangle and the depth key is
// evaluated with explicitly rounded FP32 operations in a fixed order, so that
// the tile lists are reproducible bit for bit on any IEEE machine.
#include "gs_internal.cuh"

namespace gs {

// Real SH with Condon-Shortley phase; constants are the closed forms
// K0 = 1/(2 sqrt(pi)), K1 = sqrt(3/(4 pi)), K2a = sqrt(15/pi)/2,
// K2b = sqrt(5/pi)/4, K2c = sqrt(15/pi)/4, K3a = sqrt(35/(2 pi))/4,
// K3b = sqrt(105/pi)/2, K3c = sqrt(21/(2 pi))/4, K3d = sqrt(7/pi)/4,
// K3e = sqrt(105/pi)/4.
constexpr float K0 = 0.28209479177387814f;
constexpr float K1 = 0.4886025119029199f;
constexpr float K2a = 1.0925484305920792f;
constexpr float K2b = 0.31539156525252005f;
constexpr float K2c = 0.5462742152960396f;
constexpr float K3a = 0.5900435899266435f;
constexpr float K3b = 2.890611442640554f;
constexpr float K3c = 0.4570457994644658f;
constexpr float K3d = 0.3731763325901154f;
constexpr float K3e = 1.445305721320277f;

__device__ inline void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = K0;
  Y[1] = -K1 * y;
  Y[2] = K1 * z;
  Y[3] = -K1 * x;
  Y[4] = K2a * x * y;
  Y[5] = -K2a * y * z;
  Y[6] = K2b * (3.f * z * z - 1.f);
  Y[7] = -K2a * x * z;
  Y[8] = K2c * (x * x - y * y);
  Y[9] = -K3a * y * (3.f * x * x - y * y);
  Y[10] = K3b * x * y * z;
  Y[11] = -K3c * y * (5.f * z * z - 1.f);
  Y[12] = K3d * z * (5.f * z * z - 3.f);
  Y[13] = -K3c * x * (5.f * z * z - 1.f);
  Y[14] = K3e * z * (x * x - y * y);
  Y[15] = -K3a * x * (x * x - 3.f * y * y);
}

// d Y_k / d (x, y, z) of the polynomials above.
__device__ inline void sh_basis_grad(float x, float y, float z, float (*dY)[3]) {
  dY[0][0] = 0.f; dY[0][1] = 0.f; dY[0][2] = 0.f;
  dY[1][0] = 0.f; dY[1][1] = -K1; dY[1][2] = 0.f;
  dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = K1;
  dY[3][0] = -K1; dY[3][1] = 0.f; dY[3][2] = 0.f;
  dY[4][0] = K2a * y; dY[4][1] = K2a * x; dY[4][2] = 0.f;
  dY[5][0] = 0.f; dY[5][1] = -K2a * z; dY[5][2] = -K2a * y;
  dY[6][0] = 0.f; dY[6][1] = 0.f; dY[6][2] = 6.f * K2b * z;
  dY[7][0] = -K2a * z; dY[7][1] = 0.f; dY[7][2] = -K2a * x;
  dY[8][0] = 2.f * K2c * x; dY[8][1] = -2.f * K2c * y; dY[8][2] = 0.f;
  dY[9][0] = -6.f * K3a * x * y; dY[9][1] = -K3a * (3.f * x * x - 3.f * y * y); dY[9][2] = 0.f;
  dY[10][0] = K3b * y * z; dY[10][1] = K3b * x * z; dY[10][2] = K3b * x * y;
  dY[11][0] = 0.f; dY[11][1] = -K3c * (5.f * z * z - 1.f); dY[11][2] = -10.f * K3c * y * z;
  dY[12][0] = 0.f; dY[12][1] = 0.f; dY[12][2] = K3d * (15.f * z * z - 3.f);
  dY[13][0] = -K3c * (5.f * z * z - 1.f); dY[13][1] = 0.f; dY[13][2] = -10.f * K3c * x * z;
  dY[14][0] = 2.f * K3e * x * z; dY[14][1] = -2.f * K3e * y * z; dY[14][2] = K3e * (x * x - y * y);
  dY[15][0] = -K3a * (3.f * x * x - 3.f * y * y); dY[15][1] = 6.f * K3a * x * y; dY[15][2] = 0.f;
}

// Quantities of one entry that both passes need, in plain FP32 (any rounding).
struct Geo {
  float xc[3], z, iz, tc;
  float txc, tyc;
  bool clx, cly;       // x/z or y/z clamped inside J
  float qn[4], qnorm;  // normalised quaternion and |q|
  float Rq[3][3];
  float M[3][3];       // Rq diag(s)
  float j00, j02, j11, j12, J2[3];
  float T[3][3];       // J W
  float G[3][3];       // J W Rq S
  float A00, A01, A11, det, ca, cb, cc;
  float b0, b1, q0, q1, p0, p1;
  float mv[3], mlen, n[3];
};

__device__ inline void geo_forward(const ViewDev& V, const float m[3], const float s[3],
                                   const float qin[4], float lowpass, Geo& g) {
  for (int i = 0; i < 3; ++i)
    g.xc[i] = V.R[3 * i] * m[0] + V.R[3 * i + 1] * m[1] + V.R[3 * i + 2] * m[2] + V.t[i];
  g.z = g.xc[2];
  g.iz = 1.f / g.z;
  g.tc = sqrtf(g.xc[0] * g.xc[0] + g.xc[1] * g.xc[1] + g.xc[2] * g.xc[2]);
  float tx = g.xc[0] * g.iz, ty = g.xc[1] * g.iz;
  g.clx = !(tx > V.lim[0] && tx < V.lim[1]);
  g.cly = !(ty > V.lim[2] && ty < V.lim[3]);
  g.txc = fminf(fmaxf(tx, V.lim[0]), V.lim[1]);
  g.tyc = fminf(fmaxf(ty, V.lim[2]), V.lim[3]);

  float n2 = qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3];
  g.qnorm = sqrtf(n2);
  float r = 1.f / g.qnorm;
  float w = qin[0] * r, x = qin[1] * r, y = qin[2] * r, z = qin[3] * r;
  g.qn[0] = w; g.qn[1] = x; g.qn[2] = y; g.qn[3] = z;
  g.Rq[0][0] = 1.f - 2.f * (y * y + z * z);
  g.Rq[0][1] = 2.f * (x * y - w * z);
  g.Rq[0][2] = 2.f * (x * z + w * y);
  g.Rq[1][0] = 2.f * (x * y + w * z);
  g.Rq[1][1] = 1.f - 2.f * (x * x + z * z);
  g.Rq[1][2] = 2.f * (y * z - w * x);
  g.Rq[2][0] = 2.f * (x * z - w * y);
  g.Rq[2][1] = 2.f * (y * z + w * x);
  g.Rq[2][2] = 1.f - 2.f * (x * x + y * y);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) g.M[i][k] = g.Rq[i][k] * s[k];

  g.j00 = V.fx * g.iz;
  g.j02 = -V.fx * g.txc * g.iz;
  g.j11 = V.fy * g.iz;
  g.j12 = -V.fy * g.tyc * g.iz;
  float it = 1.f / g.tc;
  g.J2[0] = g.xc[0] * it; g.J2[1] = g.xc[1] * it; g.J2[2] = g.xc[2] * it;
  for (int k = 0; k < 3; ++k) {
    g.T[0][k] = g.j00 * V.R[k] + g.j02 * V.R[6 + k];
    g.T[1][k] = g.j11 * V.R[3 + k] + g.j12 * V.R[6 + k];
    g.T[2][k] = g.J2[0] * V.R[k] + g.J2[1] * V.R[3 + k] + g.J2[2] * V.R[6 + k];
  }
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k)
      g.G[i][k] = g.T[i][0] * g.M[0][k] + g.T[i][1] * g.M[1][k] + g.T[i][2] * g.M[2][k];
  auto dot3 = [](const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
  g.A00 = dot3(g.G[0], g.G[0]) + lowpass;
  g.A11 = dot3(g.G[1], g.G[1]) + lowpass;
  g.A01 = dot3(g.G[0], g.G[1]);
  g.b0 = dot3(g.G[0], g.G[2]);
  g.b1 = dot3(g.G[1], g.G[2]);
  g.det = g.A00 * g.A11 - g.A01 * g.A01;
  float id = 1.f / g.det;
  g.ca = g.A11 * id;
  g.cb = -g.A01 * id;
  g.cc = g.A00 * id;
  g.q0 = -(g.ca * g.b0 + g.cb * g.b1);
  g.q1 = -(g.cb * g.b0 + g.cc * g.b1);
  float zt = g.z * it;
  g.p0 = zt * g.q0;
  g.p1 = zt * g.q1;
  g.mv[0] = -(g.q0 * g.j00 + g.J2[0]);
  g.mv[1] = -(g.q1 * g.j11 + g.J2[1]);
  g.mv[2] = -(g.q0 * g.j02 + g.q1 * g.j12 + g.J2[2]);
  g.mlen = sqrtf(dot3(g.mv, g.mv));
  float im = 1.f / g.mlen;
  g.n[0] = g.mv[0] * im; g.n[1] = g.mv[1] * im; g.n[2] = g.mv[2] * im;
}

constexpr int kPreThreads = 128;   // entries per block-chunk of the per-Gaussian kernels

// Chunk b of the frame: up to kPreThreads consecutive Gaussians of one view.
struct Chunk {
  int view;
  int n;          // entries in the chunk
  int64_t g0;     // first Gaussian (scene index)
  int64_t e0;     // first entry
};

__device__ inline Chunk chunk_of(const FrameDev* fd, int b) {
  int lo = 0, hi = fd->n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (fd->chunk_off[mid] <= b) lo = mid; else hi = mid - 1;
  }
  Chunk c;
  c.view = lo;
  c.g0 = (int64_t)(b - fd->chunk_off[lo]) * kPreThreads;
  const int64_t n = fd->scenes[fd->views[lo].scene].n;
  c.n = (int)min((int64_t)kPreThreads, n - c.g0);
  c.e0 = fd->entry_off[lo] + c.g0;
  return c;
}

template <typename T> __host__ __device__ constexpr int dtype_code() { return sizeof(T) == 4 ? GS_F32 : GS_BF16; }

// Coalesced copy of a chunk's contiguous parameter block into shared memory,
// widened to FP32; element i goes to dst[(i / group) * stride + i % group].
// 16-byte vector loads, four in flight per thread, when the source is aligned.
template <int GROUP, int STRIDE>
__device__ inline void put_elem(float* dst, int i, float v, int* bad) {
  dst[(i / GROUP) * STRIDE + i % GROUP] = v;
  if (bad && !(fabsf(v) <= 3.402823466e38f)) bad[i / GROUP] = 1;   // nan or inf
}

template <typename T, int GROUP, int STRIDE>
__device__ inline void stage(const T* __restrict__ src, int count, float* __restrict__ dst,
                             int* bad = nullptr) {
  constexpr int PER = 16 / sizeof(T);   // elements per 16-byte vector
  int done = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const int nv = count / PER;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    for (int base = 0; base < nv; base += 4 * (int)blockDim.x) {
      uint4 r[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int f = base + k * blockDim.x + threadIdx.x;
        if (f < nv) r[k] = __ldg(s4 + f);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int f = base + k * blockDim.x + threadIdx.x;
        if (f >= nv) continue;
        const uint32_t w[4] = {r[k].x, r[k].y, r[k].z, r[k].w};
        if (sizeof(T) == 4) {
#pragma unroll
          for (int c = 0; c < 4; ++c) put_elem<GROUP, STRIDE>(dst, PER * f + c, __uint_as_float(w[c]), bad);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            put_elem<GROUP, STRIDE>(dst, PER * f + 2 * c, __uint_as_float(w[c] << 16), bad);
            put_elem<GROUP, STRIDE>(dst, PER * f + 2 * c + 1, __uint_as_float(w[c] & 0xFFFF0000u), bad);
          }
        }
      }
    }
    done = nv * PER;
  }
  for (int i = done + threadIdx.x; i < count; i += blockDim.x) put_elem<GROUP, STRIDE>(dst, i, ldf(src, i), bad);
}

template <typename T>
__device__ inline void load_quat(const T* q, int64_t g, float out[4]);
template <> __device__ inline void load_quat<float>(const float* q, int64_t g, float out[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(q) + g);
  out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <> __device__ inline void load_quat<__nv_bfloat16>(const __nv_bfloat16* q, int64_t g, float out[4]) {
  const uint2 v = __ldg(reinterpret_cast<const uint2*>(q) + g);
  out[0] = __uint_as_float(v.x << 16); out[1] = __uint_as_float(v.x & 0xFFFF0000u);
  out[2] = __uint_as_float(v.y << 16); out[3] = __uint_as_float(v.y & 0xFFFF0000u);
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
template <typename T, int D>
__global__ void __launch_bounds__(kPreThreads, 4)
k_preprocess(const FrameDev* __restrict__ fd, void* __restrict__ ws, Layout L) {
  constexpr int K = (D + 1) * (D + 1), SHS = 3 * K + 1;
  __shared__ float s_sh[kPreThreads * SHS];
  __shared__ float s_m[kPreThreads * 3], s_s[kPreThreads * 3], s_o[kPreThreads];
  __shared__ int s_bad[kPreThreads];
  Header* hdr = at<Header>(ws, L.hdr);
  float4* rec = at<float4>(ws, L.rec);
  short4* rect = at<short4>(ws, L.rect);
  uint32_t* key = at<uint32_t>(ws, L.key);
  uint32_t* touched = at<uint32_t>(ws, L.touched);
  const float lp = fd->lowpass, C = fd->ext_c, amin = fd->alpha_min;
  const int sx = fd->tile_shift_x, sy = fd->tile_shift_y;
  int nonfinite = 0;
  for (int bi = blockIdx.x; bi < fd->n_chunks; bi += gridDim.x) {
    const Chunk ch = chunk_of(fd, bi);
    const ViewDev& V = fd->views[ch.view];
    const SceneDev& S = fd->scenes[V.scene];
    if (S.dtype != dtype_code<T>() || S.sh_degree != D) continue;
    __syncthreads();
    s_bad[threadIdx.x] = 0;
    __syncthreads();
    stage<T, 3, 3>(static_cast<const T*>(S.means) + 3 * ch.g0, 3 * ch.n, s_m, s_bad);
    stage<T, 3, 3>(static_cast<const T*>(S.scales) + 3 * ch.g0, 3 * ch.n, s_s, s_bad);
    stage<T, 1, 1>(static_cast<const T*>(S.opacities) + ch.g0, ch.n, s_o, s_bad);
    stage<T, 3 * K, SHS>(static_cast<const T*>(S.sh) + 3 * K * ch.g0, 3 * K * ch.n, s_sh, s_bad);
    __syncthreads();
    const int t = threadIdx.x;
    if (t >= ch.n) continue;
    const int64_t e = ch.e0 + t;
    float m[3], s[3], q[4];
    for (int k = 0; k < 3; ++k) { m[k] = s_m[3 * t + k]; s[k] = s_s[3 * t + k]; }
    load_quat<T>(static_cast<const T*>(S.quats), ch.g0 + t, q);
    const float o = s_o[t];
    const float* sh = s_sh + t * SHS;

    // finiteness of every input: staged arrays were checked on load
    float chk = 0.f;
    for (int k = 0; k < 4; ++k) chk += q[k] * 0.f;   // inf * 0 and nan * 0 are nan
    const bool finite = chk == 0.f && s_bad[t] == 0;

    // ---- exactly rounded decision chain ----------------------------------
    float xc[3];
    for (int i = 0; i < 3; ++i)
      xc[i] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(V.R[3 * i], m[0]), __fmul_rn(V.R[3 * i + 1], m[1])),
                                  __fmul_rn(V.R[3 * i + 2], m[2])), V.t[i]);
    const float z = xc[2];
    bool valid = finite && (z > V.near_plane);
    const float iz = __fdiv_rn(1.f, z);
    const float tx = __fmul_rn(xc[0], iz), ty = __fmul_rn(xc[1], iz);
    const float u = __fadd_rn(__fmul_rn(V.fx, tx), V.cx);
    const float v = __fadd_rn(__fmul_rn(V.fy, ty), V.cy);
    const float n2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(q[0], q[0]), __fmul_rn(q[1], q[1])),
                                         __fmul_rn(q[2], q[2])), __fmul_rn(q[3], q[3]));
    valid = valid && (n2 > 0.f);
    const float rn = __fdiv_rn(1.f, __fsqrt_rn(n2));
    const float w = __fmul_rn(q[0], rn), x = __fmul_rn(q[1], rn), y = __fmul_rn(q[2], rn),
                zq = __fmul_rn(q[3], rn);
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(zq, zq);
    const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, zq), yz = __fmul_rn(y, zq);
    const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, zq);
    float Rq[3][3];
    Rq[0][0] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(yy, zz)));
    Rq[0][1] = __fmul_rn(2.f, __fsub_rn(xy, wz));
    Rq[0][2] = __fmul_rn(2.f, __fadd_rn(xz, wy));
    Rq[1][0] = __fmul_rn(2.f, __fadd_rn(xy, wz));
    Rq[1][1] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, zz)));
    Rq[1][2] = __fmul_rn(2.f, __fsub_rn(yz, wx));
    Rq[2][0] = __fmul_rn(2.f, __fsub_rn(xz, wy));
    Rq[2][1] = __fmul_rn(2.f, __fadd_rn(yz, wx));
    Rq[2][2] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, yy)));
    float M[3][3];
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) M[i][k] = __fmul_rn(Rq[i][k], s[k]);
    const float txc = fminf(fmaxf(tx, V.lim[0]), V.lim[1]);
    const float tyc = fminf(fmaxf(ty, V.lim[2]), V.lim[3]);
    const float j00 = __fmul_rn(V.fx, iz);
    const float j02 = __fmul_rn(-__fmul_rn(V.fx, txc), iz);
    const float j11 = __fmul_rn(V.fy, iz);
    const float j12 = __fmul_rn(-__fmul_rn(V.fy, tyc), iz);
    float T0[3], T1[3];
    for (int k = 0; k < 3; ++k) {
      T0[k] = __fadd_rn(__fmul_rn(j00, V.R[k]), __fmul_rn(j02, V.R[6 + k]));
      T1[k] = __fadd_rn(__fmul_rn(j11, V.R[3 + k]), __fmul_rn(j12, V.R[6 + k]));
    }
    float G0[3], G1[3];
    for (int k = 0; k < 3; ++k) {
      G0[k] = __fadd_rn(__fadd_rn(__fmul_rn(T0[0], M[0][k]), __fmul_rn(T0[1], M[1][k])),
                        __fmul_rn(T0[2], M[2][k]));
      G1[k] = __fadd_rn(__fadd_rn(__fmul_rn(T1[0], M[0][k]), __fmul_rn(T1[1], M[1][k])),
                        __fmul_rn(T1[2], M[2][k]));
    }
    const float A00x = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(G0[0], G0[0]), __fmul_rn(G0[1], G0[1])),
                                           __fmul_rn(G0[2], G0[2])), lp);
    const float A11x = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(G1[0], G1[0]), __fmul_rn(G1[1], G1[1])),
                                           __fmul_rn(G1[2], G1[2])), lp);
    const float ex = __fsqrt_rn(__fmul_rn(C, A00x));
    const float ey = __fsqrt_rn(__fmul_rn(C, A11x));
    const float xlo = __fsub_rn(__fsub_rn(u, ex), 0.5f), xhi = __fsub_rn(__fadd_rn(u, ex), 0.5f);
    const float ylo = __fsub_rn(__fsub_rn(v, ey), 0.5f), yhi = __fsub_rn(__fadd_rn(v, ey), 0.5f);
    valid = valid && (xhi >= 0.f) && (xlo <= (float)(V.width - 1)) && (yhi >= 0.f) &&
            (ylo <= (float)(V.height - 1)) && (o >= amin);
    int i0 = 0, i1 = -1, j0 = 0, j1 = -1;
    if (valid) {
      i0 = (int)fmaxf(0.f, ceilf(xlo));
      i1 = (int)fminf((float)(V.width - 1), floorf(xhi));
      j0 = (int)fmaxf(0.f, ceilf(ylo));
      j1 = (int)fminf((float)(V.height - 1), floorf(yhi));
      valid = (i0 <= i1) && (j0 <= j1);
    }

    // ---- the rest of the record (ordinary FP32, from the chain's values) ----
    float conic[3] = {0.f, 0.f, 0.f}, pp[2] = {0.f, 0.f}, nn[3] = {0.f, 0.f, 0.f};
    float rgb[3] = {0.f, 0.f, 0.f};
    if (valid) {
      const float tc = sqrtf(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);
      const float it = 1.f / tc;
      const float J2[3] = {xc[0] * it, xc[1] * it, xc[2] * it};   // third row of J: d|x|/dx
      float G2[3], T2[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) T2[k] = J2[0] * V.R[k] + J2[1] * V.R[3 + k] + J2[2] * V.R[6 + k];
#pragma unroll
      for (int k = 0; k < 3; ++k) G2[k] = T2[0] * M[0][k] + T2[1] * M[1][k] + T2[2] * M[2][k];
      const float A01 = G0[0] * G1[0] + G0[1] * G1[1] + G0[2] * G1[2];
      const float b0 = G0[0] * G2[0] + G0[1] * G2[1] + G0[2] * G2[2];
      const float b1 = G1[0] * G2[0] + G1[1] * G2[1] + G1[2] * G2[2];
      const float det = A00x * A11x - A01 * A01;
      const float id = 1.f / det;
      conic[0] = A11x * id;
      conic[1] = -A01 * id;
      conic[2] = A00x * id;
      // q = -b^T A^-1: first two entries of q_hat (Eq. 13); p = (z/t) q (Eq. 15)
      const float q0 = -(conic[0] * b0 + conic[1] * b1);
      const float q1 = -(conic[1] * b0 + conic[2] * b1);
      const float zt = z * it;
      pp[0] = zt * q0;
      pp[1] = zt * q1;
      // n = J^T n', n' = -(q, 1) (Eq. 21-22), normalised
      const float mv0 = -(q0 * j00 + J2[0]);
      const float mv1 = -(q1 * j11 + J2[1]);
      const float mv2 = -(q0 * j02 + q1 * j12 + J2[2]);
      const float im = rsqrtf(mv0 * mv0 + mv1 * mv1 + mv2 * mv2);
      nn[0] = mv0 * im; nn[1] = mv1 * im; nn[2] = mv2 * im;
      valid = (det > 0.f) && isfinite(conic[0]) && isfinite(conic[1]) && isfinite(conic[2]) &&
              isfinite(pp[0]) && isfinite(pp[1]) && isfinite(nn[0]) && isfinite(nn[1]) && isfinite(nn[2]);
      float d[3] = {m[0] - V.campos[0], m[1] - V.campos[1], m[2] - V.campos[2]};
      float il = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      float Y[16];
      sh_basis(d[0] * il, d[1] * il, d[2] * il, Y);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float acc = 0.5f;
#pragma unroll
        for (int j = 0; j < K; ++j) acc += Y[j] * sh[3 * j + c];
        rgb[c] = fmaxf(acc, 0.f);
      }
    }
    if (!finite) ++nonfinite;
    if (valid) {
      float4* r = rec + 4 * e;
      // sigma beyond which alpha < alpha_min (with a margin far above FP32 error):
      // lets the compositing skip a splat for a whole block of pixels
      const float cut = logf(o / amin) * 1.0001f + 1e-4f;
      r[0] = make_float4(u, v, conic[0], conic[1]);
      r[1] = make_float4(conic[2], o, cut, z);
      r[2] = make_float4(pp[0], pp[1], nn[0], nn[1]);
      r[3] = make_float4(nn[2], rgb[0], rgb[1], rgb[2]);
      rect[e] = make_short4((short)i0, (short)i1, (short)j0, (short)j1);
      key[e] = __float_as_uint(z);
      touched[e] = (uint32_t)(((i1 >> sx) - (i0 >> sx) + 1) * ((j1 >> sy) - (j0 >> sy) + 1));
    } else {
      rect[e] = make_short4(0, -1, 0, -1);
      key[e] = kInvalidKey;
      touched[e] = 0u;
    }
  }
  for (int o = 16; o > 0; o >>= 1) nonfinite += __shfl_xor_sync(0xFFFFFFFFu, nonfinite, o);
  if ((threadIdx.x & 31) == 0 && nonfinite) {
    atomicAdd(&hdr->n_nonfinite, (unsigned long long)nonfinite);
    set_status(hdr, GS_ERR_NUMERIC);
  }
}

// ---------------------------------------------------------------------------
// Backward: d(record) -> d(means, scales, quats, opacities, sh)
// ---------------------------------------------------------------------------
// Writes a staged gradient block: plain stores if the scene has one view, else
// atomic adds (the buffers were zeroed first).  Stores go out as 16-byte
// vectors when the destination is aligned.
template <int GROUP, int STRIDE>
__device__ inline float get_elem(const float* src, int i) {
  return src[(i / GROUP) * STRIDE + i % GROUP];
}

template <int GROUP, int STRIDE>
__device__ inline void unstage(const float* __restrict__ src, int count, float* __restrict__ dst, bool store) {
  if (!dst) return;
  if (!store) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
      const float v = get_elem<GROUP, STRIDE>(src, i);
      if (v != 0.f) atomicAdd(dst + i, v);
    }
    return;
  }
  int done = 0;
  if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
    const int nv = count / 4;
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int f = threadIdx.x; f < nv; f += blockDim.x)
      d4[f] = make_float4(get_elem<GROUP, STRIDE>(src, 4 * f), get_elem<GROUP, STRIDE>(src, 4 * f + 1),
                          get_elem<GROUP, STRIDE>(src, 4 * f + 2), get_elem<GROUP, STRIDE>(src, 4 * f + 3));
    done = nv * 4;
  }
  for (int i = done + threadIdx.x; i < count; i += blockDim.x) dst[i] = get_elem<GROUP, STRIDE>(src, i);
}

template <typename T, int D>
__global__ void __launch_bounds__(kPreThreads, 3)
k_preprocess_bwd(const FrameDev* __restrict__ fd, void* __restrict__ ws, Layout L, GradPtrs gp) {
  constexpr int K = (D + 1) * (D + 1), SHS = 3 * K + 1;
  __shared__ float s_sh[kPreThreads * SHS];   // coefficients in, their gradients out
  __shared__ float s_m[kPreThreads * 3], s_s[kPreThreads * 3], s_o[kPreThreads];
  __shared__ float s_gm[kPreThreads * 3], s_gs[kPreThreads * 3], s_gq[kPreThreads * 4];
  const uint32_t* key = at<uint32_t>(ws, L.key);
  const float4* g2d = at<float4>(ws, L.grad2d);
  const float lp = fd->lowpass;
  for (int bi = blockIdx.x; bi < fd->n_chunks; bi += gridDim.x) {
    const Chunk ch = chunk_of(fd, bi);
    const ViewDev& V = fd->views[ch.view];
    const SceneDev& S = fd->scenes[V.scene];
    if (S.dtype != dtype_code<T>() || S.sh_degree != D) continue;
    const gs_scene_grads& Dg = gp.g[V.scene];
    const bool store = S.n_views == 1;  // else the buffers were zeroed and we add
    __syncthreads();
    stage<T, 3, 3>(static_cast<const T*>(S.means) + 3 * ch.g0, 3 * ch.n, s_m);
    stage<T, 3, 3>(static_cast<const T*>(S.scales) + 3 * ch.g0, 3 * ch.n, s_s);
    stage<T, 3 * K, SHS>(static_cast<const T*>(S.sh) + 3 * K * ch.g0, 3 * K * ch.n, s_sh);
    __syncthreads();
    const int t = threadIdx.x;
    float* sh = s_sh + t * SHS;
    float gm[3] = {0.f, 0.f, 0.f}, gsc[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, go = 0.f;
    const int64_t e = ch.e0 + t;
    if (t < ch.n && key[e] == kInvalidKey) {
#pragma unroll
      for (int j = 0; j < 3 * K; ++j) sh[j] = 0.f;
    } else if (t < ch.n) {
      float m[3], s[3], q[4];
      for (int k = 0; k < 3; ++k) { m[k] = s_m[3 * t + k]; s[k] = s_s[3 * t + k]; }
      load_quat<T>(static_cast<const T*>(S.quats), ch.g0 + t, q);
      Geo g;
      geo_forward(V, m, s, q, lp, g);
      const float4 ga = g2d[4 * e], gb4 = g2d[4 * e + 1], gc4 = g2d[4 * e + 2], gd4 = g2d[4 * e + 3];
      const float gu = ga.x, gv = ga.y, gca = ga.z, gcb = ga.w;
      const float gcc = gb4.x, gz = gb4.w;
      go = gb4.y;
      const float gp0 = gc4.x, gp1 = gc4.y, gn[3] = {gc4.z, gc4.w, gd4.x};
      const float grgb[3] = {gd4.y, gd4.z, gd4.w};

      // ---- colour: rgb = max(sum Y_j c_j + 1/2, 0) ----------------------------
      {
        float d[3] = {m[0] - V.campos[0], m[1] - V.campos[1], m[2] - V.campos[2]};
        float il = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        float dir[3] = {d[0] * il, d[1] * il, d[2] * il};
        float Y[16], dY[16][3];
        sh_basis(dir[0], dir[1], dir[2], Y);
        sh_basis_grad(dir[0], dir[1], dir[2], dY);
        float val[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
          for (int k = 0; k < 3; ++k) val[k] += Y[j] * sh[3 * j + k];
        float gval[3];
        for (int k = 0; k < 3; ++k) gval[k] = val[k] > 0.f ? grgb[k] : 0.f;
        float gdir[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const float gY = sh[3 * j] * gval[0] + sh[3 * j + 1] * gval[1] + sh[3 * j + 2] * gval[2];
          gdir[0] += gY * dY[j][0]; gdir[1] += gY * dY[j][1]; gdir[2] += gY * dY[j][2];
#pragma unroll
          for (int k = 0; k < 3; ++k) sh[3 * j + k] = Y[j] * gval[k];
        }
        float dd = dir[0] * gdir[0] + dir[1] * gdir[1] + dir[2] * gdir[2];
        for (int k = 0; k < 3; ++k) gm[k] += (gdir[k] - dir[k] * dd) * il;
      }
      // ---- p = (z/t) q -----------------------------------------------------------
      const float it = 1.f / g.tc;
      const float zt = g.z * it;
      float gq0 = zt * gp0, gq1 = zt * gp1;
      const float qgp = g.q0 * gp0 + g.q1 * gp1;
      const float gz_tot = gz + qgp * it;
      const float gtc = -g.z * it * it * qgp;
      // ---- n = mv / |mv|, mv = -(q0 J0 + q1 J1 + J2) ---------------------------------
      const float ndg = g.n[0] * gn[0] + g.n[1] * gn[1] + g.n[2] * gn[2];
      const float iml = 1.f / g.mlen;
      float gmv[3];
      for (int k = 0; k < 3; ++k) gmv[k] = (gn[k] - g.n[k] * ndg) * iml;
      gq0 += -(g.j00 * gmv[0] + g.j02 * gmv[2]);
      gq1 += -(g.j11 * gmv[1] + g.j12 * gmv[2]);
      float gj00 = -g.q0 * gmv[0], gj02 = -g.q0 * gmv[2];
      float gj11 = -g.q1 * gmv[1], gj12 = -g.q1 * gmv[2];
      float gJ2[3] = {-gmv[0], -gmv[1], -gmv[2]};
      // ---- q = -C b --------------------------------------------------------------------
      const float gca_t = gca - gq0 * g.b0;
      const float gcb_t = gcb - (gq0 * g.b1 + gq1 * g.b0);
      const float gcc_t = gcc - gq1 * g.b1;
      const float gb0 = -(g.ca * gq0 + g.cb * gq1);
      const float gb1 = -(g.cb * gq0 + g.cc * gq1);
      // ---- C = A^-1: dA = -C dC C (symmetric, off-diagonal counted once) ---------------
      const float h = 0.5f * gcb_t;
      const float X00 = g.ca * gca_t + g.cb * h, X01 = g.ca * h + g.cb * gcc_t;
      const float X10 = g.cb * gca_t + g.cc * h, X11 = g.cb * h + g.cc * gcc_t;
      const float gA00 = -(X00 * g.ca + X01 * g.cb);
      const float gA01 = -(X00 * g.cb + X01 * g.cc);
      const float gA11 = -(X10 * g.cb + X11 * g.cc);
      // ---- Sigma' = G G^T ----------------------------------------------------------------
      const float gS01 = 2.f * gA01;
      float gG[3][3];
      for (int k = 0; k < 3; ++k) {
        gG[0][k] = 2.f * gA00 * g.G[0][k] + gS01 * g.G[1][k] + gb0 * g.G[2][k];
        gG[1][k] = 2.f * gA11 * g.G[1][k] + gS01 * g.G[0][k] + gb1 * g.G[2][k];
        gG[2][k] = gb0 * g.G[0][k] + gb1 * g.G[1][k];
      }
      // ---- G = T M --------------------------------------------------------------------------
      float gT[3][3], gM[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          gT[i][j] = gG[i][0] * g.M[j][0] + gG[i][1] * g.M[j][1] + gG[i][2] * g.M[j][2];
          gM[i][j] = g.T[0][i] * gG[0][j] + g.T[1][i] * gG[1][j] + g.T[2][i] * gG[2][j];
        }
      // ---- T = J W ----------------------------------------------------------------------------
      for (int k = 0; k < 3; ++k) {
        gj00 += gT[0][k] * V.R[k];
        gj02 += gT[0][k] * V.R[6 + k];
        gj11 += gT[1][k] * V.R[3 + k];
        gj12 += gT[1][k] * V.R[6 + k];
        gJ2[0] += gT[2][k] * V.R[k];
        gJ2[1] += gT[2][k] * V.R[3 + k];
        gJ2[2] += gT[2][k] * V.R[6 + k];
      }
      // ---- M = Rq diag(s) ----------------------------------------------------------------------
      float gR[3][3];
      for (int k = 0; k < 3; ++k) {
        gsc[k] = gM[0][k] * g.Rq[0][k] + gM[1][k] * g.Rq[1][k] + gM[2][k] * g.Rq[2][k];
        for (int i = 0; i < 3; ++i) gR[i][k] = gM[i][k] * s[k];
      }
      // ---- Rq(qn) and normalisation --------------------------------------------------------------
      {
        const float w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
        float gqn[4];
        gqn[0] = 2.f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
        gqn[1] = 2.f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.f * x * gR[1][1] - w * gR[1][2] +
                        z * gR[2][0] + w * gR[2][1] - 2.f * x * gR[2][2]);
        gqn[2] = 2.f * (-2.f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                        w * gR[2][0] + z * gR[2][1] - 2.f * y * gR[2][2]);
        gqn[3] = 2.f * (-2.f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2.f * z * gR[1][1] +
                        y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
        const float qd = w * gqn[0] + x * gqn[1] + y * gqn[2] + z * gqn[3];
        const float iq = 1.f / g.qnorm;
        for (int k = 0; k < 4; ++k) gq[k] = (gqn[k] - g.qn[k] * qd) * iq;
      }
      // ---- J(x_c), t_c, u, v, z --------------------------------------------------------------------
      float gx[3] = {0.f, 0.f, 0.f};
      const float iz = g.iz, iz2 = iz * iz;
      gx[2] += -V.fx * iz2 * gj00 - V.fy * iz2 * gj11;
      if (!g.clx) {   // j02 = -fx x / z^2
        gx[0] += -V.fx * iz2 * gj02;
        gx[2] += 2.f * V.fx * g.xc[0] * iz2 * iz * gj02;
      } else {        // j02 = -fx L / z
        gx[2] += V.fx * g.txc * iz2 * gj02;
      }
      if (!g.cly) {
        gx[1] += -V.fy * iz2 * gj12;
        gx[2] += 2.f * V.fy * g.xc[1] * iz2 * iz * gj12;
      } else {
        gx[2] += V.fy * g.tyc * iz2 * gj12;
      }
      const float jd = g.J2[0] * gJ2[0] + g.J2[1] * gJ2[1] + g.J2[2] * gJ2[2];
      for (int k = 0; k < 3; ++k) gx[k] += (gJ2[k] - g.J2[k] * jd) * it + gtc * g.J2[k];
      gx[0] += gu * V.fx * iz;
      gx[1] += gv * V.fy * iz;
      gx[2] += -(gu * V.fx * g.xc[0] + gv * V.fy * g.xc[1]) * iz2 + gz_tot;
      for (int k = 0; k < 3; ++k) gm[k] += V.R[k] * gx[0] + V.R[3 + k] * gx[1] + V.R[6 + k] * gx[2];
    }
    for (int k = 0; k < 3; ++k) { s_gm[3 * t + k] = gm[k]; s_gs[3 * t + k] = gsc[k]; }
    for (int k = 0; k < 4; ++k) s_gq[4 * t + k] = gq[k];
    s_o[t] = go;
    __syncthreads();
    unstage<3, 3>(s_gm, 3 * ch.n, Dg.dmeans ? Dg.dmeans + 3 * ch.g0 : nullptr, store);
    unstage<3, 3>(s_gs, 3 * ch.n, Dg.dscales ? Dg.dscales + 3 * ch.g0 : nullptr, store);
    unstage<4, 4>(s_gq, 4 * ch.n, Dg.dquats ? Dg.dquats + 4 * ch.g0 : nullptr, store);
    unstage<1, 1>(s_o, ch.n, Dg.dopacities ? Dg.dopacities + ch.g0 : nullptr, store);
    unstage<3 * K, SHS>(s_sh, 3 * K * ch.n, Dg.dsh ? Dg.dsh + 3 * K * ch.g0 : nullptr, store);
  }
}

// ---------------------------------------------------------------------------
// Launchers: one launch per (dtype, SH degree) present in the frame
// ---------------------------------------------------------------------------
static int grid_chunks(int n_chunks) {
  int b = n_chunks < 1 ? 1 : n_chunks;
  return b > 148 * 16 ? 148 * 16 : b;
}

template <typename T>
static void launch_fwd_t(int deg, const FrameDev* fd, void* ws, const Layout& L, int grid, cudaStream_t s) {
  switch (deg) {
    case 0: k_preprocess<T, 0><<<grid, kPreThreads, 0, s>>>(fd, ws, L); break;
    case 1: k_preprocess<T, 1><<<grid, kPreThreads, 0, s>>>(fd, ws, L); break;
    case 2: k_preprocess<T, 2><<<grid, kPreThreads, 0, s>>>(fd, ws, L); break;
    default: k_preprocess<T, 3><<<grid, kPreThreads, 0, s>>>(fd, ws, L); break;
  }
}

template <typename T>
static void launch_bwd_t(int deg, const FrameDev* fd, void* ws, const Layout& L, const GradPtrs& gp,
                         int grid, cudaStream_t s) {
  switch (deg) {
    case 0: k_preprocess_bwd<T, 0><<<grid, kPreThreads, 0, s>>>(fd, ws, L, gp); break;
    case 1: k_preprocess_bwd<T, 1><<<grid, kPreThreads, 0, s>>>(fd, ws, L, gp); break;
    case 2: k_preprocess_bwd<T, 2><<<grid, kPreThreads, 0, s>>>(fd, ws, L, gp); break;
    default: k_preprocess_bwd<T, 3><<<grid, kPreThreads, 0, s>>>(fd, ws, L, gp); break;
  }
}

// Bit (4 * dtype + degree) set for every kind of scene that a view renders.
static unsigned kinds(const FrameDev& hf) {
  unsigned k = 0;
  for (int v = 0; v < hf.n_views; ++v) {
    const SceneDev& S = hf.scenes[hf.views[v].scene];
    if (S.n > 0) k |= 1u << (4 * S.dtype + S.sh_degree);
  }
  return k;
}

cudaError_t launch_preprocess(void* ws, const Layout& L, const FrameDev& hf, cudaStream_t s) {
  const FrameDev* fd = at<FrameDev>(ws, L.frame);
  const unsigned k = kinds(hf);
  const int grid = grid_chunks(hf.n_chunks);
  for (int deg = 0; deg < 4; ++deg) {
    if (k & (1u << (4 * GS_F32 + deg))) launch_fwd_t<float>(deg, fd, ws, L, grid, s);
    if (k & (1u << (4 * GS_BF16 + deg))) launch_fwd_t<__nv_bfloat16>(deg, fd, ws, L, grid, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(void* ws, const Layout& L, const FrameDev& hf, const GradPtrs& gp,
                                  cudaStream_t s) {
  const FrameDev* fd = at<FrameDev>(ws, L.frame);
  const unsigned k = kinds(hf);
  const int grid = grid_chunks(hf.n_chunks);
  for (int deg = 0; deg < 4; ++deg) {
    if (k & (1u << (4 * GS_F32 + deg))) launch_bwd_t<float>(deg, fd, ws, L, gp, grid, s);
    if (k & (1u << (4 * GS_BF16 + deg))) launch_bwd_t<__nv_bfloat16>(deg, fd, ws, L, gp, grid, s);
  }
  return cudaGetLastError();
}

}  // namespace gs
