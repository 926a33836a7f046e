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
#include <algorithm>

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

// (gx, gy, gz) = sum_k gY_k dY_k/d(x, y, z) for the first K polynomials above
// (the transposed Jacobian of sh_basis applied to gY).
template <int K>
__device__ inline void sh_basis_vjp(float x, float y, float z, const float* gY, float* out) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (K > 1) {
    gy -= K1 * gY[1];
    gz += K1 * gY[2];
    gx -= K1 * gY[3];
  }
  if (K > 4) {
    gx += K2a * y * gY[4]; gy += K2a * x * gY[4];
    gy -= K2a * z * gY[5]; gz -= K2a * y * gY[5];
    gz += 6.f * K2b * z * gY[6];
    gx -= K2a * z * gY[7]; gz -= K2a * x * gY[7];
    gx += 2.f * K2c * x * gY[8]; gy -= 2.f * K2c * y * gY[8];
  }
  if (K > 9) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gx -= 6.f * K3a * x * y * gY[9]; gy -= K3a * (3.f * xx - 3.f * yy) * gY[9];
    gx += K3b * y * z * gY[10]; gy += K3b * x * z * gY[10]; gz += K3b * x * y * gY[10];
    gy -= K3c * (5.f * zz - 1.f) * gY[11]; gz -= 10.f * K3c * y * z * gY[11];
    gz += K3d * (15.f * zz - 3.f) * gY[12];
    gx -= K3c * (5.f * zz - 1.f) * gY[13]; gz -= 10.f * K3c * x * z * gY[13];
    gx += 2.f * K3e * x * z * gY[14]; gy -= 2.f * K3e * y * z * gY[14]; gz += K3e * (xx - yy) * gY[14];
    gx -= K3a * (3.f * xx - 3.f * yy) * gY[15]; gy += 6.f * K3a * x * y * gY[15];
  }
  out[0] = gx; out[1] = gy; out[2] = gz;
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

// Element i of a shared-memory array of T, widened to FP32.
template <typename T> __device__ inline float lds(const T* p, int i);
template <> __device__ inline float lds<float>(const float* p, int i) { return p[i]; }
template <> __device__ inline float lds<__nv_bfloat16>(const __nv_bfloat16* p, int i) {
  return __bfloat162float(p[i]);
}
// The same through a volatile pointer: the compiler neither caches nor reuses it.
template <typename T> __device__ inline float lds_volatile(const T* p, int i);
template <> __device__ inline float lds_volatile<float>(const float* p, int i) {
  return reinterpret_cast<const volatile float*>(p)[i];
}
template <> __device__ inline float lds_volatile<__nv_bfloat16>(const __nv_bfloat16* p, int i) {
  return __uint_as_float((uint32_t)reinterpret_cast<const volatile unsigned short*>(p)[i] << 16);
}

// Global loads of one Gaussian's parameters, widened to FP32.
template <typename T>
__device__ inline void load_gauss(const SceneDev& S, int64_t g, float m[3], float s[3], float q[4], float& o);
template <>
__device__ inline void load_gauss<float>(const SceneDev& S, int64_t g, float m[3], float s[3], float q[4],
                                         float& o) {
  const float* mp = static_cast<const float*>(S.means) + 3 * g;
  const float* sp = static_cast<const float*>(S.scales) + 3 * g;
  for (int k = 0; k < 3; ++k) { m[k] = __ldg(mp + k); s[k] = __ldg(sp + k); }
  const float* qp = static_cast<const float*>(S.quats) + 4 * g;
  if ((reinterpret_cast<uintptr_t>(qp) & 15) == 0) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(qp));
    q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
  } else {
    for (int k = 0; k < 4; ++k) q[k] = __ldg(qp + k);
  }
  o = __ldg(static_cast<const float*>(S.opacities) + g);
}
template <>
__device__ inline void load_gauss<__nv_bfloat16>(const SceneDev& S, int64_t g, float m[3], float s[3], float q[4],
                                                 float& o) {
  const __nv_bfloat16* mp = static_cast<const __nv_bfloat16*>(S.means) + 3 * g;
  const __nv_bfloat16* sp = static_cast<const __nv_bfloat16*>(S.scales) + 3 * g;
  const __nv_bfloat16* qp = static_cast<const __nv_bfloat16*>(S.quats) + 4 * g;
  for (int k = 0; k < 3; ++k) { m[k] = __bfloat162float(mp[k]); s[k] = __bfloat162float(sp[k]); }
  for (int k = 0; k < 4; ++k) q[k] = __bfloat162float(qp[k]);
  o = __bfloat162float(static_cast<const __nv_bfloat16*>(S.opacities)[g]);
}

// A Gaussian's 3K SH coefficients, widened to FP32 (16-byte loads when aligned).
template <typename T, int K>
__device__ inline void load_sh(const SceneDev& S, int64_t g, float* c) {
  const T* p = static_cast<const T*>(S.sh) + 3 * K * g;
  constexpr int PER = 16 / (int)sizeof(T);
  if ((3 * K) % PER == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
    for (int f = 0; f < 3 * K / PER; ++f) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + f);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (sizeof(T) == 4) {
          c[PER * f + k] = __uint_as_float(w[k]);
        } else {
          c[PER * f + 2 * k] = __uint_as_float(w[k] << 16);
          c[PER * f + 2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 3 * K; ++j) c[j] = ldf(p, j);
  }
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
// GEO: forward-only geometry (alpha, depth, normal); SH coefficients are not
// read and the colour is left 0.  One launch covers every SH degree.
template <typename T, int D, bool GEO>
__global__ void __launch_bounds__(kPreThreads, 5)
k_preprocess(const FrameDev* __restrict__ fd, void* __restrict__ ws, Layout L) {
  pdl_wait();
  pdl_trigger();
  constexpr int K = (D + 1) * (D + 1);
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
    if (S.dtype != dtype_code<T>() || (!GEO && S.sh_degree != D)) continue;
    const int t = threadIdx.x;
    if (t >= ch.n) continue;
    const int64_t e = ch.e0 + t, g = ch.g0 + t;
    float m[3], s[3], q[4], o;
    load_gauss<T>(S, g, m, s, q, o);
    if (S.filter_var) filter3d_apply(__ldg(S.filter_var + g), s, o);   // Mip-Splatting 3D filter
    float chk = 0.f;   // inf * 0 and nan * 0 are nan
    for (int k = 0; k < 3; ++k) chk += m[k] * 0.f + s[k] * 0.f;
    for (int k = 0; k < 4; ++k) chk += q[k] * 0.f;
    chk += o * 0.f;
    const bool finite = chk == 0.f;
    if (!finite) ++nonfinite;
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
      // SH coefficients are read only for entries that survive the culling
      float c[3 * K];
      if constexpr (!GEO) {
        load_sh<T, K>(S, g, c);
        float shchk = 0.f;
#pragma unroll
        for (int j = 0; j < 3 * K; ++j) shchk += c[j] * 0.f;
        if (shchk != 0.f) { valid = false; ++nonfinite; }
        // the colour at once, so the SH registers are free before the geometry
        float d[3] = {m[0] - V.campos[0], m[1] - V.campos[1], m[2] - V.campos[2]};
        float il = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        float Y[16];
        sh_basis(d[0] * il, d[1] * il, d[2] * il, Y);
#pragma unroll
        for (int ch3 = 0; ch3 < 3; ++ch3) {
          float acc = 0.5f;
#pragma unroll
          for (int j = 0; j < K; ++j) acc += Y[j] * c[3 * j + ch3];
          rgb[ch3] = fmaxf(acc, 0.f);
        }
      }
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
      valid = valid && (det > 0.f) && isfinite(conic[0]) && isfinite(conic[1]) && isfinite(conic[2]) &&
              isfinite(pp[0]) && isfinite(pp[1]) && isfinite(nn[0]) && isfinite(nn[1]) && isfinite(nn[2]);
    }
    if (valid) {
      float4* r = rec + 4 * e;
      // the conic times log2(e), diagonal halved: the compositing evaluates
      // sigma log2(e) directly and exp(-sigma) as a power of two
      constexpr float kL2E = 1.44269504088896341f;   // log2(e)
      r[0] = make_float4(u, v, conic[0] * (0.5f * kL2E), conic[1] * kL2E);
      r[1] = make_float4(conic[2] * (0.5f * kL2E), o, nn[1], nn[2]);
      r[2] = make_float4(pp[0], pp[1], z, 0.f);
      r[3] = make_float4(rgb[0], rgb[1], rgb[2], nn[0]);
      rect[e] = make_short4((short)i0, (short)i1, (short)j0, (short)j1);
      key[e] = __float_as_uint(z);
      touched[e] = (uint32_t)(((i1 >> sx) - (i0 >> sx) + 1) * ((j1 >> sy) - (j0 >> sy) + 1)) |
                   (uint32_t)(rgb[0] > 0.f) << kTouchedBits | (uint32_t)(rgb[1] > 0.f) << (kTouchedBits + 1) |
                   (uint32_t)(rgb[2] > 0.f) << (kTouchedBits + 2);
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
// FILT: the scene carries Mip-Splatting 3D filter variances.
template <typename T, int D, bool FILT>
__global__ void __launch_bounds__(kPreThreads, 5)
k_preprocess_bwd(const FrameDev* __restrict__ fd, void* __restrict__ ws, Layout L, GradPtrs gp) {
  pdl_wait();
  pdl_trigger();
  constexpr int K = (D + 1) * (D + 1);
  const uint32_t* touched = at<uint32_t>(ws, L.touched);
  const float4* g2d = at<float4>(ws, L.grad2d);
  const float lp = fd->lowpass;
  // Single-view scenes store their gradients through shared memory: each thread
  // writes its rows there, then the block writes the chunk's contiguous
  // gradient ranges with coalesced stores (the SH rows as 16-byte pieces).
  constexpr int R4 = (3 * K) / 4;                  // float4s of one SH row
  constexpr bool STAGE_SH = (3 * K) % 4 == 0;
  constexpr int R4P = STAGE_SH ? (R4 | 1) : 1;     // odd row stride: no bank conflicts
  __shared__ float4 s_sh[kPreThreads * R4P];
  __shared__ float s_m[3 * kPreThreads], s_s[3 * kPreThreads], s_o[kPreThreads];
  __shared__ float4 s_q[kPreThreads];
  for (int bi = blockIdx.x; bi < fd->n_chunks; bi += gridDim.x) {
    const Chunk ch = chunk_of(fd, bi);
    const ViewDev& V = fd->views[ch.view];
    const SceneDev& S = fd->scenes[V.scene];
    if (S.dtype != dtype_code<T>() || S.sh_degree != D || (S.filter_var != nullptr) != FILT) continue;
    const int t = threadIdx.x;
    const bool act = t < ch.n;
    const gs_scene_grads& Dg = gp.g[V.scene];
    const bool store = S.n_views == 1;  // else the buffers were zeroed and we add
    const bool stage_sh = STAGE_SH && store && Dg.dsh &&
                          (reinterpret_cast<uintptr_t>(Dg.dsh) & 15) == 0;   // block-uniform
    auto put = [&](float* dst, int64_t i, float v) {
      if (store) dst[i] = v;
      else if (v != 0.f) atomicAdd(dst + i, v);
    };
    const int64_t e = ch.e0 + (act ? t : 0), g = ch.g0 + (act ? t : 0);
    float gm[3] = {0.f, 0.f, 0.f}, gsc[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, go = 0.f;
    const uint32_t tw = act ? touched[e] : 0u;   // 0: culled; else tiles and the colour clamps
    if ((tw & kTouchedMask) == 0u) {
      if (stage_sh) {
#pragma unroll
        for (int f = 0; f < R4; ++f) s_sh[t * R4P + f] = make_float4(0.f, 0.f, 0.f, 0.f);
      } else if (act && store && Dg.dsh) {
        float* dst = Dg.dsh + 3 * K * g;
        for (int j = 0; j < 3 * K; ++j) dst[j] = 0.f;
      }
    } else {
      float m[3], s[3], q[4], o;
      load_gauss<T>(S, g, m, s, q, o);
      const float s0[3] = {s[0], s[1], s[2]};
      const float fv = FILT ? __ldg(S.filter_var + g) : 0.f;
      if (FILT) filter3d_apply(fv, s, o);   // s, o: filtered scales and opacity
      // ---- colour first (its registers are free again before the geometry):
      // rgb = max(sum_j Y_j c_j + 1/2, 0); the forward noted in the entry's
      // touched word which channels were above 0 (the others are clamped)
      {
        const float4 grgb4 = g2d[4 * e + 3];
        const float gval[3] = {(tw >> kTouchedBits) & 1u ? grgb4.x : 0.f,
                               (tw >> (kTouchedBits + 1)) & 1u ? grgb4.y : 0.f,
                               (tw >> (kTouchedBits + 2)) & 1u ? grgb4.z : 0.f};
        const float d[3] = {m[0] - V.campos[0], m[1] - V.campos[1], m[2] - V.campos[2]};
        const float il = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const float dir[3] = {d[0] * il, d[1] * il, d[2] * il};
        float Y[16], gY[16];
        sh_basis(dir[0], dir[1], dir[2], Y);
        {
          float c[3 * K];
          load_sh<T, K>(S, g, c);
#pragma unroll
          for (int j = 0; j < K; ++j) gY[j] = c[3 * j] * gval[0] + c[3 * j + 1] * gval[1] + c[3 * j + 2] * gval[2];
        }
        float gdir[3];
        sh_basis_vjp<K>(dir[0], dir[1], dir[2], gY, gdir);
        const float dd = dir[0] * gdir[0] + dir[1] * gdir[1] + dir[2] * gdir[2];
        for (int k = 0; k < 3; ++k) gm[k] += (gdir[k] - dir[k] * dd) * il;
        // dL/dc_jk = Y_j gval_k
        if (stage_sh) {
#pragma unroll
          for (int f = 0; f < R4; ++f) {
            float v4[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) v4[c] = Y[(4 * f + c) / 3] * gval[(4 * f + c) % 3];
            s_sh[t * R4P + f] = make_float4(v4[0], v4[1], v4[2], v4[3]);
          }
        } else if (Dg.dsh) {
          float* dst = Dg.dsh + 3 * K * g;
#pragma unroll
          for (int j = 0; j < K; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) put(dst, 3 * j + k, Y[j] * gval[k]);
        }
      }
      Geo geo;
      geo_forward(V, m, s, q, lp, geo);
      const Geo& gg = geo;
      const float4 ga = g2d[4 * e], gb4 = g2d[4 * e + 1], gc4 = g2d[4 * e + 2], gd4 = g2d[4 * e + 3];
      // the compositing backward leaves sums linear in the conic, p and o:
      // (S gs dx, S gs dy, S gs dx^2, S gs dx dy, S gs dy^2, S gs, -, S sd), gs = dL/dsigma;
      // sigma = (c_a dx^2 + c_c dy^2) / 2 + c_b dx dy, alpha = o exp(-sigma), d = z + p . Delta
      const float gz = gb4.w;
      const float gu = gg.ca * ga.x + gg.cb * ga.y + gg.p0 * gz;
      const float gv = gg.cb * ga.x + gg.cc * ga.y + gg.p1 * gz;
      const float gca = 0.5f * ga.z, gcb = ga.w, gcc = 0.5f * gb4.x;
      go = -gb4.y / o;
      const float gp0 = gc4.x, gp1 = gc4.y, gn[3] = {gd4.w, gc4.z, gc4.w};

      // ---- p = (z/t) q -----------------------------------------------------------
      const float it = 1.f / gg.tc;
      const float zt = gg.z * it;
      float gq0 = zt * gp0, gq1 = zt * gp1;
      const float qgp = gg.q0 * gp0 + gg.q1 * gp1;
      const float gz_tot = gz + qgp * it;
      const float gtc = -gg.z * it * it * qgp;
      // ---- n = mv / |mv|, mv = -(q0 J0 + q1 J1 + J2) ---------------------------------
      const float ndg = gg.n[0] * gn[0] + gg.n[1] * gn[1] + gg.n[2] * gn[2];
      const float iml = 1.f / gg.mlen;
      float gmv[3];
      for (int k = 0; k < 3; ++k) gmv[k] = (gn[k] - gg.n[k] * ndg) * iml;
      gq0 += -(gg.j00 * gmv[0] + gg.j02 * gmv[2]);
      gq1 += -(gg.j11 * gmv[1] + gg.j12 * gmv[2]);
      float gj00 = -gg.q0 * gmv[0], gj02 = -gg.q0 * gmv[2];
      float gj11 = -gg.q1 * gmv[1], gj12 = -gg.q1 * gmv[2];
      float gJ2[3] = {-gmv[0], -gmv[1], -gmv[2]};
      // ---- q = -C b --------------------------------------------------------------------
      const float gca_t = gca - gq0 * gg.b0;
      const float gcb_t = gcb - (gq0 * gg.b1 + gq1 * gg.b0);
      const float gcc_t = gcc - gq1 * gg.b1;
      const float gb0 = -(gg.ca * gq0 + gg.cb * gq1);
      const float gb1 = -(gg.cb * gq0 + gg.cc * gq1);
      // ---- C = A^-1: dA = -C dC C (symmetric, off-diagonal counted once) ---------------
      const float h = 0.5f * gcb_t;
      const float X00 = gg.ca * gca_t + gg.cb * h, X01 = gg.ca * h + gg.cb * gcc_t;
      const float X10 = gg.cb * gca_t + gg.cc * h, X11 = gg.cb * h + gg.cc * gcc_t;
      const float gA00 = -(X00 * gg.ca + X01 * gg.cb);
      const float gA01 = -(X00 * gg.cb + X01 * gg.cc);
      const float gA11 = -(X10 * gg.cb + X11 * gg.cc);
      // ---- Sigma' = G G^T ----------------------------------------------------------------
      const float gS01 = 2.f * gA01;
      float gG[3][3];
      for (int k = 0; k < 3; ++k) {
        gG[0][k] = 2.f * gA00 * gg.G[0][k] + gS01 * gg.G[1][k] + gb0 * gg.G[2][k];
        gG[1][k] = 2.f * gA11 * gg.G[1][k] + gS01 * gg.G[0][k] + gb1 * gg.G[2][k];
        gG[2][k] = gb0 * gg.G[0][k] + gb1 * gg.G[1][k];
      }
      // ---- G = T M --------------------------------------------------------------------------
      float gT[3][3], gM[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          gT[i][j] = gG[i][0] * gg.M[j][0] + gG[i][1] * gg.M[j][1] + gG[i][2] * gg.M[j][2];
          gM[i][j] = gg.T[0][i] * gG[0][j] + gg.T[1][i] * gG[1][j] + gg.T[2][i] * gG[2][j];
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
        gsc[k] = gM[0][k] * gg.Rq[0][k] + gM[1][k] * gg.Rq[1][k] + gM[2][k] * gg.Rq[2][k];
        for (int i = 0; i < 3; ++i) gR[i][k] = gM[i][k] * s[k];
      }
      // ---- Rq(qn) and normalisation --------------------------------------------------------------
      {
        const float w = gg.qn[0], x = gg.qn[1], y = gg.qn[2], z = gg.qn[3];
        float gqn[4];
        gqn[0] = 2.f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
        gqn[1] = 2.f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.f * x * gR[1][1] - w * gR[1][2] +
                        z * gR[2][0] + w * gR[2][1] - 2.f * x * gR[2][2]);
        gqn[2] = 2.f * (-2.f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                        w * gR[2][0] + z * gR[2][1] - 2.f * y * gR[2][2]);
        gqn[3] = 2.f * (-2.f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2.f * z * gR[1][1] +
                        y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
        const float qd = w * gqn[0] + x * gqn[1] + y * gqn[2] + z * gqn[3];
        const float iq = 1.f / gg.qnorm;
        for (int k = 0; k < 4; ++k) gq[k] = (gqn[k] - gg.qn[k] * qd) * iq;
      }
      // ---- J(x_c), t_c, u, v, z --------------------------------------------------------------------
      float gx[3] = {0.f, 0.f, 0.f};
      const float iz = gg.iz, iz2 = iz * iz;
      gx[2] += -V.fx * iz2 * gj00 - V.fy * iz2 * gj11;
      if (!gg.clx) {   // j02 = -fx x / z^2
        gx[0] += -V.fx * iz2 * gj02;
        gx[2] += 2.f * V.fx * gg.xc[0] * iz2 * iz * gj02;
      } else {        // j02 = -fx L / z
        gx[2] += V.fx * gg.txc * iz2 * gj02;
      }
      if (!gg.cly) {
        gx[1] += -V.fy * iz2 * gj12;
        gx[2] += 2.f * V.fy * gg.xc[1] * iz2 * iz * gj12;
      } else {
        gx[2] += V.fy * gg.tyc * iz2 * gj12;
      }
      const float jd = gg.J2[0] * gJ2[0] + gg.J2[1] * gJ2[1] + gg.J2[2] * gJ2[2];
      for (int k = 0; k < 3; ++k) gx[k] += (gJ2[k] - gg.J2[k] * jd) * it + gtc * gg.J2[k];
      gx[0] += gu * V.fx * iz;
      gx[1] += gv * V.fy * iz;
      gx[2] += -(gu * V.fx * gg.xc[0] + gv * V.fy * gg.xc[1]) * iz2 + gz_tot;
      for (int k = 0; k < 3; ++k) gm[k] += V.R[k] * gx[0] + V.R[3 + k] * gx[1] + V.R[6 + k] * gx[2];
      // ---- 3D filter: s~ = sqrt(s^2 + v), o' = o prod s/s~ ------------------------------------------
      if (FILT) {
        float rp = 1.f;
        for (int k = 0; k < 3; ++k) rp *= s0[k] / s[k];
        for (int k = 0; k < 3; ++k)
          gsc[k] = gsc[k] * (s0[k] / s[k]) + go * o * fv / (s0[k] * s[k] * s[k]);
        go *= rp;
      }
    }
    if (store) {
      for (int k = 0; k < 3; ++k) { s_m[3 * t + k] = gm[k]; s_s[3 * t + k] = gsc[k]; }
      s_q[t] = make_float4(gq[0], gq[1], gq[2], gq[3]);
      s_o[t] = go;
      __syncthreads();
      const int n = ch.n;
      if (Dg.dmeans) for (int i = t; i < 3 * n; i += kPreThreads) Dg.dmeans[3 * ch.g0 + i] = s_m[i];
      if (Dg.dscales) for (int i = t; i < 3 * n; i += kPreThreads) Dg.dscales[3 * ch.g0 + i] = s_s[i];
      if (Dg.dquats)
        for (int i = t; i < 4 * n; i += kPreThreads) Dg.dquats[4 * ch.g0 + i] = (&s_q[0].x)[i];
      if (Dg.dopacities && act) Dg.dopacities[ch.g0 + t] = s_o[t];
      if constexpr (STAGE_SH) {
        if (stage_sh) {
          float4* dst = reinterpret_cast<float4*>(Dg.dsh + 3 * K * ch.g0);
          for (int f = t; f < R4 * n; f += kPreThreads) dst[f] = s_sh[(f / R4) * R4P + f % R4];
        }
      }
      __syncthreads();   // the staging rows are rewritten by the next chunk
    } else if (act) {
      if (Dg.dmeans) for (int k = 0; k < 3; ++k) put(Dg.dmeans, 3 * g + k, gm[k]);
      if (Dg.dscales) for (int k = 0; k < 3; ++k) put(Dg.dscales, 3 * g + k, gsc[k]);
      if (Dg.dquats) for (int k = 0; k < 4; ++k) put(Dg.dquats, 4 * g + k, gq[k]);
      if (Dg.dopacities) put(Dg.dopacities, g, go);
    }
  }
}

// ---------------------------------------------------------------------------
// Mip-Splatting 3D filter variance from the cameras: v = c min_n (z_n / f_n)^2
// over the views n of the scene in which the centre is in front of the near
// plane and projects inside the image widened by 15 % on each side; Gaussians
// seen by no view get the largest v of the seen ones.  Pass 1 writes v (or -1)
// and folds the maximum into the header; pass 2 fills the unseen.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_filter3d(const FrameDev* __restrict__ fd, void* __restrict__ ws, Layout L, int scene,
                           float scale, float* __restrict__ out) {
  const SceneDev& S = fd->scenes[scene];
  Header* hdr = at<Header>(ws, L.hdr);
  const T* mp = static_cast<const T*>(S.means);
  float vmax = 0.f;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < S.n; g += (int64_t)gridDim.x * blockDim.x) {
    const float m0 = ldf<T>(mp, 3 * g), m1 = ldf<T>(mp, 3 * g + 1), m2 = ldf<T>(mp, 3 * g + 2);
    float best = 3.4e38f;
    bool seen = false;
    for (int v = 0; v < fd->n_views; ++v) {
      const ViewDev& V = fd->views[v];
      if (V.scene != scene) continue;
      const float x = V.R[0] * m0 + V.R[1] * m1 + V.R[2] * m2 + V.t[0];
      const float y = V.R[3] * m0 + V.R[4] * m1 + V.R[5] * m2 + V.t[1];
      const float z = V.R[6] * m0 + V.R[7] * m1 + V.R[8] * m2 + V.t[2];
      if (!(z > V.near_plane)) continue;
      const float u = V.fx * x / z + V.cx, w = V.fy * y / z + V.cy;
      const float mw = 0.15f * V.width, mh = 0.15f * V.height;
      if (u >= -mw && u <= V.width + mw && w >= -mh && w <= V.height + mh) {
        const float r = z / V.fx;
        best = fminf(best, r * r);
        seen = true;
      }
    }
    const float val = seen ? scale * best : -1.f;
    out[g] = val;
    vmax = fmaxf(vmax, val);
  }
  for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xFFFFFFFFu, vmax, o));
  if ((threadIdx.x & 31) == 0 && vmax > 0.f) atomicMax(&hdr->filter_max, __float_as_uint(vmax));
}

__global__ void k_filter3d_fill(const FrameDev* __restrict__ fd, void* __restrict__ ws, Layout L, int scene,
                                float* __restrict__ out) {
  const int64_t n = fd->scenes[scene].n;
  const float fill = __uint_as_float(at<Header>(ws, L.hdr)->filter_max);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    if (out[g] < 0.f) out[g] = fill;
}

cudaError_t launch_filter3d(void* ws, const Layout& L, const FrameDev& hf, int scene, float scale, float* out,
                            cudaStream_t s) {
  const int64_t n = hf.scenes[scene].n;
  if (n == 0) return cudaSuccess;
  const FrameDev* fd = at<FrameDev>(ws, L.frame);
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
  if (hf.scenes[scene].dtype == GS_BF16)
    k_filter3d<__nv_bfloat16><<<grid, 256, 0, s>>>(fd, ws, L, scene, scale, out);
  else
    k_filter3d<float><<<grid, 256, 0, s>>>(fd, ws, L, scene, scale, out);
  k_filter3d_fill<<<grid, 256, 0, s>>>(fd, ws, L, scene, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers: one launch per (dtype, SH degree) present in the frame
// ---------------------------------------------------------------------------
static int grid_chunks(int n_chunks) {
  int b = n_chunks < 1 ? 1 : n_chunks;
  return b > 148 * 32 ? 148 * 32 : b;
}

template <typename T>
static cudaError_t fwd_t(int deg, const FrameDev* fd, void* ws, const Layout& L, int grid, cudaStream_t s) {
  switch (deg) {
    case 0: launch_pdl(k_preprocess<T, 0, false>, grid, kPreThreads, 0, s, fd, ws, L); break;
    case 1: launch_pdl(k_preprocess<T, 1, false>, grid, kPreThreads, 0, s, fd, ws, L); break;
    case 2: launch_pdl(k_preprocess<T, 2, false>, grid, kPreThreads, 0, s, fd, ws, L); break;
    default: launch_pdl(k_preprocess<T, 3, false>, grid, kPreThreads, 0, s, fd, ws, L); break;
  }
  return cudaGetLastError();
}

template <typename T, bool FILT>
static cudaError_t bwd_t(int deg, const FrameDev* fd, void* ws, const Layout& L, const GradPtrs& gp, int grid,
                         cudaStream_t s) {
  switch (deg) {
    case 0: launch_pdl(k_preprocess_bwd<T, 0, FILT>, grid, kPreThreads, 0, s, fd, ws, L, gp); break;
    case 1: launch_pdl(k_preprocess_bwd<T, 1, FILT>, grid, kPreThreads, 0, s, fd, ws, L, gp); break;
    case 2: launch_pdl(k_preprocess_bwd<T, 2, FILT>, grid, kPreThreads, 0, s, fd, ws, L, gp); break;
    default: launch_pdl(k_preprocess_bwd<T, 3, FILT>, grid, kPreThreads, 0, s, fd, ws, L, gp); break;
  }
  return cudaGetLastError();
}

// Bit (4 * dtype + degree), plus 8 when the scene is filtered, set for every
// kind of scene that a view renders.
static unsigned kinds(const FrameDev& hf) {
  unsigned k = 0;
  for (int v = 0; v < hf.n_views; ++v) {
    const SceneDev& S = hf.scenes[hf.views[v].scene];
    if (S.n > 0) k |= 1u << (4 * S.dtype + S.sh_degree + (S.filter_var ? 8 : 0));
  }
  return k;
}

cudaError_t launch_preprocess(void* ws, const Layout& L, const FrameDev& hf, cudaStream_t s) {
  const FrameDev* fd = at<FrameDev>(ws, L.frame);
  const unsigned k0 = kinds(hf);
  const unsigned k = (k0 | (k0 >> 8)) & 0xFFu;   // the forward reads the filter at run time
  const int grid = grid_chunks(hf.n_chunks);
  cudaError_t e = cudaSuccess;
  if (hf.geometry_only) {   // one launch per dtype, SH not read
    if (k & (0xFu << (4 * GS_F32))) launch_pdl(k_preprocess<float, 0, true>, grid, kPreThreads, 0, s, fd, ws, L);
    if (k & (0xFu << (4 * GS_BF16)))
      launch_pdl(k_preprocess<__nv_bfloat16, 0, true>, grid, kPreThreads, 0, s, fd, ws, L);
    return cudaGetLastError();
  }
  for (int deg = 0; deg < 4 && e == cudaSuccess; ++deg) {
    if (k & (1u << (4 * GS_F32 + deg))) e = fwd_t<float>(deg, fd, ws, L, grid, s);
    if (e == cudaSuccess && (k & (1u << (4 * GS_BF16 + deg)))) e = fwd_t<__nv_bfloat16>(deg, fd, ws, L, grid, s);
  }
  return e;
}

cudaError_t launch_preprocess_bwd(void* ws, const Layout& L, const FrameDev& hf, const GradPtrs& gp,
                                  cudaStream_t s) {
  const FrameDev* fd = at<FrameDev>(ws, L.frame);
  const unsigned k = kinds(hf);
  const int grid = grid_chunks(hf.n_chunks);
  cudaError_t e = cudaSuccess;
  for (int deg = 0; deg < 4 && e == cudaSuccess; ++deg) {
    if (k & (1u << (4 * GS_F32 + deg))) e = bwd_t<float, false>(deg, fd, ws, L, gp, grid, s);
    if (e == cudaSuccess && (k & (1u << (4 * GS_BF16 + deg))))
      e = bwd_t<__nv_bfloat16, false>(deg, fd, ws, L, gp, grid, s);
    if (e == cudaSuccess && (k & (1u << (8 + 4 * GS_F32 + deg)))) e = bwd_t<float, true>(deg, fd, ws, L, gp, grid, s);
    if (e == cudaSuccess && (k & (1u << (8 + 4 * GS_BF16 + deg))))
      e = bwd_t<__nv_bfloat16, true>(deg, fd, ws, L, gp, grid, s);
  }
  return e;
}

}  // namespace gs
