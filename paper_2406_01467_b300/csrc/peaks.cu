// Throughput probes of the units the compositing kernels run on: FP32 fused
// multiply-add (scalar and packed FP32x2), the MUFU base-2 exponential, and
// shared-memory reads.  The paper has no counterpart; these give the measured
// denominators of the compositing rooflines on the GPU the library runs on.
//
// Each probe is a resident wave of blocks whose threads run long chains of the
// one operation with enough independent chains per thread to hide its latency,
// so the launch time is set by that unit's throughput.  The caller times the
// launch (CUDA events) and divides the work it reports by the time.
#include "gs_internal.cuh"

namespace gs {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;    // independent dependency chains per thread
constexpr int kUnroll = 16;   // operations per chain per loop trip

__device__ inline float probe_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The sink store happens only for a value the chains never produce; it keeps
// the compiler from removing them.
__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma(float* sink, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 1e-3f + i;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = __fmaf_rn(a[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.2345f) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma2(float* sink, int iters, float b, float c) {
  float2 a[kChains];
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, i * 0.5f);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
  if (s == -1.2345f) sink[0] = s;
}

// x -> 2^-x stays in (0, 1] from a start in [0, 1]: no overflow, no denormals.
__global__ void __launch_bounds__(kProbeThreads) k_probe_ex2(float* sink, int iters) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (threadIdx.x & 31) * (1.f / 32.f) + i * 0.01f;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = probe_ex2(-a[i]);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.2345f) sink[0] = s;
}

// 16-byte shared-memory reads, lane l of every warp reading consecutive
// float4s (512 bytes per warp instruction, no bank conflict); the address
// moves every read so no load is loop invariant.
constexpr int kProbeSmemVec = 1024;   // float4s of the block's buffer (16 KB)

__global__ void __launch_bounds__(kProbeThreads) k_probe_lds(float* sink, int iters) {
  __shared__ float4 buf[kProbeSmemVec];
  for (int i = threadIdx.x; i < kProbeSmemVec; i += kProbeThreads)
    buf[i] = make_float4(i * 1e-3f, 1.f, 2.f, 3.f);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int base = threadIdx.x & (kProbeSmemVec - 1);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const float4 v = buf[(base + u * 32) & (kProbeSmemVec - 1)];
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    base = (base + kUnroll * 32 + 32) & (kProbeSmemVec - 1);
  }
  const float s = acc.x + acc.y + acc.z + acc.w;
  if (s == -1.2345f) sink[0] = s;
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_peak_probe(int32_t kind, int32_t iters, float* sink, int64_t* work, void* stream) {
  if (iters < 1 || iters > (1 << 24)) return set_error(GS_ERR_INVALID_ARG, "iters must be in [1, 2^24]");
  if (!sink || !work) return set_error(GS_ERR_INVALID_ARG, "sink and work must not be NULL");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(GS_ERR_CUDA, "gs_peak_probe: %s", cudaGetErrorString(e));
  int per_sm = 1;
  const void* fn = nullptr;
  switch (kind) {
    case GS_PEAK_FFMA: fn = (const void*)k_probe_ffma; break;
    case GS_PEAK_FFMA2: fn = (const void*)k_probe_ffma2; break;
    case GS_PEAK_EX2: fn = (const void*)k_probe_ex2; break;
    case GS_PEAK_LDS128: fn = (const void*)k_probe_lds; break;
    default: return set_error(GS_ERR_INVALID_ARG, "unknown probe kind %d", kind);
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kProbeThreads, 0);
  if (e != cudaSuccess) return set_error(GS_ERR_CUDA, "gs_peak_probe: %s", cudaGetErrorString(e));
  const int blocks = sms * std::max(per_sm, 1);
  const int64_t threads = int64_t(blocks) * kProbeThreads;
  const int64_t per_thread = int64_t(iters) * kUnroll;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (kind) {
    case GS_PEAK_FFMA:
      k_probe_ffma<<<blocks, kProbeThreads, 0, s>>>(sink, iters, 0.999f, 1e-3f);
      *work = threads * per_thread * kChains;          // FMAs
      break;
    case GS_PEAK_FFMA2:
      k_probe_ffma2<<<blocks, kProbeThreads, 0, s>>>(sink, iters, 0.999f, 1e-3f);
      *work = threads * per_thread * kChains * 2;      // FMAs (two per instruction)
      break;
    case GS_PEAK_EX2:
      k_probe_ex2<<<blocks, kProbeThreads, 0, s>>>(sink, iters);
      *work = threads * per_thread * kChains;          // exponentials
      break;
    default:
      k_probe_lds<<<blocks, kProbeThreads, 0, s>>>(sink, iters);
      *work = threads * per_thread * 16;               // bytes read
      break;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GS_ERR_CUDA, "gs_peak_probe launch: %s", cudaGetErrorString(e));
  return GS_OK;
}
