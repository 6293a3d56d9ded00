// tode_peak.cu -- micro-benchmark kernels that measure the denominators of
// the solver kernels' rooflines on the running GPU: the FP32 and FP64 FMA
// rates, the MUFU rates of ex2.approx and tanh.approx (the transcendental
// unit the dopri5 controller's power and the MLP field's tanh use), and an
// empty kernel for the launch and graph-replay rates.  Each arithmetic
// kernel runs UNROLL independent dependency chains per thread so that the
// pipe, not the latency of one chain, is the limit; the result is written
// to a sink so the compiler keeps the work.  The caller times the launch
// (CUDA events on its stream) and divides the operation count by the time.
#include "tode_internal.h"

namespace tode {

constexpr int PEAK_UNROLL = 8;

__global__ void k_peak_fma32(int iters, float* sink) {
  float a[PEAK_UNROLL];
#pragma unroll
  for (int u = 0; u < PEAK_UNROLL; ++u) a[u] = (float)(threadIdx.x + u) * 1e-3f;
  const float m = 0.999f, c = 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u) a[u] = __fmaf_rn(a[u], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int u = 0; u < PEAK_UNROLL; ++u) s += a[u];
  if (s == 12345.0f) sink[threadIdx.x] = s;  // never true; keeps the chains
}

// FP32x2: Blackwell's paired FMA (two IEEE FMAs per issue), the form the
// linear field's products use
__global__ void k_peak_ffma2(int iters, float* sink) {
  float2 a[PEAK_UNROLL];
#pragma unroll
  for (int u = 0; u < PEAK_UNROLL; ++u)
    a[u] = make_float2((float)(threadIdx.x + u) * 1e-3f, (float)(threadIdx.x - u) * 1e-3f);
  const float2 m = make_float2(0.999f, 0.998f), c = make_float2(1e-4f, 2e-4f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u) a[u] = __ffma2_rn(a[u], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int u = 0; u < PEAK_UNROLL; ++u) s += a[u].x + a[u].y;
  if (s == 12345.0f) sink[threadIdx.x] = s;
}

__global__ void k_peak_fma64(int iters, float* sink) {
  double a[PEAK_UNROLL];
#pragma unroll
  for (int u = 0; u < PEAK_UNROLL; ++u) a[u] = (double)(threadIdx.x + u) * 1e-3;
  const double m = 0.999, c = 1e-4;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u) a[u] = __fma_rn(a[u], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < PEAK_UNROLL; ++u) s += a[u];
  if (s == 12345.0) sink[threadIdx.x] = (float)s;
}

__global__ void k_peak_ex2(int iters, float* sink) {
  float a[PEAK_UNROLL];
#pragma unroll
  for (int u = 0; u < PEAK_UNROLL; ++u) a[u] = -(float)(threadIdx.x % 7 + u) * 1e-2f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[u]));
      a[u] = -y;  // stays in (-1, 0]: no overflow
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int u = 0; u < PEAK_UNROLL; ++u) s += a[u];
  if (s == 12345.0f) sink[threadIdx.x] = s;
}

__global__ void k_peak_tanh(int iters, float* sink) {
  float a[PEAK_UNROLL];
#pragma unroll
  for (int u = 0; u < PEAK_UNROLL; ++u) a[u] = (float)(threadIdx.x % 5 + u) * 0.1f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u) {
      float y;
      asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(a[u]));
      a[u] = y;
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int u = 0; u < PEAK_UNROLL; ++u) s += a[u];
  if (s == 12345.0f) sink[threadIdx.x] = s;
}

__global__ void k_peak_empty() {}

}  // namespace tode

extern "C" tode_err tode_peak_kernel(int kind, int grid, int block, int iters, float* sink,
                                     void* stream) {
  if (grid < 1 || block < 1 || block > 1024 || iters < 0 || (kind != TODE_PEAK_EMPTY && !sink))
    return TODE_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  switch (kind) {
    case TODE_PEAK_FMA32: tode::k_peak_fma32<<<grid, block, 0, st>>>(iters, sink); break;
    case TODE_PEAK_FFMA2: tode::k_peak_ffma2<<<grid, block, 0, st>>>(iters, sink); break;
    case TODE_PEAK_FMA64: tode::k_peak_fma64<<<grid, block, 0, st>>>(iters, sink); break;
    case TODE_PEAK_EX2: tode::k_peak_ex2<<<grid, block, 0, st>>>(iters, sink); break;
    case TODE_PEAK_TANH: tode::k_peak_tanh<<<grid, block, 0, st>>>(iters, sink); break;
    case TODE_PEAK_EMPTY: tode::k_peak_empty<<<grid, block, 0, st>>>(); break;
    default: return TODE_EINVAL;
  }
  TODE_CUDA_TRY(cudaGetLastError());
  return TODE_OK;
}
