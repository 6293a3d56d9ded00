// tode_tc_gemm.cu -- tode_tc_gemm: the MLP field's tensor-core building block
// on its own (C = A * B^T, BF16 inputs, FP32 accumulation in tensor memory),
// so that the operand layout, descriptors and tensor-memory conventions can be
// checked against a plain matrix product.
#include "tode_internal.h"
#include "tode_tc.cuh"

namespace tode {

// flags bit 0: A given as [K][M] row-major and fed MN-major; bit 1: the same
// for B ([K][N]); bit 2: swap the two core-matrix strides of MN-major
// operands (which descriptor field is which is what this probe checks).
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B, float* C, int M,
              int N, int K, int flags, int32_t* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  // MN-major probes keep A and B 100 KB apart so that either reading of the
  // descriptor's two stride fields stays inside this CTA's allocation
  unsigned char* sA = smem;  // 128 x K
  unsigned char* sB = smem + ((flags & 7) ? (size_t)102400 : (size_t)128 * K * 2);  // N x K
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const bool a_mn = flags & 1, b_mn = flags & 2, swap = flags & 4;
  // operands into the core-matrix layout: K-major tiles are [rows][K]; an
  // MN-major operand is stored as the [K][rows] tile it was given, i.e. its
  // M (or N) index runs along the core matrices' 16-byte rows
  for (int e = tid; e < M * K; e += 128) {
    if (a_mn) {
      const int k = e / 128, m = e % 128;
      *reinterpret_cast<uint16_t*>(sA + tc::cm_offset(k, m, 128)) = A[e];
    } else {
      const int row = e / K, k = e % K;
      *reinterpret_cast<uint16_t*>(sA + tc::cm_offset(row, k, K)) = A[e];
    }
  }
  for (int e = tid; e < N * K; e += 128) {
    if (b_mn) {
      const int k = e / N, n = e % N;
      *reinterpret_cast<uint16_t*>(sB + tc::cm_offset(k, n, N)) = B[e];
    } else {
      const int row = e / K, k = e % K;
      *reinterpret_cast<uint16_t*>(sB + tc::cm_offset(row, k, K)) = B[e];
    }
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_base;
  if (M == 64) {
    // M = 64: mark every lane first, so the dump shows where the 64 rows land
    float mark[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) mark[j] = -12345.0f;
    for (int c = 0; c < N; c += 16) tc::tmem_st16(tbase + ((uint32_t)(warp * 32) << 16) + c, mark);
    tc::tmem_wait_st();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }

  if (tid == 0) {
    const uint32_t idesc = tc::idesc_bf16_f32(M, N, a_mn, b_mn);
    const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
    for (int kk = 0; kk < K / 16; ++kk) {
      // K-major: next K slice is 2 core matrices (256 B) along K.  MN-major:
      // 2 groups of 8 K-rows, each MN*16 bytes.
      uint64_t da, db;
      if (a_mn) {
        const uint32_t kst = (uint32_t)M * 16, mst = 128;
        da = swap ? tc::smem_desc(a0 + kk * 2 * kst, kst, mst)
                  : tc::smem_desc(a0 + kk * 2 * kst, mst, kst);
      } else {
        da = tc::smem_desc(a0 + kk * 256, 128, K * 16);
      }
      if (b_mn) {
        const uint32_t kst = (uint32_t)N * 16, nst = 128;
        db = swap ? tc::smem_desc(b0 + kk * 2 * kst, kst, nst)
                  : tc::smem_desc(b0 + kk * 2 * kst, nst, kst);
      } else {
        db = tc::smem_desc(b0 + kk * 256, 128, K * 16);
      }
      tc::mma_bf16(tbase, da, db, idesc, kk > 0);
    }
    tc::mma_commit(&mbar);
  }
  const bool ok = tc::mbar_wait(&mbar, 0);
  if (!ok && lane == 0) atomicExch(err, 1);
  tc::fence_after_sync();
  if (ok && M == 64 && (flags & 8)) {
    // the 16x32bx2 access shape: thread t's 16 values go to C[warp*32 + t][0:16]
    float v[16];
    tc::tmem_ld16x2<32>(tbase + ((uint32_t)(warp * 32) << 16), v);
    tc::tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 16; ++j) C[(size_t)(warp * 32 + lane) * N + j] = v[j];
  } else if (ok) {
    const int row = warp * 32 + lane;
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) C[(size_t)row * N + c + j] = v[j];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

}  // namespace tode

extern "C" tode_err tode_tc_gemm(const void* A, const void* B, float* C, int M, int N, int K,
                                 int flags, int32_t* err, void* stream) {
  if (!A || !B || !C || !err) return TODE_EINVAL;
  if ((M != 128 && M != 64) || N < 16 || N > 256 || N % 16 || K < 16 || K > 256 || K % 16)
    return TODE_EINVAL;
  if (M == 64 && (flags & 1)) return TODE_EINVAL;
  if (flags & ~15) return TODE_EINVAL;
  if ((flags & 8) && (M != 64 || N < 48)) return TODE_EINVAL;
  const int lay = flags & 7;  // operand-layout flags
  if (lay && (K > 128 || N > 144)) return TODE_EINVAL;
  const size_t smem = lay ? (size_t)215040 : (size_t)(128 + N) * K * 2;
  cudaError_t e = cudaFuncSetAttribute(tode::k_tc_gemm,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return TODE_ECUDA;
  }
  tode::k_tc_gemm<<<1, 128, smem, (cudaStream_t)stream>>>((const uint16_t*)A, (const uint16_t*)B,
                                                          C, M, N, K, flags, err);
  if (cudaGetLastError() != cudaSuccess) return TODE_ECUDA;
  return TODE_OK;
}
