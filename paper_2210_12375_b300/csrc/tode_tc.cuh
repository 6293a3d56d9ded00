// tode_tc.cuh -- Blackwell (sm_103a) tensor-core building blocks in inline
// PTX: tensor-memory allocation, tcgen05.mma (kind::f16, BF16 x BF16 -> FP32
// in TMEM), commit to an mbarrier, tensor-memory loads, bulk copies into
// shared memory, and bounded mbarrier waits.
//
// Operand layout in shared memory ("core-matrix", K-major, no swizzle): a
// rows x K tile (rows = M for A, N for B) is cut into 8-row x 8-element core
// matrices of 128 contiguous bytes (row r of a core matrix at r*16 bytes).
// Core matrices adjacent along K are LBO = 128 bytes apart, 8-row groups are
// SBO = K*16 bytes apart, so element (row, k) of a tile with K columns sits
// at  (row/8)*K*16 + (k/8)*128 + (row%8)*16 + (k%8)*2  bytes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tode {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) in a core-matrix tile with K columns
__host__ __device__ __forceinline__ uint32_t cm_offset(int row, int k, int K) {
  return (uint32_t)((row >> 3) * K * 16 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices along K), stride byte offset (between 8-row
// groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // version
  return d;                // base offset 0, layout SWIZZLE_NONE (0)
}

// Descriptor of an MN-major operand stored as a core-matrix tile whose rows
// are the K index (a [K][MN] tile): the leading-dimension field takes the
// stride between groups of 8 K-rows (MN*16 bytes), the stride field the
// 128-byte step between 8-element MN chunks (measured on sm_103a; the other
// assignment gives wrong products).
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t saddr, uint32_t k8_stride,
                                                 uint32_t mn8_stride = 128) {
  return smem_desc(saddr, k8_stride, mn8_stride);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, N/8
// and M/16 fields; a_mn / b_mn select the MN-major operand layout (the
// operand's M or N index runs along the 16-byte rows of its core matrices).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N, bool a_mn = false,
                                                      bool b_mn = false) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------- TMEM
// Whole-warp operations.
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(smem_dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> visible to the tensor cores
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db,
                                         uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}
// Arrive once on the mbarrier when all prior MMAs of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns of this warp's lane quarter.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
// 32 lanes x 32 bits, one column of this warp's lane quarter.
__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr) : "memory");
  return __uint_as_float(r);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 16 lanes x 32 bits, twice: threads 0-15 read lanes 0-15 of the warp's lane
// quarter at columns [c, c+16), threads 16-31 the same lanes at columns
// [c+SPLIT, c+SPLIT+16) -- the access shape of an M = 64 accumulator, whose
// rows occupy lanes 0-15 of each quarter.
template <int SPLIT>
__device__ __forceinline__ void tmem_ld16x2(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.16x32bx2.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16], %17;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr), "n"(SPLIT)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
// 32 lanes x 32 bits, 16 consecutive columns: this warp's lane quarter.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for the phase with the given parity; gives up after ~budget cycles
// and returns false (the caller records an error and winds down).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity,
                                          long long budget = 2000000000LL) {
  const long long t0 = clock64();
  while (!mbar_try_wait(mbar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}
// try_wait with a suspend-time hint (ns): a thread whose phase has not
// completed sleeps up to the hint instead of spinning, so threads that wait
// out a whole GEMM chain leave the issue slots to the ones that work.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* mbar, uint32_t parity,
                                                   uint32_t hint_ns) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n\t"
      "selp.b32 %0, 1, 0, P;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(mbar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return done != 0;
}
// As mbar_wait, sleeping between polls (for waits that span many MMAs).
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* mbar, uint32_t parity,
                                                long long budget = 2000000000LL) {
  const long long t0 = clock64();
  while (!mbar_try_wait_hint(mbar, parity, 200)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of
// 16), completing on the mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes,
                                         uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

// ---------------------------------------------------------------- CTA pairs
// A 2-CTA cluster whose M = 256 MMAs span both SMs (cta_group::2): CTA r
// holds rows 128r .. 128r+127 of A and half of B's N columns at the same
// shared-memory offsets, and its tensor memory receives its own 128 rows of
// D.  One thread of CTA 0 issues the pair's MMAs.  Every tcgen05 operation of
// a kernel that uses these takes the same cta_group, so the pair kernels
// allocate, commit and free through the functions below.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// all threads of both CTAs; release / acquire at cluster scope
__device__ __forceinline__ void cluster_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::
          : "memory");
}
// the same shared-memory variable in CTA `cta` of the cluster
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t cta) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_u32(p)), "r"(cta));
  return ra;
}
__device__ __forceinline__ int ld_peer_s32(const int* p, uint32_t cta) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(peer_addr(p, cta)) : "memory");
  return v;
}
// one arrival on the mbarrier at this address in CTA `cta`, ordered after
// this thread's earlier memory operations at cluster scope
__device__ __forceinline__ void mbar_arrive_peer(uint64_t* mbar, uint32_t cta) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                   peer_addr(mbar, cta))
               : "memory");
}
// bounded wait with cluster-scope acquire (arrivals from the peer CTA)
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* mbar, uint32_t parity,
                                                  long long budget = 2000000000LL) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}
// whole warp, in each CTA of the pair
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* smem_dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(smem_dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// D[tmem] (+)= A B^T over the pair (idesc with M = 256), from CTA 0
__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem_d, uint64_t da, uint64_t db,
                                              uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}
// once the pair's earlier MMAs complete: one arrival on the mbarrier at this
// offset in both CTAs ...
__device__ __forceinline__ void mma_commit_pair_both(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
      "[%0], %1;" ::"r"(smem_u32(mbar)),
      "h"((uint16_t)3)
      : "memory");
}
// 2-D tensor-map copy of one box at (x, y) into this CTA's shared memory,
// completing on the mbarrier at shared::cluster address `mbar` -- this CTA's
// or, for CTA 1 of a pair, CTA 0's (the pair's cta_group::2 form).  x times
// the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tensor_g2s_pair(void* smem_dst, const void* tmap, int x, int y,
                                                uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
// ... or in the issuing CTA only
__device__ __forceinline__ void mma_commit_pair_local(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}

}  // namespace tc
}  // namespace tode
