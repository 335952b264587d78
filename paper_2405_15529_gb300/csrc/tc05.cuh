// tc05.cuh -- inline-PTX helpers for the 5th-generation tensor cores of
// sm_103a (tcgen05): tensor-memory allocation, shared-memory matrix
// descriptors, kind::tf32 MMAs with an FP32 accumulator in tensor memory,
// commits to an mbarrier with a time-bounded wait, and tensor-memory loads.
//
// Operand layout used throughout: K-major, no swizzle.  A tile of R rows by
// K 32-bit elements is stored as "core matrices" of 8 rows x 16 bytes
// (4 elements), 128 contiguous bytes each; the core matrix holding rows
// 8a..8a+7 and elements 4b..4b+3 starts at a * SBO + b * LBO with
// LBO = 128 and SBO = (K / 4) * 128.  One kind::tf32 MMA consumes K = 8,
// i.e. two core matrices along K: the descriptor of the next K-slice starts
// 256 bytes further.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace pylom {
namespace tc05 {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of an R x K K-major tile (K a multiple of 4)
__device__ __forceinline__ uint32_t cm_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * ((K >> 2) * 128) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor (tcgen05 version, no swizzle)
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D f32, A and B tf32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc, bool acc) {
  const uint32_t a = acc ? 1u : 0u;
  asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               :: "r"(dtmem), "l"(da), "l"(db), "r"(idesc), "r"(a));
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for phase `parity` of the mbarrier; gives up after limit_ns (default
// kWaitLimitNs) and returns false (the caller records PYLOM_ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  const unsigned long long t0 = global_ns();
  // suspend-time hint: a waiting thread sleeps in try_wait until the phase
  // completes or the hint runs out, instead of spinning on issue slots that
  // the block's other warps need (at most 1 ms, so the limit still holds)
  const uint32_t hint_ns = (uint32_t)(limit_ns / 8 < 1000000ull ? limit_ns / 8 : 1000000ull);
  while (true) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity), "r"(hint_ns) : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// One thread: arm the mbarrier for `bytes` of TMA traffic and arrive on it.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}

// TMA: the 2-D box at (x, y) of the tensor map (x the contiguous dimension;
// x times the element size must be a multiple of 16 bytes) into shared
// memory at dst, completing `bytes` on the mbarrier.  This GPU's memory
// only; no cluster multicast.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int32_t x, int32_t y, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      :: "r"(smem_u32(dst)), "l"((uint64_t)tmap), "r"(x), "r"(y), "r"(smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make this thread's generic-proxy shared-memory writes visible to the tensor cores
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// whole warp: allocate ncols (power of two >= 32) tensor-memory columns,
// address written to *dst (shared)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(dst)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols));
}

// warp w (w = 0..3) reads its 32 lanes (rows 32w..32w+31) x 16 columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// 3xTF32 split: x = hi + lo with hi exactly representable in TF32
// (10 explicit mantissa bits, round to nearest) and lo the FP32 remainder.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

}  // namespace tc05
}  // namespace pylom
