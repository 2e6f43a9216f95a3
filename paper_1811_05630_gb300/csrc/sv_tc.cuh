// sv_tc.cuh — the tcgen05 (5th-generation tensor core) pieces the fused pass uses for dense
// 4- and 5-qubit gates: shared-memory operand layout and descriptors, MMA issue, completion
// through an mbarrier with a bounded wait, and tensor-memory loads. Inline PTX for sm_103a.
//
// Operands are FP16 matrices in the no-swizzle K-major layout: "core matrices" of 8 rows by
// 8 K-elements (16 bytes per row, 128 bytes each); core matrices adjacent in K lie 128 bytes
// apart (the descriptor's leading byte offset) and 8-row groups (K / 8) * 128 bytes apart (its
// stride byte offset). An MMA of kind::f16 with M = 128 rows and N columns multiplies A
// (M x 16) by B (N x 16, also K-major) and adds into an FP32 accumulator in tensor memory:
// row r in lane r, column n in column base + n.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>

namespace sv {

constexpr int kTcDigits = 7;     // balanced base-512 digits of a 62-bit coefficient
constexpr int kTcM = 128;        // tuples per MMA (rows of A)
constexpr int kTcN = 32;         // output columns per accumulator
constexpr int kTcCols = 256;     // tensor-memory columns a CTA holds (two CTAs fit an SM's 512)
constexpr int kTcMaxAcc = 8;     // accumulators of kTcN columns
constexpr long long kTcWaitLimit = 1ll << 24;  // mbarrier polls before the wait gives up

// Element (r, k) of an R x kdim K-major operand tile.
__host__ __device__ __forceinline__ int tc_tile_index(int r, int k, int kdim) {
  return ((r >> 3) * (kdim >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (8-row) byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, FP16 A and B, both K-major, M x N.
__device__ __forceinline__ uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) += / = A (desc) x B (desc)^T over K = 16. One thread issues it.
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

// Arrive on the mbarrier once every MMA issued before by this thread has completed.
__device__ __forceinline__ void tc_commit(unsigned long long* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      tc_smem_u32(mbar)));
}

__device__ __forceinline__ void tc_mbar_init(unsigned long long* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(mbar)));
  asm volatile("fence.mbarrier_init.release.cluster;");
}

// Wait for phase `parity` of the mbarrier to complete, polling at most `limit` times.
// Returns false when the limit ran out.
__device__ __forceinline__ bool tc_wait_bounded(unsigned long long* mbar, uint32_t parity, long long limit) {
  const uint32_t a = tc_smem_u32(mbar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity));
    if (done) return true;
  }
  return false;
}

// The tensor-core pass's wait: at most kTcWaitLimit polls.
__device__ __forceinline__ bool tc_wait(unsigned long long* mbar, uint32_t parity) {
  return tc_wait_bounded(mbar, parity, kTcWaitLimit);
}

// Generic-proxy writes of operand tiles become visible to the tensor cores' (async) proxy.
__device__ __forceinline__ void tc_fence_operands() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Four consecutive FP32 columns of this warp's 32 lanes (lane quarter from the address),
// issued without waiting: the registers are valid after tc_ld_wait().
__device__ __forceinline__ void tc_ld4(uint32_t taddr, uint32_t v[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tc_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Tensor-memory columns for the CTA (one warp; the base address lands in *dst).
__device__ __forceinline__ void tc_alloc(uint32_t* dst) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(dst)),
               "r"(kTcCols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols));
}

}  // namespace sv
