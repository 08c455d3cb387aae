// Fifth-generation tensor-core helpers (tcgen05, sm_100 family): tensor-memory
// allocation, shared-memory operand descriptors, MMA issue and completion,
// tensor-memory loads.  Inline PTX only.
//
// Operands are bf16, K-major, without swizzle.  An operand of R rows and K
// columns (K a multiple of 16) is stored as 8x8 core matrices (8 rows of 16
// bytes, 128 contiguous bytes); the 8-row groups are outermost and the K chunks
// of 8 elements inside them:
//     byte(r, k) = (r / 8) * (K/8) * 128 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
// i.e. leading-dimension byte offset (between K chunks) 128 and stride byte
// offset (between 8-row groups) (K/8) * 128.  One MMA consumes K = 16 (two
// chunks); the next K step starts 256 bytes further.
//
// Accumulators are FP32 in tensor memory: for M = 128 and one CTA, row r of the
// product lives in TMEM lane r and column c in the allocation's column c.  Warp w
// of a warpgroup reads lanes 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mdk {
namespace tc {

__host__ __device__ constexpr uint32_t op_offset(int r, int k, int kc) {
    return (uint32_t)((r >> 3) * kc * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading- and stride-
// dimension byte offsets, descriptor version 1, no swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc_raw(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// K-major operand as above: LBO = 128 between K chunks, SBO = group_chunks * 128
// between 8-row groups (group_chunks = kc for one piece, or the chunks of all
// pieces stored in one 8-row group).
__device__ __forceinline__ uint64_t smem_desc_kmajor(uint32_t saddr, uint32_t group_chunks) {
    return smem_desc_raw(saddr, 128u, group_chunks * 128u);
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t kc) {
    return smem_desc_kmajor(saddr, kc);
}
// MN-major operand (M contiguous inside the 16-byte rows of a core matrix, the
// rows of a core matrix 8 consecutive K): for this major-ness the leading-
// dimension byte offset is the stride between 8-deep K groups (mg * 128 here,
// mg = 8-element M groups of the operand) and the stride-dimension byte
// offset the stride between 8-element M groups (128 here).
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t saddr, uint32_t mg) {
    return smem_desc_raw(saddr, mg * 128u, 128u);
}

// Instruction descriptor of kind::f16: bf16 A and B (both K-major; bit 15
// set makes A MN-major), FP32 accumulator, M x N (M = 128; N a multiple of 16
// up to 256).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Tensor-memory allocation of `ncols` columns (a power of two >= 32), written to
// *dst (shared memory).  Warp-collective: one full warp executes it.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "r"(ncols)
                 : "memory");
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
// Make this thread's generic-proxy shared-memory stores visible to the tensor
// core (async proxy); a CTA barrier follows before the MMA is issued.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D (tmem) = A * B^T (+ D when accumulate != 0), one elected thread.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The mbarrier receives one arrival when every MMA this thread issued so far
// has completed.
__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            (uint32_t)__cvta_generic_to_shared(bar))
        : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// x = hi + lo with hi = bf16(x) and lo = bf16(x - hi), both rounded to nearest;
// hi*b + lo*b carries about 16 significant bits of x.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

}  // namespace tc
}  // namespace mdk
