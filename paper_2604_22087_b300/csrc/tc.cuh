// Blackwell (sm_100-family, here sm_103a) tensor-core helpers: TMEM allocation, tcgen05.mma
// with shared-memory operand descriptors, commit to an mbarrier, bounded mbarrier waits and
// TMEM -> register loads.  Inline PTX only; one CTA = 4 warps = 128 threads, where thread t
// owns row t of a 128-row accumulator (TMEM lane t).
//
// Operand layout in shared memory: K-major, no swizzle.  A [R rows][K] tile of 16-bit values
// is stored as 8-row x 16-byte "core matrices"; core matrix (row block rb, k block kb) lives at
// ((rb * (K/8)) + kb) * 128 bytes, element (r, k) at that base + (r%8)*16 + (k%8)*2.  The
// descriptor's leading byte offset is the step between core matrices along K (128 B) and the
// stride byte offset the step between 8-row blocks ((K/8)*128 B).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace jetsci {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (r, k) in a K-major no-swizzle tile with K columns (16-bit elements).
__host__ __device__ __forceinline__ uint32_t core_offset(int r, int k, int K) {
    return (uint32_t)((((r >> 3) * (K >> 3)) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (no swizzle).  Bits: [0,14) addr>>4, [16,30) LBO>>4,
// [32,46) SBO>>4, [46,48) version = 1, [49,52) base offset 0, [52] LBO mode 0, [61,64) swizzle 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both operands K-major.
// Bits: [4,6) D format (1 = F32), [7,10) A format (1 = BF16), [10,13) B format (1 = BF16),
// [15] A major, [16] B major (0 = K), [17,23) N >> 3, [24,29) M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::tf32: TF32 x TF32 -> FP32 (format code 2), both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Makes generic-proxy shared-memory writes visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_smem_to_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D[tmem] = A * B^T (+ D if accumulate), A from desc a (M x K), B from desc b (N x K).
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the mbarrier when all previously issued tcgen05.mma of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

// One arrival on an mbarrier from a thread (completes its phase when the expected count is 1).
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    uint64_t state;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_addr(mbar)) : "memory");
    (void)state;
}

// Makes a freshly initialised mbarrier visible to the async proxy (tensor-core commits).
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Waits for the given phase with an iteration cap; returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t phase, uint32_t max_iter = (1u << 24)) {
    for (uint32_t it = 0; it < max_iter; it++)
        if (mbar_try_wait(mbar, phase)) return true;
    return false;
}

// 32 lanes x 32 bit x 16 columns: thread t of the warp gets lane (warp%4)*32 + t.  The load
// and its wait are one asm statement: the destination registers are undefined until the wait,
// and a separate statement would let the compiler copy them in between.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

// TMEM address of column `col` in the lane quarter of the calling warp (the column must be
// the same for all 32 threads of the warp: tcgen05.ld is warp-collective).
__device__ __forceinline__ uint32_t tmem_lane_addr(uint32_t base, int col) {
    const uint32_t quarter = (threadIdx.x >> 5) & 3;
    return base + ((quarter * 32u) << 16) + (uint32_t)col;
}

// Bulk asynchronous copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// shared to global memory, in this thread's current bulk group; make the shared-memory writes
// visible to the async proxy first (fence_smem_to_async).
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_addr(ssrc)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until the thread's bulk groups have finished reading their shared-memory source.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Waits until the thread's bulk groups have completed (their writes performed).
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void st_bf16(unsigned char *tile, int r, int k, int K, float x) {
    *reinterpret_cast<__nv_bfloat16 *>(tile + core_offset(r, k, K)) = __float2bfloat16_rn(x);
}

__device__ __forceinline__ float ld_bf16(const unsigned char *tile, int r, int k, int K) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(tile + core_offset(r, k, K)));
}

// Issues D = A(128 x K) * B(N x K)^T as K/16 MMAs of K = 16 (BF16), from one thread.
__device__ __forceinline__ void gemm_bf16_128xN(uint32_t d_tmem, const unsigned char *A, const unsigned char *B,
                                                int N, int K) {
    const uint32_t a0 = smem_addr(A), b0 = smem_addr(B);
    const uint32_t sbo = (uint32_t)(K >> 3) * 128u;
    const uint32_t id = idesc_bf16(128, N);
    for (int kk = 0; kk < K / 16; kk++) {
        uint64_t da = smem_desc(a0 + kk * 256u, 128u, sbo);
        uint64_t db = smem_desc(b0 + kk * 256u, 128u, sbo);
        mma_bf16(d_tmem, da, db, id, kk > 0 ? 1u : 0u);
    }
}

}  // namespace tc
}  // namespace jetsci
