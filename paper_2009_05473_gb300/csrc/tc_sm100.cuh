// Inline-PTX wrappers for the fifth-generation tensor cores of the sm_100 family
// (tcgen05: MMA issued by one thread, accumulators in tensor memory), for
// mbarriers and for bulk global->shared copies.
//
// Operands are K-major without swizzle: 8 x 8 "core matrices" of 16-bit elements,
// each 8 rows of 16 contiguous bytes (128 bytes).  A shared-memory descriptor gives
// the start address, the byte distance between core matrices adjacent along K (LBO)
// and along M or N (SBO).  One tcgen05.mma of kind::f16 multiplies an M x 16 slice of
// A by a 16 x N slice of B^T (B stored N x K, K-major) into an M x N FP32 block of
// tensor memory (M = 128: row i in lane i, column j in column j).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace sfw {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// K-major, no swizzle; addresses and offsets in bytes (multiples of 16).
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the sm_100 family; base offset 0, no swizzle
    return d;
}

// K-major with the 128-byte swizzle: atoms of 8 rows x 64 elements (1024 bytes, 1024-byte
// aligned), 8-row groups SBO = 1024 bytes apart; the start address of a K = 16 slice moves by
// 32 bytes inside an atom (the swizzle applies to the absolute address bits).
__device__ __forceinline__ uint64_t desc_kmajor_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                  // leading byte offset: unused by this layout
    d |= (uint64_t)(1024u >> 4) << 32;       // stride byte offset: 8-row groups
    d |= (uint64_t)1 << 46;                  // descriptor version of the sm_100 family
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16 with bf16 A and B (both K-major) and FP32 accumulation.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4)                          // D format: FP32
           | (1u << 7)                        // A format: bf16
           | (1u << 10)                       // B format: bf16
           | ((uint32_t)(N >> 3) << 17)       // N / 8
           | ((uint32_t)(M >> 4) << 24);      // M / 16
}

// Instruction descriptor of kind::tf32 (A and B FP32 in memory, read as tf32; both K-major)
// with FP32 accumulation.
__host__ __device__ constexpr uint32_t idesc_tf32_f32(int M, int N) {
    return (1u << 4)                          // D format: FP32
           | (2u << 7)                        // A format: tf32
           | (2u << 10)                       // B format: tf32
           | ((uint32_t)(N >> 3) << 17)       // N / 8
           | ((uint32_t)(M >> 4) << 24);      // M / 16
}

// Tensor memory: allocation and release by one whole warp; the address lands in *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 :: "r"(smem_addr(slot)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(taddr), "r"(ncols)
                 : "memory");
}

// D (+)= A B^T for one K = 16 slice; issued by a single thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate) : "memory");
}
// D (+)= A B^T for one K = 8 slice of tf32 operands (32 bytes of a 128-byte row).
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate) : "memory");
}
// The mbarrier at bar receives one arrival once every earlier tcgen05 op of this thread is done.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 :: "r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// Generic-proxy shared-memory writes made visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// 16 consecutive FP32 columns of this warp's 32 lanes of tensor memory (one lane per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                 "%12, %13, %14, %15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without the wait: several may be in flight before one tmem_wait_ld.
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                 "%12, %13, %14, %15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// ---- mbarriers (shared::cta) and bulk copies
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" :: "r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the completion of the phase of parity `parity`; false if it did not come.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int max_polls = 1 << 20) {
    for (int it = 0; it < max_polls; ++it) {
        uint32_t done = 0;
        asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, q;\n}\n"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
// Named barrier `id` over `count` threads that also returns, to every one of them, whether any
// passed true: a decision all of them take together (e.g. to stop on an abort flag that other
// warps may set at any moment).
template <int id, int count>
__device__ __forceinline__ bool bar_sync_or(bool v) {
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
                 " selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r) : "r"((uint32_t)v), "n"(id), "n"(count) : "memory");
    return r != 0;
}
// A 3-D box of a tiled tensor map into shared memory (x in elements, a multiple of 16 bytes);
// completes on bar with the box's bytes (out-of-range elements read as zero).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* tmap, int x, int y, int z, uint32_t bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];\n"
                 :: "r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(bar) : "memory");
}
// bytes (multiple of 16) from global src to shared dst (both 16-byte aligned); completes on bar.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// 8 bytes from global to shared by an asynchronous copy (completed by cp_async_wait_all).
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" :: "r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Byte offset of element (row, k) in a K-major, no-swizzle operand of `rows` rows whose
// core matrices are ordered row group fastest: LBO = rows * 16 bytes, SBO = 128 bytes.
__host__ __device__ inline uint32_t kmajor_offset(int row, int k, int rows) {
    return (uint32_t)(k >> 3) * (uint32_t)(rows * 16) + (uint32_t)(row >> 3) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// Byte offset of element (row, k) in a K-major operand with the 128-byte swizzle: atoms of
// 8 rows x 64 elements ordered row group fastest ((rows / 8) atoms per 64 columns of K); the
// 16-byte chunk c of row r sits at chunk c ^ (r mod 8).
__host__ __device__ inline uint32_t sw128_offset(int row, int k, int rows) {
    return (uint32_t)(k >> 6) * (uint32_t)(rows >> 3) * 1024u + (uint32_t)(row >> 3) * 1024u +
           (uint32_t)(row & 7) * 128u + ((uint32_t)(((k >> 3) & 7) ^ (row & 7)) << 4) + (uint32_t)(k & 7) * 2u;
}
// Start address of the K = 16 slice ks of such an operand.
__host__ __device__ inline uint32_t sw128_slice(int ks, int rows) {
    return (uint32_t)(ks >> 2) * (uint32_t)(rows >> 3) * 1024u + (uint32_t)(ks & 3) * 32u;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(bar) : "memory");
}

}  // namespace tc
}  // namespace sfw
