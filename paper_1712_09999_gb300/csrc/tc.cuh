// 5th-generation tensor cores (tcgen05): tensor-memory allocation, shared-memory
// operand descriptors, the TF32 MMA, its completion signal and tensor-memory loads.
//
// Operand layout used throughout: K-major with the 64-byte swizzle. A matrix of
// `rows` x 16 TF32 values occupies rows of 64 bytes; the 16-byte group g of row r
// sits at g ^ ((r >> 1) & 3); 8-row groups are 512 bytes apart. This is exactly
// the shared-memory image a bulk tensor copy with CU_TENSOR_MAP_SWIZZLE_64B
// writes for a box of 16 floats x rows, so such a box is an operand as it lands.
// An MMA step consumes K = 8 (32 bytes of each row): the second step of a
// 16-wide tile starts 32 bytes further.
#pragma once
#include <cstdint>

namespace pasd {

// Instruction descriptor of tcgen05.mma kind::tf32: FP32 accumulate, TF32 A and B,
// both K-major, shape M x N (M = 128: N a multiple of 16 up to 256).
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
    return (1u << 4)                          // D format: F32
           | (2u << 7) | (2u << 10)           // A, B format: TF32
           | ((uint32_t)(N >> 3) << 17)       // N / 8
           | ((uint32_t)(M >> 4) << 24);      // M / 16
}

// Shared-memory descriptor of a K-major operand with the 64-byte swizzle
// (start address, leading offset 16 B (unused by swizzled K-major layouts),
// 512 B between 8-row groups, descriptor version 1, swizzle code 4).
__device__ __forceinline__ uint64_t tc_desc_sw64(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// D (+)= A B^T on the tensor cores; issued by one thread. `acc` = 0 overwrites D.
__device__ __forceinline__ void tc_mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// Arrive once on `bar` when every MMA this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Tensor-memory allocation (one full warp): the base address is written to *dst.
// `ncols` is a power of two >= 32.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive 32-bit columns of this thread's tensor-memory lane (warp w of
// a warpgroup reads lanes 32w .. 32w + 31; lane bits are 31..16 of the address).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x rounded to the nearest TF32 value (low 13 bits zero; ties away from zero).
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// Two-term TF32 split: hi = rn(x), lo = rn(x - hi) (x - hi is exact), so
// x = hi + lo up to 2^-24 |x|.
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
    hi = tf32_rn(x);
    lo = tf32_rn(x - hi);
}

}  // namespace pasd
