// Bulk tensor loads (TMA) and mbarriers: the PTX the streaming kernels share,
// and the host-side tensor-map encoder.
#pragma once
#include <cuda.h>
#include <cstdint>

namespace pasd {

// Polls of a bounded mbarrier wait: far above any real copy time (a copy that
// never lands makes the kernel record PASD_ERR_TIMEOUT and return).
constexpr uint32_t kWaitPolls = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait: gives up after `limit` polls (each try_wait may suspend briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Orders this thread's later bulk tensor copies through the tensor map at `map`
// (in global memory, written before the launch) after that write.
__device__ __forceinline__ void tensormap_acquire(const void* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(map) : "memory");
}
// Copies a kernel-argument struct from global to shared memory (all threads of
// the CTA, 4-byte words), then synchronises the CTA.
template <class T>
__device__ __forceinline__ void load_args_to_smem(T* dst, const T* src) {
    static_assert(sizeof(T) % 4 == 0, "argument structs are word multiples");
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
    __syncthreads();
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Tiled bulk tensor load of rank R (coordinates innermost first) into shared
// memory, completing on `bar` with the box's byte count.
template <int R>
__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, uint64_t* bar, const int* c) {
    const uint32_t d = smem_u32(dst), b = smem_u32(bar);
    const uint64_t m = reinterpret_cast<uint64_t>(map);
    if (R == 1)
        asm volatile("cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3}], [%2];\n"
                     ::"r"(d), "l"(m), "r"(b), "r"(c[0]) : "memory");
    else if (R == 2)
        asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n"
                     ::"r"(d), "l"(m), "r"(b), "r"(c[0]), "r"(c[1]) : "memory");
    else if (R == 3)
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];\n"
                     ::"r"(d), "l"(m), "r"(b), "r"(c[0]), "r"(c[1]), "r"(c[2]) : "memory");
    else if (R == 4)
        asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];\n"
                     ::"r"(d), "l"(m), "r"(b), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]) : "memory");
    else
        asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6, %7}], [%2];\n"
                     ::"r"(d), "l"(m), "r"(b), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]) : "memory");
}

// Host: encodes a tiled float32 tensor map over a dense C-order array.
// dims and box are given innermost first; `swizzle` is one of
// CU_TENSOR_MAP_SWIZZLE_{NONE,32B,64B,128B}. Returns false (with a message in
// err) when the driver entry point is missing or refuses the map.
bool encode_tiled_f32(CUtensorMap* m, const float* base, int rank, const uint64_t* dims, const uint32_t* box,
                      CUtensorMapSwizzle swizzle, char* err, size_t errlen, const char* what);

}  // namespace pasd
