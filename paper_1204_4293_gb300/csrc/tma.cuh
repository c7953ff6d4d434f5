// tma.cuh -- bulk tensor copies (TMA) into shared memory with an mbarrier,
// and the host-side encoding of their tensor maps.
//
// A kernel initialises one mbarrier (one arrival), thread 0 announces the
// bytes and issues the copies, and every thread polls the barrier's phase.
// The poll is bounded: if the bytes never arrive the CTA leaves together and
// sets this translation unit's wait-error flag, which fm_device_error reads.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched from the driver at run time)
#include <cudaTypedefs.h>

#include "common.cuh"

namespace fm {

// one flag per translation unit (no relocatable device code)
static __device__ int g_wait_error;

constexpr int kMaxWaitIters = 1 << 20;  // bound on polls of one set of copies

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// first 128-byte aligned address at or after p (bulk tensor copy destinations)
template <typename T> __device__ __forceinline__ T *align128(void *p)
{
    return reinterpret_cast<T *>(static_cast<unsigned char *>(p) + ((128 - (smem_u32(p) & 127)) & 127));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// box of a 3-D tensor map at (x, y, z) into shared memory (128-byte aligned)
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
// box of a 5-D tensor map at (c0 .. c4) into shared memory (128-byte aligned)
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}
// box of shared memory (128-byte aligned, written by this CTA's threads and
// made visible to the async proxy with fence_async_smem) to a 3-D tensor map
// at (x, y, z) >= 0; completion tracked by the issuing thread's bulk group
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int x, int y, int z, const void *src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the issuing thread waits until its committed bulk stores are complete
// (their shared-memory sources read and their writes performed); the CTA
// must not exit before the sources have been read
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// every thread polls phase `parity` of bar; false (for the whole CTA) when
// the bound ran out, after flagging it.  Every thread of the CTA must call it.
// A few blocking polls (try_wait may suspend the thread for a system-defined
// time) and then non-blocking polls 64 ns apart, so that a wait that runs out
// ends after about 2^20 x 64 ns = 0.07 s whatever that suspend time is.
__device__ __forceinline__ bool tma_wait_all(uint64_t *bar, uint32_t parity)
{
    bool done = false;
    for (int it = 0; it < 8 && !done; ++it) done = mbar_try_wait(bar, parity);
    for (int it = 0; it < kMaxWaitIters && !done; ++it) {
        __nanosleep(64);
        done = mbar_test_wait(bar, parity);
    }
    if (__syncthreads_or(!done)) {
        if (threadIdx.x == 0) atomicExch(&g_wait_error, 1);
        return false;
    }
    return true;
}

// Host: this translation unit's wait-error flag (read, optionally cleared);
// -1 if the device cannot be queried.
static inline int wait_error_flag(bool clear)
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_wait_error, sizeof(int)) != cudaSuccess) return -1;
    if (clear && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_wait_error, &z, sizeof(int));
    }
    return v;
}

// Host: 3-D fp32 tensor map, dims innermost first, strides (bytes) of dims 1
// and 2, box per dim.  False when the driver's encoder is missing or refuses
// the layout (then the caller loads without it).
bool encode_map3d_f32(CUtensorMap *map, const void *base, const uint64_t dims[3], const uint64_t strides[2],
                      const uint32_t box[3]);
// the same for rank 5 (strides of dims 1..4)
bool encode_map5d_f32(CUtensorMap *map, const void *base, const uint64_t dims[5], const uint64_t strides[4],
                      const uint32_t box[5]);

}  // namespace fm
