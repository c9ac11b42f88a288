// Shared-memory barriers and tensor-memory-accelerator copies for the streaming
// stencil kernels: mbarrier init / expect_tx / arrive, a parity wait bounded by
// %globaltimer (on expiry the caller raises the device flag and returns; nothing
// spins forever), a tiled cp.async.bulk.tensor load and a plain cp.async.bulk load,
// both completing on an mbarrier.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "oed_internal.cuh"

namespace oed {

// host: tensor map over the [2 nsolve][nz][xp] FP32 planes of one wavefield level,
// copy boxes of bx columns by bz rows (stream_tma.cu)
bool tma_make_map(CUtensorMap *map, void *base, const Geometry &g, int nsolve, int bx, int bz);

// host: tensor map over one level in the paired layout (oed_internal.cuh), as a 4-D tensor
// (floats of a half row, the two halves, rows, solves), copy boxes of bslots slots of both
// halves by bz rows (stream_tma.cu)
bool tma_make_paired_map(CUtensorMap *map, void *base, const Geometry &g, int nsolve, int bslots, int bz);

constexpr unsigned long long kWaitLimitNs = 2000000000ULL;   // 2 s per wait

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(bar)),
                 "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"((unsigned)__cvta_generic_to_shared(bar))
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase with the given parity, bounded by limit_ns; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          unsigned long long limit_ns = kWaitLimitNs)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, int x, int y, int z,
                                          uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"((unsigned)__cvta_generic_to_shared(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z),
        "r"((unsigned)__cvta_generic_to_shared(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load4(void *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                          uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::
            "r"((unsigned)__cvta_generic_to_shared(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w),
        "r"((unsigned)__cvta_generic_to_shared(bar))
        : "memory");
}

// 1-D bulk copy global -> shared, completion on an mbarrier (16-byte aligned, size a
// multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes), "r"((unsigned)__cvta_generic_to_shared(bar))
                 : "memory");
}

}  // namespace oed
