// pic_tma.cuh -- tensor-memory-accelerator (TMA) staging for the field
// stencils: tiled bulk tensor copies from this GPU's global memory into shared
// memory, completed on mbarriers, with bounded waits.
//
// A wait on an mbarrier never spins without a limit: it polls up to a time
// budget (globaltimer, nanoseconds) and reports failure, after which the
// kernel records ERR_TIMEOUT in the device error word and stops issuing work.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "pic_internal.cuh"

namespace pic {

// time budget of one mbarrier wait (a stage of a plane pipeline lands in
// microseconds; two seconds means the copy will not come)
constexpr uint64_t kWaitBudgetNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make barrier initialisation and earlier generic-proxy shared-memory
// accesses visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one arrival that also announces the bytes the copies of this phase bring
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// true once the phase with the given parity has completed; false after the
// time budget (from t0) is spent
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t t0, uint64_t budget_ns)
{
    const uint32_t a = smem_addr(bar);
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > budget_ns) return false;
    }
}

// tiled 4D bulk tensor copy of the box at (c0, c1, c2, c3) into shared
// memory, completing on bar; c0 (innermost) times the element size must be a
// multiple of 16 bytes, the others may be negative or beyond the extent
// (those elements are filled with zeros)
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

// host: a 4D tiled tensor map of `count` contiguous arrays of extents
// (n0, n1, n2) (innermost first) of elem-byte elements, box (b0, b1, 1, count);
// false if the driver entry point is missing or the shape breaks a rule
bool encode_map_4d(CUtensorMap *map, const void *base, int elem, uint64_t n0, uint64_t n1, uint64_t n2,
                   uint64_t count, uint32_t b0, uint32_t b1);

}  // namespace pic
