// mbarrier and TMA primitives (inline PTX) for the tensor-core halfspace kernel.
// Every wait is bounded.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "rrs_internal.h"

namespace rrs {
namespace async {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity to complete: gives up after
// about a second of SM clock, or as soon as any CTA of the grid has flagged a
// timeout in the shared error word.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const int* err, bool honor_grid_abort = true)
{
    const long long t0 = clock64();
    for (uint32_t i = 0;; ++i) {
        if (mbar_test(bar, parity)) return true;
        if ((i & 255u) == 255u) {
            if (clock64() - t0 > 2000000000LL) return false;
            if (honor_grid_abort && (*(volatile const int*)err & ERR_TIMEOUT)) return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace async
}  // namespace rrs
