// Grid-wide barrier of a cooperative launch, with a bounded wait: used by
// the persistent superstep loops (sell.cu, msssp.cu).
#pragma once

#include "gxp_internal.hpp"

namespace gxp {

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Barrier of all CTAs of a cooperative grid: arrival counter and generation
// (the last CTA to arrive resets the counter, then releases the next
// generation). A wait that runs past timeout_ns, or any wait when `force`
// (an injected fault), sets kErrTimeout and gives up; the caller then
// returns. Returns false when this CTA gave up or another one had.
__device__ inline bool grid_barrier(GridBar* b, uint32_t n_ctas, uint64_t timeout_ns, bool force, uint32_t* err) {
    __shared__ uint32_t s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t gen = ld_acquire_gpu(&b->gen);
        __threadfence();
        uint32_t ok = 1u;
        if (atomicAdd(&b->count, 1u) == n_ctas - 1u) {
            b->count = 0u;   // the others wait on gen, not on the counter
            st_release_gpu(&b->gen, gen + 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (ld_acquire_gpu(&b->gen) == gen) {
                if (force || global_ns() - t0 > timeout_ns) {
                    atomicOr(err, kErrTimeout);
                    ok = 0u;
                    break;
                }
                __nanosleep(64);
            }
            __threadfence();
        }
        if (ok && (ld_acquire_gpu(err) & kErrTimeout)) ok = 0u;   // another CTA gave up
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0u;
}

}  // namespace gxp
