// Grid-wide barrier of the cooperative kernels (single_solve.cu,
// single_solve64.cu, batch_tail.cu): every CTA of the launch must be
// co-resident.  bar[0] counts the arrivals of the current barrier, bar[1] is
// its generation.  Thread 0 of each CTA arrives with an acquire-release atomic
// (its release covers the CTA's stores, ordered before it by __syncthreads);
// the last CTA to arrive resets the count and publishes the next generation
// with a release store; the others poll the generation with acquire loads.
// Every wait has a deadline: past it the kernel's error word is set to
// RELU_QP_ERR_TIMEOUT and the barrier returns false in every thread of the CTA
// (also when another CTA has already set the error word), and the caller
// returns from the kernel.
#pragma once

#include "../../include/relu_qp.h"

namespace rq {

__device__ __forceinline__ long long grid_sync_timer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err, long long timeout_ns, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (gridDim.x > 1) {
            unsigned gen, arrived;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(bar + 1) : "memory");
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
            if (arrived == gridDim.x - 1) {
                asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(bar), "r"(0u) : "memory");
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 1), "r"(gen + 1u) : "memory");
            } else {
                const long long t0 = grid_sync_timer();
                while (true) {
                    unsigned v;
                    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar + 1) : "memory");
                    if (v != gen) break;
                    if (grid_sync_timer() - t0 > timeout_ns) {
                        atomicExch(err, RELU_QP_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        if (*((volatile int*)err) != 0) ok = 0;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

}  // namespace rq
