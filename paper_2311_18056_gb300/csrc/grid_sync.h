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
//
// The arrival and wait logic is written once (barrier_arrive_wait) over a
// policy of memory operations: the device policy below uses PTX atomics at GPU
// scope and %globaltimer; diag.cu instantiates it with host atomics so that
// host threads can exercise the same logic, deadline included.
#pragma once

#include "../../include/relu_qp.h"

namespace rq {

// One arrival of `expected` participants on bar (count, generation); false if
// the wait passed timeout_ns (err set to RELU_QP_ERR_TIMEOUT) or err was
// already set by another participant.
#pragma nv_exec_check_disable
template <class Ops>
__host__ __device__ inline bool barrier_arrive_wait(Ops& o, unsigned* bar, int* err, unsigned expected,
                                                    long long timeout_ns) {
    bool ok = true;
    const unsigned gen = o.load_relaxed(bar + 1);
    const unsigned arrived = o.fetch_add_acq_rel(bar, 1u);
    if (arrived == expected - 1u) {
        o.store_relaxed(bar, 0u);
        o.store_release(bar + 1, gen + 1u);
    } else {
        const long long t0 = o.now_ns();
        while (true) {
            if (o.load_acquire(bar + 1) != gen) break;
            if (o.now_ns() - t0 > timeout_ns) {
                o.set_error(err, RELU_QP_ERR_TIMEOUT);
                ok = false;
                break;
            }
            o.relax();
        }
    }
    if (o.load_error(err) != 0) ok = false;
    return ok;
}

#ifdef __CUDACC__
__device__ __forceinline__ long long grid_sync_timer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Device policy of barrier_arrive_wait: atomics at GPU scope.
struct GridSyncDeviceOps {
    __device__ __forceinline__ unsigned load_relaxed(const unsigned* p) {
        unsigned v;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        return v;
    }
    __device__ __forceinline__ unsigned fetch_add_acq_rel(unsigned* p, unsigned v) {
        unsigned old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
        return old;
    }
    __device__ __forceinline__ void store_relaxed(unsigned* p, unsigned v) {
        asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
    }
    __device__ __forceinline__ void store_release(unsigned* p, unsigned v) {
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
    }
    __device__ __forceinline__ unsigned load_acquire(const unsigned* p) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        return v;
    }
    __device__ __forceinline__ long long now_ns() { return grid_sync_timer(); }
    __device__ __forceinline__ void relax() {}
    __device__ __forceinline__ void set_error(int* err, int code) { atomicExch(err, code); }
    __device__ __forceinline__ int load_error(const int* err) { return *((const volatile int*)err); }
};

// Barrier over `expected` CTAs (gridDim.x for the kernels' own barriers).
__device__ __forceinline__ bool grid_sync_n(unsigned* bar, int* err, long long timeout_ns, int* s_ok,
                                            unsigned expected) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (expected > 1) {
            GridSyncDeviceOps o;
            ok = barrier_arrive_wait(o, bar, err, expected, timeout_ns) ? 1 : 0;
        } else if (*((volatile int*)err) != 0) {
            ok = 0;
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err, long long timeout_ns, int* s_ok) {
    return grid_sync_n(bar, err, timeout_ns, s_ok, gridDim.x);
}
#endif

}  // namespace rq
