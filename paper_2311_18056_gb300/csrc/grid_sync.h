// Grid-wide barrier of the cooperative kernels (single_solve.cu,
// single_solve64.cu, batch_tail.cu): every CTA of the launch must be
// co-resident.  bar[0] counts every arrival of the launch (zeroed before the
// launch, never reset during it); each CTA keeps the number of barriers it has
// passed (its epoch), so barrier e is complete once the count reaches
// e * expected.  Thread 0 of each CTA arrives with a release reduction (no
// return value to wait for; the release covers the CTA's stores, ordered before
// it by __syncthreads) and polls the count with acquire loads, each issued
// together with a relaxed load of the error word.  Every wait has a deadline:
// past it the kernel's error word is set to RELU_QP_ERR_TIMEOUT; a CTA that
// sees the error word set leaves at once, and the barrier returns false in
// every thread of the CTA, so the caller returns from the kernel.
//
// The arrival and wait logic is written once (barrier_arrive_wait) over a
// policy of memory operations: the device policy below uses PTX atomics at GPU
// scope and %globaltimer; diag.cu instantiates it with host atomics so that
// host threads can exercise the same logic, deadline included.
#pragma once

#include "../../include/relu_qp.h"

namespace rq {

// One arrival of `expected` participants on the arrival counter *count;
// `epoch` is the caller's number of barriers passed on it.  False if the wait
// passed timeout_ns (err set to RELU_QP_ERR_TIMEOUT) or another participant
// has set err.
#pragma nv_exec_check_disable
template <class Ops>
__host__ __device__ inline bool barrier_arrive_wait(Ops& o, unsigned* count, int* err, unsigned expected,
                                                    unsigned& epoch, long long timeout_ns) {
    const unsigned target = (++epoch) * expected;   // modulo 2^32, as the count
    o.add_release(count, 1u);
    long long t0 = 0;
    bool timing = false;
    while (true) {
        const int e = o.load_error(err);
        const unsigned v = o.load_acquire(count);
        if (e != 0) return false;
        if (static_cast<int>(v - target) >= 0) return true;
        const long long t = o.now_ns();
        if (!timing) {
            t0 = t;
            timing = true;
        } else if (t - t0 > timeout_ns) {
            o.set_error(err, RELU_QP_ERR_TIMEOUT);
            return false;
        }
        o.relax();
    }
}

#ifdef __CUDACC__
__device__ __forceinline__ long long grid_sync_timer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Device policy of barrier_arrive_wait: atomics at GPU scope.
struct GridSyncDeviceOps {
    __device__ __forceinline__ void add_release(unsigned* p, unsigned v) {
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
    }
    __device__ __forceinline__ unsigned load_acquire(const unsigned* p) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        return v;
    }
    __device__ __forceinline__ int load_error(const int* p) {
        int v;
        asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        return v;
    }
    __device__ __forceinline__ long long now_ns() { return grid_sync_timer(); }
    __device__ __forceinline__ void relax() {}
    __device__ __forceinline__ void set_error(int* err, int code) { atomicExch(err, code); }
};

// Per-CTA state of the grid barrier, in shared memory: `epoch` (read and
// written by thread 0 only) counts the barriers the CTA has passed; `ok` carries
// thread 0's verdict to the CTA.  grid_sync_init runs once at kernel start.
struct GridSyncState {
    unsigned epoch;
    int ok;
};

__device__ __forceinline__ void grid_sync_init(GridSyncState* s) {
    if (threadIdx.x == 0) s->epoch = 0u;
}

// Barrier over `expected` CTAs (gridDim.x for the kernels' own barriers).
__device__ __forceinline__ bool grid_sync_n(unsigned* bar, int* err, long long timeout_ns, GridSyncState* s,
                                            unsigned expected) {
    __syncthreads();
    if (threadIdx.x == 0) {
        GridSyncDeviceOps o;
        int ok = 1;
        if (expected > 1)
            ok = barrier_arrive_wait(o, bar, err, expected, s->epoch, timeout_ns) ? 1 : 0;
        else if (o.load_error(err) != 0)
            ok = 0;
        s->ok = ok;
    }
    __syncthreads();
    return s->ok != 0;
}

__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err, long long timeout_ns, GridSyncState* s) {
    return grid_sync_n(bar, err, timeout_ns, s, gridDim.x);
}
#endif

}  // namespace rq
