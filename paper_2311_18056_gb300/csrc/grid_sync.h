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
// The same header holds the barrier of the kernels that run as one
// thread-block cluster (cluster_barrier, below), which waits on mbarriers.
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

// ---- one thread-block cluster instead of a cooperative grid ----
__device__ __forceinline__ uint32_t cl_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_smem(const void* ptr) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
// shared::cluster address of the shared::cta address `addr` in CTA `rank`
__device__ __forceinline__ uint32_t cl_mapa(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_st(uint32_t cluster_addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(cluster_addr), "f"(v) : "memory");
}
__device__ __forceinline__ void cl_arrive(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool cl_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// hardware barrier of every thread of the cluster (no deadline: only where every CTA is
// known to arrive, at the start and at the end of a kernel)
__device__ __forceinline__ void cl_sync_hw() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Barrier of the CTAs of one cluster with a deadline.  Every CTA has an
// mbarrier expecting C arrivals per phase; lane q of warp 0 arrives (release at
// cluster scope) on CTA q's, and thread 0 waits (acquire) on its own with a
// deadline, leaving early once another CTA has set the error word.  Each CTA
// arrives once per barrier on every mbarrier, so no CTA passes barrier k before
// every CTA has arrived at it, and a CTA's own mbarrier is never more than one
// phase ahead of it (the parity wait cannot miss a phase).  A CTA that gives up
// must not exit before its partners: the kernel ends with cl_sync_hw, which
// every CTA reaches because every wait before it has a deadline.
struct ClusterBarrier {
    uint32_t bar;     // this CTA's mbarrier (shared::cta address)
    uint32_t phase;   // barriers passed
    int C;            // CTAs of the cluster
};

// Initialise (all threads) with `extra` arrivals per phase beyond the C CTAs
// (0 in the kernels; the deadline diagnostics use 1: a barrier that never
// completes); ends with a hardware cluster barrier, so every mbarrier is
// initialised before any remote arrival.
__device__ __forceinline__ void cluster_barrier_init(ClusterBarrier& cb, unsigned long long* mbar, unsigned extra) {
    cb.C = (int)cl_size();
    cb.bar = cl_smem(mbar);
    cb.phase = 0u;
    if (threadIdx.x == 0)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n fence.mbarrier_init.release.cluster;" ::"r"(cb.bar),
                     "r"((unsigned)cb.C + extra)
                     : "memory");
    cl_sync_hw();
}

__device__ __forceinline__ bool cluster_barrier(ClusterBarrier& cb, int* err, long long timeout_ns, GridSyncState* s) {
    __syncthreads();
    if (threadIdx.x < (unsigned)cb.C) cl_arrive(cl_mapa(cb.bar, threadIdx.x));
    if (threadIdx.x == 0) {
        int ok = 1;
        const long long t0 = grid_sync_timer();
        while (!cl_try(cb.bar, cb.phase & 1u)) {
            int e;
            asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(e) : "l"(err) : "memory");
            if (e != 0) {
                ok = 0;
                break;
            }
            if (grid_sync_timer() - t0 > timeout_ns) {
                atomicExch(err, RELU_QP_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        s->ok = ok;
    }
    ++cb.phase;
    __syncthreads();
    return s->ok != 0;
}
#endif

}  // namespace rq
