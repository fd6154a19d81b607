// Deadline diagnostics.  Every device-side wait of the library (the grid
// barrier of the cooperative kernels, the mbarrier waits and the layer-counter
// wait of the tensor-core kernels) gives up at a deadline and reports
// RELU_QP_ERR_TIMEOUT instead of hanging.  These entry points make each kind
// of wait run out on purpose, with a short deadline, so that a test can check
// that the wait returns, that the status reaches the host, and that the CUDA
// context is still usable afterwards.  Nothing here faults, traps or spins
// without a bound.
//
// relu_qp_diag_host_barrier runs the grid barrier's arrival/wait logic
// (barrier_arrive_wait in grid_sync.h, the same template the kernels use) on
// host threads, so that it can be tested without a GPU.
#include "batch.h"
#include "grid_sync.h"

#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

namespace rq {

namespace {

// Cooperative launch of `grid` CTAs that meet at a barrier expecting
// `expected` arrivals: expected = grid passes; expected = grid + 1 makes every
// CTA wait for an arrival that never comes, until the deadline.
__global__ void diag_grid_kernel(unsigned* bar, int* err, unsigned expected, long long timeout_ns) {
    __shared__ GridSyncState s_ok;
    grid_sync_init(&s_ok);
    grid_sync_n(bar, err, timeout_ns, &s_ok, expected);
}

// One cluster of CTAs that meet `rounds` times at the cluster barrier, whose
// mbarriers expect `extra` arrivals more than there are CTAs (extra = 1: every
// CTA waits until the deadline); every CTA then reaches the final hardware
// cluster barrier (no CTA exits while a partner may still arrive on its
// mbarrier).
__global__ void diag_cluster_kernel(int* err, unsigned extra, int rounds, long long timeout_ns) {
    __shared__ GridSyncState s_ok;
    __shared__ __align__(8) unsigned long long s_bar;
    ClusterBarrier cb{0u, 0u, 1};
    cluster_barrier_init(cb, &s_bar, extra);
    for (int k = 0; k < rounds; ++k)
        if (!cluster_barrier(cb, err, timeout_ns, &s_ok)) break;
    __syncthreads();
    cl_sync_hw();
}

// Host policy of barrier_arrive_wait: C++ atomics on the same words.
struct HostOps {
    void add_release(unsigned* p, unsigned v) { __atomic_fetch_add(p, v, __ATOMIC_RELEASE); }
    unsigned load_acquire(const unsigned* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
    int load_error(const int* err) { return __atomic_load_n(err, __ATOMIC_RELAXED); }
    long long now_ns() {
        return std::chrono::duration_cast<std::chrono::nanoseconds>(
                   std::chrono::steady_clock::now().time_since_epoch())
            .count();
    }
    void relax() { std::this_thread::yield(); }
    void set_error(int* err, int code) { __atomic_store_n(err, code, __ATOMIC_SEQ_CST); }
};

}  // namespace

}  // namespace rq

extern "C" {

int relu_qp_diag_device_wait(int kind, long long timeout_ns, int* status, double* ms) {
    if (kind < 0 || kind > 5 || timeout_ns < 1000 || timeout_ns > 1000000000LL || !status)
        return RELU_QP_ERR_INVALID;
    *status = 0;
    if (ms) *ms = 0.0;
    int dev = 0, sms = 0, coop = 0, clus = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&clus, cudaDevAttrClusterLaunch, dev) != cudaSuccess) {
        cudaGetLastError();
        return RELU_QP_ERR_CUDA;
    }
    int* words = nullptr;   // [0] error, [1] site, [2] counter, [3] pad, [4] barrier arrivals, [5] pad
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = RELU_QP_OK;
    if (cudaMalloc(&words, 8 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return RELU_QP_ERR_OOM;
    }
    cudaMemset(words, 0, 8 * sizeof(int));
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, 0);
    if (kind <= 1) {
        if (!coop) {
            rc = RELU_QP_ERR_UNSUPPORTED;
        } else {
            // a few CTAs, one per SM at most: every one is co-resident
            const int grid = sms < 8 ? sms : 8;
            unsigned* bar = reinterpret_cast<unsigned*>(words + 4);
            int* err = words;
            unsigned expected = (unsigned)grid + (kind == 0 ? 1u : 0u);
            long long ns = timeout_ns;
            void* args[] = {&bar, &err, &expected, &ns};
            if (cudaLaunchCooperativeKernel((const void*)rq::diag_grid_kernel, dim3(grid), dim3(64), args, 0, 0) !=
                cudaSuccess)
                rc = RELU_QP_ERR_CUDA;
        }
    } else if (kind <= 3) {
        rc = rq::tc_diag_wait(kind - 2, words, timeout_ns, 0);
    } else if (!clus) {
        rc = RELU_QP_ERR_UNSUPPORTED;
    } else {
        // a cluster of 2 CTAs: kind 4 one arrival short, kind 5 three complete rounds
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(2);
        cfg.blockDim = dim3(64);
        cfg.stream = 0;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int* err = words;
        const unsigned extra = kind == 4 ? 1u : 0u;
        const int rounds = kind == 4 ? 1 : 3;
        const long long ns = timeout_ns;
        if (cudaLaunchKernelEx(&cfg, rq::diag_cluster_kernel, err, extra, rounds, ns) != cudaSuccess)
            rc = RELU_QP_ERR_CUDA;
    }
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = RELU_QP_ERR_CUDA;
    if (rc == RELU_QP_OK) {
        int h[2] = {0, 0};
        if (cudaMemcpy(h, words, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) rc = RELU_QP_ERR_CUDA;
        *status = h[0];
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (ms) *ms = t;
    }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(words);
    return rc;
}

int relu_qp_diag_host_barrier(int threads, int extra, int rounds, long long timeout_ns, int* timeouts,
                              double* ms) {
    if (threads < 1 || threads > 64 || extra < 0 || extra > 64 || rounds < 1 || rounds > 100000 ||
        timeout_ns < 1000 || timeout_ns > 10000000000LL || !timeouts)
        return RELU_QP_ERR_INVALID;
    unsigned bar[2] = {0u, 0u};
    int err = 0;
    std::atomic<int> n_timeout{0};
    const unsigned expected = (unsigned)(threads + extra);
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([&]() {
            rq::HostOps o;
            unsigned epoch = 0;
            for (int r = 0; r < rounds; ++r) {
                if (!rq::barrier_arrive_wait(o, bar, &err, expected, epoch, timeout_ns)) {
                    n_timeout.fetch_add(1);
                    return;
                }
            }
        });
    for (auto& th : pool) th.join();
    *timeouts = n_timeout.load();
    if (ms) *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return err == 0 || err == RELU_QP_ERR_TIMEOUT ? RELU_QP_OK : RELU_QP_ERR_CUDA;
}

}  // extern "C"
