// tcgen05 (5th-generation tensor core) backend of the batched layer.
//
// Each layer is T[slot, r] = sum_k S[slot, k] Wt[r, k] for a 128-slot x BN-row
// tile, with S and Wt given as BF16 parts and the FP32 accumulator in TMEM:
//   refined layers   S = d_hi + d_lo (d = s - s_ref), Wt = w1 + w2:
//                    T = d_hi w1 + d_hi w2 + d_lo w1                 (3 MMAs / k-step)
//   accurate layers  S = s1 + s2 + s3, Wt = w1 + w2 + w3 (3-way splits):
//                    T = s1 w1 + s1 w2 + s2 w1 + s1 w3 + s2 w2 + s3 w1 (6 MMAs / k-step)
// The residual products [P; A] x and A^T lam_std (and, optionally, the first
// layer of every chunk) use the accurate form; the layers the refined one
// (see batch.cu).
//
// Accumulation by significance: the tensor core adds into its FP32
// accumulator with truncation, so every MMA that lands on a large partial sum
// costs up to one unit in its last place, biased in one direction.  The hi*hi
// product goes to one TMEM accumulator and every correction product (2^-9 of
// it or smaller) to a second one; the epilogue adds the two in FP32.  This
// keeps the truncation of the ~K/16 correction MMAs 2^-9 smaller.
//
// Warp roles (320 threads): warp 0 issues TMA loads (128B-swizzled K-major
// tiles, one mbarrier per stage), warp 1 allocates TMEM and one lane issues
// the MMAs, warps 2-9 run the epilogue: each reads its 32 TMEM lanes (one slot
// per thread; warps w and w+4 share a lane quadrant and split the columns)
// and applies the element-wise layer of batch.h, 16 rows at a time.  Every
// mbarrier wait has a deadline; on expiry the kernel records an error, waits
// (bounded) for its own copies and MMAs, frees TMEM and returns.
#include "batch.h"

#include <cuda.h>

#include <algorithm>
#include <type_traits>
#include <cstring>
#include <vector>

namespace rq {

namespace {

constexpr int kThreadsTC = 320;   // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kBK = 64;                        // bf16 elements per 128-byte swizzled row
constexpr int kTileBytesA = kSlotTile * 128;   // one A part: 128 rows x 128 B
constexpr long long kWaitNs = 1000000000LL;    // 1 s deadline for any single wait

enum Mode { MODE_LAYER_REFINED = 0, MODE_LAYER_ACCURATE = 1, MODE_CHECK1 = 2, MODE_CHECK2 = 3 };

struct TcArgs {
    int num_kb;        // k-blocks of 64
    int k_off;         // first column (x coordinate) of both operands
    int a_row[3];      // row offset of each A part in the operand tensor (+ slot0)
    int b_row[3];      // row offset of each B part in the weight tensor (+ row0)
    int b_rho_stride;  // LAYER: rows between bank entries in the weight tensor
    int rows;          // valid output rows (R for layers, n for the check)
    int* err;          // device error word
};

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
// a wait gave up: error word err[0], and err[1] = which wait (first one wins)
enum WaitSite : int {
    WS_PROD_EMPTY = 1, WS_PROD_SYNC, WS_MMA_FULL, WS_MMA_ACC, WS_EPI_ACC, WS_EPI_RECV, WS_DRAIN_READY, WS_DRAIN_FREE
};
__device__ __forceinline__ void wait_failed(int* err, int site) {
    atomicCAS(err + 1, 0, site);
    atomicExch(err, RELU_QP_ERR_TIMEOUT);
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ long long gtime() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase with the given parity to complete; false after the
// deadline.  (The deadline is checked after every unsuccessful try_wait,
// which itself blocks for a while; a tight loop of tries between clock reads
// made every pipeline hand-off several times slower.)
__device__ __forceinline__ bool mbar_wait_ns(uint32_t bar, uint32_t parity, long long ns) {
    const long long t0 = gtime();
    while (!mbar_try(bar, parity))
        if (gtime() - t0 > ns) return false;
    return true;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) { return mbar_wait_ns(bar, parity, kWaitNs); }

// Wait (acquire at GPU scope) until the counter reaches target; false after ns.
__device__ __forceinline__ bool wait_counter_geq(const unsigned* ctr, unsigned target, long long ns) {
    const long long t0 = gtime();
    while (true) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) return true;
        if (gtime() - t0 > ns) return false;
    }
}

// The same for a long wait by a thread that is not on the critical path: poll
// every `ns` nanoseconds so that the polling does not slow down the barrier
// operations of the producer and MMA threads.
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t bar, uint32_t parity, unsigned ns) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = gtime();
    while (true) {
        __nanosleep(ns);
        if (mbar_try(bar, parity)) return true;
        if (gtime() - t0 > kWaitNs) return false;
    }
}

// Programmatic dependent launch: let the next kernel of the stream start its
// set-up, and wait until the previous kernel's results are visible (a no-op
// for a kernel launched without the programmatic-serialisation attribute).
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // version
    d |= (uint64_t)2 << 61;              // SWIZZLE_128B
    return d;
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// two 16-column loads (the two significance accumulators) behind one wait
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float (&v)[16], float (&w)[16]) {
    uint32_t r[16], s[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]),
          "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11]), "=r"(s[12]), "=r"(s[13]), "=r"(s[14]), "=r"(s[15])
        : "r"(tb));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v[i] = __uint_as_float(r[i]);
        w[i] = __uint_as_float(s[i]);
    }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// --- thread-block cluster (K-split pair) helpers ---
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of the variable at shared::cta address `addr` in CTA `rank`
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster4(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// arrive (release at cluster scope) on an mbarrier of another CTA of the cluster
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// wait (acquire at cluster scope) with a deadline, polling every `ns` nanoseconds
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, unsigned ns) {
    const long long t0 = gtime();
    while (!mbar_try_cluster(bar, parity)) {
        if (gtime() - t0 > kWaitNs) return false;
        if (ns) __nanosleep(ns);
    }
    return true;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__host__ __device__ constexpr int tmem_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512; }

template <int NA, int NB, int BN, int STAGES, int KS>
struct TcSmem {
    static constexpr int kA = NA * kTileBytesA;
    static constexpr int kB = NB * BN * 128;
    static constexpr int kStage = kA + kB;
    // epilogue transpose buffers (8 warps); the drained (3-part) modes read their
    // sums transposed from the drain buffer and need none
    static constexpr int kXpose = NA == 3 ? 0 : 8 * 32 * 17 * 4;
    // the partners' partial sums of this CTA's columns: KS - 1 buffers of [128 slots][BN / KS
    // columns], 16-byte chunks swizzled by slot
    static constexpr int kRecv = KS > 1 ? (KS - 1) * kSlotTile * (BN / KS) * 4 : 0;
    // 3-part modes: FP32 running sums of the drained accumulators, per epilogue warp
    // [32 lanes][BN / 2 + 1] (padded rows)
    static constexpr int kDrain = NA == 3 ? 8 * 32 * (BN / 2 + 1) * 4 : 0;
    static constexpr int kBytes = STAGES * kStage + kXpose + kRecv + kDrain + 1024 /* align */ + 256 /* barriers */;
};

// ---------------------------------------------------------------------------
// producer and MMA loops: separate (not inlined) functions, so that the few
// values they carry stay in registers whatever the epilogue's register
// pressure is; both return false when a wait passed its deadline
// ---------------------------------------------------------------------------
// bar0: full barriers [0, S), empty barriers [S, 2S); stage s at sbase + s * kStage.
// The weight tiles (B) never change between launches, so the tiles of the first
// stages are requested before griddep_wait, i.e. while the previous kernel of
// the stream may still run; the operand tiles (A), which that kernel writes,
// only after it.
// Operand tiles of the slot groups in use: the active QPs of a tile fill its
// slots from the first one on, so the 32-slot groups with work are a prefix
// (bit g of gmask); a full tile takes one 128-row box, a partial one a 32-row
// box per group.  Rows of idle groups keep stale values; their MMA rows only
// feed the outputs of empty slots, which the epilogue discards.
template <int NA>
__device__ __forceinline__ void load_operand(const CUtensorMap* tmA, const CUtensorMap* tmA32, uint32_t st, int k0,
                                             const int (&arow)[3], unsigned gmask, uint32_t full) {
    if (gmask == 0xFu) {
#pragma unroll
        for (int a = 0; a < NA; ++a) tma_load_2d(st + a * kTileBytesA, tmA, k0, arow[a], full);
    } else {
#pragma unroll
        for (int a = 0; a < NA; ++a)
            for (int g = 0; g < 4; ++g)
                if ((gmask >> g) & 1u) tma_load_2d(st + a * kTileBytesA + g * 4096, tmA32, k0, arow[a] + 32 * g, full);
    }
}

template <int NA>
__device__ __forceinline__ uint32_t operand_bytes(unsigned gmask) {
    return (uint32_t)(NA * __popc(gmask) * 4096);
}

template <int NA, int NB, int BN, int STAGES, int KSTAGE, int KA>
__device__ __noinline__ bool produce(const CUtensorMap* tmA, const CUtensorMap* tmA32, const CUtensorMap* tmB,
                                     uint32_t sbase, uint32_t bar0, int nkb, int koff, int a0, int a1, int a2, int b0,
                                     int b1, int b2, unsigned gmask, int& issued) {
    const int arow[3] = {a0, a1, a2}, brow[3] = {b0, b1, b2};
    const uint32_t tx = (uint32_t)(KSTAGE - KA) + operand_bytes<NA>(gmask);
    const int pre = nkb < STAGES ? nkb : STAGES;   // stages start empty
    for (int kb = 0; kb < pre; ++kb) {
        const uint32_t full = bar0 + 8 * kb;
        mbar_expect_tx(full, tx);
        const uint32_t st = sbase + kb * KSTAGE;
#pragma unroll
        for (int b = 0; b < NB; ++b) tma_load_2d(st + KA + b * BN * 128, tmB, kb * kBK + koff, brow[b], full);
    }
    griddep_wait();
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        const uint32_t full = bar0 + 8 * s;
        const uint32_t st = sbase + s * KSTAGE;
        const int k0 = kb * kBK + koff;
        if (kb >= pre) {
            if (!mbar_wait(bar0 + 8 * (STAGES + s), ph ^ 1)) return false;
            mbar_expect_tx(full, tx);
#pragma unroll
            for (int b = 0; b < NB; ++b) tma_load_2d(st + KA + b * BN * 128, tmB, k0, brow[b], full);
        }
        load_operand<NA>(tmA, tmA32, st, k0, arow, gmask, full);
        issued = kb + 1;
    }
    return true;
}

// One layer of the persistent chunk kernel: as produce(), with the stage
// ring continuing across layers (k-block g0 + kb uses stage (g0 + kb) % S),
// and the operand tiles requested only once every CTA of this slot tile has
// released the previous layer (its counter reached `target`; sync == nullptr:
// wait for the previous kernel of the stream instead).
template <int NB, int BN, int STAGES, int KSTAGE, int KA>
__device__ __noinline__ bool produce_layer(const CUtensorMap* tmA, const CUtensorMap* tmA32, const CUtensorMap* tmB,
                                           uint32_t sbase, uint32_t bar0, int nkb, int koff, int g0, int a0, int a1,
                                           int b0, int b1, unsigned gmask, const unsigned* sync, unsigned target,
                                           int own_lo, int own_n, uint32_t own_bar, uint32_t own_par, int& issued,
                                           bool& sync_failed) {
    const int brow[2] = {b0, b1}, arow[3] = {a0, a1, 0};
    const uint32_t tx = (uint32_t)(KSTAGE - KA) + operand_bytes<2>(gmask);
    const int pre = nkb < STAGES ? nkb : STAGES;
    // k blocks in the order own_lo, own_lo + 1, ... (wrapping): the first own_n of them hold only
    // rows this CTA's own epilogue wrote
    auto kb_at = [&](int i) { return (i + own_lo) % nkb; };
    for (int i = 0; i < pre; ++i) {
        const int gk = g0 + i, s = gk % STAGES;
        if (!mbar_wait(bar0 + 8 * (STAGES + s), ((gk / STAGES) & 1) ^ 1)) return false;
        const uint32_t full = bar0 + 8 * s;
        mbar_expect_tx(full, tx);
#pragma unroll
        for (int b = 0; b < NB; ++b)
            tma_load_2d(sbase + s * KSTAGE + KA + b * BN * 128, tmB, kb_at(i) * kBK + koff, brow[b], full);
    }
    if (!sync) griddep_wait();
    bool own_ready = !sync || own_n == 0, tile_ready = !sync;
    for (int i = 0; i < nkb; ++i) {
        const int gk = g0 + i, s = gk % STAGES;
        const uint32_t full = bar0 + 8 * s;
        const uint32_t st = sbase + s * KSTAGE;
        const int k0 = kb_at(i) * kBK + koff;
        if (i >= pre) {
            if (!mbar_wait(bar0 + 8 * (STAGES + s), ((gk / STAGES) & 1) ^ 1)) return false;
            mbar_expect_tx(full, tx);
#pragma unroll
            for (int b = 0; b < NB; ++b) tma_load_2d(st + KA + b * BN * 128, tmB, k0, brow[b], full);
        }
        if (i < own_n && !own_ready) {
            // rows this CTA wrote itself: its epilogue warps have stored them and fenced
            // them for the async proxy before arriving on own_bar
            if (!mbar_wait(own_bar, own_par)) {
                sync_failed = true;
                return false;
            }
            asm volatile("fence.proxy.async.global;" ::: "memory");
            own_ready = true;
        } else if (i >= own_n && !tile_ready) {
            if (!wait_counter_geq(sync, target, kWaitNs)) {
                sync_failed = true;
                return false;
            }
            // the operand was written by generic stores of other CTAs; order them before the TMA reads
            asm volatile("fence.proxy.async.global;" ::: "memory");
            tile_ready = true;
        }
        load_operand<2>(tmA, tmA32, st, k0, arow, gmask, full);
        issued = gk + 1;
    }
    return true;
}

template <int BN, int STAGES, int KSTAGE, int KA>
__device__ __noinline__ bool issue_layer(uint32_t sbase, uint32_t bar0, uint32_t tmem, int nkb, int g0) {
    constexpr uint32_t IDESC = idesc_bf16(BN);
    const uint64_t d0 = sdesc(sbase);
    for (int kb = 0; kb < nkb; ++kb) {
        const int gk = g0 + kb, s = gk % STAGES;
        if (!mbar_wait(bar0 + 8 * s, (gk / STAGES) & 1)) return false;
        fence_after();
        const uint64_t da = d0 + (uint64_t)((s * KSTAGE) >> 4);
        const uint64_t db = da + (uint64_t)(KA >> 4);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
                // (d_hi, w1) -> accumulator 0; (d_hi, w2), (d_lo, w1) -> accumulator 1
                const int ia = pr == 2 ? 1 : 0, ib = pr == 1 ? 1 : 0;
                const uint64_t ad = da + (uint64_t)((ia * kTileBytesA + kk * 32) >> 4);
                const uint64_t bd = db + (uint64_t)((ib * BN * 128 + kk * 32) >> 4);
                const bool first = kb == 0 && kk == 0 && pr <= 1;
                mma_bf16(tmem + (pr == 0 ? 0 : BN), ad, bd, IDESC, first ? 0u : 1u);
            }
        }
        mma_commit(bar0 + 8 * (STAGES + s));
    }
    return true;
}

// Descriptors are formed once; a stage, part or 16-element k step is a
// constant byte offset, i.e. an add of offset / 16 to the address field
// (shared addresses stay below 2^18, so the 14-bit field cannot carry).
template <int NPROD, int BN, int STAGES, int KSTAGE, int KA>
__device__ __noinline__ bool issue_mmas(uint32_t sbase, uint32_t bar0, uint32_t tmem, int nkb) {
    constexpr uint32_t IDESC = idesc_bf16(BN);
    const uint64_t d0 = sdesc(sbase);
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(bar0 + 8 * s, ph)) return false;
        fence_after();
        const uint64_t da = d0 + (uint64_t)((s * KSTAGE) >> 4);
        const uint64_t db = da + (uint64_t)(KA >> 4);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
            for (int pr = 0; pr < NPROD; ++pr) {
                // product list: (0,0) | (0,1) (1,0) (0,2) (1,1) (2,0)
                const int ia = pr == 0 ? 0 : pr == 1 ? 0 : pr == 2 ? 1 : pr == 3 ? 0 : pr == 4 ? 1 : 2;
                const int ib = pr == 0 ? 0 : pr == 1 ? 1 : pr == 2 ? 0 : pr == 3 ? 2 : pr == 4 ? 1 : 0;
                const uint64_t ad = da + (uint64_t)((ia * kTileBytesA + kk * 32) >> 4);
                const uint64_t bd = db + (uint64_t)((ib * BN * 128 + kk * 32) >> 4);
                const bool first = kb == 0 && kk == 0 && pr <= 1;   // first MMA of either accumulator
                mma_bf16(tmem + (pr == 0 ? 0 : BN), ad, bd, IDESC, first ? 0u : 1u);
            }
        }
        mma_commit(bar0 + 8 * (STAGES + s));
    }
    return true;
}

// 3-part modes (accurate layer, residual products): the products of k-block kb
// go into a fresh accumulator pair in TMEM buffer kb & 1 (columns
// [2 BN (kb & 1), 2 BN (kb & 1) + 2 BN)), committed to kready[kb & 1]; the
// epilogue warps add every k-block's pair into FP32 running sums (round to
// nearest) and release the buffer through drained[kb & 1].  The tensor core's
// truncating accumulation then spans the 4 MMA steps of one k-block instead of
// the whole dot product.
template <int BN, int STAGES, int KSTAGE, int KA>
__device__ __noinline__ bool issue_mmas_drain(uint32_t sbase, uint32_t bar0, uint32_t tmem, int nkb, uint32_t kready0,
                                              uint32_t drained0) {
    constexpr uint32_t IDESC = idesc_bf16(BN);
    const uint64_t d0 = sdesc(sbase);
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES;
        const int b = kb & 1;
        if (!mbar_wait(bar0 + 8 * s, (kb / STAGES) & 1)) return false;
        if (kb >= 2 && !mbar_wait(drained0 + 8 * b, ((kb >> 1) - 1) & 1)) return false;
        fence_after();
        const uint64_t da = d0 + (uint64_t)((s * KSTAGE) >> 4);
        const uint64_t db = da + (uint64_t)(KA >> 4);
        const uint32_t tb = tmem + (uint32_t)(2 * BN * b);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
            for (int pr = 0; pr < 6; ++pr) {
                const int ia = pr == 0 ? 0 : pr == 1 ? 0 : pr == 2 ? 1 : pr == 3 ? 0 : pr == 4 ? 1 : 2;
                const int ib = pr == 0 ? 0 : pr == 1 ? 1 : pr == 2 ? 0 : pr == 3 ? 2 : pr == 4 ? 1 : 0;
                const uint64_t ad = da + (uint64_t)((ia * kTileBytesA + kk * 32) >> 4);
                const uint64_t bd = db + (uint64_t)((ib * BN * 128 + kk * 32) >> 4);
                const bool first = kk == 0 && pr <= 1;   // fresh pair for every k-block
                mma_bf16(tb + (pr == 0 ? 0 : BN), ad, bd, IDESC, first ? 0u : 1u);
            }
        }
        mma_commit(bar0 + 8 * (STAGES + s));
        mma_commit(kready0 + 8 * b);
    }
    return true;
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
// float offset of (slot, col) in a receive buffer of OWN columns: the 16-byte
// chunk index is XORed with the low bits of the slot, so the rows a warp
// writes or reads at one column spread over the banks (OWN is 16 or a
// multiple of 32)
template <int OWN>
__device__ __forceinline__ int recv_off(int slot, int col) {
    constexpr int SW = OWN / 4 >= 8 ? 7 : OWN / 4 - 1;
    return slot * OWN + ((((col >> 2) ^ (slot & SW))) << 2) + (col & 3);
}

// The epilogue of one tile for the epilogue warp `warp` (2..9): waits for the
// accumulators (barrier bar_acc, phase parity par_acc), exchanges the K-split
// partial sums with the partners (bar_recv / par_recv), and applies the
// element-wise part of the mode to this warp's columns.  Returns false after a
// deadline (the error is recorded).
template <int MODE, int BN, int KS>
__device__ __forceinline__ bool tile_epilogue(const BatchParams& p, const TcArgs& g, int warp, int lane, int rank,
                                              int slot0, int row0, int ri, uint32_t tmem, float* xpose, float* recv,
                                              uint32_t bar_acc, uint32_t par_acc, uint32_t bar_recv,
                                              uint32_t par_recv, int* s_fail, float* drain = nullptr, int nkb = 0,
                                              uint32_t kready0 = 0, uint32_t drained0 = 0) {
    constexpr int OWN = BN / KS;
    constexpr int HALVES = OWN >= 32 ? 2 : 1;
    constexpr int PER = OWN / HALVES;
    constexpr bool DRAIN = MODE != MODE_LAYER_REFINED;
    // drained modes with a K split: every epilogue warp drains its share of all BN
    // columns over this CTA's k range (DW columns from dbeg), sends the partners
    // their columns' partial sums, and the warps that hold this CTA's own columns
    // add the KS partials in rank order in place
    constexpr bool DSPLIT = DRAIN && KS > 1;
    constexpr int DW = DSPLIT ? BN / HALVES : PER;
    const int q = warp & 3;                         // TMEM lane quadrant of this warp
    const int half = (warp - 2) >> 2;               // which half of this CTA's columns
    const int slot = slot0 + q * 32 + lane;
    const int qp = p.perm[slot];
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    // whole 16-row pieces are transposed so that lane = 4 * (slot % 8) + (row
    // group): pass `pass` handles rows cg..cg+3 of the QP of slot pass * 8 +
    // lane / 4, and a warp's 128-bit accesses cover 8 QPs' contiguous 64-byte
    // row segments.  Refined layers transpose through a per-warp shared-memory
    // buffer; the drained modes read the other slots' sums where they are.
    const int cg = (lane & 3) * 4;
    int qq[4];
#pragma unroll
    for (int pass = 0; pass < 4; ++pass) qq[pass] = __shfl_sync(0xffffffffu, qp, pass * 8 + (lane >> 2));
    const int own0 = rank * OWN;
    const int dbeg = DSPLIT ? half * DW : own0 + half * PER;   // first drained column of this warp
    const bool holds_own = !DSPLIT || (own0 >= dbeg && own0 < dbeg + DW);
    // the columns this warp finalises (none for a split warp that only sends)
    const int cbeg = DSPLIT ? own0 : own0 + half * PER;
    const int cend = holds_own ? cbeg + (DSPLIT ? OWN : PER) : cbeg;
    const bool n_aligned = (p.n & 3) == 0;
    auto whole_at = [&](int c0) {
        const int r0 = row0 + c0;
        return MODE <= MODE_LAYER_ACCURATE && r0 + 16 <= g.rows && (r0 + 16 <= p.n || (r0 >= p.n && n_aligned));
    };
    // residual products: 16-row pieces of rows of x only or of A x only take the
    // transposed path as well (the drained sums of every slot of the warp are in
    // shared memory, so the transposition needs no extra buffer)
    constexpr bool CHECK = MODE == MODE_CHECK1 || MODE == MODE_CHECK2;
    auto check_whole_at = [&](int c0) {
        const int r0 = row0 + c0;
        return CHECK && r0 + 16 <= g.rows && (r0 + 16 <= p.n || (r0 >= p.n && n_aligned));
    };
    float mx[4][4];   // per pass (QP): the residual maxima of the transposed pieces
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) mx[a][b] = 0.f;
    // refined layers: the lighter refined-only inputs (flags never hold EPI_REBASE)
    using Piece = typename std::conditional<MODE == MODE_LAYER_REFINED, Chunk4R, Chunk4>::type;
    Piece in[4];
    float rs[4] = {1.f, 1.f, 1.f, 1.f}, rs_next[4] = {1.f, 1.f, 1.f, 1.f};
    // inputs of one 4-row piece of the 16-column chunk at c0 (pass = QP group)
    auto load_pass = [&](int c0, int pass) {
        if (qq[pass] >= 0) chunk4_load(p, qq[pass], ri, row0 + c0 + cg, in[pass]);
    };
    auto load_rs = [&](int c0, float (&dst)[4]) {
        const int r0 = row0 + c0 + cg;
        if (r0 >= p.n) ld4(p.rs + (r0 - p.n), dst);
    };
    // the inputs of the first chunk load while the MMAs run
    if (cend > cbeg && whole_at(cbeg)) {
        load_rs(cbeg, rs);
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) load_pass(cbeg, pass);
    }
    // one lane per warp polls the accumulator barrier (sleeping between
    // polls) for the whole main loop; then every lane observes the
    // completed phase itself
    bool ready = true;
    // this warp's running sums [lane][DW] (drained modes)
    float* dsum = DRAIN ? drain + (warp - 2) * 32 * (DW + 1) + lane * (DW + 1) : nullptr;
    if (DRAIN) {
#pragma unroll
        for (int c = 0; c < DW; ++c) dsum[c] = 0.f;
        for (int kb = 0; kb < nkb && ready; ++kb) {
            const int b = kb & 1;
            const uint32_t par = (kb >> 1) & 1;
            if (lane == 0) ready = mbar_wait_sleep(kready0 + 8 * b, par, 64);
            ready = __shfl_sync(0xffffffffu, ready, 0);
            if (ready) ready = mbar_wait(kready0 + 8 * b, par);
            ready = __all_sync(0xffffffffu, ready);
            if (!ready) break;
            fence_after();
            const uint32_t tb = tl + (uint32_t)(2 * BN * b);
#pragma unroll
            for (int c = 0; c < DW; c += 16) {
                float v[16], w[16];
                tmem_ld16x2(tb + dbeg + c, tb + BN + dbeg + c, v, w);
#pragma unroll
                for (int t = 0; t < 16; ++t) dsum[c + t] += v[t] + w[t];
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(drained0 + 8 * b);
        }
    } else {
        if (lane == 0) ready = mbar_wait_sleep(bar_acc, par_acc, 256);
        ready = __shfl_sync(0xffffffffu, ready, 0);
        if (ready) ready = mbar_wait(bar_acc, par_acc);
        ready = __all_sync(0xffffffffu, ready);
        if (ready) fence_after();
    }
    if (DSPLIT) {
        // partial sums of the partners' columns (those this warp drained) go to row
        // (q * 32 + lane) of buffer j of each partner's receive area
        const int srow = q * 32 + lane;
        for (int pk = 0; pk < KS; ++pk) {
            if (pk == rank) continue;
            const int pc0 = pk * OWN;
            if (pc0 < dbeg || pc0 >= dbeg + DW) continue;   // not drained here
            const int j = rank < pk ? rank : rank - 1;
            const uint32_t dst = mapa(smem_u32(recv + j * kSlotTile * OWN), (uint32_t)pk);
            if (ready) {
#pragma unroll
                for (int c = 0; c < OWN; c += 4)
                    st_cluster4(dst + 4u * (uint32_t)recv_off<OWN>(srow, c), dsum[pc0 - dbeg + c],
                                dsum[pc0 - dbeg + c + 1], dsum[pc0 - dbeg + c + 2], dsum[pc0 - dbeg + c + 3]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(mapa(bar_recv, (uint32_t)pk));
        }
        bool got = true;
        if (holds_own) {
            if (lane == 0) got = mbar_wait_cluster(bar_recv, par_recv, 64);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (got) got = mbar_wait_cluster(bar_recv, par_recv, 0);
            got = __all_sync(0xffffffffu, got);
            if (!got && ready && lane == 0) { wait_failed(g.err, WS_EPI_RECV); *s_fail = 1; }
            if (got && ready) {
                // own columns: the KS partials added in rank order, written back in place
#pragma unroll
                for (int c = 0; c < OWN; c += 4) {
                    float tot[4];
#pragma unroll
                    for (int k = 0; k < KS; ++k) {
                        float part[4];
                        if (k == rank) {
#pragma unroll
                            for (int t = 0; t < 4; ++t) part[t] = dsum[own0 - dbeg + c + t];
                        } else {
                            const float* rb = recv + (k < rank ? k : k - 1) * kSlotTile * OWN;
                            const float4 o = *reinterpret_cast<const float4*>(rb + recv_off<OWN>(srow, c));
                            part[0] = o.x;
                            part[1] = o.y;
                            part[2] = o.z;
                            part[3] = o.w;
                        }
#pragma unroll
                        for (int t = 0; t < 4; ++t) tot[t] = k == 0 ? part[t] : tot[t] + part[t];
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) dsum[own0 - dbeg + c + t] = tot[t];
                }
            }
        }
        ready = ready && got;
    }
    if (KS > 1 && !DRAIN) {
        // send every partner its columns of this warp's TMEM lanes: row (q * 32 + lane)
        // of buffer j of the partner's receive area (j = this CTA's index among the
        // partner's senders), columns half * PER ...
        const int srow = q * 32 + lane;
        for (int pk = 0; pk < KS; ++pk) {
            if (pk == rank) continue;
            const int j = rank < pk ? rank : rank - 1;
            const int pc0 = pk * OWN + half * PER;
            const uint32_t dst = mapa(smem_u32(recv + j * kSlotTile * OWN), (uint32_t)pk);
            if (ready) {
#pragma unroll
                for (int c = 0; c < PER; c += 16) {
                    float v[16], w[16];
                    tmem_ld16x2(tl + pc0 + c, tl + BN + pc0 + c, v, w);
#pragma unroll
                    for (int t = 0; t < 16; t += 4)
                        st_cluster4(dst + 4u * (uint32_t)recv_off<OWN>(srow, half * PER + c + t), v[t] + w[t],
                                    v[t + 1] + w[t + 1], v[t + 2] + w[t + 2], v[t + 3] + w[t + 3]);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(mapa(bar_recv, (uint32_t)pk));
        }
        // the partners' partial sums of this CTA's columns
        bool got = true;
        if (lane == 0) got = mbar_wait_cluster(bar_recv, par_recv, 64);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got) got = mbar_wait_cluster(bar_recv, par_recv, 0);
        got = __all_sync(0xffffffffu, got);
        if (!got && ready && lane == 0) { wait_failed(g.err, WS_EPI_RECV); *s_fail = 1; }
        ready = ready && got;
    }
    if (!ready) {
        if (lane == 0) { wait_failed(g.err, DRAIN ? WS_DRAIN_READY : WS_EPI_ACC); *s_fail = 1; }
    } else {
        float ra = 0.f, rb = 0.f, rc = 0.f, rd = 0.f;
        // inputs of the next whole chunk load pass by pass as this chunk's
        // passes finish, so that a memory round trip overlaps a chunk of work
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
            const int r0 = row0 + c0;
            const bool whole = whole_at(c0);
            const int cn = c0 + 16;
            const bool next_whole = cn < cend && whole_at(cn);
            if (next_whole) load_rs(cn, rs_next);
            if (CHECK && check_whole_at(c0)) {
                // lane = 4 * (slot % 8) + row group: rows r0 + cg .. + 3 of the slot
                // pass * 8 + lane / 4, read from that slot's drained sums
                __syncwarp();
                const float* wsum = drain + (warp - 2) * 32 * (DW + 1);
#pragma unroll
                for (int pass = 0; pass < 4; ++pass) {
                    const int sl = pass * 8 + (lane >> 2);
                    if (qq[pass] < 0) continue;
                    const float* src = wsum + sl * (DW + 1) + (c0 - dbeg) + cg;
                    const float a4[4] = {src[0], src[1], src[2], src[3]};
                    if (MODE == MODE_CHECK1)
                        check1_4(p, slot0 + q * 32 + sl, qq[pass], ri, r0 + cg, a4, mx[pass][0], mx[pass][1],
                                 mx[pass][2], mx[pass][3]);
                    else
                        check2_4(p, qq[pass], r0 + cg, a4, mx[pass][0], mx[pass][1]);
                }
                continue;
            }
            float v[16];
            if (DRAIN) {
#pragma unroll
                for (int t = 0; t < 16; ++t) v[t] = dsum[c0 - dbeg + t];
            } else {
                float w[16];
                tmem_ld16x2(tl + c0, tl + BN + c0, v, w);
#pragma unroll
                for (int t = 0; t < 16; ++t) v[t] += w[t];
            }
            if (KS > 1 && !DRAIN) {
                // partial sums of ranks 0 .. KS-1 added in rank order
                float tot[16];
#pragma unroll
                for (int k = 0; k < KS; ++k) {
                    float part[16];
                    if (k == rank) {
#pragma unroll
                        for (int t = 0; t < 16; ++t) part[t] = v[t];
                    } else {
                        const float* rb = recv + (k < rank ? k : k - 1) * kSlotTile * OWN;
#pragma unroll
                        for (int t = 0; t < 16; t += 4) {
                            const float4 o =
                                *reinterpret_cast<const float4*>(rb + recv_off<OWN>(q * 32 + lane, c0 - own0 + t));
                            part[t] = o.x;
                            part[t + 1] = o.y;
                            part[t + 2] = o.z;
                            part[t + 3] = o.w;
                        }
                    }
#pragma unroll
                    for (int t = 0; t < 16; ++t) tot[t] = k == 0 ? part[t] : tot[t] + part[t];
                }
#pragma unroll
                for (int t = 0; t < 16; ++t) v[t] = tot[t];
            }
            if (whole) {
                // the source rows: this warp's transpose buffer (refined), or the
                // drained sums, which already hold every slot of the warp
                const float* base;
                int stride, off;
                if (DRAIN) {
                    base = drain + (warp - 2) * 32 * (DW + 1);
                    stride = DW + 1;
                    off = c0 - dbeg;
                } else {
                    float* xb = xpose + (warp - 2) * 32 * 17;       // [32 slots][16 rows]
#pragma unroll
                    for (int t = 0; t < 16; ++t) xb[lane * 17 + t] = v[t];
                    base = xb;
                    stride = 17;
                    off = 0;
                }
                __syncwarp();
#pragma unroll
                for (int pass = 0; pass < 4; ++pass) {
                    const int sl = pass * 8 + (lane >> 2);          // slot within the warp's 32
                    if (qq[pass] >= 0) {
                        float a4[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t) a4[t] = base[sl * stride + off + cg + t];
                        chunk4_apply(p, slot0 + q * 32 + sl, qq[pass], ri, r0 + cg, a4, in[pass], rs);
                    }
                    if (next_whole) load_pass(cn, pass);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) rs[k] = rs_next[k];
                __syncwarp();
                continue;
            }
            if (qp >= 0) {
#pragma unroll 4
                for (int t = 0; t < 16; ++t) {
                    const int r = r0 + t;
                    if (r >= g.rows) continue;
                    if (MODE == MODE_CHECK1) check1_elem(p, slot, qp, ri, r, v[t], ra, rb, rc, rd);
                    else if (MODE == MODE_CHECK2) check2_elem(p, qp, r, v[t], ra, rb);
                    else layer_elem(p, slot, qp, ri, r, v[t]);
                }
            }
            if (next_whole) {
#pragma unroll
                for (int pass = 0; pass < 4; ++pass) load_pass(cn, pass);
#pragma unroll
                for (int k = 0; k < 4; ++k) rs[k] = rs_next[k];
            }
        }
        if (qp >= 0) {
            if (MODE == MODE_CHECK1) {
                red_slot(p.RED, qp, RW_RP, ra);
                red_slot(p.RED, qp, RW_AX, rb);
                red_slot(p.RED, qp, RW_Z, rc);
                red_slot(p.RED, qp, RW_PX, rd);
            } else if (MODE == MODE_CHECK2) {
                red_slot(p.RED, qp, RW_RD, ra);
                red_slot(p.RED, qp, RW_ATL, rb);
            }
        }
        if (CHECK) {
            // the transposed pieces: the 4 lanes of a slot (lane & 3 = row group)
            // combine their maxima, then one of them adds them to the QP's words
#pragma unroll
            for (int pass = 0; pass < 4; ++pass) {
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    float v = mx[pass][b];
                    v = nmax(v, __shfl_xor_sync(0xffffffffu, v, 1));
                    v = nmax(v, __shfl_xor_sync(0xffffffffu, v, 2));
                    mx[pass][b] = v;
                }
                if ((lane & 3) == 0 && qq[pass] >= 0) {
                    if (MODE == MODE_CHECK1) {
                        red_slot(p.RED, qq[pass], RW_RP, mx[pass][0]);
                        red_slot(p.RED, qq[pass], RW_AX, mx[pass][1]);
                        red_slot(p.RED, qq[pass], RW_Z, mx[pass][2]);
                        red_slot(p.RED, qq[pass], RW_PX, mx[pass][3]);
                    } else {
                        red_slot(p.RED, qq[pass], RW_RD, mx[pass][0]);
                        red_slot(p.RED, qq[pass], RW_ATL, mx[pass][1]);
                    }
                }
            }
        }
    }
    return ready;
}

// KS = 2 or 4 (refined layers): the KS CTAs of a cluster split the k-blocks
// into KS fixed ranges; after its main loop each CTA sends every partner the
// partial sums of that partner's BN / KS columns (into the partner's shared
// memory) and finalises its own columns, adding the KS partial sums in rank
// order.  The ranges and the order depend only on the problem and KS; the tuner
// picks KS per number of active slot tiles, so in the BF16 split form a QP's
// rounding may depend on the size of its batch (within the form's tolerance).
template <int MODE, int BN, int STAGES, int KS>
__global__ void __launch_bounds__(kThreadsTC, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA32,
                   const __grid_constant__ CUtensorMap tmB, BatchParams p, TcArgs g) {
    constexpr int NA = MODE == MODE_LAYER_REFINED ? 2 : 3;
    constexpr int NB = NA;
    constexpr int NPROD = NA == 2 ? 3 : 6;
    constexpr int ACC = 2;   // significance accumulators of BN columns each
    constexpr bool DRAIN = MODE != MODE_LAYER_REFINED;
    constexpr int TCOLS = tmem_cols((DRAIN ? 2 : 1) * ACC * BN);   // drained modes: two buffers
    constexpr int OWN = BN / KS;        // columns this CTA finalises
    constexpr int HALVES = OWN >= 32 ? 2 : 1;   // epilogue warps per TMEM lane quadrant
    constexpr int PER = OWN / HALVES;   // columns per epilogue warp
    static_assert(KS == 1 || KS == 2 || KS == 4, "K split of 1, 2 or 4");
    static_assert(PER % 16 == 0, "the epilogue works on 16-column pieces");
    using L = TcSmem<NA, NB, BN, STAGES, KS>;

    const int tile = blockIdx.y;
    if (tile >= p.counters[CNT_TILES]) return;     // uniform over the CTA (and the cluster)
    // the partial-sum exchange addresses KS CTAs of a cluster: refuse any other launch shape
    if (KS > 1 && cluster_size() != (uint32_t)KS) {
        if (threadIdx.x == 0) atomicExch(g.err, RELU_QP_ERR_CUDA);
        return;
    }
    const int slot0 = tile * kSlotTile;
    const int rank = KS > 1 ? (int)cluster_rank() : 0;
    const int row0 = (blockIdx.x / KS) * BN;
    const int ri = p.tile_rho[tile];
    // k-blocks of this CTA: [kb_begin, kb_begin + kb_count)
    const int kb_begin = rank * g.num_kb / KS;
    const int kb_count = (rank + 1) * g.num_kb / KS - kb_begin;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* xpose = reinterpret_cast<float*>(smem + STAGES * L::kStage);
    float* recv = reinterpret_cast<float*>(smem + STAGES * L::kStage + L::kXpose);
    float* drain = reinterpret_cast<float*>(smem + STAGES * L::kStage + L::kXpose + L::kRecv);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * L::kStage + L::kXpose + L::kRecv + L::kDrain);
    // bars[0..S) full, bars[S..2S) empty, bars[2S] accumulator ready, bars[2S+1] partners'
    // partial sums received (KS > 1), bars[2S+2..2S+3] k-block buffer ready, bars[2S+4..2S+5]
    // buffer drained (3-part modes); then the TMEM address
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 6);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[STAGES + s]), 1);
        }
        mbar_init(smem_u32(&bars[2 * STAGES]), 1);
        // one arrival per sending epilogue warp of every partner (refined: every warp;
        // drained with a K split: the 4 warps that drained this CTA's columns)
        mbar_init(smem_u32(&bars[2 * STAGES + 1]), (KS > 1 ? KS - 1 : 1) * 4 * (DRAIN ? 1 : HALVES));
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bars[2 * STAGES + 2 + b]), 1);
            mbar_init(smem_u32(&bars[2 * STAGES + 4 + b]), 4 * HALVES);   // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    // the partners' barriers are initialised before anything is sent to them
    if (KS > 1) cluster_sync();
    const uint32_t tmem = *tmem_holder;
    // the next kernel of the stream may be scheduled once every CTA got here
    griddep_launch();

    if (warp == 0) {
        // ------------------------- TMA producer -------------------------
        if (lane == 0) {
            prefetch_map(&tmA);
            prefetch_map(&tmA32);
            prefetch_map(&tmB);
            unsigned gmask = 0;
            for (int gr = 0; gr < 4; ++gr)
                if (p.perm[slot0 + 32 * gr] >= 0) gmask |= 1u << gr;
            int arow[3] = {0, 0, 0}, brow[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < NA; ++a) arow[a] = g.a_row[a] + slot0;
#pragma unroll
            for (int b = 0; b < NB; ++b) brow[b] = g.b_row[b] + ri * g.b_rho_stride + row0;
            int issued = 0;
            const bool ok = produce<NA, NB, BN, STAGES, L::kStage, L::kA>(
                &tmA, &tmA32, &tmB, smem_u32(smem), smem_u32(bars), kb_count, g.k_off + kb_begin * kBK, arow[0],
                arow[1], arow[2], brow[0], brow[1], brow[2], gmask, issued);
            if (!ok) {
                wait_failed(g.err, WS_PROD_EMPTY);
                s_fail = 1;
                // wait (bounded) for the copies already in flight
                for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
                    mbar_wait(smem_u32(&bars[kb % STAGES]), (kb / STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        // ------------------------- MMA issuer -------------------------
        if (lane == 0) {
            const bool ok =
                DRAIN ? issue_mmas_drain<BN, STAGES, L::kStage, L::kA>(smem_u32(smem), smem_u32(bars), tmem, kb_count,
                                                                      smem_u32(&bars[2 * STAGES + 2]),
                                                                      smem_u32(&bars[2 * STAGES + 4]))
                      : issue_mmas<NPROD, BN, STAGES, L::kStage, L::kA>(smem_u32(smem), smem_u32(bars), tmem,
                                                                       kb_count);
            // (also after a failure: MMAs already issued must land before TMEM is freed)
            mma_commit(smem_u32(&bars[2 * STAGES]));
            // keep TMEM alive until the MMAs have landed
            if (!mbar_wait(smem_u32(&bars[2 * STAGES]), 0) || !ok) {
                wait_failed(g.err, ok ? WS_MMA_ACC : WS_MMA_FULL);
                s_fail = 1;
            }
        }
        __syncwarp();
    } else if (HALVES == 2 || warp < 6) {
        // ------------------------- epilogue -------------------------
        // the previous kernel's writes (the carried r, the state) are read and the
        // operand it read is overwritten: wait for it
        griddep_wait();
        tile_epilogue<MODE, BN, KS>(p, g, warp, lane, rank, slot0, row0, ri, tmem, xpose, recv,
                                    smem_u32(&bars[2 * STAGES]), 0, smem_u32(&bars[2 * STAGES + 1]), 0, &s_fail,
                                    drain, kb_count, smem_u32(&bars[2 * STAGES + 2]), smem_u32(&bars[2 * STAGES + 4]));
    }
    fence_before();
    __syncthreads();
    // no CTA of a cluster leaves while another may still address its shared memory
    if (KS > 1) cluster_sync();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Persistent chunk: the refined layers 1 .. nl of one chunk in one launch.
// Every CTA keeps its (slot tile, row block, k range) for all layers, so the
// set-up (barriers, TMEM, tensor maps) happens once and the weight tiles of a
// layer are requested while the previous layer still finishes.  Layer j reads
// operand pair (j - 1) & 1 and writes pair j & 1 (both written only by the
// epilogues of the CTAs of the same slot tile): after its epilogue a CTA adds
// one to the tile's counter, and a producer requests the operand of layer j
// only once the counter shows every CTA of the tile done with layer j - 1.  The
// counters start at zero and the tile's last CTA puts them back to zero at the
// end (launches are in stream order, without programmatic overlap).
// That also orders the reuse of TMEM and of the receive buffers (a partner
// sends layer j's partial sums only after all of layer j - 1 is done).  The
// CTAs of a tile must be co-resident: the host launches it only when the grid
// is at most one CTA per SM and nothing else of the handle runs beside it;
// every wait has a deadline.
// ---------------------------------------------------------------------------
struct ChunkArgs {
    int nl;                    // refined layers of the chunk (1 .. nl)
    unsigned last_flags;       // extra flags of layer nl (EPI_LAST, EPI_CHECK)
    __nv_bfloat16* OP;         // operand parts: pair 0 = parts 0, 1; pair 1 = parts 2, 3
    size_t opart;              // elements per part
    int slots;                 // rows per part in the operand tensor map
    unsigned* sync;            // per slot tile: CTAs done with layers so far (zero at launch), then
                               // at sync + done_off the CTAs done with the whole launch
    int done_off;
    int ncols;                 // resident-weight kernel: slots in the MMA's N (a multiple of 16)
};

template <int BN, int STAGES, int KS>
__global__ void __launch_bounds__(kThreadsTC, 1)
    tc_chunk_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA32,
                    const __grid_constant__ CUtensorMap tmB, BatchParams p, TcArgs g, ChunkArgs c) {
    constexpr int TCOLS = tmem_cols(2 * BN);
    constexpr int OWN = BN / KS;
    constexpr int HALVES = OWN >= 32 ? 2 : 1;
    constexpr int PER = OWN / HALVES;
    static_assert(KS == 1 || KS == 2 || KS == 4, "K split of 1, 2 or 4");
    static_assert(PER % 16 == 0, "the epilogue works on 16-column pieces");
    using L = TcSmem<2, 2, BN, STAGES, KS>;

    const int tile = blockIdx.y;
    if (tile >= p.counters[CNT_TILES]) return;     // uniform over the CTA (and the cluster)
    if (KS > 1 && cluster_size() != (uint32_t)KS) {
        if (threadIdx.x == 0) atomicExch(g.err, RELU_QP_ERR_CUDA);
        return;
    }
    const int slot0 = tile * kSlotTile;
    const int rank = KS > 1 ? (int)cluster_rank() : 0;
    const int row0 = (blockIdx.x / KS) * BN;
    const int ri = p.tile_rho[tile];
    const int kb_begin = rank * g.num_kb / KS;
    const int kb_count = (rank + 1) * g.num_kb / KS - kb_begin;
    const unsigned nct = gridDim.x;                // CTAs of this slot tile

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* xpose = reinterpret_cast<float*>(smem + STAGES * L::kStage);
    float* recv = reinterpret_cast<float*>(smem + STAGES * L::kStage + L::kXpose);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * L::kStage + L::kXpose + L::kRecv);
    // bars[2S] accumulator ready, bars[2S+1] partners' partial sums received,
    // bars[2S+2] accumulator consumed (the epilogue warps read all of a layer's TMEM),
    // bars[2S+3] this CTA's rows of the layer stored (for its producer's own k blocks)
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
    int& s_fail = *reinterpret_cast<int*>(tmem_holder + 1);   // in the dynamic area: no static shared memory

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[STAGES + s]), 1);
        }
        mbar_init(smem_u32(&bars[2 * STAGES]), 1);
        mbar_init(smem_u32(&bars[2 * STAGES + 1]), (KS > 1 ? KS - 1 : 1) * 4 * HALVES);
        mbar_init(smem_u32(&bars[2 * STAGES + 2]), 4 * HALVES);   // one arrival per epilogue warp
        mbar_init(smem_u32(&bars[2 * STAGES + 3]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (KS > 1) cluster_sync();
    const uint32_t tmem = *tmem_holder;
    griddep_launch();

    if (warp == 0) {
        // ------------------------- TMA producer -------------------------
        if (lane == 0) {
            prefetch_map(&tmA);
            prefetch_map(&tmA32);
            prefetch_map(&tmB);
            unsigned gmask = 0;
            for (int gr = 0; gr < 4; ++gr)
                if (p.perm[slot0 + 32 * gr] >= 0) gmask |= 1u << gr;
            const int b0 = g.b_row[0] + ri * g.b_rho_stride + row0, b1 = g.b_row[1] + ri * g.b_rho_stride + row0;
            // without a K split, the k blocks made only of this CTA's own rows are loaded first,
            // after its own epilogue and before the tile's counter; every other k block
            // still waits for the whole tile (which also keeps each layer's epilogue from
            // overwriting an operand buffer another CTA may still read)
            const int own_lo = KS == 1 ? (row0 + kBK - 1) / kBK : 0;
            const int own_hi = KS == 1 ? min(row0 + BN, g.rows) / kBK : 0;
            const int own_n = (KS == 1 && own_hi > own_lo && own_hi - own_lo < kb_count) ? own_hi - own_lo : 0;
            int issued = 0;
            bool sync_failed = false;
            for (int j = 1; j <= c.nl; ++j) {
                if (*(volatile int*)&s_fail) break;
                const int a0 = 2 * ((j - 1) & 1) * c.slots + slot0;
                const bool ok = produce_layer<2, BN, STAGES, L::kStage, L::kA>(
                    &tmA, &tmA32, &tmB, smem_u32(smem), smem_u32(bars), kb_count, g.k_off + kb_begin * kBK,
                    (j - 1) * kb_count, a0, a0 + c.slots, b0, b1, gmask, j == 1 ? nullptr : c.sync + tile,
                    (unsigned)(j - 1) * nct, own_n ? own_lo : 0, own_n, smem_u32(&bars[2 * STAGES + 3]),
                    (uint32_t)((j - 2) & 1), issued, sync_failed);
                if (!ok) {
                    wait_failed(g.err, sync_failed ? WS_PROD_SYNC : WS_PROD_EMPTY);
                    s_fail = 1;
                    break;
                }
            }
            // wait (bounded) for the copies still in flight
            for (int gk = (issued > STAGES ? issued - STAGES : 0); gk < issued; ++gk)
                mbar_wait(smem_u32(&bars[gk % STAGES]), (gk / STAGES) & 1);
        }
    } else if (warp == 1) {
        // ------------------------- MMA issuer -------------------------
        if (lane == 0) {
            int commits = 0;
            for (int j = 1; j <= c.nl; ++j) {
                if (*(volatile int*)&s_fail) break;
                // the accumulators of layer j - 1 must have been read by every epilogue
                // warp before layer j writes them (this also keeps the ready barrier
                // from completing a phase the epilogue has not seen)
                if (j > 1 && !mbar_wait(smem_u32(&bars[2 * STAGES + 2]), (uint32_t)((j - 2) & 1))) {
                    wait_failed(g.err, WS_MMA_ACC);
                    s_fail = 1;
                    break;
                }
                fence_after();
                const bool ok = issue_layer<BN, STAGES, L::kStage, L::kA>(smem_u32(smem), smem_u32(bars), tmem,
                                                                        kb_count, (j - 1) * kb_count);
                // committed also after a failure, so that the MMAs already issued are waited for
                mma_commit(smem_u32(&bars[2 * STAGES]));
                ++commits;
                if (!ok) {
                    wait_failed(g.err, WS_MMA_FULL);
                    s_fail = 1;
                    break;
                }
            }
            // keep TMEM alive until the last MMAs have landed
            if (commits > 0 && !mbar_wait(smem_u32(&bars[2 * STAGES]), (commits - 1) & 1)) {
                wait_failed(g.err, WS_MMA_ACC);
                s_fail = 1;
            }
        }
        __syncwarp();
    } else if (HALVES == 2 || warp < 6) {
        // ------------------------- epilogue -------------------------
        griddep_wait();
        constexpr int kEpiThreads = 32 * 4 * HALVES;
        for (int j = 1; j <= c.nl; ++j) {
            BatchParams q = p;
            q.flags = EPI_REFINE | (j == c.nl ? c.last_flags : 0u);
            q.Dhi = c.OP + (size_t)(2 * (j & 1)) * c.opart;
            q.Dlo = q.Dhi + c.opart;
            tile_epilogue<MODE_LAYER_REFINED, BN, KS>(q, g, warp, lane, rank, slot0, row0, ri, tmem, xpose, recv,
                                                      smem_u32(&bars[2 * STAGES]), (uint32_t)((j - 1) & 1),
                                                      smem_u32(&bars[2 * STAGES + 1]), (uint32_t)((j - 1) & 1),
                                                      &s_fail);
            // this warp has read all of layer j's accumulators
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars[2 * STAGES + 2]));
            // release this CTA's part of layer j: its operand and state stores, then
            // its TMEM reads, before the tile's counter moves on
            asm volatile("fence.proxy.async.global;" ::: "memory");
            fence_before();
            // barrier of the epilogue warps that also ORs their view of the failure
            // flag, so that all of them leave the loop together or none does
            const int mine = *(volatile int*)&s_fail;
            int any;
            asm volatile(
                "{\n .reg .pred pi, po;\n setp.ne.s32 pi, %1, 0;\n"
                " bar.red.or.pred po, 1, %2, pi;\n selp.s32 %0, 1, 0, po;\n}\n"
                : "=r"(any)
                : "r"(mine), "r"(kEpiThreads)
                : "memory");
            if (any) break;
            if (warp == 2 && lane == 0) {
                // this CTA's rows of layer j are stored (each epilogue thread fenced them for the
                // async proxy before the barrier above): its producer may load them
                if (j < c.nl) mbar_arrive(smem_u32(&bars[2 * STAGES + 3]));
                if (j < c.nl) {
                    // a release at GPU scope: it orders this CTA's stores of layer j (those of the
                    // other epilogue warps through the barrier above) before the counter's increment
                    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(c.sync + tile) : "memory");
                } else {
                    __threadfence();
                    // after the last layer nobody waits on the counter: the tile's last CTA
                    // to get here puts it (and the done count) back to zero for the next launch
                    const unsigned done = atomicAdd(c.sync + c.done_off + tile, 1u) + 1u;
                    if (done == nct) {
                        atomicExch(c.sync + tile, 0u);
                        atomicExch(c.sync + c.done_off + tile, 0u);
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (KS > 1) cluster_sync();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Resident-weight chunk kernel: the refined layers 1 .. nl of a chunk when a
// single slot tile holds at most NS active QPs (the middle and end of a
// batched solve, when few QPs are left).
//
// The roles of the operands are swapped: the MMA's M = 128 rows are rows of
// the layer Wt and its N = NS columns are the QP slots, so that a CTA's rows
// of Wt, over its k range, stay in shared memory for the whole chunk and each
// layer only loads the (small) operand of the slots.  A cluster of 8 CTAs
// shares a block of 128 rows and splits k into 8 ranges (<= 4 k-blocks each:
// w1 and w2 of 128 rows x 256 k are 128 KB); every CTA sends its partial sums
// of rows 16 r .. 16 r + 15 to rank r through distributed shared memory, and
// rank r adds the 8 partials in rank order and applies the element-wise layer
// (chunk4_apply) to its 16 rows x NS slots.  Layers are ordered by the tile's
// counter as in tc_chunk_kernel (release after the epilogue, acquire before
// the next operand load); every wait has a deadline.
// Warps: 0 TMA, 1 MMA (one lane), 2-5 epilogue (warp w reads TMEM lanes of
// quadrant w % 4).
// ---------------------------------------------------------------------------
constexpr int kSmallKS = 8;                          // K split over a cluster of 8 CTAs
constexpr int kSmallRows = 128;                      // rows of Wt per CTA (the MMA M dimension)
constexpr int kSmallMaxKb = 4;                       // k-blocks per CTA at most
constexpr int kSmallOwn = kSmallRows / kSmallKS;     // rows each CTA finalises
constexpr int kSmallThreads = 192;

template <int NS>
struct SmallSmem {
    static constexpr int kWPart = kSmallRows * 128;                 // one k-block of one weight part
    static constexpr int kOpPart = NS * 128;                        // one k-block of one operand part
    static constexpr int kW = 2 * kSmallMaxKb * kWPart;
    static constexpr int kOp = 2 * kSmallMaxKb * kOpPart;
    static constexpr int kRecv = kSmallKS * kSmallOwn * NS * 4;      // [sender][16 rows][NS slots] FP32
    static constexpr int kBytes = kW + kOp + kRecv + 1024 /* align */ + 256 /* barriers */;
};

// float offset of (row, slot) in one sender's [16 rows][NS] block of the
// receive buffer: the 16-byte chunk index is XORed with the row, so that the
// 16 rows a half-warp writes at one slot land in different banks
template <int NS>
__device__ __forceinline__ int small_off(int row, int slot) {
    constexpr int MASK = NS / 4 - 1;
    return row * NS + ((((slot >> 2) ^ (row & MASK))) << 2) + (slot & 3);
}

template <int NS>
__global__ void __launch_bounds__(kSmallThreads, 1)
    tc_small_kernel(const __grid_constant__ CUtensorMap tmA32, const __grid_constant__ CUtensorMap tmW,
                    BatchParams p, TcArgs g, ChunkArgs c) {
    static_assert(NS == 32 || NS == 64, "32 or 64 slots");
    using L = SmallSmem<NS>;
    constexpr int TCOLS = tmem_cols(2 * NS);
    if (cluster_size() != (uint32_t)kSmallKS) {
        if (threadIdx.x == 0) atomicExch(g.err, RELU_QP_ERR_CUDA);
        return;
    }
    const int tile = 0;                                 // the single active slot tile
    const int slot0 = 0;
    const int rank = (int)cluster_rank();
    const int row0 = (blockIdx.x / kSmallKS) * kSmallRows;
    const int ri = p.tile_rho[tile];
    const int kb_begin = rank * g.num_kb / kSmallKS;
    const int kb_count = (rank + 1) * g.num_kb / kSmallKS - kb_begin;
    const unsigned nct = gridDim.x;

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sW = smem;
    uint8_t* sOp = smem + L::kW;
    float* recv = reinterpret_cast<float*>(smem + L::kW + L::kOp);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kW + L::kOp + L::kRecv);
    // bars: 0 weights loaded, 1 operand loaded, 2 accumulators ready, 3 accumulators
    // consumed, 4 partials received; then the TMEM address and the failure flag
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 5);
    int& s_fail = *reinterpret_cast<int*>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        mbar_init(smem_u32(&bars[2]), 1);
        mbar_init(smem_u32(&bars[3]), 4);             // one arrival per epilogue warp
        mbar_init(smem_u32(&bars[4]), kSmallKS);      // one arrival per sender CTA
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    cluster_sync();        // every partner's barriers are initialised before anything is sent
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        // ------------------------- TMA producer -------------------------
        if (lane == 0) {
            prefetch_map(&tmA32);
            prefetch_map(&tmW);
            // the weight slice, once: parts w1, w2 of rows row0 .. row0 + 127, this CTA's k-blocks
            const uint32_t wfull = smem_u32(&bars[0]);
            mbar_expect_tx(wfull, (uint32_t)(2 * kb_count * L::kWPart));
            for (int b = 0; b < kb_count; ++b)
                for (int part = 0; part < 2; ++part)
                    tma_load_2d(smem_u32(sW + (part * kSmallMaxKb + b) * L::kWPart), &tmW,
                                (kb_begin + b) * kBK, g.b_row[part] + ri * g.b_rho_stride + row0, wfull);
            const uint32_t opfull = smem_u32(&bars[1]);
            int loads = 0;
            for (int j = 1; j <= c.nl; ++j) {
                if (*(volatile int*)&s_fail) break;
                if (j > 1) {
                    // every CTA of the tile is done with layer j - 1 (which also means this
                    // CTA's MMAs of layer j - 1 have read the operand buffer)
                    if (!wait_counter_geq(c.sync + tile, (unsigned)(j - 1) * nct, kWaitNs)) {
                        wait_failed(g.err, WS_PROD_SYNC);
                        s_fail = 1;
                        break;
                    }
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
                const int a0 = 2 * ((j - 1) & 1) * c.slots + slot0;
                mbar_expect_tx(opfull, (uint32_t)(2 * kb_count * ((c.ncols + 31) / 32) * 4096));
                for (int b = 0; b < kb_count; ++b)
                    for (int part = 0; part < 2; ++part)
                        for (int gr = 0; gr < (c.ncols + 31) / 32; ++gr)
                            tma_load_2d(smem_u32(sOp + (part * kSmallMaxKb + b) * L::kOpPart + gr * 4096), &tmA32,
                                        (kb_begin + b) * kBK, a0 + part * c.slots + 32 * gr, opfull);
                ++loads;
            }
            // the copies in flight land before the CTA may exit (bounded waits)
            if (loads > 0) mbar_wait(opfull, (uint32_t)((loads - 1) & 1));
            mbar_wait(wfull, 0);
        }
    } else if (warp == 1) {
        // ------------------------- MMA issuer -------------------------
        if (lane == 0) {
            const uint32_t IDESC = idesc_bf16(c.ncols);
            int commits = 0;
            bool ok = mbar_wait(smem_u32(&bars[0]), 0);
            if (!ok) {
                wait_failed(g.err, WS_MMA_FULL);
                s_fail = 1;
            }
            for (int j = 1; ok && j <= c.nl; ++j) {
                if (*(volatile int*)&s_fail) break;
                if (j > 1 && !mbar_wait(smem_u32(&bars[3]), (uint32_t)((j - 2) & 1))) {
                    wait_failed(g.err, WS_MMA_ACC);
                    s_fail = 1;
                    break;
                }
                if (!mbar_wait(smem_u32(&bars[1]), (uint32_t)((j - 1) & 1))) {
                    wait_failed(g.err, WS_MMA_FULL);
                    s_fail = 1;
                    break;
                }
                fence_after();
                const uint64_t dw = sdesc(smem_u32(sW)), dop = sdesc(smem_u32(sOp));
                for (int b = 0; b < kb_count; ++b) {
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
                        for (int pr = 0; pr < 3; ++pr) {
                            // (w1, d_hi) -> accumulator 0; (w2, d_hi), (w1, d_lo) -> accumulator 1
                            const int iw = pr == 1 ? 1 : 0, io = pr == 2 ? 1 : 0;
                            const uint64_t ad = dw + (uint64_t)(((iw * kSmallMaxKb + b) * L::kWPart + kk * 32) >> 4);
                            const uint64_t bd = dop + (uint64_t)(((io * kSmallMaxKb + b) * L::kOpPart + kk * 32) >> 4);
                            const bool first = b == 0 && kk == 0 && pr <= 1;
                            mma_bf16(tmem + (pr == 0 ? 0 : NS), ad, bd, IDESC, first ? 0u : 1u);
                        }
                    }
                }
                mma_commit(smem_u32(&bars[2]));
                ++commits;
            }
            if (commits > 0 && !mbar_wait(smem_u32(&bars[2]), (uint32_t)((commits - 1) & 1))) {
                wait_failed(g.err, WS_MMA_ACC);
                s_fail = 1;
            }
        }
        __syncwarp();
    } else {
        // ------------------------- epilogue (warps 2-5) -------------------------
        const int q = warp & 3;                       // TMEM lane quadrant: rows 32 q .. 32 q + 31
        const int et = (warp - 2) * 32 + lane;        // 0 .. 127
        // the element this thread finalises: slot es, rows fr0 .. fr0 + 7 of the block
        const int es = et >> 1;
        const int fr = rank * kSmallOwn + (et & 1) * 8;          // row within the 128-row block
        const int fr0 = row0 + fr;
        const bool mine = es < c.ncols;
        const int eqp = mine ? p.perm[slot0 + es] : -1;
        const bool n_aligned = (p.n & 3) == 0;
        auto whole4 = [&](int r0) { return r0 + 4 <= g.rows && (r0 + 4 <= p.n || (r0 >= p.n && n_aligned)); };
        // sender side: lane = row 32 q + lane of the block; rows 16 o .. 16 o + 15 go to rank o
        const int srow = q * 32 + lane;
        const int owner = srow / kSmallOwn;
        const uint32_t recv_remote = mapa(smem_u32(recv), (uint32_t)owner);
        for (int j = 1; j <= c.nl; ++j) {
            BatchParams pj = p;
            pj.flags = EPI_REFINE | (j == c.nl ? c.last_flags : 0u);
            pj.Dhi = c.OP + (size_t)(2 * (j & 1)) * c.opart;
            pj.Dlo = pj.Dhi + c.opart;
            // this thread's inputs load while the MMAs run
            Chunk4R in[2];
            if (eqp >= 0) {
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2)
                    if (whole4(fr0 + 4 * h2)) chunk4_load(pj, eqp, ri, fr0 + 4 * h2, in[h2]);
            }
            // the accumulators of layer j
            bool ready = true;
            if (lane == 0) ready = mbar_wait_sleep(smem_u32(&bars[2]), (uint32_t)((j - 1) & 1), 128);
            ready = __shfl_sync(0xffffffffu, ready, 0);
            if (ready) ready = mbar_wait(smem_u32(&bars[2]), (uint32_t)((j - 1) & 1));
            ready = __all_sync(0xffffffffu, ready);
            if (ready) {
                fence_after();
                const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
                // partial sums of this CTA's k range for row srow, all NS slots -> rank owner,
                // into its receive slot `rank` at row srow % 16
                const uint32_t dst = recv_remote + 4u * (uint32_t)(rank * kSmallOwn * NS);
                const int rw = srow % kSmallOwn;
                for (int c0 = 0; c0 < c.ncols; c0 += 16) {
                    float v[16], w[16];
                    tmem_ld16x2(tl + c0, tl + NS + c0, v, w);
#pragma unroll
                    for (int t = 0; t < 16; t += 4)
                        st_cluster4(dst + 4u * (uint32_t)small_off<NS>(rw, c0 + t), v[t] + w[t], v[t + 1] + w[t + 1],
                                    v[t + 2] + w[t + 2], v[t + 3] + w[t + 3]);
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars[3]));          // this warp's TMEM reads are done
            // lanes 0 and 16 announce their half-warp's rows to the two owners
            if ((lane & 15) == 0) mbar_arrive_cluster(mapa(smem_u32(&bars[4]), (uint32_t)owner));
            bool got = ready;
            if (got) {
                if (lane == 0) got = mbar_wait_cluster(smem_u32(&bars[4]), (uint32_t)((j - 1) & 1), 64);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (got) got = mbar_wait_cluster(smem_u32(&bars[4]), (uint32_t)((j - 1) & 1), 0);
                got = __all_sync(0xffffffffu, got);
            }
            if (!ready || !got) {
                if (lane == 0) {
                    wait_failed(g.err, ready ? WS_EPI_RECV : WS_EPI_ACC);
                    s_fail = 1;
                }
            } else if (eqp >= 0) {
                // the 8 partials of rows fr .. fr + 7, slot es, added in rank order
                float acc[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float tsum = 0.f;
#pragma unroll
                    for (int k = 0; k < kSmallKS; ++k) {
                        const float v = recv[k * kSmallOwn * NS + small_off<NS>((fr - rank * kSmallOwn) + i, es)];
                        tsum = k == 0 ? v : tsum + v;
                    }
                    acc[i] = tsum;
                }
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int r0 = fr0 + 4 * h2;
                    if (whole4(r0)) {
                        float rs4[4] = {1.f, 1.f, 1.f, 1.f};
                        if (r0 >= p.n) ld4(p.rs + (r0 - p.n), rs4);
                        const float a4[4] = {acc[4 * h2], acc[4 * h2 + 1], acc[4 * h2 + 2], acc[4 * h2 + 3]};
                        chunk4_apply(pj, slot0 + es, eqp, ri, r0, a4, in[h2], rs4);
                    } else {
                        for (int t = 0; t < 4; ++t)
                            if (r0 + t < g.rows) layer_elem(pj, slot0 + es, eqp, ri, r0 + t, acc[4 * h2 + t]);
                    }
                }
            }
            // release this CTA's part of layer j (operand and state stores) before the
            // tile's counter moves on; the epilogue warps leave the loop together
            asm volatile("fence.proxy.async.global;" ::: "memory");
            fence_before();
            const int mine_fail = *(volatile int*)&s_fail;
            int any;
            asm volatile(
                "{\n .reg .pred pi, po;\n setp.ne.s32 pi, %1, 0;\n"
                " bar.red.or.pred po, 1, %2, pi;\n selp.s32 %0, 1, 0, po;\n}\n"
                : "=r"(any)
                : "r"(mine_fail), "r"(128)
                : "memory");
            if (any) break;
            if (warp == 2 && lane == 0) {
                if (j < c.nl) {
                    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(c.sync + tile) : "memory");
                } else {
                    __threadfence();
                    const unsigned done = atomicAdd(c.sync + c.done_off + tile, 1u) + 1u;
                    if (done == nct) {
                        atomicExch(c.sync + tile, 0u);
                        atomicExch(c.sync + c.done_off + tile, 0u);
                    }
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    cluster_sync();        // no CTA leaves while a partner may still write into its shared memory
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Deadline diagnostics: the waits above, made to run out on purpose.  kind 0:
// an mbarrier that nothing arrives on (mbar_wait_ns); kind 1: a layer counter
// that nothing increments (wait_counter_geq).  The waiting thread gives up at
// its deadline and records RELU_QP_ERR_TIMEOUT in err[0] (err[1] = the kind +
// 1), as the kernels above do; nothing faults or hangs.
// ---------------------------------------------------------------------------
__global__ void tc_diag_wait_kernel(int kind, const unsigned* ctr, int* err, long long ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const bool ok = kind == 0 ? mbar_wait_ns(smem_u32(&bar), 0, ns) : wait_counter_geq(ctr, 1u, ns);
    if (!ok) {
        atomicCAS(err + 1, 0, kind + 1);
        atomicExch(err, RELU_QP_ERR_TIMEOUT);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// tile widths (rows of Wt per CTA) of the refined layer; the 3-part modes use 64
constexpr int kLayerBN[] = {16, 32, 64, 96, 128, 160, 192, 256};
constexpr int kNumLayerBN = sizeof(kLayerBN) / sizeof(int);

int bn_index(int bn) {
    for (int i = 0; i < kNumLayerBN; ++i)
        if (kLayerBN[i] == bn) return i;
    return -1;
}

struct TcState {
    EncodeTiledFn encode = nullptr;
    LayerCfg cfg{1, 128};                // refined layer: K split and width when no table is set
    std::vector<LayerCfg> cfg_by_tiles;  // [t] = the tuned configuration for t active slot tiles
    bool chunk_ok = true;                // persistent chunk kernel usable (cleared after a refused launch)
    bool small_ok = true;                // resident-weight chunk kernel usable (cleared after a refused launch)
    bool small_use = false;              // the tuner found it faster for one slot tile of few QPs
    int small_clusters = -1;             // clusters of it that fit co-resident (-1: not asked yet)
    int* err = nullptr;                  // = counters + CNT_ERR
    // encoded maps, keyed by box rows
    CUtensorMap opnd_map[2], ck_map[2];  // operand tensors, boxes of 128 and of 32 slot rows
    CUtensorMap wb_map[kNumLayerBN];     // weights, box rows kLayerBN[i]
    CUtensorMap wcb_map[3];              // check matrix, box rows 64, 128 and 96
};

int encode_2d(relu_qp_t h, TcState* st, CUtensorMap* map, void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {kBK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = st->encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, RELU_QP_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return RELU_QP_OK;
}

template <int MODE, int BN, int KS>
constexpr int stages_for() {
    using L1 = TcSmem<MODE == MODE_LAYER_REFINED ? 2 : 3, MODE == MODE_LAYER_REFINED ? 2 : 3, BN, 1, KS>;
    constexpr int budget = 227 * 1024 - 512;   // opt-in maximum less the static shared memory
    constexpr int s = (budget - 1024 - 256 - L1::kXpose - L1::kRecv - L1::kDrain) / L1::kStage;
    return s > 4 ? 4 : s;
}

// pdl: launch with programmatic stream serialisation, so that this kernel's
// set-up and first weight loads overlap the end of the previous kernel in the
// stream (the kernel waits for that kernel's results before it touches them)
template <int MODE, int BN, int KS>
int launch_tc(relu_qp_t h, const CUtensorMap* a, const CUtensorMap& b, const BatchParams& p, const TcArgs& g,
              int tiles, bool pdl) {
    constexpr int S = stages_for<MODE, BN, KS>();
    static_assert(S >= 2, "not enough shared memory for two stages");
    using L = TcSmem<MODE == MODE_LAYER_REFINED ? 2 : 3, MODE == MODE_LAYER_REFINED ? 2 : 3, BN, S, KS>;
    auto kern = tc_gemm_kernel<MODE, BN, S, KS>;
    RQ_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes));
    const dim3 grid(KS * ceil_div(g.rows, BN), tiles);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreadsTC);
    cfg.dynamicSmemBytes = L::kBytes;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (KS > 1) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = KS;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    if (pdl) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    RQ_CUDA(h, cudaLaunchKernelEx(&cfg, kern, a[0], a[1], b, p, g));
    return RELU_QP_OK;
}

template <int BN, int KS>
int launch_chunk(relu_qp_t h, const CUtensorMap* a, const CUtensorMap& b, const BatchParams& p, const TcArgs& g,
                 const ChunkArgs& c, int tiles_y) {
    constexpr int S = stages_for<MODE_LAYER_REFINED, BN, KS>();
    using L = TcSmem<2, 2, BN, S, KS>;
    auto kern = tc_chunk_kernel<BN, S, KS>;
    RQ_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(KS * ceil_div(g.rows, BN), tiles_y);
    cfg.blockDim = dim3(kThreadsTC);
    cfg.dynamicSmemBytes = L::kBytes;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    int na = 0;
    if (KS > 1) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = KS;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    // no programmatic dependent launch: the layer counters must be at zero (stream
    // order after the previous launch and the host's reset) before any CTA starts
    cfg.attrs = attr;
    cfg.numAttrs = na;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a[0], a[1], b, p, g, c);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RELU_QP_ERR_UNSUPPORTED;     // the caller falls back to one launch per layer
    }
    return RELU_QP_OK;
}

// (K split, width) pairs the persistent chunk kernel is built for
bool chunk_has(int ks, int bn) {
    if (ks == 4) return bn == 64 || bn == 128;
    if (ks == 2) return bn == 64 || bn == 128 || bn == 192;
    return ks == 1 && (bn == 16 || bn == 32 || bn == 64 || bn == 96 || bn == 128);
}

int dispatch_chunk(relu_qp_t h, int bn, int ks, const CUtensorMap* wmaps, const BatchParams& p, const TcArgs& g,
                   const CUtensorMap* a, const ChunkArgs& c, int tiles_y) {
    if (ks == 4) {
        switch (bn) {
            case 64: return launch_chunk<64, 4>(h, a, wmaps[2], p, g, c, tiles_y);
            case 128: return launch_chunk<128, 4>(h, a, wmaps[4], p, g, c, tiles_y);
        }
    } else if (ks == 2) {
        switch (bn) {
            case 64: return launch_chunk<64, 2>(h, a, wmaps[2], p, g, c, tiles_y);
            case 128: return launch_chunk<128, 2>(h, a, wmaps[4], p, g, c, tiles_y);
            case 192: return launch_chunk<192, 2>(h, a, wmaps[6], p, g, c, tiles_y);
        }
    } else {
        switch (bn) {
            case 16: return launch_chunk<16, 1>(h, a, wmaps[0], p, g, c, tiles_y);
            case 32: return launch_chunk<32, 1>(h, a, wmaps[1], p, g, c, tiles_y);
            case 64: return launch_chunk<64, 1>(h, a, wmaps[2], p, g, c, tiles_y);
            case 96: return launch_chunk<96, 1>(h, a, wmaps[3], p, g, c, tiles_y);
            case 128: return launch_chunk<128, 1>(h, a, wmaps[4], p, g, c, tiles_y);
        }
    }
    return RELU_QP_ERR_UNSUPPORTED;
}

template <int NS>
int launch_small(relu_qp_t h, const CUtensorMap& a32, const CUtensorMap& w128, const BatchParams& p,
                 const TcArgs& g, const ChunkArgs& c) {
    using L = SmallSmem<NS>;
    auto kern = tc_small_kernel<NS>;
    RQ_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(kSmallKS * ceil_div(g.rows, kSmallRows), 1);
    cfg.blockDim = dim3(kSmallThreads);
    cfg.dynamicSmemBytes = L::kBytes;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kSmallKS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a32, w128, p, g, c);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RELU_QP_ERR_UNSUPPORTED;     // the caller uses the other chunk kernel
    }
    return RELU_QP_OK;
}

// Refined layer widths by K split: KS = 4 takes 64 and 128 (each CTA
// finalises 16 or 32 columns; wider tiles leave no room for the three receive
// buffers), KS = 2 takes 64, 128 and 192 (BN = 256 would not leave room for
// the receive buffer), KS = 1 any width of kLayerBN (BN / 2 columns per warp).
int dispatch_refined(relu_qp_t h, int bn, int ks, const CUtensorMap* wmaps, const BatchParams& p, const TcArgs& g,
                     const CUtensorMap* a, int tiles, bool pdl) {
    constexpr int M = MODE_LAYER_REFINED;
    if (ks == 4) {
        switch (bn) {
            case 64: return launch_tc<M, 64, 4>(h, a, wmaps[2], p, g, tiles, pdl);
            case 128: return launch_tc<M, 128, 4>(h, a, wmaps[4], p, g, tiles, pdl);
            default: return fail(h, RELU_QP_ERR_INVALID, "unsupported tile width " + std::to_string(bn));
        }
    }
    if (ks == 2) {
        switch (bn) {
            case 64: return launch_tc<M, 64, 2>(h, a, wmaps[2], p, g, tiles, pdl);
            case 128: return launch_tc<M, 128, 2>(h, a, wmaps[4], p, g, tiles, pdl);
            case 192: return launch_tc<M, 192, 2>(h, a, wmaps[6], p, g, tiles, pdl);
            default: return fail(h, RELU_QP_ERR_INVALID, "unsupported tile width " + std::to_string(bn));
        }
    }
    switch (bn) {
        case 16: return launch_tc<M, 16, 1>(h, a, wmaps[0], p, g, tiles, pdl);
        case 32: return launch_tc<M, 32, 1>(h, a, wmaps[1], p, g, tiles, pdl);
        case 64: return launch_tc<M, 64, 1>(h, a, wmaps[2], p, g, tiles, pdl);
        case 96: return launch_tc<M, 96, 1>(h, a, wmaps[3], p, g, tiles, pdl);
        case 128: return launch_tc<M, 128, 1>(h, a, wmaps[4], p, g, tiles, pdl);
        case 160: return launch_tc<M, 160, 1>(h, a, wmaps[5], p, g, tiles, pdl);
        case 192: return launch_tc<M, 192, 1>(h, a, wmaps[6], p, g, tiles, pdl);
        case 256: return launch_tc<M, 256, 1>(h, a, wmaps[7], p, g, tiles, pdl);
        default: return fail(h, RELU_QP_ERR_INVALID, "unsupported tile width " + std::to_string(bn));
    }
}

// 3-part modes: b64 / b96 are the weight maps with 64- and 96-row boxes.  The
// drained accumulation keeps FP32 sums of BN / 2 columns per epilogue warp in
// shared memory, which leaves room for two pipeline stages at BN = 64 or 96.
// BN = 96 when it turns two waves of CTAs over the active slot tiles into one
// (the full batch: 25 row blocks of 64 x 8 tiles = 200 CTAs, of 96: 136); the
// tile width does not change any output's arithmetic (the k order is fixed).
template <int MODE>
int dispatch_3part(relu_qp_t h, int active_tiles, const CUtensorMap& b64, const CUtensorMap& b96,
                   const BatchParams& p, const TcArgs& g, const CUtensorMap* a, int tiles) {
    const long long w64 = (long long)ceil_div(g.rows, 64) * active_tiles;
    const long long w96 = (long long)ceil_div(g.rows, 96) * active_tiles;
    // few active tiles: the k-blocks of every tile split over a cluster of 4 or 2 CTAs
    // (at least 2 k-blocks each) while the CTAs still fit one wave
    if (4 * w64 <= h->num_sms && g.num_kb >= 8) return launch_tc<MODE, 64, 4>(h, a, b64, p, g, tiles, false);
    if (2 * w64 <= h->num_sms && g.num_kb >= 4) return launch_tc<MODE, 64, 2>(h, a, b64, p, g, tiles, false);
    if (w64 > h->num_sms && w96 <= h->num_sms) return launch_tc<MODE, 96, 1>(h, a, b96, p, g, tiles, false);
    return launch_tc<MODE, 64, 1>(h, a, b64, p, g, tiles, false);
}

}  // namespace

int tc_prepare(relu_qp_t h) {
    BatchWork& w = h->bw;
    TcState* st = new (std::nothrow) TcState();
    if (!st) return fail(h, RELU_QP_ERR_OOM, "host allocation failed");
    w.tc = st;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    RQ_CUDA(h, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (!fn || q != cudaDriverEntryPointSuccess)
        return fail(h, RELU_QP_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
    st->encode = reinterpret_cast<EncodeTiledFn>(fn);
    st->err = w.counters + CNT_ERR;
    st->cfg = LayerCfg{w.ldk / kBK >= 4 ? 2 : 1, w.ldk / kBK >= 4 ? 128 : 64};
    for (int i = 0; i < 2; ++i) {
        RQ_TRY(encode_2d(h, st, &st->opnd_map[i], w.OPND, 7ull * w.slots, w.ldk, i == 0 ? kSlotTile : 32));
        RQ_TRY(encode_2d(h, st, &st->ck_map[i], w.CK, 3ull * w.slots, w.ldkc, i == 0 ? kSlotTile : 32));
    }
    for (int i = 0; i < kNumLayerBN; ++i)
        RQ_TRY(encode_2d(h, st, &st->wb_map[i], w.WB, (uint64_t)h->nr * 3 * w.Rpad, w.ldk, kLayerBN[i]));
    for (int i = 0; i < 3; ++i)
        RQ_TRY(encode_2d(h, st, &st->wcb_map[i], w.WCB, 3ull * w.npad, w.ldkc, i == 2 ? 96 : 64 << i));
    return RELU_QP_OK;
}

void tc_release(relu_qp_t h) {
    delete static_cast<TcState*>(h->bw.tc);
    h->bw.tc = nullptr;
}

// (K split, width) pairs of the refined layer: a split needs two k-blocks per rank;
// KS = 4 takes widths 64 and 128 (each CTA finalises 16 or 32 columns, and wider
// tiles leave no room for the receive buffers), KS = 2 takes 64, 128 and 192, no
// split any width of kLayerBN
bool cfg_ok(relu_qp_t h, LayerCfg c) {
    const int nkb = h->bw.ldk / kBK;
    if (c.ks == 4) return nkb >= 8 && (c.bn == 64 || c.bn == 128);
    if (c.ks == 2) return nkb >= 4 && (c.bn == 64 || c.bn == 128 || c.bn == 192);
    return c.ks == 1 && bn_index(c.bn) >= 0;
}

int tc_layer_cfgs(relu_qp_t h, std::vector<LayerCfg>& out) {
    out.clear();
    for (int ks : {1, 2, 4})
        for (int i = 0; i < kNumLayerBN; ++i)
            if (cfg_ok(h, LayerCfg{ks, kLayerBN[i]})) out.push_back(LayerCfg{ks, kLayerBN[i]});
    return (int)out.size();
}

int tc_set_layer_cfg(relu_qp_t h, LayerCfg c) {
    TcState* st = static_cast<TcState*>(h->bw.tc);
    if (!cfg_ok(h, c)) return fail(h, RELU_QP_ERR_INVALID, "unsupported refined-layer configuration");
    st->cfg = c;
    st->cfg_by_tiles.clear();
    return RELU_QP_OK;
}

int tc_set_layer_table(relu_qp_t h, const std::vector<LayerCfg>& by_tiles) {
    TcState* st = static_cast<TcState*>(h->bw.tc);
    for (size_t t = 1; t < by_tiles.size(); ++t)
        if (!cfg_ok(h, by_tiles[t])) return fail(h, RELU_QP_ERR_INVALID, "unsupported refined-layer configuration");
    st->cfg_by_tiles = by_tiles;
    return RELU_QP_OK;
}

LayerCfg cfg_for(const TcState* st, int active_tiles) {
    if (st->cfg_by_tiles.empty()) return st->cfg;
    return st->cfg_by_tiles[std::max(1, std::min<int>(active_tiles, (int)st->cfg_by_tiles.size() - 1))];
}

int tc_layer(relu_qp_t h, const BatchParams& p, int operand_set, int tiles, int active_tiles, bool pdl) {
    BatchWork& w = h->bw;
    TcState* st = static_cast<TcState*>(w.tc);
    TcArgs g{};
    g.num_kb = w.ldk / kBK;
    g.rows = h->R;
    g.err = st->err;
    g.b_rho_stride = 3 * w.Rpad;
    for (int b = 0; b < 3; ++b) g.b_row[b] = b * w.Rpad;
    if (operand_set < 0) {   // accurate: s1, s2, s3 are parts 4..6
        for (int a = 0; a < 3; ++a) g.a_row[a] = (4 + a) * w.slots;
        return dispatch_3part<MODE_LAYER_ACCURATE>(h, active_tiles, st->wb_map[2], st->wb_map[3], p, g,
                                                   st->opnd_map, tiles);
    }
    // the configuration tuned for this many active slot tiles
    const LayerCfg c = cfg_for(st, active_tiles);
    g.a_row[0] = (2 * operand_set) * w.slots;
    g.a_row[1] = (2 * operand_set + 1) * w.slots;
    return dispatch_refined(h, c.bn, c.ks, st->wb_map, p, g, st->opnd_map, tiles, pdl);
}

int tc_chunk(relu_qp_t h, const BatchParams& p, int nl, unsigned last_flags, int active_tiles) {
    BatchWork& w = h->bw;
    TcState* st = static_cast<TcState*>(w.tc);
    if (!st->chunk_ok || nl < 1 || active_tiles < 1) return RELU_QP_ERR_UNSUPPORTED;
    const LayerCfg lc = cfg_for(st, active_tiles);
    const int bn = lc.bn;
    if (!chunk_has(lc.ks, bn)) return RELU_QP_ERR_UNSUPPORTED;
    const int tiles_y = std::min(active_tiles, w.slots / kSlotTile);
    // all CTAs of the active tiles co-resident, one per SM
    if ((long long)lc.ks * ceil_div(h->R, bn) * tiles_y > h->num_sms) return RELU_QP_ERR_UNSUPPORTED;
    TcArgs g{};
    g.num_kb = w.ldk / kBK;
    g.rows = h->R;
    g.err = st->err;
    g.b_rho_stride = 3 * w.Rpad;
    for (int b = 0; b < 3; ++b) g.b_row[b] = b * w.Rpad;
    ChunkArgs c{};
    c.nl = nl;
    c.last_flags = last_flags;
    c.OP = static_cast<__nv_bfloat16*>(w.OPND);
    c.opart = (size_t)w.slots * w.ldk;
    c.slots = w.slots;
    c.sync = w.chunk_sync;
    c.done_off = w.slots / kSlotTile;
    const int rc = dispatch_chunk(h, bn, lc.ks, st->wb_map, p, g, st->opnd_map, c, tiles_y);
    if (rc == RELU_QP_ERR_UNSUPPORTED) st->chunk_ok = false;   // launch refused: not again for this handle
    return rc;
}

void tc_disable_chunk(relu_qp_t h) { static_cast<TcState*>(h->bw.tc)->chunk_ok = false; }

// Clusters of the resident-weight kernel (its larger instantiation) that the
// GPU can hold at once; every CTA of a launch must be co-resident, since the
// layers are ordered by a counter the CTAs wait on.
int small_clusters_fit(relu_qp_t h) {
    auto kern = tc_small_kernel<64>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SmallSmem<64>::kBytes) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(kSmallKS * ceil_div(h->R, kSmallRows), 1);
    cfg.blockDim = dim3(kSmallThreads);
    cfg.dynamicSmemBytes = SmallSmem<64>::kBytes;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kSmallKS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void*)kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

bool tc_small_eligible(relu_qp_t h, int active, int active_tiles) {
    const BatchWork& w = h->bw;
    TcState* st = static_cast<TcState*>(w.tc);
    if (!st || !st->small_ok || !w.chunk_sync || active_tiles != 1 || active < 1 || active > 64) return false;
    const int nkb = w.ldk / kBK;
    if (ceil_div(nkb, kSmallKS) > kSmallMaxKb || nkb < kSmallKS) return false;
    if ((long long)kSmallKS * ceil_div(h->R, kSmallRows) > h->num_sms) return false;
    if (st->small_clusters < 0) st->small_clusters = small_clusters_fit(h);
    return st->small_clusters >= ceil_div(h->R, kSmallRows);
}

void tc_small_set(relu_qp_t h, bool use) { static_cast<TcState*>(h->bw.tc)->small_use = use; }
bool tc_small_chosen(relu_qp_t h) { return static_cast<const TcState*>(h->bw.tc)->small_use; }

int tc_small(relu_qp_t h, const BatchParams& p, int nl, unsigned last_flags, int active, int active_tiles) {
    BatchWork& w = h->bw;
    TcState* st = static_cast<TcState*>(w.tc);
    if (nl < 1 || !tc_small_eligible(h, active, active_tiles)) return RELU_QP_ERR_UNSUPPORTED;
    TcArgs g{};
    g.num_kb = w.ldk / kBK;
    g.rows = h->R;
    g.err = st->err;
    g.b_rho_stride = 3 * w.Rpad;
    for (int b = 0; b < 3; ++b) g.b_row[b] = b * w.Rpad;
    ChunkArgs c{};
    c.nl = nl;
    c.last_flags = last_flags;
    c.OP = static_cast<__nv_bfloat16*>(w.OPND);
    c.opart = (size_t)w.slots * w.ldk;
    c.slots = w.slots;
    c.sync = w.chunk_sync;
    c.done_off = w.slots / kSlotTile;
    c.ncols = std::max(16, (active + 15) / 16 * 16);   // the MMA's N covers the active slots
    const int rc = active <= 32 ? launch_small<32>(h, st->opnd_map[1], st->wb_map[4], p, g, c)
                                : launch_small<64>(h, st->opnd_map[1], st->wb_map[4], p, g, c);
    if (rc == RELU_QP_ERR_UNSUPPORTED) st->small_ok = false;   // launch refused: not again for this handle
    return rc;
}

int tc_check(relu_qp_t h, const BatchParams& p, int phase, int tiles, int active_tiles) {
    BatchWork& w = h->bw;
    TcState* st = static_cast<TcState*>(w.tc);
    TcArgs g{};
    g.num_kb = (phase == 1 ? w.n64 : w.m64) / kBK;
    g.k_off = phase == 1 ? 0 : w.n64;
    g.rows = phase == 1 ? h->n + h->m : h->n;
    g.err = st->err;
    g.b_rho_stride = 0;
    for (int a = 0; a < 3; ++a) {
        g.a_row[a] = a * w.slots;
        g.b_row[a] = a * w.npad;
    }
    if (phase == 1)
        return dispatch_3part<MODE_CHECK1>(h, active_tiles, st->wcb_map[0], st->wcb_map[2], p, g, st->ck_map, tiles);
    return dispatch_3part<MODE_CHECK2>(h, active_tiles, st->wcb_map[0], st->wcb_map[2], p, g, st->ck_map, tiles);
}

// Launch tc_diag_wait_kernel on `stream` with the words at dev (>= 4 ints,
// zeroed by the caller); the caller synchronises and reads err = dev[0..1].
int tc_diag_wait(int kind, int* dev, long long ns, cudaStream_t stream) {
    tc_diag_wait_kernel<<<1, 32, 0, stream>>>(kind, reinterpret_cast<const unsigned*>(dev + 2), dev, ns);
    return cudaGetLastError() == cudaSuccess ? RELU_QP_OK : RELU_QP_ERR_CUDA;
}

int tc_error(relu_qp_t h, int* site) {
    TcState* st = static_cast<TcState*>(h->bw.tc);
    if (!st) return 0;
    int e[2] = {0, 0};
    cudaMemcpy(e, st->err, sizeof(e), cudaMemcpyDeviceToHost);
    if (e[0]) cudaMemset(st->err, 0, sizeof(e));
    if (site) *site = e[1];
    return e[0];
}

}  // namespace rq
