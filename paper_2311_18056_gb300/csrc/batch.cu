// Batched online stage of Algorithm 1: B QPs sharing P and A (so every W_rho
// of the bank) with their own q, l, u, warm start and penalty index.
//
// One chunk = check_interval layers (25 by default, Sec. III-C).  Every layer
// is one GEMM over the active slots with the element-wise layer in its
// epilogue (batch.h).  At the end of a chunk the residuals of Eqs. primal and
// dual are formed per QP, the decision kernel applies the stop test and the
// penalty rule of Eq. rho_update (nearest bank entry, Sec. III-C), converged
// QPs leave the batch, and the rest are regrouped so that a 128-slot tile
// holds QPs of one bank entry only.  The host reads one counter per chunk.
//
// Backends: FP32 on the CUDA cores (this file) and BF16 hi+lo split operands
// on the tcgen05 tensor cores (batch_tc.cu) with FP32 accumulation.  In the
// split form the first layer of a chunk is an accurate (3-way split) product
// that stores c = Wt s_ref + b, and the other layers apply the 2-way split
// only to the increment: t = c + Wt (s - s_ref).
#include "batch.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <thread>
#include <new>

namespace rq {

namespace {

inline int __float_as_int_host(float f) {
    int i;
    std::memcpy(&i, &f, sizeof(i));
    return i;
}

struct W32Ptrs {
    const float* w[RQ_MAX_RHO];
};

// C[i][j] = alpha * sum_k X[i][k] W[j][k] + (off ? off[j] : 0), bounds-checked
// (problem updates; not on the per-layer path).
__global__ void __launch_bounds__(256) sgemm_nt_kernel(int M, int N, int K, const float* __restrict__ X, int ldx,
                                                       const float* __restrict__ W, int ldw, float alpha,
                                                       const float* __restrict__ off, float* __restrict__ C,
                                                       int ldc) {
    __shared__ float Xs[16][64 + 4];
    __shared__ float Ws[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            const int row = e >> 4, k = e & 15;
            const int gi = i0 + row, gj = j0 + row, gk = k0 + k;
            Xs[k][row] = (gi < M && gk < K) ? X[(size_t)gi * ldx + gk] : 0.f;
            Ws[k][row] = (gj < N && gk < K) ? W[(size_t)gj * ldw + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                a[t] = Xs[k][ty + 16 * t];
                b[t] = Ws[k][tx + 16 * t];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + ty + 16 * u;
        if (i >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int j = j0 + tx + 16 * v;
            if (j >= N) continue;
            C[(size_t)i * ldc + j] = alpha * acc[u][v] + (off ? off[j] : 0.f);
        }
    }
}

// Shared main loop of the FP32 batched kernels: a TS-slot x TR-row tile of
// sum_k X[slot, k] W[row, k] over k in [kbeg, kend) (rows of X and W have
// leading dimension ld, zero padded to a multiple of 64).  256 threads: thread
// (ty, tx) = (tid / 16, tid % 16) accumulates slots ty + 16 i (i < TS / 16) and
// rows tx + 16 j (j < TR / 16).  Every 16-wide k step is summed, in k order,
// into a fresh partial that is then added to the running sum: with
// multipliers of ~1e3 the terms of these dot products cancel heavily, and one
// long sequential FP32 sum would lose ~sqrt(K) units in the last place of its
// largest partial sum (measured: dual residuals off by 1e-3 on the humanoid
// workload).  The arithmetic of an output does not depend on TS or TR.
// k tiles stream through a STAGES-deep cp.async pipeline into shared memory
// laid out [slot or row][k] with a padded stride, so that the copies run
// ahead of the arithmetic by STAGES - 1 steps.
template <int TS, int TR>
struct F32Tile {
    static constexpr int SA = TS / 16, RA = TR / 16;
    static constexpr int LDS = 20;           // padded k stride in floats (80 bytes, 16-byte aligned)
    static constexpr int STAGES = 4;
    static constexpr int XS = TS * LDS, WS = TR * LDS;
    static constexpr int BYTES = STAGES * (XS + WS) * 4;
};

__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool valid) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int TS, int TR>
__device__ __forceinline__ void fp32_tile(const float* __restrict__ X, const float* __restrict__ W, int ld,
                                          int kbeg, int kend, int nrows, int slot0, int row0,
                                          float (&acc)[TS / 16][TR / 16]) {
    using T = F32Tile<TS, TR>;
    extern __shared__ __align__(16) float fsm[];
    float* Xs = fsm;
    float* Ws = fsm + T::STAGES * T::XS;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < T::SA; ++a)
#pragma unroll
        for (int b = 0; b < T::RA; ++b) acc[a][b] = 0.f;
    // one k tile: TS rows of X and TR rows of W, 4 chunks of 16 bytes each
    auto load = [&](int stage, int k0) {
        for (int e = threadIdx.x; e < 4 * (TS + TR); e += 256) {
            const int c = e & 3;
            if (e < 4 * TS) {
                const int sl = e >> 2;
                cp_async16(Xs + stage * T::XS + sl * T::LDS + 4 * c, X + (size_t)(slot0 + sl) * ld + k0 + 4 * c, true);
            } else {
                const int rw = (e - 4 * TS) >> 2;
                const bool ok = row0 + rw < nrows;
                cp_async16(Ws + stage * T::WS + rw * T::LDS + 4 * c,
                           ok ? W + (size_t)(row0 + rw) * ld + k0 + 4 * c : W, ok);
            }
        }
    };
#pragma unroll
    for (int s = 0; s < T::STAGES - 1; ++s) {
        if (kbeg + 16 * s < kend) load(s, kbeg + 16 * s);
        cp_async_commit();
    }
    int it = 0;
    for (int k0 = kbeg; k0 < kend; k0 += 16, ++it) {
        cp_async_wait<T::STAGES - 2>();
        __syncthreads();
        const int kn = k0 + 16 * (T::STAGES - 1);
        if (kn < kend) load((it + T::STAGES - 1) % T::STAGES, kn);
        cp_async_commit();
        const float* xs = Xs + (it % T::STAGES) * T::XS;
        const float* ws = Ws + (it % T::STAGES) * T::WS;
        float part[T::SA][T::RA];
#pragma unroll
        for (int a = 0; a < T::SA; ++a)
#pragma unroll
            for (int b = 0; b < T::RA; ++b) part[a][b] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 16; kk += 4) {
            float4 xa[T::SA], wb[T::RA];
#pragma unroll
            for (int a = 0; a < T::SA; ++a) xa[a] = *reinterpret_cast<const float4*>(xs + (ty + 16 * a) * T::LDS + kk);
#pragma unroll
            for (int b = 0; b < T::RA; ++b) wb[b] = *reinterpret_cast<const float4*>(ws + (tx + 16 * b) * T::LDS + kk);
#pragma unroll
            for (int a = 0; a < T::SA; ++a)
#pragma unroll
                for (int b = 0; b < T::RA; ++b) {
                    part[a][b] = fmaf(xa[a].x, wb[b].x, part[a][b]);
                    part[a][b] = fmaf(xa[a].y, wb[b].y, part[a][b]);
                    part[a][b] = fmaf(xa[a].z, wb[b].z, part[a][b]);
                    part[a][b] = fmaf(xa[a].w, wb[b].w, part[a][b]);
                }
        }
#pragma unroll
        for (int a = 0; a < T::SA; ++a)
#pragma unroll
            for (int b = 0; b < T::RA; ++b) acc[a][b] += part[a][b];
    }
    cp_async_wait<0>();
}

// Slot range of a CTA: TS-slot sub-tiles of the 128-slot tiles; a sub-tile
// with no active QP has nothing to do (the active QPs of a bank group fill
// its slots from the first one on, so perm of the first slot decides).
template <int TS>
__device__ __forceinline__ bool fp32_slots(const BatchParams& p, int& tile, int& slot0) {
    tile = (blockIdx.y * TS) / kSlotTile;
    slot0 = blockIdx.y * TS;
    if (tile >= p.counters[CNT_TILES]) return false;
    return TS == kSlotTile || p.perm[slot0] >= 0;
}

// One layer for every active slot tile (FP32 backend, and the accurate first
// layer of a chunk in the BF16 split form).
template <int TS, int TR>
__global__ void __launch_bounds__(256) batch_layer_fp32_kernel(BatchParams p, W32Ptrs wp) {
    int tile, slot0;
    if (!fp32_slots<TS>(p, tile, slot0)) return;
    const int ri = p.tile_rho[tile];
    const int row0 = blockIdx.x * TR;
    float acc[TS / 16][TR / 16];
    fp32_tile<TS, TR>(p.Sin, wp.w[ri], p.ldk, 0, p.ldk, p.R, slot0, row0, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < TS / 16; ++a) {
        const int slot = slot0 + ty + 16 * a;
        const int qp = p.perm[slot];
        if (qp < 0) continue;
#pragma unroll
        for (int b = 0; b < TR / 16; ++b) {
            const int r = row0 + tx + 16 * b;
            if (r < p.R) layer_elem(p, slot, qp, ri, r, acc[a][b]);
        }
    }
}

// max over the 16 threads of a half warp that share ty (NaN kept)
__device__ __forceinline__ float half_warp_max(float v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v = nmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Residual products (FP32 backend).  Phase 1: [P; A] x over the x columns of
// the check operand; phase 2: A^T lam_std over its multiplier columns.
template <int TS, int TR>
__global__ void __launch_bounds__(256) batch_check_fp32_kernel(BatchParams p, const float* __restrict__ Wc, int phase) {
    int tile, slot0;
    if (!fp32_slots<TS>(p, tile, slot0)) return;
    const int ri = p.tile_rho[tile];
    const int row0 = blockIdx.x * TR;
    const int rows = phase == 1 ? p.n + p.m : p.n;
    float acc[TS / 16][TR / 16];
    if (phase == 1)
        fp32_tile<TS, TR>(p.CK32, Wc, p.ldkc, 0, p.n64, rows, slot0, row0, acc);
    else
        fp32_tile<TS, TR>(p.CK32, Wc, p.ldkc, p.n64, p.ldkc, rows, slot0, row0, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < TS / 16; ++a) {
        const int slot = slot0 + ty + 16 * a;
        const int qp = p.perm[slot];     // the same in the 16 threads of a half warp
        float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f;
        if (qp >= 0) {
#pragma unroll
            for (int b = 0; b < TR / 16; ++b) {
                const int r = row0 + tx + 16 * b;
                if (r >= rows) continue;
                if (phase == 1) check1_elem(p, slot, qp, ri, r, acc[a][b], r0, r1, r2, r3);
                else check2_elem(p, qp, r, acc[a][b], r0, r1);
            }
        }
        r0 = half_warp_max(r0);
        r1 = half_warp_max(r1);
        r2 = half_warp_max(r2);
        r3 = half_warp_max(r3);
        if (qp < 0 || tx != 0) continue;
        if (phase == 1) {
            red_slot(p.RED, qp, RW_RP, r0);
            red_slot(p.RED, qp, RW_AX, r1);
            red_slot(p.RED, qp, RW_Z, r2);
            red_slot(p.RED, qp, RW_PX, r3);
        } else {
            red_slot(p.RED, qp, RW_RD, r0);
            red_slot(p.RED, qp, RW_ATL, r1);
        }
    }
}

// Launch helpers: the full-width tile (128 slots x 64 rows) while more than
// two slot tiles are active, else 32 x 32 sub-tiles, which skip the empty
// slots of the last tile of a bank group and give the convergence tail more
// CTAs.
template <int TS, int TR>
int launch_layer32(relu_qp_t h, const BatchParams& q, const W32Ptrs& wp, int tiles_max) {
    auto k = batch_layer_fp32_kernel<TS, TR>;
    RQ_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, F32Tile<TS, TR>::BYTES));
    k<<<dim3(ceil_div(h->R, TR), tiles_max * (kSlotTile / TS)), 256, F32Tile<TS, TR>::BYTES, h->stream>>>(q, wp);
    RQ_CUDA(h, cudaGetLastError());
    return RELU_QP_OK;
}

int layer32(relu_qp_t h, const BatchParams& q, const W32Ptrs& wp, int tiles_max, int active) {
    if (ceil_div(active, kSlotTile) <= 2) return launch_layer32<32, 32>(h, q, wp, tiles_max);
    return launch_layer32<128, 64>(h, q, wp, tiles_max);
}

template <int TS, int TR>
int launch_check32(relu_qp_t h, const BatchParams& q, const float* Wc, int tiles_max, int phase) {
    auto k = batch_check_fp32_kernel<TS, TR>;
    RQ_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, F32Tile<TS, TR>::BYTES));
    const int rows = phase == 1 ? h->n + h->m : h->n;
    k<<<dim3(ceil_div(rows, TR), tiles_max * (kSlotTile / TS)), 256, F32Tile<TS, TR>::BYTES, h->stream>>>(q, Wc,
                                                                                                         phase);
    RQ_CUDA(h, cudaGetLastError());
    return RELU_QP_OK;
}

int check32(relu_qp_t h, const BatchParams& q, const float* Wc, int tiles_max, int active, int phase) {
    if (ceil_div(active, kSlotTile) <= 2) return launch_check32<32, 32>(h, q, Wc, tiles_max, phase);
    return launch_check32<128, 64>(h, q, Wc, tiles_max, phase);
}

// Stop test and penalty rule per QP (one 128-thread block per QP: thread 0
// decides, the block copies the outputs of a finished QP or rebases lam' on a
// bank switch).
constexpr int kDecideThreads = 128;

// by_slot: one block per slot of the tiles in use (QP = perm[slot], padding
// slots return), which covers every active QP; else one block per QP id.
__global__ void __launch_bounds__(kDecideThreads) batch_decide_kernel(BatchParams p, DecideArgs d, int by_slot) {
    const int qp = by_slot ? p.perm[blockIdx.x] : (int)blockIdx.x;
    if (qp < 0 || qp >= d.B) return;
    __shared__ int s_act, s_nri;    // s_act: -1 not active, 0 continue, 1 finished, 2 bank switch
    unsigned* red = p.RED + (size_t)qp * RW_WORDS;
    if (threadIdx.x == 0) {
        int act = -1, nri = 0;
        if (d.status[qp] == QP_ACTIVE) {
            const unsigned w[RW_WORDS] = {red[0], red[1], red[2], red[3], red[4], red[5], red[6], red[7]};
            act = decide_qp(p, d, qp, w, nri);
        }
        s_act = act;
        s_nri = nri;
    }
    __syncthreads();
    const int act = s_act;
    if (act < 0) return;
    if (act == 1) {
        for (int k = threadIdx.x; k < p.n; k += kDecideThreads) d.XO[(size_t)qp * p.n + k] = p.Y[(size_t)qp * p.ldn + k];
        for (int i = threadIdx.x; i < p.m; i += kDecideThreads) {
            d.ZO[(size_t)qp * p.m + i] = p.Z[(size_t)qp * p.ldm + i];
            d.LO[(size_t)qp * p.m + i] = p.LSTD[(size_t)qp * p.ldm + i];
        }
    } else if (act == 2) {
        // rebase lam' so that the next layer is standard ADMM with the new rho
        const int nri = s_nri;
        for (int i = threadIdx.x; i < p.m; i += kDecideThreads) {
            const size_t o = (size_t)qp * p.ldm + i;
            const float rho_i = (float)(p.rhod[nri] * (double)p.rs[i]);
            p.LAM[o] = lam_standard(p.LSTD[o], -rho_i, p.AY[o] - p.Z[o]);
        }
    }
    if (threadIdx.x < RW_WORDS) red[threadIdx.x] = 0u;
}

// Regroup the active QPs by bank index: slots [base_g, base_g + count_g) hold
// group g in increasing QP id, each group padded to a multiple of 128 slots.
__global__ void __launch_bounds__(1024) batch_assign_kernel(int B, int slots, int nr, const int* __restrict__ status,
                                                            const int* __restrict__ rho_idx, int* perm,
                                                            int* tile_rho, int* counters) {
    __shared__ int cnt[RQ_MAX_RHO], base[RQ_MAX_RHO], warp_cnt[32], run;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int s = tid; s < slots; s += blockDim.x) perm[s] = -1;
    if (tid < RQ_MAX_RHO) cnt[tid] = 0;
    __syncthreads();
    for (int qp = tid; qp < B; qp += blockDim.x)
        if (status[qp] == QP_ACTIVE) atomicAdd(&cnt[rho_idx[qp]], 1);
    __syncthreads();
    if (tid == 0) {
        int off = 0, t = 0, tot = 0;
        for (int g = 0; g < nr; ++g) {
            base[g] = off;
            const int tiles = (cnt[g] + kSlotTile - 1) / kSlotTile;
            for (int k = 0; k < tiles; ++k) tile_rho[t++] = g;
            off += tiles * kSlotTile;
            tot += cnt[g];
        }
        counters[CNT_TILES] = t;
        counters[CNT_ACTIVE] = tot;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int g = 0; g < nr; ++g) {
        if (cnt[g] == 0) continue;
        for (int c0 = 0; c0 < B; c0 += blockDim.x) {
            const int qp = c0 + tid;
            const bool flag = qp < B && status[qp] == QP_ACTIVE && rho_idx[qp] == g;
            const unsigned ball = __ballot_sync(0xffffffffu, flag);
            if (lane == 0) warp_cnt[warp] = __popc(ball);
            __syncthreads();
            if (tid == 0) {
                int acc = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    const int c = warp_cnt[w];
                    warp_cnt[w] = acc;
                    acc += c;
                }
                run = acc;
            }
            __syncthreads();
            if (flag) perm[base[g] + warp_cnt[warp] + __popc(ball & lt)] = qp;
            __syncthreads();
            if (tid == 0) base[g] += run;
            __syncthreads();
        }
    }
}

// Operand of the first layer of a chunk: s = [x; 2 rho z - lam'] per slot, in
// FP32 or as a 3-way BF16 split; padding slots get zeros.  One thread per 4
// consecutive columns of a slot.
__global__ void batch_fill_kernel(BatchParams p, const int* __restrict__ rho_idx, float* S32, __nv_bfloat16* T,
                                  size_t part) {
    const int q4 = p.ldk >> 2;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int slot = (int)(e / q4);
    const int k0 = (int)(e % q4) * 4;
    if (slot >= p.counters[CNT_TILES] * kSlotTile) return;
    const int qp = p.perm[slot];
    const int ri = qp >= 0 ? rho_idx[qp] : 0;
    float v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int k = k0 + t;
        v[t] = 0.f;
        if (qp >= 0) {
            if (k < p.n) {
                v[t] = p.Y[(size_t)qp * p.ldn + k];
            } else if (k < p.R) {
                const int i = k - p.n;
                const size_t o = (size_t)qp * p.ldm + i;
                v[t] = next_operand(p.rho[ri] * p.rs[i], p.Z[o], p.LAM[o]);
            }
        }
    }
    const size_t o = (size_t)slot * p.ldk + k0;
    if (S32) {
        st4(S32 + o, v);
    } else {
        __nv_bfloat16 a[4], b[4], c[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) split3(v[t], a[t], b[t], c[t]);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            T[o + t] = a[t];
            T[o + t + part] = b[t];
            T[o + t + 2 * part] = c[t];
        }
    }
}

// Start state per QP: x given (Y) or 0, z = A x (AY holds A x for warm starts),
// lam' = lam_warm (staged in LSTD) or 0.
__global__ void batch_init_kernel(BatchParams p, int B, int warm, int lam_given, const int* __restrict__ rw,
                                  int rho0, int* status, int* rho_idx, int* iters, int* nsw) {
    const int qp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (qp >= p.cap) return;
    if (lane == 0) {
        status[qp] = qp < B ? QP_ACTIVE : QP_UNUSED;
        rho_idx[qp] = (qp < B && rw) ? rw[qp] : rho0;
        iters[qp] = 0;
        nsw[qp] = 0;
    }
    if (lane < RW_WORDS) p.RED[(size_t)qp * RW_WORDS + lane] = 0u;
    if (qp >= B) return;
    for (int i = lane; i < p.m; i += 32) {
        const size_t o = (size_t)qp * p.ldm + i;
        const float ax = warm ? p.AY[o] : 0.f;
        p.AY[o] = ax;
        p.Z[o] = ax;
        p.LAM[o] = lam_given ? p.LSTD[o] : 0.f;
    }
    if (!warm)
        for (int k = lane; k < p.n; k += 32) p.Y[(size_t)qp * p.ldn + k] = 0.f;
}

// out[r] = max_k |X[r][k] f[k]| (f = nullptr: 1).
__global__ void row_absmax_kernel(const float* __restrict__ X, int rows, int cols, int ld,
                                  const float* __restrict__ f, float* out) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    float v = 0.f;
    for (int k = lane; k < cols; k += 32) v = fmaxf(v, fabsf(f ? X[(size_t)r * ld + k] * f[k] : X[(size_t)r * ld + k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) out[r] = v;
}

// X[r][k] *= f[k] for rows [0, rows): the problem scaling's maps between the
// original and the scaled problem's data and iterates.
__global__ void scale_rows_kernel(float* X, int rows, int cols, int ld, const float* __restrict__ f) {
    const size_t total = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), k = (int)(e % cols);
        X[(size_t)r * ld + k] *= f[k];
    }
}

// Check matrix [[P, A^T], [A, 0]] in FP32: x columns [0, n64), multiplier
// columns [n64, n64 + m64); rows [0, n) for P and A^T, [n, n + m) for A.
__global__ void build_wc32_kernel(const float* __restrict__ P32, const float* __restrict__ A32, int ldp,
                                  const float* __restrict__ At32, int ldt, int n, int m, int n64, int ldkc,
                                  float* __restrict__ Wc) {
    const size_t total = (size_t)(n + m) * ldkc;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / ldkc), k = (int)(e % ldkc);
        float v = 0.f;
        if (j < n) {
            if (k < n) v = P32[(size_t)j * ldp + k];
            else if (k >= n64 && k < n64 + m) v = At32[(size_t)j * ldt + (k - n64)];
        } else if (k < n) {
            v = A32[(size_t)(j - n) * ldp + k];
        }
        Wc[e] = v;
    }
}

int sgemm_nt(relu_qp_t h, int M, int N, int K, const float* X, int ldx, const float* W, int ldw, float alpha,
             const float* off, float* C, int ldc) {
    if (M <= 0 || N <= 0) return RELU_QP_OK;
    dim3 grid(ceil_div(N, 64), ceil_div(M, 64));
    sgemm_nt_kernel<<<grid, 256, 0, h->stream>>>(M, N, K, X, ldx, W, ldw, alpha, off, C, ldc);
    RQ_CUDA(h, cudaGetLastError());
    ++h->launches;
    return RELU_QP_OK;
}

BatchParams base_params(relu_qp_t h) {
    BatchWork& w = h->bw;
    BatchParams p{};
    p.n = h->n;
    p.m = h->m;
    p.R = h->R;
    p.ldn = w.ldn;
    p.ldm = w.ldm;
    p.ldR = w.ldR;
    p.ldk = w.ldk;
    p.n64 = w.n64;
    p.ldkc = w.ldkc;
    p.cap = w.cap;
    p.slots = w.slots;
    p.nr = h->nr;
    for (int r = 0; r < h->nr; ++r) {
        p.rho[r] = (float)h->be[r].rho;
        p.rhod[r] = h->be[r].rho;
        p.logrho[r] = std::log(h->be[r].rho);
    }
    p.rs = h->rs32;
    p.rsx = h->sc_rx;
    p.rsz = h->sc_z;
    p.Y = w.Y; p.Z = w.Z; p.LAM = w.LAM; p.AY = w.AY; p.RR = w.RR; p.LSTD = w.LSTD; p.C = w.C; p.SREF = w.SREF; p.PY = w.PY;
    p.L = w.L; p.U = w.U; p.Q = w.Q; p.BIAS = w.BIAS; p.QN = w.QN;
    p.perm = w.perm; p.tile_rho = w.tile_rho; p.counters = w.counters; p.RED = w.RED;
    return p;
}

int scale_rows(relu_qp_t h, float* X, int rows, int cols, int ld, const float* f) {
    if (!f || rows <= 0 || cols <= 0) return RELU_QP_OK;
    const size_t total = (size_t)rows * cols;
    const int g = (int)std::min<size_t>((total + 255) / 256, 4096);
    scale_rows_kernel<<<g, 256, 0, h->stream>>>(X, rows, cols, ld, f);
    RQ_CUDA(h, cudaGetLastError());
    ++h->launches;
    return RELU_QP_OK;
}

int copy_rows_in(relu_qp_t h, float* dst, int ld, const float* src, int rows, int cols) {
    if (rows <= 0 || cols <= 0) return RELU_QP_OK;
    RQ_CUDA(h, cudaMemcpy2DAsync(dst, sizeof(float) * ld, src, sizeof(float) * cols, sizeof(float) * cols, rows,
                                 cudaMemcpyDefault, h->stream));
    return RELU_QP_OK;
}

}  // namespace

// Device bytes per QP slot of a batched handle: the arrays batch_alloc sizes by
// max_batch (per-QP state, bias rows of every bank entry, outputs, records) and
// the share of the slot-indexed operands (cap slots of the slots rows).
size_t batch_slot_bytes(relu_qp_t h) {
    const BatchWork& w = h->bw;
    const size_t mm = h->m > 0 ? h->m : 1, f = sizeof(float);
    size_t b = 3 * w.ldn * f + f;                       // Y, Q, PY, QN
    b += 7 * w.ldm * f;                                 // Z, LAM, AY, RR, LSTD, L, U
    b += (size_t)h->nr * w.ldR * f;                     // BIAS
    b += (h->n + 2 * mm) * f;                           // XO, ZO, LO
    b += RW_WORDS * sizeof(unsigned) + 6 * sizeof(int); // RED, rho_idx, status, iters, nsw, rp, rd
    b += sizeof(int);                                   // perm
    if (w.prec == RELU_QP_PREC_BF16X3) {
        b += 2 * w.ldR * f;                             // C, SREF
        b += w.ldk * f + w.ldkc * f;                    // S32, CK32
        b += 2 * (7 * (size_t)w.ldk + 3 * (size_t)w.ldkc);   // BF16 operand parts and check operand
    } else {
        b += 2 * w.ldk * f + w.ldkc * f;                // S32 pair, CK32
    }
    return b;
}

int batch_alloc(relu_qp_t h) {
    BatchWork& w = h->bw;
    const int n = h->n, m = h->m, R = h->R, nr = h->nr;
    const int mm = m > 0 ? m : 1;
    w.cap = h->opts.max_batch;
    w.prec = h->opts.batch_precision;
    w.slots = (int)round_up(w.cap, kSlotTile) + nr * kSlotTile;
    w.ldn = (int)round_up(n, 4);
    w.ldm = (int)round_up(mm, 4);
    w.ldR = (int)round_up(R, 4);
    w.ldk = h->ldw;
    w.n64 = (int)round_up(n, 64);
    w.m64 = (int)round_up(mm, 64);
    w.ldkc = w.n64 + w.m64;
    w.Rpad = (int)round_up(R, 256);
    w.npad = (int)round_up(n + m, 256);
    const size_t cap = w.cap;
    RQ_TRY(alloc(h, &w.Y, cap * w.ldn));
    RQ_TRY(alloc(h, &w.Q, cap * w.ldn));
    RQ_TRY(alloc(h, &w.PY, cap * w.ldn));
    RQ_TRY(alloc(h, &w.QN, cap));
    RQ_TRY(alloc(h, &w.Z, cap * w.ldm));
    RQ_TRY(alloc(h, &w.LAM, cap * w.ldm));
    RQ_TRY(alloc(h, &w.AY, cap * w.ldm));
    RQ_TRY(alloc(h, &w.RR, cap * w.ldm));
    RQ_TRY(alloc(h, &w.LSTD, cap * w.ldm));
    RQ_TRY(alloc(h, &w.L, cap * w.ldm));
    RQ_TRY(alloc(h, &w.U, cap * w.ldm));
    RQ_TRY(alloc(h, &w.BIAS, (size_t)nr * cap * w.ldR));
    RQ_TRY(alloc(h, &w.XO, cap * n));
    RQ_TRY(alloc(h, &w.ZO, cap * mm));
    RQ_TRY(alloc(h, &w.LO, cap * mm));
    RQ_TRY(alloc(h, &w.RED, cap * RW_WORDS));
    RQ_TRY(alloc(h, &w.rho_idx, cap));
    RQ_TRY(alloc(h, &w.status, cap));
    RQ_TRY(alloc(h, &w.iters, cap));
    RQ_TRY(alloc(h, &w.nsw, cap));
    RQ_TRY(alloc(h, &w.rp, cap));
    RQ_TRY(alloc(h, &w.rd, cap));
    RQ_TRY(alloc(h, &w.perm, (size_t)w.slots));
    RQ_TRY(alloc(h, &w.tile_rho, (size_t)w.slots / kSlotTile));
    RQ_TRY(alloc(h, &w.counters, CNT_WORDS));
    if (w.prec == RELU_QP_PREC_BF16X3) {
        RQ_TRY(alloc(h, &w.C, cap * w.ldR));
        RQ_TRY(alloc(h, &w.SREF, cap * w.ldR));
        RQ_TRY(alloc(h, &w.S32, (size_t)w.slots * w.ldk));   // FP32 operand of the accurate layer
        RQ_TRY(alloc(h, &w.CK32, (size_t)w.slots * w.ldkc));  // FP32 check operand
        RQ_TRY(alloc(h, &w.Wc32, (size_t)(n + m) * w.ldkc));
        RQ_TRY(dev_alloc(h, &w.OPND, sizeof(uint16_t) * 7 * (size_t)w.slots * w.ldk + 1024));
        RQ_TRY(dev_alloc(h, &w.CK, sizeof(uint16_t) * 3 * (size_t)w.slots * w.ldkc + 1024));
        RQ_TRY(dev_alloc(h, &w.WB, sizeof(uint16_t) * (size_t)nr * 3 * w.Rpad * w.ldk + 1024));
        RQ_TRY(dev_alloc(h, &w.WCB, sizeof(uint16_t) * 3 * (size_t)w.npad * w.ldkc + 1024));
        RQ_TRY(alloc(h, &w.chunk_sync, 2 * (size_t)w.slots / kSlotTile));   // layer counters, done counters
        RQ_CUDA(h, cudaMemset(w.chunk_sync, 0, sizeof(unsigned) * 2 * (w.slots / kSlotTile)));
    } else {
        RQ_TRY(alloc(h, &w.S32, 2 * (size_t)w.slots * w.ldk));
        RQ_TRY(alloc(h, &w.CK32, (size_t)w.slots * w.ldkc));
        RQ_TRY(alloc(h, &w.Wc32, (size_t)(n + m) * w.ldkc));
    }
    RQ_TRY(batch_tail_alloc(h));
    RQ_CUDA(h, cudaMallocHost(reinterpret_cast<void**>(&w.cnt_host), sizeof(int) * CNT_WORDS));
    RQ_CUDA(h, cudaEventCreateWithFlags(&w.ev_cnt, cudaEventDisableTiming));
    return RELU_QP_OK;
}

// Tuning layout: the first `active_tiles` tiles hold `per_tile` QPs each (a prefix
// of the tile, as the regrouping leaves it).
__global__ void tune_perm_kernel(int slots, int cap, int active_tiles, int per_tile, int* perm, int* tile_rho,
                                 int* counters) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < slots; s += gridDim.x * blockDim.x) {
        const bool in = s / kSlotTile < active_tiles && s % kSlotTile < per_tile && s < cap;
        perm[s] = in ? s : -1;
        if (s % kSlotTile == 0) tile_rho[s / kSlotTile] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counters[CNT_TILES] = active_tiles;
        counters[CNT_ACTIVE] = min(cap, active_tiles * per_tile);
    }
}

// Choose the refined layer's configuration (K split over a cluster, tile
// width) for every number of active slot tiles by timing what a chunk would
// run: the persistent chunk kernel where the tiles fit one wave, else one
// launch per layer.  Counts of one or two tiles are timed with tiles that hold
// 48 QPs each (the convergence tail); larger counts with full tiles.  State
// values do not matter here; every buffer the layers touch is re-initialised by
// the next solve.  RELU_QP_TUNE_LOG=1 prints the measurements to stderr.
int tc_tune(relu_qp_t h) {
    BatchWork& w = h->bw;
    BatchParams p = base_params(h);
    const size_t opart = (size_t)w.slots * w.ldk;
    __nv_bfloat16* OP = static_cast<__nv_bfloat16*>(w.OPND);
    p.flags = EPI_REFINE;
    p.Dhi = OP + 2 * opart;
    p.Dlo = OP + 3 * opart;
    p.CK = static_cast<__nv_bfloat16*>(w.CK);
    const int tiles = w.slots / kSlotTile;
    const char* log_env = std::getenv("RELU_QP_TUNE_LOG");
    const bool log = log_env && log_env[0] == '1';
    std::vector<LayerCfg> cfgs;
    tc_layer_cfgs(h, cfgs);
    // measured tile counts: every count up to 8, then every 4th up to 32, then every 16th
    std::vector<int> counts;
    for (int t = 1; t <= tiles; ++t)
        if (t <= 8 || (t <= 32 && t % 4 == 0) || t % 16 == 0 || t == tiles) counts.push_back(t);
    std::vector<LayerCfg> table(tiles + 1, cfgs[0]);
    for (int t : counts) {
        const int per_tile = t <= 2 ? 48 : kSlotTile;
        tune_perm_kernel<<<ceil_div(w.slots, 256), 256, 0, h->stream>>>(w.slots, w.cap, t, per_tile, w.perm,
                                                                         w.tile_rho, w.counters);
        RQ_CUDA(h, cudaGetLastError());
        float best = 1e30f;
        LayerCfg best_c = cfgs[0];
        for (const LayerCfg& c : cfgs) {
            RQ_TRY(tc_set_layer_cfg(h, c));
            float ms = 0.f;
            int layers = 0;
            bool chunked = false;
            if (w.chunk_sync) {
                RQ_CUDA(h, cudaMemsetAsync(w.chunk_sync, 0, sizeof(unsigned) * 2 * tiles, h->stream));
                const int rc = tc_chunk(h, p, 2, 0u, t);    // warm-up (and eligibility)
                if (rc == RELU_QP_OK) {
                    RQ_CUDA(h, cudaMemsetAsync(w.chunk_sync, 0, sizeof(unsigned) * 2 * tiles, h->stream));
                    RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
                    RQ_TRY(tc_chunk(h, p, 8, 0u, t));
                    RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
                    layers = 8;
                    chunked = true;
                } else if (rc != RELU_QP_ERR_UNSUPPORTED) {
                    return rc;
                }
            }
            if (!chunked) {
                RQ_TRY(tc_layer(h, p, 0, tiles, t));
                RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
                RQ_TRY(tc_layer(h, p, 0, tiles, t));
                for (int rep = 1; rep < 4; ++rep) RQ_TRY(tc_layer(h, p, 0, tiles, t, true));
                RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
                layers = 4;
            }
            RQ_CUDA(h, cudaEventSynchronize(h->ev1));
            int site = 0;
            if (tc_error(h, &site))
                return fail(h, RELU_QP_ERR_TIMEOUT,
                            "tensor-core wait " + std::to_string(site) + " passed its deadline while tuning (tiles " +
                                std::to_string(t) + ", ks " + std::to_string(c.ks) + ", bn " + std::to_string(c.bn) +
                                (chunked ? ", chunk kernel)" : ", one launch per layer)"));
            RQ_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
            ms /= layers;
            if (log)
                std::fprintf(stderr, "relu_qp tune: n=%d m=%d tiles=%d qps/tile=%d ks=%d bn=%d %s us=%.2f\n", h->n,
                             h->m, t, per_tile, c.ks, c.bn, chunked ? "chunk" : "layer", 1e3f * ms);
            if (ms < best) {
                best = ms;
                best_c = c;
            }
        }
        for (int u = t; u <= tiles; ++u) table[u] = best_c;   // until the next measured count
        if (t == 1 && tc_small_eligible(h, per_tile, 1)) {
            // the resident-weight kernel for one tile of few QPs against the best tiled one
            RQ_CUDA(h, cudaMemsetAsync(w.chunk_sync, 0, sizeof(unsigned) * 2 * tiles, h->stream));
            int rc = tc_small(h, p, 2, 0u, per_tile, 1);
            if (rc == RELU_QP_OK) {
                RQ_CUDA(h, cudaMemsetAsync(w.chunk_sync, 0, sizeof(unsigned) * 2 * tiles, h->stream));
                RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
                RQ_TRY(tc_small(h, p, 8, 0u, per_tile, 1));
                RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
                RQ_CUDA(h, cudaEventSynchronize(h->ev1));
                int site = 0;
                if (tc_error(h, &site))
                    return fail(h, RELU_QP_ERR_TIMEOUT, "tensor-core wait " + std::to_string(site) +
                                                            " passed its deadline while tuning (resident-weight kernel)");
                float ms = 0.f;
                RQ_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
                ms /= 8;
                if (log)
                    std::fprintf(stderr, "relu_qp tune: n=%d m=%d tiles=1 qps/tile=%d resident-weight us=%.2f\n", h->n,
                                 h->m, per_tile, 1e3f * ms);
                tc_small_set(h, ms < best);
            } else if (rc != RELU_QP_ERR_UNSUPPORTED) {
                return rc;
            }
        }
    }
    tune_perm_kernel<<<ceil_div(w.slots, 256), 256, 0, h->stream>>>(w.slots, w.cap, tiles, kSlotTile, w.perm,
                                                                     w.tile_rho, w.counters);
    RQ_CUDA(h, cudaGetLastError());
    RQ_TRY(tc_set_layer_table(h, table));
    if (log) {
        std::fprintf(stderr, "relu_qp tune: chose (ks, bn) by active tiles:");
        for (int t = 1; t <= tiles; ++t) std::fprintf(stderr, " (%d,%d)", table[t].ks, table[t].bn);
        std::fprintf(stderr, "\n");
    }
    if (tc_error(h)) return fail(h, RELU_QP_ERR_TIMEOUT, "tensor-core kernel wait passed its deadline while tuning");
    RQ_CUDA(h, cudaMemsetAsync(w.RED, 0, sizeof(unsigned) * (size_t)w.cap * RW_WORDS, h->stream));
    RQ_CUDA(h, cudaMemsetAsync(w.counters, 0, sizeof(int) * CNT_WORDS, h->stream));
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return RELU_QP_OK;
}

void batch_release(relu_qp_t h) {
    if (h->bw.tc) tc_release(h);
    if (h->bw.cnt_host) cudaFreeHost(h->bw.cnt_host);
    if (h->bw.ev_cnt) cudaEventDestroy(h->bw.ev_cnt);
    h->bw.cnt_host = nullptr;
    h->bw.ev_cnt = nullptr;
}

// After the FP64 stage: FP32 check matrix (FP32 backend) or tensor maps and
// tile tuning (BF16 backend).
int batch_finish_setup(relu_qp_t h) {
    BatchWork& w = h->bw;
    if (w.prec == RELU_QP_PREC_BF16X3) {
        RQ_TRY(tc_prepare(h));
        RQ_TRY(tc_tune(h));
    }
    const int ldp = (int)round_up(h->n, 4), ldt = (int)round_up(h->m > 0 ? h->m : 1, 4);
    const size_t total = (size_t)(h->n + h->m) * w.ldkc;
    int g = (int)std::min<size_t>((total + 255) / 256, 8192);
    build_wc32_kernel<<<g, 256, 0, h->stream>>>(h->P32, h->A32, ldp, h->At32, ldt, h->n, h->m, w.n64, w.ldkc,
                                                w.Wc32);
    RQ_CUDA(h, cudaGetLastError());
    return RELU_QP_OK;
}

int batch_update(relu_qp_t h, int B, const float* Q, const float* L, const float* U) {
    BatchWork& w = h->bw;
    const int n = h->n, m = h->m, R = h->R;
    if (Q) RQ_TRY(copy_rows_in(h, w.Q, w.ldn, Q, B, n));
    if (L && m > 0) RQ_TRY(copy_rows_in(h, w.L, w.ldm, L, B, m));
    if (U && m > 0) RQ_TRY(copy_rows_in(h, w.U, w.ldm, U, B, m));
    // scaled handles: q -> c D q, l -> E l, u -> E u
    if (Q) RQ_TRY(scale_rows(h, w.Q, B, n, w.ldn, h->sc_q));
    if (L && m > 0) RQ_TRY(scale_rows(h, w.L, B, m, w.ldm, h->sc_e));
    if (U && m > 0) RQ_TRY(scale_rows(h, w.U, B, m, w.ldm, h->sc_e));
    if (Q) {
        for (int r = 0; r < h->nr; ++r)
            RQ_TRY(sgemm_nt(h, B, R, n, w.Q, w.ldn, h->be[r].Bop, n, 1.f, nullptr,
                            w.BIAS + (size_t)r * w.cap * w.ldR, w.ldR));
        row_absmax_kernel<<<ceil_div(B * 32, 256), 256, 0, h->stream>>>(w.Q, B, n, w.ldn, h->sc_rx, w.QN);
        RQ_CUDA(h, cudaGetLastError());
        ++h->launches;
    }
    w.B = B;
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return RELU_QP_OK;
}

int batch_set_parametric(relu_qp_t h, int nx, const double* F, const double* E, const double* l0,
                         const double* u0) {
    BatchWork& w = h->bw;
    const int n = h->n, m = h->m, R = h->R;
    if (w.nx != nx) {
        w.nx = nx;
        w.ldx = (int)round_up(nx, 4);
        RQ_TRY(alloc(h, &w.F32, (size_t)n * w.ldx));
        RQ_TRY(alloc(h, &w.Ft32, (size_t)nx * w.ldn));
        RQ_TRY(alloc(h, &w.E32, (size_t)(m > 0 ? m : 1) * w.ldx));
        RQ_TRY(alloc(h, &w.l0, (size_t)(m > 0 ? m : 1)));
        RQ_TRY(alloc(h, &w.u0, (size_t)(m > 0 ? m : 1)));
        RQ_TRY(alloc(h, &w.X0, (size_t)w.cap * w.ldx));
        for (int r = 0; r < h->nr; ++r) RQ_TRY(alloc(h, &w.G[r], (size_t)R * w.ldx));
    }
    // scaled handles: F -> c D F, E -> E E, l0 -> E l0, u0 -> E u0 (in FP64)
    const bool sc = h->scaled != 0;
    std::vector<float> f((size_t)n * w.ldx, 0.f), ft((size_t)nx * w.ldn, 0.f);
    for (int i = 0; i < n; ++i) {
        const double fi = sc ? h->sC * h->sD[i] : 1.0;
        for (int k = 0; k < nx; ++k) {
            f[(size_t)i * w.ldx + k] = (float)(fi * F[(size_t)i * nx + k]);
            ft[(size_t)k * w.ldn + i] = (float)(fi * F[(size_t)i * nx + k]);
        }
    }
    RQ_CUDA(h, cudaMemcpy(w.F32, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
    RQ_CUDA(h, cudaMemcpy(w.Ft32, ft.data(), sizeof(float) * ft.size(), cudaMemcpyHostToDevice));
    if (m > 0) {
        std::vector<float> e((size_t)m * w.ldx, 0.f), lo(m), up(m);
        for (int i = 0; i < m; ++i) {
            const double ei = sc ? h->sE[i] : 1.0;
            for (int k = 0; k < nx; ++k) e[(size_t)i * w.ldx + k] = (float)(ei * E[(size_t)i * nx + k]);
            lo[i] = (float)(ei * l0[i]);
            up[i] = (float)(ei * u0[i]);
        }
        RQ_CUDA(h, cudaMemcpy(w.E32, e.data(), sizeof(float) * e.size(), cudaMemcpyHostToDevice));
        RQ_CUDA(h, cudaMemcpy(w.l0, lo.data(), sizeof(float) * m, cudaMemcpyHostToDevice));
        RQ_CUDA(h, cudaMemcpy(w.u0, up.data(), sizeof(float) * m, cudaMemcpyHostToDevice));
    }
    for (int r = 0; r < h->nr; ++r)   // G_r = Bop_r F
        RQ_TRY(sgemm_nt(h, R, nx, n, h->be[r].Bop, n, w.Ft32, w.ldn, 1.f, nullptr, w.G[r], w.ldx));
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return RELU_QP_OK;
}

int batch_update_x0(relu_qp_t h, int B, const float* X0) {
    BatchWork& w = h->bw;
    const int n = h->n, m = h->m, R = h->R, nx = w.nx;
    RQ_TRY(copy_rows_in(h, w.X0, w.ldx, X0, B, nx));
    RQ_TRY(sgemm_nt(h, B, n, nx, w.X0, w.ldx, w.F32, w.ldx, 1.f, nullptr, w.Q, w.ldn));
    if (m > 0) {
        RQ_TRY(sgemm_nt(h, B, m, nx, w.X0, w.ldx, w.E32, w.ldx, -1.f, w.l0, w.L, w.ldm));
        RQ_TRY(sgemm_nt(h, B, m, nx, w.X0, w.ldx, w.E32, w.ldx, -1.f, w.u0, w.U, w.ldm));
    }
    for (int r = 0; r < h->nr; ++r)
        RQ_TRY(sgemm_nt(h, B, R, nx, w.X0, w.ldx, w.G[r], w.ldx, 1.f, nullptr, w.BIAS + (size_t)r * w.cap * w.ldR,
                        w.ldR));
    row_absmax_kernel<<<ceil_div(B * 32, 256), 256, 0, h->stream>>>(w.Q, B, n, w.ldn, h->sc_rx, w.QN);
    RQ_CUDA(h, cudaGetLastError());
    ++h->launches;
    w.B = B;
    return RELU_QP_OK;
}

// Regroup the active QPs among the first nqp QP indices into slots (assign)
// and write the FP32 operand of the next chunk's first layer (fill).
int regroup_slots(relu_qp_t h, const BatchParams& p, int nqp, bool assign) {
    BatchWork& w = h->bw;
    const bool bf16 = w.prec == RELU_QP_PREC_BF16X3;
    const size_t opart = (size_t)w.slots * w.ldk;
    __nv_bfloat16* OP = static_cast<__nv_bfloat16*>(w.OPND);
    if (assign) {
        batch_assign_kernel<<<1, 1024, 0, h->stream>>>(nqp, w.slots, h->nr, w.status, w.rho_idx, w.perm, w.tile_rho,
                                                       w.counters);
        RQ_CUDA(h, cudaGetLastError());
        ++h->launches;
    }
    const bool split_operand = bf16 && w.rebase_tc;
    batch_fill_kernel<<<(int)((size_t)w.slots * (w.ldk / 4) / 256 + 1), 256, 0, h->stream>>>(
        p, w.rho_idx, split_operand ? nullptr : w.S32, split_operand ? OP + 4 * opart : nullptr, opart);
    RQ_CUDA(h, cudaGetLastError());
    ++h->launches;
    return RELU_QP_OK;
}

// `len` layers of one chunk over the slots of the last regroup; with `check`
// the last layer also writes x into the check operand.  `active` is the
// number of QPs in the batch (for the tile-width choice and the FLOP count).
int run_layers(relu_qp_t h, const BatchParams& p, int len, bool check, int active, int tiles_now,
               size_t& prof_used, int j_begin = 0, int j_end = 1 << 30) {
    BatchWork& w = h->bw;
    const int R = h->R;
    const bool bf16 = w.prec == RELU_QP_PREC_BF16X3;
    const int tiles_max = w.slots / kSlotTile;
    const size_t opart = (size_t)w.slots * w.ldk;
    __nv_bfloat16* OP = static_cast<__nv_bfloat16*>(w.OPND);
    W32Ptrs wp{};
    for (int r = 0; r < h->nr; ++r) wp.w[r] = h->be[r].Wt;
    // profiling: one event pair around the refined layers of the chunk (events
    // between them would break the programmatic overlap of consecutive layers)
    const bool timed = h->prof_on && bf16 && len > 1 && prof_used + 2 <= h->prof_ev.size();
    // layer counters of the persistent chunk kernel start at zero
    if (bf16 && w.chunk_sync && len > 1 && j_end > 1)
        RQ_CUDA(h, cudaMemsetAsync(w.chunk_sync, 0, sizeof(unsigned) * 2 * tiles_max, h->stream));
    for (int j = j_begin; j < std::min(len, j_end); ++j) {
        BatchParams q = p;
        q.flags = 0;
        if (j == len - 1) q.flags |= EPI_LAST | (check ? EPI_CHECK : 0u);
        if (bf16) {
            q.flags |= EPI_REFINE | (j == 0 ? EPI_REBASE : 0u);
            q.Dhi = OP + (size_t)(2 * (j & 1)) * opart;
            q.Dlo = q.Dhi + opart;
            if (w.check_tc) q.CK = static_cast<__nv_bfloat16*>(w.CK);
            else q.CK32 = w.CK32;
            if (j == 1 && w.chunk_sync) {
                // layers 1 .. len-1 in one persistent launch when the tile's CTAs fit in one wave:
                // the resident-weight kernel for one tile of few QPs (when the tuner chose it),
                // else the tiled chunk kernel
                BatchParams qc = q;
                qc.flags = 0;
                if (timed) RQ_CUDA(h, cudaEventRecord(h->prof_ev[prof_used], h->stream));
                int rc = RELU_QP_ERR_UNSUPPORTED;
                if (tc_small_chosen(h) && tc_small_eligible(h, active, tiles_now)) {
                    rc = tc_small(h, qc, len - 1, EPI_LAST | (check ? EPI_CHECK : 0u), active, tiles_now);
                    if (rc != RELU_QP_OK && rc != RELU_QP_ERR_UNSUPPORTED) return rc;
                    if (rc == RELU_QP_OK) ++h->resident_launches;
                }
                if (rc != RELU_QP_OK) rc = tc_chunk(h, qc, len - 1, EPI_LAST | (check ? EPI_CHECK : 0u), tiles_now);
                if (rc == RELU_QP_OK) {
                    h->launches += 1;
                    h->layer_launches += len - 1;
                    h->layer_flops += (len - 1) * 2.0 * 3.0 * (double)R * (double)R * (double)active;
                    if (timed) {
                        RQ_CUDA(h, cudaEventRecord(h->prof_ev[prof_used + 1], h->stream));
                        h->prof_span_launches.push_back(len - 1);
                        prof_used += 2;
                    }
                    break;
                }
                if (rc != RELU_QP_ERR_UNSUPPORTED) return rc;
                // refused: one launch per layer below (which records the span's start again)
            }
            if (j == 0 && !w.rebase_tc) {
                // accurate layer c = Wt s_ref + b in FP32 on the CUDA cores (round to
                // nearest); the tensor core's truncating accumulation of the full
                // operand would set the fixed point's accuracy instead
                q.Sin = w.S32;
                RQ_TRY(layer32(h, q, wp, tiles_max, active));
                ++h->launches;
            } else {
                // operand set read by this layer: 4..6 = s (3-way), else pair ((j-1)&1)
                if (timed && j == 1) RQ_CUDA(h, cudaEventRecord(h->prof_ev[prof_used], h->stream));
                RQ_TRY(tc_layer(h, q, j == 0 ? -1 : ((j - 1) & 1), tiles_max,
                                tiles_now > 0 ? tiles_now : ceil_div(active, kSlotTile) + h->nr - 1, j > 0));
                ++h->launches;
                if (j > 0) {
                    ++h->layer_launches;
                    // three BF16 products of the (n+m) x (n+m) factored layer per active QP
                    h->layer_flops += 2.0 * 3.0 * (double)R * (double)R * (double)active;
                }
                if (timed && j == len - 1) {
                    RQ_CUDA(h, cudaEventRecord(h->prof_ev[prof_used + 1], h->stream));
                    h->prof_span_launches.push_back(len - 1);
                    prof_used += 2;
                }
            }
        } else {
            q.Sin = w.S32 + (size_t)(j & 1) * opart;
            q.Sout = w.S32 + (size_t)((j + 1) & 1) * opart;
            q.CK32 = w.CK32;
            const bool timed32 = h->prof_on && prof_used + 2 <= h->prof_ev.size();
            if (timed32) RQ_CUDA(h, cudaEventRecord(h->prof_ev[prof_used], h->stream));
            RQ_TRY(layer32(h, q, wp, tiles_max, active));
            ++h->launches;
            ++h->layer_launches;
            h->layer_flops += 2.0 * (double)R * (double)R * (double)active;   // one FP32 product per QP
            if (timed32) {
                RQ_CUDA(h, cudaEventRecord(h->prof_ev[prof_used + 1], h->stream));
                h->prof_span_launches.push_back(1);
                prof_used += 2;
            }
        }
    }
    return RELU_QP_OK;
}

// Residual products of a check: [P; A] x, then A^T lam_std (Eqs. primal, dual).
// tiles_now: slot tiles in use when the host knows them (> 0), else a bound
// from the active QP count is used.
int run_check(relu_qp_t h, const BatchParams& p, int active, int tiles_now) {
    BatchWork& w = h->bw;
    const int tiles_max = w.slots / kSlotTile;
    BatchParams q = p;
    if (w.prec == RELU_QP_PREC_BF16X3 && w.check_tc) {
        q.CK = static_cast<__nv_bfloat16*>(w.CK);
        const int active_tiles =
            tiles_now > 0 ? tiles_now : std::min(tiles_max, ceil_div(active, kSlotTile) + h->nr - 1);
        RQ_TRY(tc_check(h, q, 1, tiles_max, active_tiles));
        RQ_TRY(tc_check(h, q, 2, tiles_max, active_tiles));
    } else {
        q.CK32 = w.CK32;
        RQ_TRY(check32(h, q, w.Wc32, tiles_max, active, 1));
        RQ_TRY(check32(h, q, w.Wc32, tiles_max, active, 2));
    }
    h->launches += 2;
    return RELU_QP_OK;
}

int nearest_rho(relu_qp_t h, double rho) {
    int best = 0;
    double bd = 1e300;
    for (int k = 0; k < h->nr; ++k) {
        const double d = std::fabs(std::log(rho) - std::log(h->bank[k]));
        if (d < bd) { bd = d; best = k; }
    }
    return best;
}

int batch_solve(relu_qp_t h, int B, const float* Xw, const float* Lw, const int* rw, double eps_abs,
                double eps_rel, int max_iter, float* Xo, float* Zo, float* Lo, relu_qp_info* infos) {
    BatchWork& w = h->bw;
    const int n = h->n, m = h->m, R = h->R;
    const bool bf16 = w.prec == RELU_QP_PREC_BF16X3;
    BatchParams p = base_params(h);
    const int tiles_max = w.slots / kSlotTile;
    // ---- start state ----
    const int rho0 = nearest_rho(h, h->opts.rho0);
    h->prof_span_launches.clear();
    int* rw_dev = nullptr;
    if (rw) {
        RQ_CUDA(h, cudaMemcpyAsync(w.iters, rw, sizeof(int) * B, cudaMemcpyDefault, h->stream));
        rw_dev = w.iters;   // staged; batch_init copies it into rho_idx before resetting iters
    }
    // scaled handles: warm starts xb = x / D, lamb = c lam / E
    if (Xw) {
        RQ_TRY(copy_rows_in(h, w.Y, w.ldn, Xw, B, n));
        RQ_TRY(scale_rows(h, w.Y, B, n, w.ldn, h->sc_xi));
        if (m > 0) RQ_TRY(sgemm_nt(h, B, m, n, w.Y, w.ldn, h->A32, (int)round_up(n, 4), 1.f, nullptr, w.AY, w.ldm));
    }
    if (Lw && m > 0) {
        RQ_TRY(copy_rows_in(h, w.LSTD, w.ldm, Lw, B, m));
        RQ_TRY(scale_rows(h, w.LSTD, B, m, w.ldm, h->sc_li));
    }
    RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
    batch_init_kernel<<<ceil_div(w.cap * 32, 256), 256, 0, h->stream>>>(p, B, Xw != nullptr, Lw != nullptr && m > 0,
                                                                        rw_dev, rho0, w.status, w.rho_idx, w.iters,
                                                                        w.nsw);
    RQ_CUDA(h, cudaGetLastError());
    ++h->launches;
    RQ_TRY(regroup_slots(h, p, B, true));
    if (bf16) RQ_CUDA(h, cudaMemsetAsync(w.counters + CNT_ERR, 0, 2 * sizeof(int), h->stream));
    const int ci = h->opts.check_interval;
    const int chunk = ci > 0 ? ci : 25;
    int it = 0;
    int active = B;              // QPs in the batch (known to the host after each check)
    // slot tiles in use: exact at a cold start (every QP in the starting bank entry's
    // group) and after each check, an upper bound after a warm start
    int tiles_now = rw ? std::min(tiles_max, ceil_div(B, kSlotTile) + h->nr - 1) : ceil_div(B, kSlotTile);
    size_t prof_used = 0, gap_used = 0;
    bool tail_used = false;
    bool first_done = false;     // the chunk's first layer was enqueued before the host's read-back
    while (it < max_iter) {
        const int len = std::min(chunk, max_iter - it);
        const bool last_chunk = it + len == max_iter;
        const bool check = (ci > 0 && (it + len) % ci == 0) || last_chunk;
        RQ_TRY(run_layers(h, p, len, check, active, tiles_now, prof_used, first_done ? 1 : 0));
        first_done = false;
        it += len;
        if (check) {
            RQ_TRY(run_check(h, p, active, tiles_now));
            DecideArgs d{B, it, last_chunk ? 1 : 0, h->opts.adaptive_rho, eps_abs, eps_rel, w.XO, w.ZO, w.LO,
                         w.status, w.iters, w.rho_idx, w.nsw, w.rp, w.rd, 0, max_iter, nullptr, nullptr};
            // the active QPs are the ones in the slots of the last regroup: one block per slot
            const bool by_slot = tiles_now > 0 && tiles_now * kSlotTile < B;
            batch_decide_kernel<<<by_slot ? tiles_now * kSlotTile : B, kDecideThreads, 0, h->stream>>>(
                p, d, by_slot ? 1 : 0);
            RQ_CUDA(h, cudaGetLastError());
            ++h->launches;
        }
        if (last_chunk) break;
        RQ_TRY(regroup_slots(h, p, B, check));
        if (check) {
            // the host needs the active QP and slot-tile counts of the regroup (they choose
            // the next chunk's kernel); the copy is waited for through an event, and in the
            // split form the next chunk's first (accurate) layer is enqueued before the
            // wait, so that the GPU works during the round trip.  That layer stores only
            // chunk-local data (c, s_ref, r, the operand), never x, Ax, z or lam', so nothing
            // depends on it if the host then stops or hands the last QPs to the tail kernel.
            RQ_CUDA(h, cudaMemcpyAsync(w.cnt_host, w.counters, sizeof(int) * CNT_WORDS, cudaMemcpyDeviceToHost,
                                       h->stream));
            RQ_CUDA(h, cudaEventRecord(w.ev_cnt, h->stream));
            const int nlen = std::min(chunk, max_iter - it);
            if (bf16 && nlen > 1) {
                const bool ncheck = (ci > 0 && (it + nlen) % ci == 0) || it + nlen == max_iter;
                RQ_TRY(run_layers(h, p, nlen, ncheck, active, tiles_now, prof_used, 0, 1));
                first_done = true;
            }
            // profiling: how long the GPU then waits for the host
            const bool gap = h->prof_on && gap_used + 2 <= h->gap_ev.size();
            if (gap) RQ_CUDA(h, cudaEventRecord(h->gap_ev[gap_used], h->stream));
            RQ_CUDA(h, cudaEventSynchronize(w.ev_cnt));
            if (gap) {
                RQ_CUDA(h, cudaEventRecord(h->gap_ev[gap_used + 1], h->stream));
                gap_used += 2;
            }
            int cnt[CNT_WORDS];
            std::memcpy(cnt, w.cnt_host, sizeof(cnt));
            if (cnt[CNT_ERR]) break;     // reported below
            if (cnt[CNT_ACTIVE] == 0) break;
            active = cnt[CNT_ACTIVE];
            tiles_now = cnt[CNT_TILES];
            if (active <= kTailMax && w.tail_grid > 0) {
                // the few QPs left finish in one cooperative launch
                DecideArgs d{B, it, 0, h->opts.adaptive_rho, eps_abs, eps_rel, w.XO, w.ZO, w.LO, w.status, w.iters,
                             w.rho_idx, w.nsw, w.rp, w.rd, 0, max_iter, nullptr, nullptr};
                RQ_TRY(batch_tail(h, p, d, active, it, max_iter));
                tail_used = true;
                break;
            }
        }
    }
    RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    if (bf16) {
        const int e = tc_error(h);
        if (e == RELU_QP_ERR_TIMEOUT) return fail(h, e, "a tensor-core kernel wait passed its deadline");
        if (e) return fail(h, RELU_QP_ERR_CUDA, "a tensor-core kernel found a launch shape it cannot run");
    }
    if (tail_used && batch_tail_error(h))
        return fail(h, RELU_QP_ERR_TIMEOUT, "a grid barrier of the convergence-tail kernel passed its deadline");
    for (size_t e = 0; e + 1 < prof_used; e += 2) {
        float ms = 0.f;
        RQ_CUDA(h, cudaEventElapsedTime(&ms, h->prof_ev[e], h->prof_ev[e + 1]));
        h->layer_ms += ms;
        h->layer_timed += h->prof_span_launches[e / 2];
    }
    h->prof_span_launches.clear();
    for (size_t e = 0; e + 1 < gap_used; e += 2) {
        float ms = 0.f;
        RQ_CUDA(h, cudaEventElapsedTime(&ms, h->gap_ev[e], h->gap_ev[e + 1]));
        h->host_gap_ms += ms;
        ++h->host_checks;
    }
    // ---- outputs (scaled handles: x = D xb, z = zb / E, lam = E lamb / c) ----
    RQ_TRY(scale_rows(h, w.XO, B, n, n, h->sc_x));
    if (Zo && m > 0) RQ_TRY(scale_rows(h, w.ZO, B, m, m, h->sc_z));
    if (Lo && m > 0) RQ_TRY(scale_rows(h, w.LO, B, m, m, h->sc_l));
    RQ_CUDA(h, cudaMemcpyAsync(Xo, w.XO, sizeof(float) * B * n, cudaMemcpyDefault, h->stream));
    if (Zo && m > 0) RQ_CUDA(h, cudaMemcpyAsync(Zo, w.ZO, sizeof(float) * B * m, cudaMemcpyDefault, h->stream));
    if (Lo && m > 0) RQ_CUDA(h, cudaMemcpyAsync(Lo, w.LO, sizeof(float) * B * m, cudaMemcpyDefault, h->stream));
    if (infos) {
        std::vector<int> st(B), itv(B), ri(B), sw(B);
        std::vector<float> rp(B), rd(B);
        RQ_CUDA(h, cudaMemcpyAsync(st.data(), w.status, sizeof(int) * B, cudaMemcpyDeviceToHost, h->stream));
        RQ_CUDA(h, cudaMemcpyAsync(itv.data(), w.iters, sizeof(int) * B, cudaMemcpyDeviceToHost, h->stream));
        RQ_CUDA(h, cudaMemcpyAsync(ri.data(), w.rho_idx, sizeof(int) * B, cudaMemcpyDeviceToHost, h->stream));
        RQ_CUDA(h, cudaMemcpyAsync(sw.data(), w.nsw, sizeof(int) * B, cudaMemcpyDeviceToHost, h->stream));
        RQ_CUDA(h, cudaMemcpyAsync(rp.data(), w.rp, sizeof(float) * B, cudaMemcpyDeviceToHost, h->stream));
        RQ_CUDA(h, cudaMemcpyAsync(rd.data(), w.rd, sizeof(float) * B, cudaMemcpyDeviceToHost, h->stream));
        RQ_CUDA(h, cudaStreamSynchronize(h->stream));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        for (int b = 0; b < B; ++b) {
            infos[b].status = st[b];
            infos[b].iters = itv[b];
            infos[b].rho_index = ri[b];
            infos[b].rho_switches = sw[b];
            infos[b].r_prim = rp[b];
            infos[b].r_dual = rd[b];
            infos[b].solve_ms = ms;
        }
    }
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return RELU_QP_OK;
}

}  // namespace rq

// ===========================================================================
// Continuous batching (serving).  A server holds several problem families,
// each a handle with its own layer bank and batch slots.  Requests (a new
// initial state x0 for one client of one family) wait in a host queue; at
// every step each family admits waiting requests into its free QP slots
// (parametric update of q, l, u, b and a warm start from the client's last
// solution, kept on the device), runs one chunk (check_interval layers, the
// residual check, the stop test and penalty rule) on its own stream, and
// retires the QPs that finished.  Families' chunks overlap on the GPU.
// ===========================================================================
namespace rq {

namespace {

struct ServeDev {
    int *idx = nullptr, *cl = nullptr, *client_of = nullptr, *done = nullptr, *cnt = nullptr;
    float *x0c = nullptr, *Qc = nullptr, *Lc = nullptr, *Uc = nullptr, *Bc = nullptr, *AYc = nullptr, *Xc = nullptr;
    float *out = nullptr;
    float *Wx = nullptr, *Wl = nullptr;
    int *Wr = nullptr, *Wv = nullptr;
};

// Admitted request j goes to QP index idx[j]: warm start from its client's
// last solution (x, lam_std, rho index) if there is one, else cold.
__global__ void serve_admit_kernel(BatchParams p, int k, const int* __restrict__ idx, const int* __restrict__ cl,
                                   const float* __restrict__ Wx, const float* __restrict__ Wl,
                                   const int* __restrict__ Wr, const int* __restrict__ Wv, int rho0, int* status,
                                   int* rho_idx, int* iters, int* nsw, int* client_of, float* Xc) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= k) return;
    const int qp = idx[j], c = cl[j];
    const bool warm = c >= 0 && Wv[c] != 0;
    for (int t = lane; t < p.n; t += 32) {
        const float v = warm ? Wx[(size_t)c * p.ldn + t] : 0.f;
        p.Y[(size_t)qp * p.ldn + t] = v;
        Xc[(size_t)j * p.ldn + t] = v;
    }
    for (int i = lane; i < p.m; i += 32) p.LAM[(size_t)qp * p.ldm + i] = warm ? Wl[(size_t)c * p.ldm + i] : 0.f;
    if (lane == 0) {
        status[qp] = QP_ACTIVE;
        rho_idx[qp] = warm ? Wr[c] : rho0;
        iters[qp] = 0;
        nsw[qp] = 0;
        client_of[qp] = c;
    }
    if (lane < RW_WORDS) p.RED[(size_t)qp * RW_WORDS + lane] = 0u;
}

// Compact rows of the admitted requests -> their QP rows (q, l, u, every b_r,
// and z = A x for the warm start, which also seeds the carried A x).
__global__ void serve_scatter_kernel(BatchParams p, int k, const int* __restrict__ idx, const float* __restrict__ Qc,
                                     const float* __restrict__ Lc, const float* __restrict__ Uc,
                                     const float* __restrict__ Bc, const float* __restrict__ AYc, float* Q, float* L,
                                     float* U, float* BIAS, float* QN) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= k) return;
    const int qp = idx[j];
    float qn = 0.f;
    for (int t = lane; t < p.n; t += 32) {
        const float v = Qc[(size_t)j * p.ldn + t];
        Q[(size_t)qp * p.ldn + t] = v;
        qn = fmaxf(qn, fabsf(p.rsx ? v * p.rsx[t] : v));   // |q|_inf of the original problem
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qn = fmaxf(qn, __shfl_xor_sync(0xffffffffu, qn, o));
    if (lane == 0) QN[qp] = qn;
    for (int i = lane; i < p.m; i += 32) {
        const size_t o = (size_t)qp * p.ldm + i, oc = (size_t)j * p.ldm + i;
        L[o] = Lc[oc];
        U[o] = Uc[oc];
        p.AY[o] = AYc[oc];
        p.Z[o] = AYc[oc];
    }
    for (int r = 0; r < p.nr; ++r)
        for (int t = lane; t < p.R; t += 32)
            BIAS[((size_t)r * p.cap + qp) * p.ldR + t] = Bc[((size_t)r * p.cap + j) * p.ldR + t];
}

// Finished QPs: pack [x | qp, status, iters, rho, switches, r_prim, r_dual] per
// result, store the client's warm start, free the QP index.
__global__ void serve_gather_kernel(BatchParams p, const int* __restrict__ done, const int* __restrict__ cnt,
                                    const int* __restrict__ client_of, int* status, const int* __restrict__ iters,
                                    const int* __restrict__ rho_idx, const int* __restrict__ nsw,
                                    const float* __restrict__ rp, const float* __restrict__ rd,
                                    const float* __restrict__ XO, const float* __restrict__ sx, float* Wx, float* Wl,
                                    int* Wr, int* Wv, float* out, int ldo) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= *cnt) return;
    const int qp = done[j];
    const int c = client_of[qp];
    float* o = out + (size_t)j * ldo;
    // x of the original problem (x = D xb when scaled); the client's warm start stays scaled
    for (int t = lane; t < p.n; t += 32) o[t] = sx ? XO[(size_t)qp * p.n + t] * sx[t] : XO[(size_t)qp * p.n + t];
    if (c >= 0) {
        for (int t = lane; t < p.n; t += 32) Wx[(size_t)c * p.ldn + t] = p.Y[(size_t)qp * p.ldn + t];
        for (int i = lane; i < p.m; i += 32) Wl[(size_t)c * p.ldm + i] = p.LSTD[(size_t)qp * p.ldm + i];
    }
    if (lane == 0) {
        o[p.n + 0] = __int_as_float(qp);
        o[p.n + 1] = __int_as_float(status[qp]);
        o[p.n + 2] = __int_as_float(iters[qp]);
        o[p.n + 3] = __int_as_float(rho_idx[qp]);
        o[p.n + 4] = __int_as_float(nsw[qp]);
        o[p.n + 5] = rp[qp];
        o[p.n + 6] = rd[qp];
        if (c >= 0) {
            Wr[c] = rho_idx[qp];
            Wv[c] = 1;
        }
        status[qp] = QP_UNUSED;
    }
}

}  // namespace

struct ServeRequest {
    int client;
    long long tag;
    double t_submit;
    std::vector<float> x0;
};

struct ServeFamily {
    relu_qp_t h = nullptr;
    cudaStream_t stream = nullptr, saved_stream = nullptr;
    int cap = 0, clients = 0, active = 0, ldo = 0, rho0 = 0;
    std::deque<ServeRequest> queue;
    std::vector<int> free_idx;
    std::vector<long long> tag_of;
    std::vector<double> t_submit_of;
    std::vector<int> client_of;
    ServeDev d;
    float* h_x0c = nullptr;
    int *h_idx = nullptr, *h_cl = nullptr, *h_cnt = nullptr;
    float* h_out = nullptr;
    cudaEvent_t ev = nullptr;
    bool launched = false;
    std::vector<void*> dev_allocs, host_allocs;
    size_t dev_bytes = 0;          // the server's device buffers for this family
    size_t slot_bytes = 0;         // device bytes charged per admitted request
};

struct ServeResult {
    relu_qp_result r;
    std::vector<float> x;
};

}  // namespace rq

struct relu_qp_server_s {
    std::vector<rq::ServeFamily> fam;
    std::deque<rq::ServeResult> results;
    long long budget = 0;          // device-memory budget (0: slots only)
    size_t fixed = 0;              // every family's bank and fixed buffers
    size_t in_use = 0;             // bytes charged by the requests in slots
    double eps_abs = 1e-3, eps_rel = 0.0;
    int max_iter = 4000;
    std::chrono::steady_clock::time_point t0;
    std::string err;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace rq {

namespace {

int sfail(relu_qp_server_t s, int code, const std::string& msg) {
    s->err = msg;
    return code;
}

template <typename T>
int sdev(relu_qp_server_t s, ServeFamily& f, T** p, size_t count) {
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(s, RELU_QP_ERR_OOM, std::string("server device buffer: ") + cudaGetErrorString(e));
    }
    cudaMemset(q, 0, count * sizeof(T) + 16);
    f.dev_allocs.push_back(q);
    f.dev_bytes += count * sizeof(T) + 16;
    *p = static_cast<T*>(q);
    return RELU_QP_OK;
}

template <typename T>
int shost(relu_qp_server_t s, ServeFamily& f, T** p, size_t count) {
    void* q = nullptr;
    const cudaError_t e = cudaMallocHost(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(s, RELU_QP_ERR_OOM, std::string("server pinned buffer: ") + cudaGetErrorString(e));
    }
    f.host_allocs.push_back(q);
    *p = static_cast<T*>(q);
    return RELU_QP_OK;
}

#define RQ_SCUDA(s, call)                                                                        \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            return sfail((s), RELU_QP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                        \
    } while (0)

int family_launch(relu_qp_server_t s, ServeFamily& f) {
    relu_qp_t h = f.h;
    BatchWork& w = h->bw;
    const int n = h->n, m = h->m, R = h->R, nx = w.nx;
    BatchParams p = base_params(h);
    // ---- admission: a free slot, and (with a budget) room for the request's
    // slot bytes that no older waiting request of another family needs ----
    int k = (int)std::min(f.queue.size(), f.free_idx.size());
    if (s->budget > 0 && k > 0) {
        const size_t room = (size_t)s->budget - s->fixed;
        // the oldest request waiting in another family that has a free slot
        double t_old = 1e300;
        size_t b_old = 0;
        for (const auto& g : s->fam) {
            if (&g == &f || g.queue.empty() || g.free_idx.empty()) continue;
            if (g.queue.front().t_submit < t_old) {
                t_old = g.queue.front().t_submit;
                b_old = g.slot_bytes;
            }
        }
        int fit = 0;
        size_t used = s->in_use;
        while (fit < k) {
            const size_t need = used + f.slot_bytes + (f.queue[fit].t_submit > t_old ? b_old : 0);
            if (need > room) break;
            used += f.slot_bytes;
            ++fit;
        }
        k = fit;
    }
    if (k > 0) {
        s->in_use += (size_t)k * f.slot_bytes;
        for (int j = 0; j < k; ++j) {
            ServeRequest rq_ = std::move(f.queue.front());
            f.queue.pop_front();
            const int qp = f.free_idx.back();
            f.free_idx.pop_back();
            f.h_idx[j] = qp;
            f.h_cl[j] = rq_.client;
            std::memcpy(f.h_x0c + (size_t)j * w.ldx, rq_.x0.data(), sizeof(float) * nx);
            f.tag_of[qp] = rq_.tag;
            f.t_submit_of[qp] = rq_.t_submit;
            f.client_of[qp] = rq_.client;
        }
        f.active += k;
        RQ_SCUDA(s, cudaMemcpyAsync(f.d.x0c, f.h_x0c, sizeof(float) * k * w.ldx, cudaMemcpyHostToDevice, f.stream));
        RQ_SCUDA(s, cudaMemcpyAsync(f.d.idx, f.h_idx, sizeof(int) * k, cudaMemcpyHostToDevice, f.stream));
        RQ_SCUDA(s, cudaMemcpyAsync(f.d.cl, f.h_cl, sizeof(int) * k, cudaMemcpyHostToDevice, f.stream));
        serve_admit_kernel<<<ceil_div(k * 32, 256), 256, 0, f.stream>>>(p, k, f.d.idx, f.d.cl, f.d.Wx, f.d.Wl, f.d.Wr,
                                                                       f.d.Wv, f.rho0, w.status, w.rho_idx, w.iters,
                                                                       w.nsw, f.d.client_of, f.d.Xc);
        RQ_SCUDA(s, cudaGetLastError());
        ++h->launches;
        RQ_TRY(sgemm_nt(h, k, n, nx, f.d.x0c, w.ldx, w.F32, w.ldx, 1.f, nullptr, f.d.Qc, w.ldn));
        if (m > 0) {
            RQ_TRY(sgemm_nt(h, k, m, nx, f.d.x0c, w.ldx, w.E32, w.ldx, -1.f, w.l0, f.d.Lc, w.ldm));
            RQ_TRY(sgemm_nt(h, k, m, nx, f.d.x0c, w.ldx, w.E32, w.ldx, -1.f, w.u0, f.d.Uc, w.ldm));
            RQ_TRY(sgemm_nt(h, k, m, n, f.d.Xc, w.ldn, h->A32, (int)round_up(n, 4), 1.f, nullptr, f.d.AYc, w.ldm));
        }
        for (int r = 0; r < h->nr; ++r)
            RQ_TRY(sgemm_nt(h, k, R, nx, f.d.x0c, w.ldx, w.G[r], w.ldx, 1.f, nullptr,
                            f.d.Bc + (size_t)r * w.cap * w.ldR, w.ldR));
        serve_scatter_kernel<<<ceil_div(k * 32, 256), 256, 0, f.stream>>>(p, k, f.d.idx, f.d.Qc, f.d.Lc, f.d.Uc,
                                                                         f.d.Bc, f.d.AYc, w.Q, w.L, w.U, w.BIAS,
                                                                         w.QN);
        RQ_SCUDA(s, cudaGetLastError());
        ++h->launches;
    }
    if (f.active == 0) return RELU_QP_OK;
    // ---- one chunk ----
    const int ci = h->opts.check_interval;
    size_t prof_used = 0;
    h->prof_span_launches.clear();    // the server does not read the layer events
    RQ_TRY(regroup_slots(h, p, w.cap, true));
    RQ_TRY(run_layers(h, p, ci, true, f.active, 0, prof_used));
    RQ_TRY(run_check(h, p, f.active, 0));
    RQ_SCUDA(s, cudaMemsetAsync(f.d.cnt, 0, sizeof(int), f.stream));
    DecideArgs dd{w.cap, 0, 0, h->opts.adaptive_rho, s->eps_abs, s->eps_rel, w.XO, w.ZO, w.LO,
                  w.status, w.iters, w.rho_idx, w.nsw, w.rp, w.rd, ci, s->max_iter, f.d.done, f.d.cnt};
    batch_decide_kernel<<<w.cap, kDecideThreads, 0, f.stream>>>(p, dd, 0);
    RQ_SCUDA(s, cudaGetLastError());
    serve_gather_kernel<<<ceil_div(w.cap * 32, 256), 256, 0, f.stream>>>(
        p, f.d.done, f.d.cnt, f.d.client_of, w.status, w.iters, w.rho_idx, w.nsw, w.rp, w.rd, w.XO, h->sc_x, f.d.Wx,
        f.d.Wl, f.d.Wr, f.d.Wv, f.d.out, f.ldo);
    RQ_SCUDA(s, cudaGetLastError());
    h->launches += 2;
    RQ_SCUDA(s, cudaMemcpyAsync(f.h_cnt, f.d.cnt, sizeof(int), cudaMemcpyDeviceToHost, f.stream));
    RQ_SCUDA(s, cudaMemcpyAsync(f.h_cnt + 1, w.counters, sizeof(int) * CNT_WORDS, cudaMemcpyDeviceToHost, f.stream));
    RQ_SCUDA(s, cudaMemcpyAsync(f.h_out, f.d.out, sizeof(float) * (size_t)w.cap * f.ldo, cudaMemcpyDeviceToHost,
                                f.stream));
    RQ_SCUDA(s, cudaEventRecord(f.ev, f.stream));
    f.launched = true;
    return RELU_QP_OK;
}

int family_collect(relu_qp_server_t s, ServeFamily& f, int fi) {
    if (!f.launched) return RELU_QP_OK;
    f.launched = false;
    RQ_SCUDA(s, cudaEventSynchronize(f.ev));   // complete already when called from server_step
    const double t = s->now();
    if (f.h_cnt[1 + CNT_ERR]) return sfail(s, RELU_QP_ERR_TIMEOUT, "a tensor-core kernel wait passed its deadline");
    const int cnt = f.h_cnt[0];
    const int n = f.h->n;
    for (int j = 0; j < cnt; ++j) {
        const float* o = f.h_out + (size_t)j * f.ldo;
        ServeResult res;
        const int qp = __float_as_int_host(o[n + 0]);
        res.r.tag = f.tag_of[qp];
        res.r.family = fi;
        res.r.client = f.client_of[qp];
        res.r.status = __float_as_int_host(o[n + 1]);
        res.r.iters = __float_as_int_host(o[n + 2]);
        res.r.rho_index = __float_as_int_host(o[n + 3]);
        res.r.rho_switches = __float_as_int_host(o[n + 4]);
        res.r.r_prim = o[n + 5];
        res.r.r_dual = o[n + 6];
        res.r.t_submit = f.t_submit_of[qp];
        res.r.t_done = t;
        res.x.assign(o, o + n);
        s->results.push_back(std::move(res));
        f.free_idx.push_back(qp);
        --f.active;
        s->in_use -= std::min(s->in_use, f.slot_bytes);
    }
    return RELU_QP_OK;
}

}  // namespace

int server_create(relu_qp_server_t* out, relu_qp_t const* families, int nf, const int* clients, double eps_abs,
                  double eps_rel, int max_iter) {
    relu_qp_server_t s = new (std::nothrow) relu_qp_server_s;
    if (!s) return RELU_QP_ERR_OOM;
    *out = s;
    s->eps_abs = eps_abs;
    s->eps_rel = eps_rel;
    s->max_iter = max_iter;
    s->t0 = std::chrono::steady_clock::now();
    s->fam.resize(nf);
    for (int fi = 0; fi < nf; ++fi) {
        ServeFamily& f = s->fam[fi];
        relu_qp_t h = families[fi];
        BatchWork& w = h->bw;
        f.h = h;
        f.cap = w.cap;
        f.clients = clients ? clients[fi] : 0;
        f.ldo = h->n + 8;
        f.rho0 = nearest_rho(h, h->opts.rho0);
        f.tag_of.assign(f.cap, 0);
        f.t_submit_of.assign(f.cap, 0.0);
        f.client_of.assign(f.cap, -1);
        for (int q = f.cap - 1; q >= 0; --q) f.free_idx.push_back(q);
        // smaller problems get higher stream priorities, so that their short chunks
        // do not queue behind the grids of a family of large problems
        int rank = 0;
        for (int g = 0; g < nf; ++g)
            if (families[g]->R < h->R || (families[g]->R == h->R && g < fi)) ++rank;
        int prio_lo = 0, prio_hi = 0;
        RQ_SCUDA(s, cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        // (numerically lower = higher priority: the smallest family gets prio_hi)
        const int prio = std::min(prio_lo, prio_hi + rank);
        RQ_SCUDA(s, cudaStreamCreateWithPriority(&f.stream, cudaStreamNonBlocking, prio));
        RQ_SCUDA(s, cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming));
        f.saved_stream = h->stream;
        h->stream = f.stream;
        // families share the GPU: no persistent (one-wave, co-resident) chunk kernels
        if (h->bw.tc) tc_disable_chunk(h);
        const size_t cap = f.cap, cl = f.clients > 0 ? f.clients : 1;
        RQ_TRY(sdev(s, f, &f.d.idx, cap));
        RQ_TRY(sdev(s, f, &f.d.cl, cap));
        RQ_TRY(sdev(s, f, &f.d.client_of, cap));
        RQ_TRY(sdev(s, f, &f.d.done, cap));
        RQ_TRY(sdev(s, f, &f.d.cnt, 4));
        RQ_TRY(sdev(s, f, &f.d.x0c, cap * w.ldx));
        RQ_TRY(sdev(s, f, &f.d.Qc, cap * w.ldn));
        RQ_TRY(sdev(s, f, &f.d.Xc, cap * w.ldn));
        RQ_TRY(sdev(s, f, &f.d.Lc, cap * w.ldm));
        RQ_TRY(sdev(s, f, &f.d.Uc, cap * w.ldm));
        RQ_TRY(sdev(s, f, &f.d.AYc, cap * w.ldm));
        RQ_TRY(sdev(s, f, &f.d.Bc, (size_t)h->nr * cap * w.ldR));
        RQ_TRY(sdev(s, f, &f.d.out, cap * f.ldo));
        RQ_TRY(sdev(s, f, &f.d.Wx, cl * w.ldn));
        RQ_TRY(sdev(s, f, &f.d.Wl, cl * w.ldm));
        RQ_TRY(sdev(s, f, &f.d.Wr, cl));
        RQ_TRY(sdev(s, f, &f.d.Wv, cl));
        RQ_TRY(shost(s, f, &f.h_x0c, cap * w.ldx));
        RQ_TRY(shost(s, f, &f.h_idx, cap));
        RQ_TRY(shost(s, f, &f.h_cl, cap));
        RQ_TRY(shost(s, f, &f.h_cnt, 8));
        RQ_TRY(shost(s, f, &f.h_out, cap * f.ldo));
        // every QP index starts free
        batch_init_kernel<<<ceil_div(w.cap * 32, 256), 256, 0, f.stream>>>(base_params(h), 0, 0, 0, nullptr, f.rho0,
                                                                           w.status, w.rho_idx, w.iters, w.nsw);
        RQ_SCUDA(s, cudaGetLastError());
        RQ_SCUDA(s, cudaMemsetAsync(w.counters, 0, sizeof(int) * CNT_WORDS, f.stream));
        RQ_SCUDA(s, cudaStreamSynchronize(f.stream));
        // memory accounting: a request occupies one QP slot of the handle plus its rows of the
        // server's compact buffers (x0, q, x, l, u, A x, b of every bank entry, the result row)
        const size_t fl = sizeof(float);
        const size_t serve_slot = (w.ldx + 2 * w.ldn + 3 * w.ldm + (size_t)h->nr * w.ldR + f.ldo) * fl +
                                  4 * sizeof(int);
        f.slot_bytes = batch_slot_bytes(h) + serve_slot;
        const size_t fam_fixed = h->dev_bytes + f.dev_bytes;
        const size_t fam_slots = (size_t)f.cap * f.slot_bytes;
        s->fixed += fam_fixed > fam_slots ? fam_fixed - fam_slots : 0;
    }
    return RELU_QP_OK;
}

int server_set_budget(relu_qp_server_t s, long long bytes) {
    size_t one = 0;   // room for one request of every family, so that none waits forever
    for (const auto& f : s->fam) one = std::max(one, f.slot_bytes);
    if (bytes > 0 && (size_t)bytes < s->fixed + one)
        return sfail(s, RELU_QP_ERR_OOM, "server budget of " + std::to_string(bytes) + " bytes is below the " +
                                             std::to_string(s->fixed) + " bytes of the families' banks and buffers "
                                             "plus one request of the largest family (" + std::to_string(one) + ")");
    s->budget = bytes;
    return RELU_QP_OK;
}

int server_family_bytes(relu_qp_server_t s, int family, long long* fixed_bytes, long long* slot_bytes) {
    const ServeFamily& f = s->fam[family];
    const size_t all = f.h->dev_bytes + f.dev_bytes, slots = (size_t)f.cap * f.slot_bytes;
    if (fixed_bytes) *fixed_bytes = (long long)(all > slots ? all - slots : 0);
    if (slot_bytes) *slot_bytes = (long long)f.slot_bytes;
    return RELU_QP_OK;
}

long long server_bytes_in_use(relu_qp_server_t s) { return (long long)s->in_use; }

int server_submit(relu_qp_server_t s, int family, int client, const float* x0, long long tag) {
    ServeFamily& f = s->fam[family];
    ServeRequest r;
    r.client = client;
    r.tag = tag;
    r.t_submit = s->now();
    r.x0.assign(x0, x0 + f.h->bw.nx);
    f.queue.push_back(std::move(r));
    return RELU_QP_OK;
}

// Families advance independently: a family with no chunk in flight admits and
// launches; one whose chunk has finished (its event has completed) retires,
// admits and launches again at once.  The call returns once some family has
// finished a chunk (or when no chunk is in flight), so a family of small
// problems is never held back by the chunk of a family of large ones.
int server_step(relu_qp_server_t s, int* active, int* waiting) {
    const size_t nf = s->fam.size();
    for (auto& f : s->fam)
        if (!f.launched) RQ_TRY(family_launch(s, f));
    bool any_in_flight = false;
    for (auto& f : s->fam) any_in_flight = any_in_flight || f.launched;
    bool progressed = !any_in_flight;
    while (!progressed) {
        for (size_t fi = 0; fi < nf; ++fi) {
            ServeFamily& f = s->fam[fi];
            if (!f.launched) continue;
            const cudaError_t q = cudaEventQuery(f.ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                cudaGetLastError();
                return sfail(s, RELU_QP_ERR_CUDA, std::string("server chunk: ") + cudaGetErrorString(q));
            }
            RQ_TRY(family_collect(s, f, (int)fi));
            RQ_TRY(family_launch(s, f));
            progressed = true;
        }
        if (!progressed) std::this_thread::yield();
    }
    int a = 0, q = 0;
    for (auto& f : s->fam) {
        a += f.active;
        q += (int)f.queue.size();
    }
    if (active) *active = a;
    if (waiting) *waiting = q;
    return RELU_QP_OK;
}

int server_poll(relu_qp_server_t s, int max_results, relu_qp_result* results, float* x_out, int x_stride) {
    int k = 0;
    while (k < max_results && !s->results.empty()) {
        ServeResult& r = s->results.front();
        if (results) results[k] = r.r;
        if (x_out) std::memcpy(x_out + (size_t)k * x_stride, r.x.data(), sizeof(float) * r.x.size());
        s->results.pop_front();
        ++k;
    }
    return k;
}

void server_destroy(relu_qp_server_t s) {
    for (auto& f : s->fam) {
        if (f.stream) cudaStreamSynchronize(f.stream);
        if (f.h) f.h->stream = f.saved_stream;
        for (void* p : f.dev_allocs) cudaFree(p);
        for (void* p : f.host_allocs) cudaFreeHost(p);
        if (f.ev) cudaEventDestroy(f.ev);
        if (f.stream) cudaStreamDestroy(f.stream);
    }
    delete s;
}

const char* server_error(relu_qp_server_t s) { return s->err.c_str(); }
int server_families(relu_qp_server_t s) { return (int)s->fam.size(); }
int server_clients(relu_qp_server_t s, int family) { return s->fam[family].clients; }
int server_nx(relu_qp_server_t s, int family) { return s->fam[family].h->bw.nx; }
double server_clock(relu_qp_server_t s) { return s->now(); }

}  // namespace rq
