// Convergence tail of a batched solve: once at most kTailMax QPs are still
// active, one cooperative kernel runs every remaining chunk of Algorithm 1 for
// them (layers, the residual checks of Eqs. primal and dual, the penalty rule
// of Eq. rho_update and the stop test), with grid barriers between the phases
// instead of a few kernel launches per layer and a host round trip per check.
//
// Arithmetic.  The layer and the residual products are FP32 on the CUDA cores
// with exactly the summation order of the tiled FP32 kernels (16-wide k steps
// summed as fresh partials, batch.cu), and the element-wise parts are the same
// functions (layer_elem, check1_elem, check2_elem, decide_qp), so for the FP32
// backend a QP's iterates do not depend on whether it finishes in the tiled
// kernels or here.  In the BF16 split backend the QPs that reach the tail
// continue in FP32 (more accurate than the split products).
//
// Work split of a layer.  CTA b owns a contiguous block of rows of Wt (cached
// in shared memory when they fit).  At the start of a chunk the live tail QPs
// are listed in compact slots, grouped by bank entry, and every layer stages
// only their operand vectors in shared memory, with every 16-float step padded
// to 20 floats so that lanes reading consecutive steps spread over the banks.
// A thread takes one step of kRG rows for all QPs of a group (code specialised
// on the group's size: each Wt value loaded feeds every QP of the group, each
// operand value kRG rows) and writes the step partials to shared memory; then
// one thread per (row, QP) adds that output's partials in step order and
// applies the element-wise part of the layer to state it keeps in registers
// for the whole chunk.  Nothing the kernel indexes at run time lives in local
// memory, which would miss in the small L1 left beside the staged data.  The
// residual products of the checks, spread over all warps of the grid, use a
// warp per row: lane l computes the steps l, l + 32, ... and lane j adds QP j's
// partials in step order.
// Every barrier wait has a deadline after which the kernel records
// RELU_QP_ERR_TIMEOUT and returns.
#include "batch.h"
#include "grid_sync.h"

#include <algorithm>

namespace rq {

namespace {

constexpr int kTailThreads = 384;   // 12 warps
constexpr int kTailWarps = kTailThreads / 32;

struct TailArgs {
    BatchParams p;              // state (QP-indexed rows), bank scalars, CK32 = CKB (Sout, flags unused)
    DecideArgs d;
    const float* W[RQ_MAX_RHO];  // FP32 Wt of every bank entry, rows of ldk floats
    const float* Wc;            // FP32 check matrix [[P, A^T], [A, 0]], rows of ldkc floats
    float* S;                   // operand double buffer [2][kTailMax][ldk]
    float* CKB;                 // check operand [kTailMax][ldkc]
    unsigned* red;              // [3][kTailMax][RW_WORDS] reduction words, rotated per check
    unsigned* bar;              // grid barrier: arrival count of the launch (+ pad word)
    int* err;                   // error word
    const int* qlist;           // [nq] QP ids
    int nq, it0, max_iter, ci;
    int rpc;                    // rows of the layer per CTA (contiguous)
    int pr;                     // rows of the layer product per pass (the step partials of a pass fit the scratch)
    int scratch;                // floats of the scratch region (step partials, the checks' round partials)
    int wcache;                 // 1: the CTA's Wt rows of one bank entry are cached in shared memory
    int regs;                   // 1: one pass, and every (row, QP) output has its own thread (state in registers)
    long long timeout_ns;
};

// Grid-wide barrier over all CTAs of the cooperative launch (grid_sync.h).
__device__ __forceinline__ bool tail_barrier(const TailArgs& a, GridSyncState* s_ok) {
    return grid_sync(a.bar, a.err, a.timeout_ns, s_ok);
}

constexpr int kStep = 16;       // k per partial (the tiled kernels' step)
constexpr int kStepPad = 20;    // floats per staged step (bank spread of 16-byte reads)

// Copy the floats [col0, col0 + cols) (multiples of 16) of every live tail QP's
// row of `src` (row stride ld) into the padded shared layout
// [j][step][kStepPad] (ops floats per QP).  Asynchronous copies (L2 -> shared,
// all in flight at once); the caller's __syncthreads follows the wait here.
__device__ __forceinline__ void stage_rows(float* sm, int ops, const float* src, int ld, int col0, int cols, int nq,
                                           const int* s_live) {
    const int c4 = cols >> 2;
    for (int e = threadIdx.x; e < nq * c4; e += blockDim.x) {
        const int j = e / c4, q = (col0 >> 2) + (e - j * c4);
        if (!s_live[j]) continue;
        const uint32_t d = static_cast<uint32_t>(
            __cvta_generic_to_shared(sm + (size_t)j * ops + (q >> 2) * kStepPad + (q & 3) * 4));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + (size_t)j * ld + 4 * q)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

constexpr int kRB = 1;          // rows per warp pass
constexpr int kPbs = 33;        // stride of a round's partials (32 steps, padded)

// kRB consecutive rows r0 .. r0 + kRB - 1 (< nrows) of a product for every
// live tail QP (warp-cooperative).  Step c of row r (k = 16 c .. 16 c + 15, c in
// [c0, c1)) for QP j is
//   part = FMA chain over k in order, starting at 0        (as fp32_tile)
// and acc_j(r) = sum of the parts in increasing c         (as fp32_tile).
// Rounds of 32 steps: lane l computes step c0 + 32 i + l of every row and QP
// (the rows' Wt values stay in registers across the QPs, each staged operand
// value feeds kRB rows), writes the partials to pb, and lane j adds QP j's
// partials of the round in step order.  acc[i] is valid in lane j < nq.
// wrow(j, r) gives QP j's row r of the matrix; rows of QPs that share the
// same matrix are loaded once.
// A row of a product matrix for one QP: `ptr` addresses step 0 of the row, and
// step c starts at ptr + c * stride (kStep in global memory, kStepPad in the
// shared-memory cache of a CTA's rows).
struct WRowRef {
    const float* ptr;
    int stride;
};

__device__ __forceinline__ float4 load_w4(const WRowRef& w, int c, int t) {
    const float4* q = reinterpret_cast<const float4*>(w.ptr + c * w.stride) + t;
    return w.stride == kStep ? __ldg(q) : *q;
}

template <class WRow>
__device__ __forceinline__ void warp_rows(const float* __restrict__ opnd, int ops, float* pb, int nq,
                                          const int* s_live, int c0, int c1, int r0, int nrows, WRow wrow,
                                          float (&acc)[kRB]) {
    const int lane = threadIdx.x & 31;
    unsigned live = 0;
    for (int j = 0; j < nq; ++j) live |= (s_live[j] ? 1u : 0u) << j;
#pragma unroll
    for (int i = 0; i < kRB; ++i) acc[i] = 0.f;
    for (int cb = c0; cb < c1; cb += 32) {
        const int c = cb + lane;
        unsigned todo = live;
        while (todo) {
            const int j0 = __ffs(todo) - 1;
            const float* w0 = wrow(j0, r0).ptr;
            unsigned same = 0;
            for (int j = j0; j < nq; ++j)
                if (((todo >> j) & 1u) && wrow(j, r0).ptr == w0) same |= 1u << j;
            todo &= ~same;
            if (c < c1) {
                float4 wv[kRB][4];
#pragma unroll
                for (int i = 0; i < kRB; ++i) {
                    const WRowRef wr = wrow(j0, r0 + i);
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        wv[i][t] = r0 + i < nrows ? load_w4(wr, c, t) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                unsigned m = same;
                while (m) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1;
                    const float* xs = opnd + (size_t)j * ops + c * kStepPad;
                    float part[kRB];
#pragma unroll
                    for (int i = 0; i < kRB; ++i) part[i] = 0.f;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const float4 xv = *reinterpret_cast<const float4*>(xs + 4 * t);
#pragma unroll
                        for (int i = 0; i < kRB; ++i) {
                            part[i] = fmaf(xv.x, wv[i][t].x, part[i]);
                            part[i] = fmaf(xv.y, wv[i][t].y, part[i]);
                            part[i] = fmaf(xv.z, wv[i][t].z, part[i]);
                            part[i] = fmaf(xv.w, wv[i][t].w, part[i]);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < kRB; ++i) pb[(i * kTailMax + j) * kPbs + lane] = part[i];
                }
            }
        }
        __syncwarp();
        if (lane < nq && ((live >> lane) & 1u)) {
            const int nc = min(32, c1 - cb);
#pragma unroll
            for (int i = 0; i < kRB; ++i) {
                const float* q = pb + (i * kTailMax + lane) * kPbs;
                if (nc == 32) {
                    // all loads first, then the additions in step order
                    float v[32];
#pragma unroll
                    for (int l = 0; l < 32; ++l) v[l] = q[l];
#pragma unroll
                    for (int l = 0; l < 32; ++l) acc[i] += v[l];
                } else {
                    for (int l = 0; l < nc; ++l) acc[i] += q[l];
                }
            }
        }
        __syncwarp();
    }
}

constexpr int kRG = 4;          // rows of one item of the layer product

// The live tail QPs of a chunk, compacted and grouped by bank entry: compact
// slot k holds tail slot j[k]; group g (QPs reading the same rows of Wt) is
// compact slots [g0[g], g0[g + 1]) with bank entry ri[g].
struct TailList {
    int nl;
    int j[kTailMax];
    int ng;
    int g0[kTailMax + 1];
    int ri[kTailMax];
};

// Copy the operand rows of the live tail QPs (floats [0, cols), a multiple of
// 16, of row j[k] of `src`, row stride ld) into compact slots k of the padded
// shared layout [k][step][kStepPad] (ops floats per slot).  As stage_rows.
__device__ __forceinline__ void stage_list(float* sm, int ops, const float* src, int ld, int cols, const TailList& L) {
    const int c4 = cols >> 2;
    for (int e = threadIdx.x; e < L.nl * c4; e += blockDim.x) {
        const int k = e / c4, q = e - k * c4;
        const uint32_t d = static_cast<uint32_t>(
            __cvta_generic_to_shared(sm + (size_t)k * ops + (q >> 2) * kStepPad + (q & 3) * 4));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + (size_t)L.j[k] * ld + 4 * q)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

// Step partials of the layer product for the CTA's local rows [rl0, rl1) and
// the NL compact slots s0 .. s0 + NL - 1 of one group.  Item (g, c) covers rows
// rl0 + kRG g .. + kRG - 1 and step c (k = 16 c .. 16 c + 15): for each row i
// and slot the FMA chain over k in order, starting at 0 (as fp32_tile), so
// every Wt value loaded feeds the NL QPs and every staged operand value kRG
// rows; NL is a template parameter, so the item's code has no per-QP tests.
// The partial goes to pbuf[((s0 + k) * (rl1 - rl0) + i) * ps + c] (ps odd: the
// owners' in-order sums read without bank conflicts).  Row rl of Wt starts at
// w0 + rl * wr and step c of it at + c * ws: the cached rows in shared memory
// (padded step layout) or the bank entry's rows in global memory, read with
// generic loads.
template <int NL>
__device__ __forceinline__ void group_partials(const float* __restrict__ opnd, int ops, float* pbuf, int ps, int rl0,
                                               int rl1, int nsteps, int s0, const float* w0, size_t wr, int ws) {
    const int npr = rl1 - rl0;
    const int ngr = (npr + kRG - 1) / kRG;
    for (int e = threadIdx.x; e < ngr * nsteps; e += blockDim.x) {
        const int g = e / nsteps, c = e - g * nsteps;
        const int rb = rl0 + g * kRG;
        float part[kRG][NL];
#pragma unroll
        for (int i = 0; i < kRG; ++i)
#pragma unroll
            for (int k = 0; k < NL; ++k) part[i][k] = 0.f;
        const float* wp[kRG];
#pragma unroll
        for (int i = 0; i < kRG; ++i) wp[i] = w0 + (size_t)(rb + i < rl1 ? rb + i : rb) * wr + (size_t)c * ws;
        const float* xs = opnd + (size_t)s0 * ops + c * kStepPad;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float4 wv[kRG];
#pragma unroll
            for (int i = 0; i < kRG; ++i) wv[i] = *(reinterpret_cast<const float4*>(wp[i]) + t);
#pragma unroll
            for (int k = 0; k < NL; ++k) {
                const float4 xv = *reinterpret_cast<const float4*>(xs + (size_t)k * ops + 4 * t);
#pragma unroll
                for (int i = 0; i < kRG; ++i) {
                    part[i][k] = fmaf(xv.x, wv[i].x, part[i][k]);
                    part[i][k] = fmaf(xv.y, wv[i].y, part[i][k]);
                    part[i][k] = fmaf(xv.z, wv[i].z, part[i][k]);
                    part[i][k] = fmaf(xv.w, wv[i].w, part[i][k]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kRG; ++i) {
            if (rb + i >= rl1) break;
#pragma unroll
            for (int k = 0; k < NL; ++k) pbuf[((size_t)(s0 + k) * npr + (rb + i - rl0)) * ps + c] = part[i][k];
        }
    }
}

// group_partials for every group of L.
__device__ __forceinline__ void layer_partials(const float* __restrict__ opnd, int ops, float* pbuf, int ps, int rl0,
                                               int rl1, int nsteps, int row_beg, const TailList& L, int cache_ri,
                                               const float* wc, int wops, const float* const* s_W, int ldk) {
    for (int g = 0; g < L.ng; ++g) {
        const int s0 = L.g0[g], n = L.g0[g + 1] - s0, ri = L.ri[g];
        const bool cached = ri == cache_ri;
        const float* w0 = cached ? wc : s_W[ri] + (size_t)row_beg * ldk;
        const size_t wr = cached ? (size_t)wops : (size_t)ldk;
        const int ws = cached ? kStepPad : kStep;
        switch (n) {
            case 1: group_partials<1>(opnd, ops, pbuf, ps, rl0, rl1, nsteps, s0, w0, wr, ws); break;
            case 2: group_partials<2>(opnd, ops, pbuf, ps, rl0, rl1, nsteps, s0, w0, wr, ws); break;
            case 3: group_partials<3>(opnd, ops, pbuf, ps, rl0, rl1, nsteps, s0, w0, wr, ws); break;
            case 4: group_partials<4>(opnd, ops, pbuf, ps, rl0, rl1, nsteps, s0, w0, wr, ws); break;
            case 5: group_partials<5>(opnd, ops, pbuf, ps, rl0, rl1, nsteps, s0, w0, wr, ws); break;
            case 6: group_partials<6>(opnd, ops, pbuf, ps, rl0, rl1, nsteps, s0, w0, wr, ws); break;
            case 7: group_partials<7>(opnd, ops, pbuf, ps, rl0, rl1, nsteps, s0, w0, wr, ws); break;
            default: group_partials<8>(opnd, ops, pbuf, ps, rl0, rl1, nsteps, s0, w0, wr, ws); break;
        }
    }
}

// Operand of the first layer of a chunk, as batch_fill_kernel: s = [x; 2 rho z - lam'].
__device__ __forceinline__ void tail_fill(const TailArgs& a, float* S, const int* s_live, const int* s_ri) {
    const BatchParams& p = a.p;
    const int total = a.nq * p.ldk;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int j = e / p.ldk, k = e - j * p.ldk;
        if (!s_live[j]) continue;
        const int qp = a.qlist[j], ri = s_ri[j];
        float v = 0.f;
        if (k < p.n) {
            v = p.Y[(size_t)qp * p.ldn + k];
        } else if (k < p.R) {
            const int i = k - p.n;
            const size_t o = (size_t)qp * p.ldm + i;
            v = next_operand(p.rho[ri] * p.rs[i], p.Z[o], p.LAM[o]);
        }
        S[(size_t)j * p.ldk + k] = v;
    }
}

__global__ void __launch_bounds__(kTailThreads, 1) batch_tail_kernel(TailArgs a) {
    extern __shared__ __align__(16) float tsm[];
    __shared__ GridSyncState s_ok;
    __shared__ int s_live[kTailMax], s_ri[kTailMax], s_act[kTailMax], s_nri[kTailMax], s_any;
    grid_sync_init(&s_ok);
    __shared__ unsigned s_red[kTailMax][RW_WORDS];
    // the launch's parameters are read in place: per-layer values (the operand the layer
    // writes, the epilogue flags) are kept in scalars
    const BatchParams& p = a.p;
    const int nq = a.nq;
    const int nsteps = (p.ldk > p.ldkc ? p.ldk : p.ldkc) / kStep;
    const int ops = nsteps * kStepPad;                       // staged floats per QP
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // scratch: the layer's step partials, or each warp's round partials in the checks
    float* pbuf = tsm + (size_t)kTailMax * ops;
    float* pb = pbuf + (size_t)warp * kRB * kTailMax * kPbs;
    // this CTA's rows of the layer, and (a.wcache) their Wt rows of one bank entry in
    // shared memory, in the padded step layout
    const int row_beg = blockIdx.x * a.rpc, row_end = min(p.R, row_beg + a.rpc);
    const int nr = max(0, row_end - row_beg);
    const int lsteps = p.ldk / kStep;                        // k steps of the layer product
    const int ps = lsteps | 1;                               // stride of an output's step partials
    const int wops = lsteps * kStepPad;                      // cached floats per row
    float* wc = pbuf + a.scratch;
    __shared__ TailList s_L;
    __shared__ const float* s_W[RQ_MAX_RHO];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int r = 0; r < RQ_MAX_RHO; ++r) s_W[r] = a.W[r];
    }
    int cache_ri = -1;
    const int gwarp = blockIdx.x * (kTailThreads / 32) + warp, nwarps = gridDim.x * (kTailThreads / 32);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    if (threadIdx.x < kTailMax) {
        const int j = threadIdx.x;
        s_live[j] = j < nq ? 1 : 0;
        s_ri[j] = j < nq ? a.d.rho_idx[a.qlist[j]] : 0;
    }
    __syncthreads();
    int cur = 0, checks = 0, it = a.it0;
    tail_fill(a, a.S, s_live, s_ri);
    if (!tail_barrier(a, &s_ok)) return;
    const int chunk = a.ci > 0 ? a.ci : 25;
    while (it < a.max_iter) {
        const int len = min(chunk, a.max_iter - it);
        const bool last_chunk = it + len == a.max_iter;
        const bool check = (a.ci > 0 && (it + len) % a.ci == 0) || last_chunk;
        // ---------------- len layers ----------------
        if (a.wcache) {
            // cache the rows of the bank entry of the first live QP (constant data)
            int ri0 = -1;
            for (int j = 0; j < nq && ri0 < 0; ++j)
                if (s_live[j]) ri0 = s_ri[j];
            if (ri0 >= 0 && ri0 != cache_ri) {
                const int c4 = p.ldk >> 2;
                for (int e = threadIdx.x; e < (row_end - row_beg) * c4; e += blockDim.x) {
                    const int rr = e / c4, q = e - rr * c4;
                    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(
                        wc + (size_t)rr * wops + (q >> 2) * kStepPad + (q & 3) * 4));
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d),
                                 "l"(s_W[ri0] + (size_t)(row_beg + rr) * p.ldk + 4 * q)
                                 : "memory");
                }
                asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
                __syncthreads();
                cache_ri = ri0;
            }
        }
        // the live QPs, compacted and grouped by bank entry, for the layer product
        if (threadIdx.x == 0) {
            TailList L{};
            for (int j = 0; j < nq; ++j) {
                if (!s_live[j]) continue;
                int g = 0;
                while (g < L.ng && L.ri[g] != s_ri[j]) ++g;
                if (g == L.ng) L.ri[L.ng++] = s_ri[j];
            }
            for (int g = 0; g < L.ng; ++g) {
                L.g0[g] = L.nl;
                for (int j = 0; j < nq; ++j)
                    if (s_live[j] && s_ri[j] == L.ri[g]) L.j[L.nl++] = j;
            }
            L.g0[L.ng] = L.nl;
            s_L = L;
        }
        __syncthreads();
        const TailList& L = s_L;
        const int nl = L.nl;
        // a.regs: thread o owns output (row row_beg + o % nr, compact slot o / nr); its state
        // (bias of the QP's bank entry, and for rows of A x the carried A x, z, lam', l, u,
        // rho_i) stays in registers for the chunk: loaded here, written back at the chunk's
        // last layer (the checks, the decision and the next chunk's fill read it from memory)
        const int ok = nr > 0 ? (int)threadIdx.x / nr : kTailMax, orl = nr > 0 ? (int)threadIdx.x % nr : 0;
        const bool own = a.regs && ok < nl;
        const int oj = own ? L.j[ok] : 0;
        const int o_qp = own ? a.qlist[oj] : 0, o_ri = own ? s_ri[oj] : 0, o_r = row_beg + orl;
        float rb = 0.f, ray = 0.f, rz = 0.f, rlam = 0.f, rlo = 0.f, rup = 0.f, rrho = 0.f;
        if (own) {
            rb = p.BIAS[((size_t)o_ri * p.cap + o_qp) * p.ldR + o_r];
            if (o_r >= p.n) {
                const size_t o = (size_t)o_qp * p.ldm + (o_r - p.n);
                ray = p.AY[o];
                rz = p.Z[o];
                rlam = p.LAM[o];
                rlo = p.L[o];
                rup = p.U[o];
                rrho = p.rho[o_ri] * p.rs[o_r - p.n];
            }
        }
        for (int jl = 0; jl < len; ++jl) {
            const float* Sc = a.S + (size_t)cur * kTailMax * p.ldk;
            float* Sout = a.S + (size_t)(cur ^ 1) * kTailMax * p.ldk;
            const bool last = jl == len - 1;
            stage_list(tsm, ops, Sc, p.ldk, p.ldk, L);
            __syncthreads();
            for (int rl0 = 0; rl0 < nr; rl0 += a.pr) {
                const int rl1 = min(nr, rl0 + a.pr), npr = rl1 - rl0;
                if (rl0 > 0) __syncthreads();   // the previous pass's sums have read pbuf
                layer_partials(tsm, ops, pbuf, ps, rl0, rl1, lsteps, row_beg, L, cache_ri, wc, wops, s_W, p.ldk);
                __syncthreads();
                // every output's partials added in step order (as fp32_tile), then the layer's
                // element-wise part
                for (int o = threadIdx.x; o < nl * npr; o += blockDim.x) {
                    const int k = o / npr, r = row_beg + rl0 + (o - k * npr), j = L.j[k];
                    const float* q = pbuf + (size_t)o * ps;
                    float acc = 0.f;
                    int c = 0;
                    for (; c + 20 <= lsteps; c += 20) {
                        // loads first, then the additions in step order
                        float v[20];
#pragma unroll
                        for (int u = 0; u < 20; ++u) v[u] = q[c + u];
#pragma unroll
                        for (int u = 0; u < 20; ++u) acc += v[u];
                    }
                    for (; c < lsteps; ++c) acc += q[c];
                    if (!a.regs) {
                        BatchParams q = p;
                        q.Sout = Sout;
                        q.flags = last ? (EPI_LAST | (check ? EPI_CHECK : 0u)) : 0u;
                        layer_elem(q, j, a.qlist[j], s_ri[j], r, acc);
                        continue;
                    }
                    // the FP32 layer of layer_elem on register state (o == threadIdx.x here)
                    const float t = acc + rb;
                    float s_new;
                    if (r < p.n) {
                        s_new = t;
                        if (last) {
                            p.Y[(size_t)o_qp * p.ldn + r] = t;
                            if (check) put_check(p, j, r, t);
                        }
                    } else {
                        float zn, ln;
                        const float rr = ax_row_carry(ray, rz, rlam, rrho);
                        ax_row_update(t, rr, rlo, rup, rrho, zn, ln, s_new);
                        ray = t;
                        rz = zn;
                        rlam = ln;
                        if (last) {
                            const size_t oo = (size_t)o_qp * p.ldm + (r - p.n);
                            p.AY[oo] = t;
                            p.Z[oo] = zn;
                            p.LAM[oo] = ln;
                        }
                    }
                    if (!last) Sout[(size_t)j * p.ldk + r] = s_new;
                }
            }
            cur ^= 1;
            if (!tail_barrier(a, &s_ok)) return;
        }
        it += len;
        if (check) {
            unsigned* slot = a.red + (size_t)(checks % 3) * kTailMax * RW_WORDS;
            if (blockIdx.x == 0)
                for (int e = threadIdx.x; e < kTailMax * RW_WORDS; e += blockDim.x)
                    a.red[(size_t)((checks + 1) % 3) * kTailMax * RW_WORDS + e] = 0u;
            ++checks;
            // phase 1: [P; A] x over the x columns of the check operand
            for (int e = threadIdx.x; e < kTailMax * RW_WORDS; e += blockDim.x) (&s_red[0][0])[e] = 0u;
            stage_rows(tsm, ops, a.CKB, p.ldkc, 0, p.n64, nq, s_live);
            __syncthreads();
            {
                float rp = 0.f, nax = 0.f, nz = 0.f, npx = 0.f;
                for (int r0 = gwarp * kRB; r0 < p.n + p.m; r0 += nwarps * kRB) {
                    float acc[kRB];
                    warp_rows(tsm, ops, pb, nq, s_live, 0, p.n64 / kStep, r0, p.n + p.m,
                              [&](int, int r) { return WRowRef{a.Wc + (size_t)r * p.ldkc, kStep}; }, acc);
                    if (lane < nq && s_live[lane])
#pragma unroll
                        for (int i = 0; i < kRB; ++i)
                            if (r0 + i < p.n + p.m)
                                check1_elem(p, lane, a.qlist[lane], s_ri[lane], r0 + i, acc[i], rp, nax, nz, npx);
                }
                if (lane < nq && s_live[lane]) {
                    atomicMax(&s_red[lane][RW_RP], __float_as_uint(fabsf(rp)));
                    atomicMax(&s_red[lane][RW_AX], __float_as_uint(fabsf(nax)));
                    atomicMax(&s_red[lane][RW_Z], __float_as_uint(fabsf(nz)));
                    atomicMax(&s_red[lane][RW_PX], __float_as_uint(fabsf(npx)));
                }
            }
            __syncthreads();
            for (int e = threadIdx.x; e < nq * RW_WORDS; e += blockDim.x)
                if ((&s_red[0][0])[e]) atomicMax(slot + e, (&s_red[0][0])[e]);
            if (!tail_barrier(a, &s_ok)) return;
            // phase 2: A^T lam_std over the multiplier columns
            for (int e = threadIdx.x; e < kTailMax * RW_WORDS; e += blockDim.x) (&s_red[0][0])[e] = 0u;
            stage_rows(tsm, ops, a.CKB, p.ldkc, p.n64, p.ldkc - p.n64, nq, s_live);
            __syncthreads();
            {
                float rd = 0.f, natl = 0.f;
                for (int r0 = gwarp * kRB; r0 < p.n; r0 += nwarps * kRB) {
                    float acc[kRB];
                    warp_rows(tsm, ops, pb, nq, s_live, p.n64 / kStep, p.ldkc / kStep, r0, p.n,
                              [&](int, int r) { return WRowRef{a.Wc + (size_t)r * p.ldkc, kStep}; }, acc);
                    if (lane < nq && s_live[lane])
#pragma unroll
                        for (int i = 0; i < kRB; ++i)
                            if (r0 + i < p.n) check2_elem(p, a.qlist[lane], r0 + i, acc[i], rd, natl);
                }
                if (lane < nq && s_live[lane]) {
                    atomicMax(&s_red[lane][RW_RD], __float_as_uint(fabsf(rd)));
                    atomicMax(&s_red[lane][RW_ATL], __float_as_uint(fabsf(natl)));
                }
            }
            __syncthreads();
            for (int e = threadIdx.x; e < nq * RW_WORDS; e += blockDim.x)
                if ((&s_red[0][0])[e]) atomicMax(slot + e, (&s_red[0][0])[e]);
            if (!tail_barrier(a, &s_ok)) return;
            // decision: every CTA reaches the same one; CTA 0 writes the per-QP records
            if (threadIdx.x < nq) {
                const int j = threadIdx.x;
                int act = -1, nri = s_ri[j];
                if (s_live[j]) {
                    unsigned w[RW_WORDS];
#pragma unroll
                    for (int k = 0; k < RW_WORDS; ++k) w[k] = __ldcg(slot + j * RW_WORDS + k);
                    DecideArgs d = a.d;
                    d.it = it;
                    d.final_iter = last_chunk ? 1 : 0;
                    if (blockIdx.x == 0) {
                        act = decide_qp(p, d, a.qlist[j], w, nri);
                    } else {
                        const Decision x = decide_eval(p, d, a.qlist[j], w, s_ri[j], 0);
                        act = x.act;
                        nri = x.nri;
                    }
                }
                s_act[j] = act;
                s_nri[j] = nri;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int any = 0;
                for (int j = 0; j < nq; ++j) {
                    if (s_act[j] == 1) s_live[j] = 0;
                    if (s_act[j] == 2) s_ri[j] = s_nri[j];
                    any |= s_live[j];
                }
                s_any = any;
            }
            __syncthreads();
            // outputs of finished QPs; lam' rebase of switched ones
            const int width = p.n > p.m ? p.n : p.m;
            for (int o = tid; o < width * nq; o += nthr) {
                const int e = o / nq, j = o - e * nq;
                const int qp = a.qlist[j];
                if (s_act[j] == 1) {
                    if (e < p.n) a.d.XO[(size_t)qp * p.n + e] = p.Y[(size_t)qp * p.ldn + e];
                    if (e < p.m) {
                        a.d.ZO[(size_t)qp * p.m + e] = p.Z[(size_t)qp * p.ldm + e];
                        a.d.LO[(size_t)qp * p.m + e] = p.LSTD[(size_t)qp * p.ldm + e];
                    }
                } else if (s_act[j] == 2 && e < p.m) {
                    const size_t oo = (size_t)qp * p.ldm + e;
                    const float rho_i = (float)(p.rhod[s_ri[j]] * (double)p.rs[e]);
                    p.LAM[oo] = lam_standard(p.LSTD[oo], -rho_i, p.AY[oo] - p.Z[oo]);
                }
            }
            if (!s_any) return;
            if (!tail_barrier(a, &s_ok)) return;
        }
        if (last_chunk) return;
        // operand of the next chunk's first layer from the state
        tail_fill(a, a.S + (size_t)cur * kTailMax * p.ldk, s_live, s_ri);
        if (!tail_barrier(a, &s_ok)) return;
    }
}

// Active QP ids in increasing order (one warp).
__global__ void tail_list_kernel(int B, const int* __restrict__ status, int* list, int cap) {
    int base = 0;
    for (int c0 = 0; c0 < B; c0 += 32) {
        const int qp = c0 + threadIdx.x;
        const bool act = qp < B && status[qp] == QP_ACTIVE;
        const unsigned ball = __ballot_sync(0xffffffffu, act);
        const int pos = base + __popc(ball & ((1u << threadIdx.x) - 1u));
        if (act && pos < cap) list[pos] = qp;
        base += __popc(ball);
    }
}

// floats of the scratch region: the step partials of `pass_rows` rows of the layer
// product [kTailMax][pass_rows][ps], or the checks' per-warp round partials
size_t tail_scratch(const BatchWork& w, int pass_rows) {
    const size_t ps = (size_t)((w.ldk / kStep) | 1);
    return std::max((size_t)kTailWarps * kRB * kTailMax * kPbs, (size_t)pass_rows * kTailMax * ps);
}

// staged operands [kTailMax][steps][kStepPad] + scratch (+ the cached Wt rows
// [rows][ldk steps][kStepPad])
size_t tail_smem(const BatchWork& w, int pass_rows, int cached_rows) {
    const size_t steps = (size_t)std::max(w.ldk, w.ldkc) / kStep;
    return ((size_t)kTailMax * steps * kStepPad + tail_scratch(w, pass_rows) +
            (size_t)cached_rows * (w.ldk / kStep) * kStepPad) *
           sizeof(float);
}

}  // namespace

int batch_tail_alloc(relu_qp_t h) {
    BatchWork& w = h->bw;
    RQ_TRY(alloc(h, &w.TS, 2 * (size_t)kTailMax * w.ldk));
    RQ_TRY(alloc(h, &w.TCK, (size_t)kTailMax * w.ldkc));
    RQ_TRY(alloc(h, &w.TRED, 3 * (size_t)kTailMax * RW_WORDS));
    RQ_TRY(alloc(h, &w.TBAR, 4));
    RQ_TRY(alloc(h, &w.TLIST, kTailMax));
    int smem_max = 0;
    RQ_CUDA(h, cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    w.tail_grid = 0;
    // one CTA per SM and (while the SMs suffice) one row of the layer per warp; the CTA's
    // rows of Wt cached in shared memory when they fit (every CTA co-resident: grid
    // barrier), and the step partials of all its rows in one pass when they fit
    const int grid = std::min(h->num_sms, ceil_div(h->R, kTailWarps));
    const int rpc = ceil_div(h->R, grid);
    for (int cache = 1; cache >= 0; --cache) {
        for (int pr = rpc;; pr = std::max(kRG, pr / 2)) {
            const size_t smem = tail_smem(w, pr, cache ? rpc : 0);
            if (smem + 1024 <= (size_t)smem_max) {
                RQ_CUDA(h, cudaFuncSetAttribute(batch_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem));
                int per_sm = 0;
                RQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_tail_kernel, kTailThreads,
                                                                         smem));
                if (per_sm >= 1) {
                    w.tail_grid = grid;
                    w.tail_rpc = rpc;
                    w.tail_pr = pr;
                    w.tail_cache = cache;
                    w.tail_smem = smem;
                    return RELU_QP_OK;
                }
            }
            if (pr <= kRG) break;
        }
    }
    return RELU_QP_OK;   // problem too large for the staged operands: no tail kernel
}

int batch_tail(relu_qp_t h, const BatchParams& p, const DecideArgs& d, int nq, int it0, int max_iter) {
    BatchWork& w = h->bw;
    if (nq <= 0 || nq > kTailMax || w.tail_grid <= 0) return fail(h, RELU_QP_ERR_INVALID, "tail size");
    tail_list_kernel<<<1, 32, 0, h->stream>>>(w.B, w.status, w.TLIST, kTailMax);
    RQ_CUDA(h, cudaGetLastError());
    RQ_CUDA(h, cudaMemsetAsync(w.TRED, 0, sizeof(unsigned) * 3 * kTailMax * RW_WORDS, h->stream));
    RQ_CUDA(h, cudaMemsetAsync(w.TBAR, 0, sizeof(unsigned) * 4, h->stream));
    TailArgs a{};
    a.p = p;
    a.p.CK32 = w.TCK;
    a.p.CK = nullptr;
    a.d = d;
    for (int r = 0; r < h->nr; ++r) a.W[r] = h->be[r].Wt;
    a.Wc = w.Wc32;
    a.S = w.TS;
    a.CKB = w.TCK;
    a.red = w.TRED;
    a.bar = w.TBAR;
    a.err = reinterpret_cast<int*>(w.TBAR + 2);
    a.qlist = w.TLIST;
    a.nq = nq;
    a.it0 = it0;
    a.max_iter = max_iter;
    a.ci = h->opts.check_interval;
    a.rpc = w.tail_rpc;
    a.pr = w.tail_pr;
    a.scratch = (int)tail_scratch(w, w.tail_pr);
    a.wcache = w.tail_cache;
    a.regs = w.tail_pr >= w.tail_rpc && w.tail_rpc * kTailMax <= kTailThreads ? 1 : 0;
    a.timeout_ns = 2000000000LL;
    void* args[] = {&a};
    RQ_CUDA(h, cudaLaunchCooperativeKernel((const void*)batch_tail_kernel, dim3(w.tail_grid), dim3(kTailThreads), args,
                                           w.tail_smem, h->stream));
    h->launches += 2;
    return RELU_QP_OK;
}

int batch_tail_error(relu_qp_t h) {
    int e = 0;
    cudaMemcpy(&e, h->bw.TBAR + 2, sizeof(int), cudaMemcpyDeviceToHost);
    return e;
}

}  // namespace rq
