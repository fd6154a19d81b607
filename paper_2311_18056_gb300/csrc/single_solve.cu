// Single-QP online stage of Algorithm 1 (Sec. III-B) in one cooperative
// kernel: the layer of Eq. gpu_update every iteration, the residuals of Eqs.
// primal and dual every check_interval layers, the penalty rule of Eq.
// rho_update with the nearest bank entry (Sec. III-C), and the stop test.
//
// Layer in factored form (the algebra is in setup_fp64.cu): with
//   s = [x; 2 rho z - lam'],   t = Wt s + b,
//   r = (Ax) - z + lam'/rho          (carried Ax from the previous layer)
//   x+ = t_x,  (Ax)+ = t_Ax,  z+ = clamp(t_Ax + r, l, u),  lam'+ = rho r,
// which equals v+ = clamp(W v + b) with v = [x; z; lam'].
//
// Work split: the R = n + m rows of Wt are cut into contiguous slices, one
// per CTA; each CTA keeps as many of its rows as fit in shared memory (the
// rest stream from L2) and its rows' state for the whole solve, and each warp
// computes up to 4 of its rows at once (coalesced 128-bit loads, one shuffle
// reduction per row).  Two launch forms, chosen by timing at setup: a
// cooperative grid, whose CTAs exchange the layer's operand through global
// memory and meet at the grid barrier, or one thread-block cluster, whose CTAs
// write each new operand entry into every CTA's shared copy and meet at a
// cluster barrier.  Every barrier wait has a deadline after which the kernel
// records RELU_QP_ERR_TIMEOUT and returns.
#include "common.h"
#include "grid_sync.h"

#include <cmath>
#include <mutex>

namespace rq {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

enum { RED_RP = 0, RED_RD, RED_AX, RED_Z, RED_PX, RED_ATL, RED_WORDS = 8 };
enum { OUT_STATUS = 0, OUT_ITERS, OUT_RHO, OUT_SWITCHES, OUT_ERR, OUT_WORDS = 8 };

struct SP {
    int n, m, R, ldw, ldp, lda, ldt, nr;
    const float* Wt[RQ_MAX_RHO];
    const float* bias[RQ_MAX_RHO];
    double rho[RQ_MAX_RHO];
    const float *P, *A, *At, *q, *l, *u, *rs;
    const float *rsx, *rsz;   // scaled problems: residual factors 1/(c D), 1/E (else nullptr)
    float *y, *z, *lam, *Ay, *s0, *s1, *Py, *Axf, *lstd;
    unsigned* red;
    unsigned* bar;
    int* out_i;
    float* out_f;
    int rho_index0, check_interval, adaptive, max_iter;
    double eps_abs, eps_rel, qnorm;
    int rows_per_cta, cached_rows, rows2_per_cta;
    long long timeout_ns;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid-wide barrier over all CTAs of the cooperative launch (grid_sync.h).
__device__ __forceinline__ bool grid_barrier(const SP& p, GridSyncState* s_ok) {
    return grid_sync(p.bar, p.out_i + OUT_ERR, p.timeout_ns, s_ok);
}

// Synchronisation between layers and phases: the grid barrier (grid form) or
// the one-cluster barrier (cluster form, grid_sync.h).
template <bool CL>
__device__ __forceinline__ bool sync_all(const SP& p, ClusterBarrier& cb, GridSyncState* gs) {
    if (!CL) return grid_barrier(p, gs);
    return cluster_barrier(cb, p.out_i + OUT_ERR, p.timeout_ns, gs);
}

// Dot product of a padded row with a padded vector in shared memory; the
// result is valid in every lane.  Rows and vectors are 16-byte aligned and
// zero padded to a multiple of 4 floats.
__device__ __forceinline__ float row_dot(const float* __restrict__ w, const float* __restrict__ s,
                                         int ld, int lane) {
    const float4* w4 = reinterpret_cast<const float4*>(w);
    const float4* s4 = reinterpret_cast<const float4*>(s);
    const int n4 = ld >> 2;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int k = lane; k < n4; k += 32) {
        const float4 a = w4[k];
        const float4 b = s4[k];
        a0 = fmaf(a.x, b.x, a0);
        a1 = fmaf(a.y, b.y, a1);
        a2 = fmaf(a.z, b.z, a2);
        a3 = fmaf(a.w, b.w, a3);
    }
    return warp_sum((a0 + a1) + (a2 + a3));
}

__device__ __forceinline__ float row_dot_global(const float* __restrict__ w, const float* __restrict__ s,
                                                int ld, int lane) {
    const float4* w4 = reinterpret_cast<const float4*>(w);
    const float4* s4 = reinterpret_cast<const float4*>(s);
    const int n4 = ld >> 2;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int k = lane; k < n4; k += 32) {
        const float4 a = __ldg(w4 + k);
        const float4 b = s4[k];
        a0 = fmaf(a.x, b.x, a0);
        a1 = fmaf(a.y, b.y, a1);
        a2 = fmaf(a.z, b.z, a2);
        a3 = fmaf(a.w, b.w, a3);
    }
    return warp_sum((a0 + a1) + (a2 + a3));
}

// Dot products of NR padded rows (w[j], in shared or global memory) with one
// padded vector in shared memory, in one pass over k: every row keeps the
// four accumulators and the reduction of row_dot, so each result has row_dot's
// bits, while the rows' loads and shuffle reductions overlap.  Results are
// valid in every lane.
template <int NR, bool LDG>
__device__ __forceinline__ void rows_dot(const float* const (&w)[NR], const float* __restrict__ s, int ld, int lane,
                                         float (&out)[NR]) {
    const float4* s4 = reinterpret_cast<const float4*>(s);
    const int n4 = ld >> 2;
    float a[NR][4];
#pragma unroll
    for (int j = 0; j < NR; ++j) a[j][0] = a[j][1] = a[j][2] = a[j][3] = 0.f;
    for (int k = lane; k < n4; k += 32) {
        const float4 b = s4[k];
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const float4* wj = reinterpret_cast<const float4*>(w[j]) + k;
            const float4 x = LDG ? __ldg(wj) : *wj;
            a[j][0] = fmaf(x.x, b.x, a[j][0]);
            a[j][1] = fmaf(x.y, b.y, a[j][1]);
            a[j][2] = fmaf(x.z, b.z, a[j][2]);
            a[j][3] = fmaf(x.w, b.w, a[j][3]);
        }
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) out[j] = warp_sum((a[j][0] + a[j][1]) + (a[j][2] + a[j][3]));
}

constexpr int kRowsILP = 4;   // rows of a warp whose dot products run together

// rows_dot for the first cnt (1 .. kRowsILP) pointers of w.  LDG: every row is in
// global memory (read-only loads); else the rows are in shared memory or mixed.
template <bool LDG>
__device__ __forceinline__ void group_dots(int cnt, const float* const (&w)[kRowsILP], const float* s, int ld,
                                           int lane, float (&acc)[kRowsILP]) {
    if (cnt == 1) {
        const float* w1[1] = {w[0]};
        float o[1];
        rows_dot<1, LDG>(w1, s, ld, lane, o);
        acc[0] = o[0];
    } else if (cnt == 2) {
        const float* w2[2] = {w[0], w[1]};
        float o[2];
        rows_dot<2, LDG>(w2, s, ld, lane, o);
        acc[0] = o[0];
        acc[1] = o[1];
    } else if (cnt == 3) {
        const float* w3[3] = {w[0], w[1], w[2]};
        float o[3];
        rows_dot<3, LDG>(w3, s, ld, lane, o);
        acc[0] = o[0];
        acc[1] = o[1];
        acc[2] = o[2];
    } else {
        rows_dot<4, LDG>(w, s, ld, lane, acc);
    }
}

// Copy `count` floats (padded length `ld`, a multiple of 4) written by other
// CTAs into shared memory, bypassing L1 so that no stale line is read.
__device__ __forceinline__ void load_shared_cg(float* dst, const float* src, int ld) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int k = threadIdx.x; k < (ld >> 2); k += blockDim.x) d4[k] = __ldcg(s4 + k);
}

__device__ void load_w_cache(const SP& p, float* wcache, int ri, int row0, int ncache) {
    const float4* src = reinterpret_cast<const float4*>(p.Wt[ri] + (size_t)row0 * p.ldw);
    float4* dst = reinterpret_cast<float4*>(wcache);
    const int total = ncache * (p.ldw >> 2);
    for (int e = threadIdx.x; e < total; e += blockDim.x) dst[e] = __ldg(src + e);
}

__device__ __forceinline__ void red_max(unsigned* slot, int word, float v) {
    atomicMax(slot + word, __float_as_uint(fabsf(v)));
}

__device__ __forceinline__ float red_get(const unsigned* slot, int word) {
    return __uint_as_float(__ldcg(slot + word));
}

// The solve.  Grid form (CL = false): a cooperative grid; the operand s of a
// layer goes through global memory (written by the rows' owners, staged into
// shared memory after the grid barrier).  Cluster form (CL = true): the launch
// is one cluster; every CTA keeps both operand buffers in shared memory and the
// owner of a row writes its new entry into every CTA's copy (distributed shared
// memory) before the cluster barrier, so a layer never touches L2 for s.
template <bool CL>
__device__ __forceinline__ void solve_body(const SP& p, float* smem, ClusterBarrier& cb, GridSyncState* gs) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = p.n, m = p.m, R = p.R;
    const int row0 = blockIdx.x * p.rows_per_cta;
    const int row1 = min(row0 + p.rows_per_cta, R);
    const int ncache = max(0, min(p.cached_rows, row1 - row0));
    float* wcache = smem;
    float* sv = smem + (size_t)p.cached_rows * p.ldw;     // ldw floats (cluster form: 2 x ldw, both operands)
    float* svk = CL ? sv + 2 * (size_t)p.ldw : sv;        // the checks' staged vector (ldw floats)
    // the state of the CTA's rows, kept in shared memory for the whole solve (the
    // global copies are still written, for the checks and the outputs): bias of the
    // bank entry in use, and for rows of A x the carried A x, z, lam', rho_i, l, u
    const int rpc = p.rows_per_cta;
    float* st_bias = sv + (CL ? 3 : 1) * (size_t)p.ldw;
    float* st_ay = st_bias + rpc;
    float* st_z = st_ay + rpc;
    float* st_lam = st_z + rpc;
    float* st_rho = st_lam + rpc;
    float* st_l = st_rho + rpc;
    float* st_u = st_l + rpc;
    const int r2_0 = blockIdx.x * p.rows2_per_cta;
    const int r2_1 = min(r2_0 + p.rows2_per_cta, n);

    int ri = p.rho_index0;
    int switches = 0, checks = 0, cur = 0;
    if (ncache > 0) load_w_cache(p, wcache, ri, row0, ncache);
    for (int r = row0 + threadIdx.x; r < row1; r += blockDim.x) {
        const int lr = r - row0;
        st_bias[lr] = __ldg(p.bias[ri] + r);
        if (r >= n) {
            const int i = r - n;
            st_ay[lr] = __ldcg(p.Ay + i);
            st_z[lr] = __ldcg(p.z + i);
            st_lam[lr] = __ldcg(p.lam + i);
            st_rho[lr] = (float)(p.rho[ri] * (double)__ldg(p.rs + i));
            st_l[lr] = __ldg(p.l + i);
            st_u[lr] = __ldg(p.u + i);
        }
    }
    if (CL) {
        // operand buffer 0 is s0; buffer 1 only needs its padding zeroed: its rows are
        // written by the partners' first layer, which may already be running (nobody
        // writes buffer 0 before every CTA has passed the first barrier)
        load_shared_cg(sv, p.s0, p.ldw);
        for (int k = R + threadIdx.x; k < p.ldw; k += blockDim.x) sv[p.ldw + k] = 0.f;
    }
    __syncthreads();

    for (int it = 1; it <= p.max_iter; ++it) {
        // ---------------- one layer: s[cur] -> s[cur^1] ----------------
        const float* scur = cur ? p.s1 : p.s0;
        float* snext = cur ? p.s0 : p.s1;
        const float* svc = CL ? sv + (size_t)cur * p.ldw : sv;
        const uint32_t svn = CL ? cl_smem(sv + (size_t)(cur ^ 1) * p.ldw) : 0u;
        if (!CL) {
            load_shared_cg(sv, scur, p.ldw);
            __syncthreads();
        }
        const float* Wg = p.Wt[ri];
        // the global copies of the rows' state are read only by the checks and the
        // outputs: written on the layers before a check and on the last one
        const bool keep = (p.check_interval > 0 && it % p.check_interval == 0) || it == p.max_iter;
        // a warp's rows rb, rb + kWarps, ... in groups of up to kRowsILP: their dot
        // products together, then lane j updates row j of the group
        for (int rb = row0 + warp; rb < row1; rb += kRowsILP * kWarps) {
            const int cnt = min(kRowsILP, (row1 - rb + kWarps - 1) / kWarps);
            // the cached rows are the first ncache of the CTA: a group is all cached, all in
            // global memory, or (once per CTA) mixed
            const int lr_first = rb - row0, lr_last = rb + (cnt - 1) * kWarps - row0;
            float acc[kRowsILP] = {0.f, 0.f, 0.f, 0.f};
            if (lr_last < ncache) {
                const float* w[kRowsILP];
#pragma unroll
                for (int j = 0; j < kRowsILP; ++j) w[j] = wcache + (size_t)(lr_first + (j < cnt ? j : 0) * kWarps) * p.ldw;
                group_dots<false>(cnt, w, svc, p.ldw, lane, acc);
            } else if (lr_first >= ncache) {
                const float* w[kRowsILP];
#pragma unroll
                for (int j = 0; j < kRowsILP; ++j) w[j] = Wg + (size_t)(rb + (j < cnt ? j : 0) * kWarps) * p.ldw;
                group_dots<true>(cnt, w, svc, p.ldw, lane, acc);
            } else {
                const float* w[kRowsILP];
#pragma unroll
                for (int j = 0; j < kRowsILP; ++j) {
                    const int r = rb + (j < cnt ? j : 0) * kWarps, lr = r - row0;
                    w[j] = lr < ncache ? wcache + (size_t)lr * p.ldw : Wg + (size_t)r * p.ldw;
                }
                group_dots<false>(cnt, w, svc, p.ldw, lane, acc);
            }
            float snew = 0.f;
            if (lane < cnt) {
                float a = acc[0];
#pragma unroll
                for (int j = 1; j < kRowsILP; ++j)
                    if (lane == j) a = acc[j];
                const int r = rb + lane * kWarps, lr = r - row0;
                const float t = a + st_bias[lr];
                if (r < n) {
                    if (keep) p.y[r] = t;
                    snew = t;
                } else {
                    const int i = r - n;
                    const float rho_i = st_rho[lr];
                    const float rr = st_ay[lr] - st_z[lr] + st_lam[lr] / rho_i;
                    const float zn = fminf(fmaxf(t + rr, st_l[lr]), st_u[lr]);
                    const float ln = rho_i * rr;
                    st_ay[lr] = t;
                    st_z[lr] = zn;
                    st_lam[lr] = ln;
                    if (keep) {
                        p.Ay[i] = t;
                        p.z[i] = zn;
                        p.lam[i] = ln;
                    }
                    snew = 2.0f * rho_i * zn - ln;
                }
                if (!CL) snext[r] = snew;
            }
            if (CL) {
                // lane q writes each row's entry into CTA q's next operand
                for (int j = 0; j < cnt; ++j) {
                    const float v = __shfl_sync(0xffffffffu, snew, j);
                    const uint32_t addr = svn + 4u * (uint32_t)(rb + j * kWarps);
                    for (int q = lane; q < cb.C; q += 32) cl_st(cl_mapa(addr, (uint32_t)q), v);
                }
            }
        }
        cur ^= 1;
        if (!sync_all<CL>(p, cb, gs)) return;

        const bool is_check = (p.check_interval > 0) && (it % p.check_interval == 0);
        const bool last = (it == p.max_iter);
        if (!is_check && !last) continue;

        // ---------------- residuals (Eqs. primal, dual) ----------------
        unsigned* slot = p.red + (checks % 3) * RED_WORDS;
        if (blockIdx.x == 0 && threadIdx.x < RED_WORDS)
            p.red[((checks + 1) % 3) * RED_WORDS + threadIdx.x] = 0u;
        ++checks;
        load_shared_cg(svk, p.y, p.ldp);
        __syncthreads();
        for (int r = row0 + warp; r < row1; r += kWarps) {
            if (r < n) {
                const float v = row_dot_global(p.P + (size_t)r * p.ldp, svk, p.ldp, lane);
                if (lane == 0) {
                    p.Py[r] = v;
                    red_max(slot, RED_PX, p.rsx ? v * p.rsx[r] : v);
                }
            } else {
                const int i = r - n;
                const float v = row_dot_global(p.A + (size_t)i * p.lda, svk, p.lda, lane);
                if (lane == 0) {
                    const float zi = p.z[i];
                    const float rho_i = (float)(p.rho[ri] * (double)__ldg(p.rs + i));
                    p.Axf[i] = v;
                    p.lstd[i] = p.lam[i] + rho_i * (v - zi);
                    const float f = p.rsz ? p.rsz[i] : 1.f;
                    red_max(slot, RED_RP, (v - zi) * f);
                    red_max(slot, RED_AX, v * f);
                    red_max(slot, RED_Z, zi * f);
                }
            }
        }
        if (!sync_all<CL>(p, cb, gs)) return;
        if (m > 0) load_shared_cg(svk, p.lstd, p.ldt);
        __syncthreads();
        for (int j = r2_0 + warp; j < r2_1; j += kWarps) {
            const float v = (m > 0) ? row_dot_global(p.At + (size_t)j * p.ldt, svk, p.ldt, lane) : 0.f;
            if (lane == 0) {
                const float f = p.rsx ? p.rsx[j] : 1.f;
                red_max(slot, RED_RD, (__ldcg(p.Py + j) + __ldg(p.q + j) + v) * f);
                red_max(slot, RED_ATL, v * f);
            }
        }
        if (!sync_all<CL>(p, cb, gs)) return;

        // ---------------- decision (identical in every CTA) ----------------
        const double rp = red_get(slot, RED_RP), rd = red_get(slot, RED_RD);
        const double nAx = red_get(slot, RED_AX), nz = red_get(slot, RED_Z);
        const double nPx = red_get(slot, RED_PX), nAtl = red_get(slot, RED_ATL);
        const bool numerical = !(isfinite(rp) && isfinite(rd) && isfinite(nPx) && isfinite(nAtl));
        const double eps_p = p.eps_abs + p.eps_rel * fmax(nAx, nz);
        const double eps_d = p.eps_abs + p.eps_rel * fmax(fmax(nPx, nAtl), p.qnorm);
        const bool converged = is_check && !numerical && rp <= eps_p && rd <= eps_d;
        if (converged || numerical || last) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                p.out_i[OUT_STATUS] = numerical ? RELU_QP_NUMERICAL
                                                : (converged ? RELU_QP_SOLVED : RELU_QP_MAX_ITER);
                p.out_i[OUT_ITERS] = it;
                p.out_i[OUT_RHO] = ri;
                p.out_i[OUT_SWITCHES] = switches;
                p.out_f[0] = (float)rp;
                p.out_f[1] = (float)rd;
            }
            return;
        }
        // refresh the carried Ax with the directly computed one
        for (int r = max(row0, n) + threadIdx.x; r < row1; r += blockDim.x) {
            const float v = p.Axf[r - n];
            p.Ay[r - n] = v;
            st_ay[r - row0] = v;
        }
        if (!p.adaptive || !is_check) continue;
        // Eq. rho_update (inf-norms, 1e-4 floors), nearest bank entry in log distance
        const double num = rp * fmax(fmax(nPx, nAtl), fmax(p.qnorm, 1e-4));
        const double den = rd * fmax(fmax(nAx, nz), 1e-4);
        int nri = ri;
        if (num > 0.0 && den > 0.0) {
            const double est = p.rho[ri] * sqrt(num / den);
            if (isfinite(est) && est > 0.0) {
                const double le = log(est);
                double best = 1e300;
                for (int k = 0; k < p.nr; ++k) {
                    const double d = fabs(le - log(p.rho[k]));
                    if (d < best) { best = d; nri = k; }
                }
            }
        }
        if (nri == ri) continue;
        // switch: rebase lam' so that the next layer is standard ADMM with the new rho
        float* scur2 = cur ? p.s1 : p.s0;
        for (int r = max(row0, n) + threadIdx.x; r < row1; r += blockDim.x) {
            const int i = r - n;
            const float rho_i = (float)(p.rho[nri] * (double)__ldg(p.rs + i));
            const float zi = p.z[i];
            const float lnew = p.lstd[i] - rho_i * (p.Axf[i] - zi);
            p.lam[i] = lnew;
            st_lam[r - row0] = lnew;
            st_rho[r - row0] = rho_i;
            const float sn = 2.0f * rho_i * zi - lnew;
            if (CL) {
                const uint32_t a = cl_smem(sv + (size_t)cur * p.ldw + r);
                for (int q = 0; q < cb.C; ++q) cl_st(cl_mapa(a, (uint32_t)q), sn);
            } else {
                scur2[r] = sn;
            }
        }
        ri = nri;
        ++switches;
        if (ncache > 0) load_w_cache(p, wcache, ri, row0, ncache);
        for (int r = row0 + threadIdx.x; r < row1; r += blockDim.x) st_bias[r - row0] = __ldg(p.bias[ri] + r);
        if (!sync_all<CL>(p, cb, gs)) return;
    }
}

template <bool CL>
__global__ void __launch_bounds__(kThreads, 1) single_solve_kernel(SP p) {
    extern __shared__ __align__(16) float smem[];
    __shared__ GridSyncState s_ok;
    __shared__ __align__(8) unsigned long long s_cbar;
    grid_sync_init(&s_ok);
    ClusterBarrier cb{0u, 0u, 1};
    if (CL) cluster_barrier_init(cb, &s_cbar, 0u);   // C arrivals per phase
    solve_body<CL>(p, smem, cb, &s_ok);
    if (CL) {
        // no CTA leaves while a partner may still write its shared memory (every
        // wait before this point has a deadline, so every CTA gets here)
        __syncthreads();
        cl_sync_hw();
    }
}

// Warm/cold start: x given (or 0), z = A x, lam' = lam (or 0), carried Ax = A x,
// s0 = [x; 2 rho z - lam'] (rho of the starting bank entry), pads zeroed.
__global__ void init_state_kernel(int n, int m, int lda, int ldw, const float* __restrict__ A,
                                  const float* __restrict__ xin, const float* __restrict__ lin,
                                  const float* __restrict__ rs, double rho, float* y, float* z,
                                  float* lam, float* Ay, float* s0, float* s1) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < ldw; r += nw) {
        if (r < n) {
            if (lane == 0) {
                const float v = xin ? xin[r] : 0.f;
                y[r] = v;
                s0[r] = v;
                s1[r] = 0.f;
            }
        } else if (r < n + m) {
            const int i = r - n;
            float v = 0.f;
            if (xin) {
                for (int k = lane; k < n; k += 32) v = fmaf(A[(size_t)i * lda + k], xin[k], v);
                v = warp_sum(v);
            }
            if (lane == 0) {
                const float li = lin ? lin[i] : 0.f;
                const float rho_i = (float)(rho * (double)rs[i]);
                z[i] = v;
                Ay[i] = v;
                lam[i] = li;
                s0[r] = 2.0f * rho_i * v - li;
                s1[r] = 0.f;
            }
        } else if (lane == 0) {
            s0[r] = 0.f;
            s1[r] = 0.f;
        }
    }
}

__global__ void matvec_rows_kernel(const float* __restrict__ M, int rows, int cols, int ld,
                                   const float* __restrict__ x, float* __restrict__ out) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < rows; r += nw) {
        float v = 0.f;
        for (int k = lane; k < cols; k += 32) v = fmaf(M[(size_t)r * ld + k], x[k], v);
        v = warp_sum(v);
        if (lane == 0) out[r] = v;
    }
}

int fill_params(relu_qp_t h, SP& p, int grid) {
    const int n = h->n, m = h->m;
    p.n = n; p.m = m; p.R = h->R; p.ldw = h->ldw;
    p.ldp = (int)round_up(n, 4);
    p.lda = (int)round_up(n, 4);
    p.ldt = (int)round_up(m > 0 ? m : 1, 4);
    p.nr = h->nr;
    for (int r = 0; r < h->nr; ++r) {
        p.Wt[r] = h->be[r].Wt;
        p.bias[r] = h->be[r].bias;
        p.rho[r] = h->be[r].rho;
    }
    p.P = h->P32; p.A = h->A32; p.At = h->At32;
    p.q = h->q32; p.l = h->l32; p.u = h->u32; p.rs = h->rs32;
    SingleWork& w = h->sw;
    p.y = w.y; p.z = w.z; p.lam = w.lam; p.Ay = w.Ay; p.s0 = w.s0; p.s1 = w.s1;
    p.Py = w.Py; p.Axf = w.Axf; p.lstd = w.lstd;
    p.red = w.red; p.bar = w.bar; p.out_i = w.out_i; p.out_f = w.out_f;
    p.rows_per_cta = ceil_div(h->R, grid);
    p.rows2_per_cta = ceil_div(n, grid);
    p.timeout_ns = 2000000000LL;
    return RELU_QP_OK;
}

// cached rows of W + the staged operand (cluster form: both operands and the checks' vector)
// + the state of the CTA's rows (7 floats per row)
size_t smem_bytes(int cached_rows, int ldw, bool cl, int rows_per_cta) {
    return (((size_t)cached_rows + (cl ? 3 : 1)) * ldw + 7 * (size_t)rows_per_cta) * sizeof(float);
}

// Largest dynamic shared memory the solve kernel may request: the opt-in
// per-block limit minus the kernel's static shared memory (of either form).
int max_shared(relu_qp_t h) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    int stat = 0;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, single_solve_kernel<false>) == cudaSuccess) stat = (int)fa.sharedSizeBytes;
    if (cudaFuncGetAttributes(&fa, single_solve_kernel<true>) == cudaSuccess && (int)fa.sharedSizeBytes > stat)
        stat = (int)fa.sharedSizeBytes;
    cudaGetLastError();
    return v - stat - 256;
}

// Shared-memory rows a CTA of a `grid`-CTA launch can cache.
int cached_rows_for(relu_qp_t h, int grid, bool cl) {
    const int rows = ceil_div(h->R, grid);
    const long budget = (long)max_shared(h) - 7L * rows * (long)sizeof(float);
    long cap = budget / (long)((size_t)h->ldw * sizeof(float)) - (cl ? 3 : 1);
    if (cap < 0) cap = 0;
    return rows < cap ? rows : (int)cap;
}

// Launch the solve kernel: a cooperative grid of `grid` CTAs, or (cluster > 1)
// one cluster of `grid` CTAs.
int launch_kernel(relu_qp_t h, SP& p, int grid, int cluster, int cached) {
    const size_t smem = smem_bytes(cached, h->ldw, cluster > 1, ceil_div(h->R, grid));
    if (cluster > 1) {
        auto k = single_solve_kernel<true>;
        RQ_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (cluster > 8) RQ_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = h->stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        RQ_CUDA(h, cudaLaunchKernelEx(&cfg, k, p));
        return RELU_QP_OK;
    }
    RQ_CUDA(h, cudaFuncSetAttribute(single_solve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    void* args[] = {&p};
    RQ_CUDA(h, cudaLaunchCooperativeKernel((const void*)single_solve_kernel<false>, dim3(grid), dim3(kThreads), args,
                                           smem, h->stream));
    return RELU_QP_OK;
}

// Whether one cluster of `c` CTAs with this shared memory can be resident.
bool cluster_fits(relu_qp_t h, int c, int cached) {
    auto k = single_solve_kernel<true>;
    const size_t smem = smem_bytes(cached, h->ldw, true, ceil_div(h->R, c));
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        (c > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
    cudaGetLastError();
    return e == cudaSuccess && n >= 1;
}

int launch(relu_qp_t h, int grid, int cluster, int cached, int rho_index, double eps_abs, double eps_rel,
           int max_iter, int check_interval, int adaptive) {
    SP p{};
    fill_params(h, p, grid);
    p.cached_rows = cached;
    p.rho_index0 = rho_index;
    p.check_interval = check_interval;
    p.adaptive = adaptive;
    p.max_iter = max_iter;
    p.eps_abs = eps_abs;
    p.eps_rel = eps_rel;
    p.qnorm = h->qnorm;
    p.rsx = h->sc_rx;
    p.rsz = h->sc_z;
    SingleWork& w = h->sw;
    RQ_CUDA(h, cudaMemsetAsync(w.red, 0, sizeof(unsigned) * 3 * RED_WORDS, h->stream));
    RQ_CUDA(h, cudaMemsetAsync(w.bar, 0, sizeof(unsigned) * 2, h->stream));
    RQ_CUDA(h, cudaMemsetAsync(w.out_i, 0, sizeof(int) * OUT_WORDS, h->stream));
    return launch_kernel(h, p, grid, cluster, cached);
}

int init_state(relu_qp_t h, const float* x, const float* lam, int rho_index) {
    SingleWork& w = h->sw;
    const int blocks = ceil_div(h->ldw * 32, 256) < 1024 ? ceil_div(h->ldw * 32, 256) : 1024;
    init_state_kernel<<<blocks, 256, 0, h->stream>>>(h->n, h->m, (int)round_up(h->n, 4), h->ldw, h->A32,
                                                      x, lam, h->rs32, h->be[rho_index].rho, w.y, w.z,
                                                      w.lam, w.Ay, w.s0, w.s1);
    RQ_CUDA(h, cudaGetLastError());
    return RELU_QP_OK;
}

}  // namespace

int compute_bias(relu_qp_t h) {
    const int blocks = ceil_div(h->R * 32, 256) < 2048 ? ceil_div(h->R * 32, 256) : 2048;
    for (int r = 0; r < h->nr; ++r) {
        matvec_rows_kernel<<<blocks, 256, 0, h->stream>>>(h->be[r].Bop, h->R, h->n, h->n, h->q32,
                                                          h->be[r].bias);
        RQ_CUDA(h, cudaGetLastError());
    }
    return RELU_QP_OK;
}

// Choose the CTA count of the cooperative launch by timing 50 fixed-rho
// layers (no checks) for each candidate that fits co-resident on the GPU.
int single_prepare(relu_qp_t h) {
    int per_sm = 0;
    // candidates: (CTAs, cluster); cluster > 1 = one cluster of that many CTAs
    std::vector<std::pair<int, int>> cands;
    for (int g = 1; g <= 4 * h->num_sms; g *= 2) cands.push_back({g, 0});
    cands.push_back({h->num_sms, 0});
    for (int c = 2; c <= 16; c *= 2) cands.push_back({c, c});
    int best_g = 1, best_cl = 0, best_c = cached_rows_for(h, 1, false);
    float best_t = 1e30f;
    for (const auto& gc : cands) {
        const int g = gc.first, cl = gc.second;
        if (g > h->R) continue;
        const int cached = cached_rows_for(h, g, cl > 1);
        if (cl > 1) {
            if (!cluster_fits(h, cl, cached)) continue;
        } else {
            // the occupancy query needs the kernel's shared-memory limit at least this large
            // (each launch below sets it to its own size)
            const size_t smem = smem_bytes(cached, h->ldw, false, ceil_div(h->R, g));
            RQ_CUDA(h, cudaFuncSetAttribute(single_solve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
            RQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, single_solve_kernel<false>, kThreads,
                                                                     smem));
            if (per_sm < 1 || g > per_sm * h->num_sms) continue;
        }
        h->sw.grid = g;
        h->sw.cluster = cl;
        RQ_TRY(init_state(h, nullptr, nullptr, 0));
        RQ_TRY(launch(h, g, cl, cached, 0, 0.0, 0.0, 10, 0, 0));   // warm-up
        RQ_TRY(init_state(h, nullptr, nullptr, 0));
        RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
        RQ_TRY(launch(h, g, cl, cached, 0, 0.0, 0.0, 50, 0, 0));
        RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
        RQ_CUDA(h, cudaStreamSynchronize(h->stream));
        int err = 0;
        RQ_CUDA(h, cudaMemcpy(&err, h->sw.out_i + OUT_ERR, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) return fail(h, RELU_QP_ERR_TIMEOUT, "a barrier deadline passed while tuning the solve");
        float ms = 0.f;
        RQ_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        if (ms < best_t) {
            best_t = ms;
            best_g = g;
            best_cl = cl;
            best_c = cached;
        }
    }
    h->sw.grid = best_g;
    h->sw.cluster = best_cl;
    h->sw.cached_rows = best_c;
    h->sw.rows_per_cta = ceil_div(h->R, best_g);
    return RELU_QP_OK;
}

int single_get_config(relu_qp_t h, int* ctas, int* cluster, int* cached_rows) {
    if (h->sw.grid <= 0) return fail(h, RELU_QP_ERR_INVALID, "the single-QP solve is not set up");
    if (ctas) *ctas = h->sw.grid;
    if (cluster) *cluster = h->sw.cluster > 1 ? h->sw.cluster : 0;
    if (cached_rows) *cached_rows = h->sw.cached_rows;
    return RELU_QP_OK;
}

int single_set_config(relu_qp_t h, int ctas, int cluster) {
    if (h->sw.grid <= 0) return fail(h, RELU_QP_ERR_INVALID, "the single-QP solve is not set up");
    if (ctas < 1 || ctas > h->R || cluster < 0 || (cluster > 1 && cluster != ctas) ||
        (cluster > 1 && cluster != 2 && cluster != 4 && cluster != 8 && cluster != 16))
        return fail(h, RELU_QP_ERR_INVALID, "ctas in [1, n + m]; cluster 0 or cluster = ctas in {2, 4, 8, 16}");
    const bool cl = cluster > 1;
    const int cached = cached_rows_for(h, ctas, cl);
    if (cl) {
        if (!cluster_fits(h, ctas, cached))
            return fail(h, RELU_QP_ERR_UNSUPPORTED, "a cluster of this size cannot be resident");
    } else {
        int per_sm = 0;
        RQ_CUDA(h, cudaFuncSetAttribute(single_solve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_bytes(cached, h->ldw, false, ceil_div(h->R, ctas))));
        RQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, single_solve_kernel<false>, kThreads,
                                                                 smem_bytes(cached, h->ldw, false, ceil_div(h->R, ctas))));
        if (per_sm < 1 || ctas > per_sm * h->num_sms)
            return fail(h, RELU_QP_ERR_UNSUPPORTED, "that many CTAs cannot be co-resident");
    }
    h->sw.grid = ctas;
    h->sw.cluster = cl ? cluster : 0;
    h->sw.cached_rows = cached;
    h->sw.rows_per_cta = ceil_div(h->R, ctas);
    return RELU_QP_OK;
}

int single_solve(relu_qp_t h, const float* x_warm, const float* lam_warm, int rho_index, double eps_abs,
                 double eps_rel, int max_iter, relu_qp_info* info) {
    SingleWork& w = h->sw;
    RQ_TRY(init_state(h, x_warm, lam_warm, rho_index));
    RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
    RQ_TRY(launch(h, w.grid, w.cluster, w.cached_rows, rho_index, eps_abs, eps_rel, max_iter,
                  h->opts.check_interval, h->opts.adaptive_rho));
    h->launches += 2;
    RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
    int oi[OUT_WORDS];
    float of[2];
    RQ_CUDA(h, cudaMemcpyAsync(oi, w.out_i, sizeof(oi), cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaMemcpyAsync(of, w.out_f, sizeof(of), cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    if (oi[OUT_ERR]) return fail(h, RELU_QP_ERR_TIMEOUT, "a barrier deadline passed in relu_qp_solve");
    if (info) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        info->status = oi[OUT_STATUS];
        info->iters = oi[OUT_ITERS];
        info->rho_index = oi[OUT_RHO];
        info->rho_switches = oi[OUT_SWITCHES];
        info->r_prim = of[0];
        info->r_dual = of[1];
        info->solve_ms = ms;
    }
    return RELU_QP_OK;
}


// ---------------------------------------------------------------------------
// Solve without allocating: the scratch of the cooperative solve lives in a
// fixed, file-scope device array instead of buffers allocated at setup.
//
// Some callers cannot allocate device memory at the time they solve: a
// real-time control loop whose cycle must not stall on cudaMalloc (which can
// synchronise the device and take unbounded time), or a host application
// whose allocator owns all device memory.  They set the problem up once (the
// layer bank is still built by relu_qp_setup) and then solve with
// relu_qp_solve_noalloc, which only launches kernels and copies.
//
// Every GPU that loads the library holds this array until the process exits.
// All calls share it, so two calls whose GPU work overlaps (on different
// streams, or from different threads) race on it; calls must be ordered.
// It keeps the contents of the last call; each call clears the parts that
// must start at zero.
// ---------------------------------------------------------------------------
namespace {

// 3 * ldw + ldp + 6 * ldt + 64 words for n + m <= kNoAllocMaxRows (see
// noalloc_words); 49152 floats = 192 KiB.
constexpr int kNoAllocMaxRows = 4096;
constexpr size_t kNoAllocWords = 49152;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
float* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;

size_t noalloc_words(int ldw, int ldp, int ldt) { return 3 * (size_t)ldw + ldp + 6 * (size_t)ldt + 64; }

// Device address of the array on the handle's device, looked up once per
// device (a host-side use of the symbol itself would not be a device address).
// The lookup is made with h->device current, whatever device the calling
// thread has made current, because the stream and every buffer of the solve
// belong to h->device.
int noalloc_scratch(relu_qp_t h, float** out) {
    const int dev = h->device;
    if (dev < 0 || dev >= kMaxDevices) return fail(h, RELU_QP_ERR_UNSUPPORTED, "device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        int cur = 0;
        RQ_CUDA(h, cudaGetDevice(&cur));
        if (cur != dev) RQ_CUDA(h, cudaSetDevice(dev));
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (cur != dev) cudaSetDevice(cur);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return fail(h, RELU_QP_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        }
        g_noalloc_ptr[dev] = static_cast<float*>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    return RELU_QP_OK;
}

// The caller's warm-start and output pointers must be device (or managed)
// memory of the handle's device: anything else would reach the kernels and
// the device-to-device copies unchecked.  NULL passes (optional arguments are
// checked by the caller).
int noalloc_check_ptr(relu_qp_t h, const void* ptr, const char* name) {
    if (!ptr) return RELU_QP_OK;
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, RELU_QP_ERR_INVALID, std::string(name) + " is not a CUDA pointer");
    }
    const bool on_device = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    if (!on_device || (a.type == cudaMemoryTypeDevice && a.device != h->device))
        return fail(h, RELU_QP_ERR_INVALID,
                    std::string(name) + " must be device FP32 memory of device " + std::to_string(h->device));
    return RELU_QP_OK;
}

}  // namespace

int single_solve_noalloc(relu_qp_t h, const float* x_warm, const float* lam_warm, int rho_index, double eps_abs,
                         double eps_rel, int max_iter, float* x_out, float* z_out, float* lam_out,
                         relu_qp_info* info) {
    const int n = h->n, m = h->m;
    const int ldp = (int)round_up(n, 4), ldt = (int)round_up(m > 0 ? m : 1, 4), ldw = h->ldw;
    if (h->R > kNoAllocMaxRows || noalloc_words(ldw, ldp, ldt) > kNoAllocWords)
        return fail(h, RELU_QP_ERR_INVALID, "relu_qp_solve_noalloc supports n + m <= " +
                                                std::to_string(kNoAllocMaxRows) + " (fixed scratch of " +
                                                std::to_string(kNoAllocWords * 4 / 1024) + " KiB)");
    RQ_TRY(noalloc_check_ptr(h, x_warm, "x_warm"));
    RQ_TRY(noalloc_check_ptr(h, lam_warm, "lam_warm"));
    RQ_TRY(noalloc_check_ptr(h, x_out, "x_out"));
    RQ_TRY(noalloc_check_ptr(h, z_out, "z_out"));
    RQ_TRY(noalloc_check_ptr(h, lam_out, "lam_out"));
    float* base = nullptr;
    RQ_TRY(noalloc_scratch(h, &base));
    // carve the scratch: vectors first (16-byte aligned offsets), then the words
    float* y = base;
    float* s0 = y + ldw;
    float* s1 = s0 + ldw;
    float* Py = s1 + ldw;
    float* z = Py + ldp;
    float* lam = z + ldt;
    float* Ay = lam + ldt;
    float* Axf = Ay + ldt;
    float* lstd = Axf + ldt;
    float* spare = lstd + ldt;            // ldt floats, unused
    unsigned* red = reinterpret_cast<unsigned*>(spare + ldt);   // 3 x 8 words
    unsigned* bar = red + 3 * RED_WORDS;                        // 2 words (+6 pad)
    int* out_i = reinterpret_cast<int*>(bar + 8);               // OUT_WORDS
    float* out_f = reinterpret_cast<float*>(out_i + OUT_WORDS); // 8 words
    SP p{};
    fill_params(h, p, h->sw.grid);
    p.y = y; p.z = z; p.lam = lam; p.Ay = Ay; p.s0 = s0; p.s1 = s1;
    p.Py = Py; p.Axf = Axf; p.lstd = lstd;
    p.red = red; p.bar = bar; p.out_i = out_i; p.out_f = out_f;
    p.cached_rows = h->sw.cached_rows;
    p.rho_index0 = rho_index;
    p.check_interval = h->opts.check_interval;
    p.adaptive = h->opts.adaptive_rho;
    p.max_iter = max_iter;
    p.eps_abs = eps_abs;
    p.eps_rel = eps_rel;
    p.qnorm = h->qnorm;
    p.rsx = h->sc_rx;
    p.rsz = h->sc_z;
    // parts that must start at zero: x and lam_std padding (read as whole
    // padded vectors by the check), reduction slots, barrier and result words
    RQ_CUDA(h, cudaMemsetAsync(y, 0, sizeof(float) * ldw, h->stream));
    RQ_CUDA(h, cudaMemsetAsync(lstd, 0, sizeof(float) * ldt, h->stream));
    RQ_CUDA(h, cudaMemsetAsync(red, 0, sizeof(unsigned) * (3 * RED_WORDS + 8) + sizeof(int) * OUT_WORDS +
                                           sizeof(float) * 8, h->stream));
    const int blocks = ceil_div(ldw * 32, 256) < 1024 ? ceil_div(ldw * 32, 256) : 1024;
    init_state_kernel<<<blocks, 256, 0, h->stream>>>(n, m, ldp, ldw, h->A32, x_warm, lam_warm, h->rs32,
                                                      h->be[rho_index].rho, y, z, lam, Ay, s0, s1);
    RQ_CUDA(h, cudaGetLastError());
    RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
    RQ_TRY(launch_kernel(h, p, h->sw.grid, h->sw.cluster, p.cached_rows));
    RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
    RQ_CUDA(h, cudaMemcpyAsync(x_out, y, sizeof(float) * n, cudaMemcpyDeviceToDevice, h->stream));
    if (z_out && m > 0) RQ_CUDA(h, cudaMemcpyAsync(z_out, z, sizeof(float) * m, cudaMemcpyDeviceToDevice, h->stream));
    if (lam_out && m > 0)
        RQ_CUDA(h, cudaMemcpyAsync(lam_out, lstd, sizeof(float) * m, cudaMemcpyDeviceToDevice, h->stream));
    int oi[OUT_WORDS];
    float of[2];
    RQ_CUDA(h, cudaMemcpyAsync(oi, out_i, sizeof(oi), cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaMemcpyAsync(of, out_f, sizeof(of), cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    if (oi[OUT_ERR]) return fail(h, RELU_QP_ERR_TIMEOUT, "a barrier deadline passed in relu_qp_solve_noalloc");
    if (info) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        info->status = oi[OUT_STATUS];
        info->iters = oi[OUT_ITERS];
        info->rho_index = oi[OUT_RHO];
        info->rho_switches = oi[OUT_SWITCHES];
        info->r_prim = of[0];
        info->r_dual = of[1];
        info->solve_ms = ms;
    }
    return RELU_QP_OK;
}

}  // namespace rq
