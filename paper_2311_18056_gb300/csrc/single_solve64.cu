// Single-QP online stage of Algorithm 1 (Sec. III-B) in FP64: the same loop as
// single_solve.cu (layer of Eq. gpu_update in factored form every iteration,
// residuals of Eqs. primal and dual every check_interval layers, penalty rule
// of Eq. rho_update with the nearest bank entry, stop test) with every
// product, state vector and residual in FP64.
//
// Why a second arithmetic: an equality row carries 1000x the penalty of an
// inequality row (Sec. II-B), so the rounding of (Ax - z) enters its
// multiplier step multiplied by up to 1000 rho every layer.  In FP32 that
// noise (~6e-8 |Ax| rho_eq) leaves the dual residual of random QPs with n/4
// equality rows near 1e-5..1e-4, above the 1e-6 tolerance of the random-QP
// benchmark (Sec. V-A); in FP64 the same noise is ~1e-16 |Ax| rho_eq.
//
// Refined form (opts.single_precision = RELU_QP_PREC_FP64R): the FP64 layer
// product is computed once per check interval (the anchor), c = Wt s_ref + b,
// and the other layers apply the FP32 bank to the increment only,
// t = c + Wt32 (s - s_ref), with the element-wise step, the state and the
// checks in FP64.  The FP32 rounding then scales with |s - s_ref|, which
// shrinks as the solve converges, and each layer costs an FP32 row product
// instead of an FP64 one (GB300's FP64 rate is ~1/60 of its FP32 rate).
//
// Work split: the R = n + m rows of Wt (FP64, R x R) are cut into contiguous
// slices, one per CTA of 16 warps; each warp produces one row at a time (lanes over the
// columns, shuffle reduction); the operand s lives in shared memory.  Rows
// stream from L2 (the FP64 bank of n + m = 3000 is 72 MB).  A grid barrier
// with a deadline separates layers.
#include "common.h"
#include "grid_sync.h"

#include <algorithm>
#include <cmath>

namespace rq {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
// operand s in shared memory: n + m doubles at most
constexpr int kMaxRows64 = 24576;

enum { RED_RP = 0, RED_RD, RED_AX, RED_Z, RED_PX, RED_ATL, RED_WORDS = 8 };
enum { OUT_STATUS = 0, OUT_ITERS, OUT_RHO, OUT_SWITCHES, OUT_ERR, OUT_WORDS = 8 };

struct SP64 {
    int n, m, R, nr;
    const double* Wt[RQ_MAX_RHO];
    const float* Wt32[RQ_MAX_RHO];   // refined form: FP32 bank, rows of ldw floats (zero padded)
    int ldw, anchor_every;
    double *c, *sref;                // refined form: anchor product and operand (R each)
    float* d32;                      // refined form: (float)(s - s_ref) of the next layer (ldw, zero padded)
    const double* bias[RQ_MAX_RHO];
    double rho[RQ_MAX_RHO];
    const double *P, *A, *At, *q, *l, *u;
    const float* rs;              // per-row penalty scale (1 or eq_scale)
    const double *rsx, *rsz;      // scaled problems: residual factors 1/(c D), 1/E (else nullptr)
    double *y, *z, *lam, *Ay, *s0, *s1, *Py, *Axf, *lstd;
    unsigned long long* red;
    unsigned* bar;
    int* out_i;
    double* out_f;
    int rho_index0, check_interval, adaptive, max_iter, rows_per_cta, rows2_per_cta;
    double eps_abs, eps_rel, qnorm;
    long long timeout_ns;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid-wide barrier over all CTAs of the cooperative launch (grid_sync.h).
__device__ __forceinline__ bool grid_barrier(const SP64& p, GridSyncState* s_ok) {
    return grid_sync(p.bar, p.out_i + OUT_ERR, p.timeout_ns, s_ok);
}

// Dot product of a row (global, read-only) with a vector in shared memory;
// the result is valid in every lane.  Eight independent loads per lane are in
// flight per step: a row streams from L2, and with one CTA of 8 warps per SM
// fewer loads in flight leave the FP64 pipe waiting on L2 latency.
__device__ __forceinline__ double row_dot(const double* __restrict__ w, const double* __restrict__ s, int len,
                                          int lane) {
    double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int k = lane;
    for (; k + 7 * 32 < len; k += 8 * 32) {
        double wv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) wv[t] = __ldg(w + k + 32 * t);
#pragma unroll
        for (int t = 0; t < 8; ++t) a[t] = fma(wv[t], s[k + 32 * t], a[t]);
    }
    for (; k < len; k += 32) a[0] = fma(__ldg(w + k), s[k], a[0]);   // at most 7 steps
    return warp_sum(((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])));
}

// FP32 row (ld floats, 16-byte aligned, zero padded) times an FP32 vector in
// shared memory; the result is valid in every lane.
__device__ __forceinline__ float row_dot32(const float* __restrict__ w, const float* __restrict__ s, int ld, int lane) {
    const float4* w4 = reinterpret_cast<const float4*>(w);
    const float4* s4 = reinterpret_cast<const float4*>(s);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int k = lane; k < (ld >> 2); k += 32) {
        const float4 a = __ldg(w4 + k);
        const float4 b = s4[k];
        a0 = fmaf(a.x, b.x, a0);
        a1 = fmaf(a.y, b.y, a1);
        a2 = fmaf(a.z, b.z, a2);
        a3 = fmaf(a.w, b.w, a3);
    }
    float v = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Vector written by other CTAs into shared memory, bypassing L1.
__device__ __forceinline__ void load_shared_cg(double* dst, const double* src, int len) {
    for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = __ldcg(src + k);
}

__device__ __forceinline__ void red_max(unsigned long long* slot, int word, double v) {
    atomicMax(slot + word, (unsigned long long)__double_as_longlong(fabs(v)));
}

__device__ __forceinline__ double red_get(const unsigned long long* slot, int word) {
    return __longlong_as_double((long long)__ldcg(slot + word));
}

template <bool REFINED>
__global__ void __launch_bounds__(kThreads, 1) single64_kernel(SP64 p) {
    extern __shared__ __align__(16) double sv[];   // R doubles (refined layers: ldw floats of the increment)
    __shared__ GridSyncState s_ok;
    grid_sync_init(&s_ok);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = p.n, m = p.m, R = p.R;
    const int row0 = blockIdx.x * p.rows_per_cta;
    const int row1 = min(row0 + p.rows_per_cta, R);
    const int r2_0 = blockIdx.x * p.rows2_per_cta;
    const int r2_1 = min(r2_0 + p.rows2_per_cta, n);

    int ri = p.rho_index0;
    int switches = 0, checks = 0, cur = 0;
    for (int it = 1; it <= p.max_iter; ++it) {
        // ---------------- one layer: s[cur] -> s[cur^1] ----------------
        const double* scur = cur ? p.s1 : p.s0;
        double* snext = cur ? p.s0 : p.s1;
        // refined form: an FP64 anchor layer at the start of every check interval (so also
        // after every bank switch), FP32 increment layers in between
        const bool anchor = !REFINED || (it - 1) % p.anchor_every == 0;
        float* dv = reinterpret_cast<float*>(sv);
        if (anchor) {
            load_shared_cg(sv, scur, R);
        } else {
            for (int k = threadIdx.x; k < p.ldw; k += blockDim.x)
                dv[k] = __ldcg(p.d32 + k);   // written by the owners of the rows in the last layer
        }
        __syncthreads();
        const double* Wg = p.Wt[ri];
        const double* bias = p.bias[ri];
        const double rho = p.rho[ri];
        for (int r = row0 + warp; r < row1; r += kWarps) {
            const double acc = anchor ? row_dot(Wg + (size_t)r * R, sv, R, lane)
                                      : (double)row_dot32(p.Wt32[ri] + (size_t)r * p.ldw, dv, p.ldw, lane);
            if (lane == 0) {
                double t;
                if (!REFINED) {
                    t = acc + __ldg(bias + r);
                } else if (anchor) {
                    t = acc + __ldg(bias + r);
                    p.c[r] = t;
                    p.sref[r] = scur[r];
                } else {
                    t = p.c[r] + acc;
                }
                if (r < n) {
                    p.y[r] = t;
                    snext[r] = t;
                    if (REFINED) p.d32[r] = (float)(t - p.sref[r]);
                } else {
                    const int i = r - n;
                    const double rho_i = rho * (double)__ldg(p.rs + i);
                    const double rr = p.Ay[i] - p.z[i] + p.lam[i] / rho_i;
                    const double zn = fmin(fmax(t + rr, __ldg(p.l + i)), __ldg(p.u + i));
                    const double ln = rho_i * rr;
                    p.Ay[i] = t;
                    p.z[i] = zn;
                    p.lam[i] = ln;
                    snext[r] = 2.0 * rho_i * zn - ln;
                    if (REFINED) p.d32[r] = (float)(snext[r] - p.sref[r]);
                }
            }
        }
        cur ^= 1;
        if (!grid_barrier(p, &s_ok)) return;

        const bool is_check = (p.check_interval > 0) && (it % p.check_interval == 0);
        const bool last = (it == p.max_iter);
        if (!is_check && !last) continue;

        // ---------------- residuals (Eqs. primal, dual) ----------------
        unsigned long long* slot = p.red + (checks % 3) * RED_WORDS;
        if (blockIdx.x == 0 && threadIdx.x < RED_WORDS) p.red[((checks + 1) % 3) * RED_WORDS + threadIdx.x] = 0ull;
        ++checks;
        load_shared_cg(sv, p.y, n);
        __syncthreads();
        for (int r = row0 + warp; r < row1; r += kWarps) {
            if (r < n) {
                const double v = row_dot(p.P + (size_t)r * n, sv, n, lane);
                if (lane == 0) {
                    p.Py[r] = v;
                    red_max(slot, RED_PX, p.rsx ? v * p.rsx[r] : v);
                }
            } else {
                const int i = r - n;
                const double v = row_dot(p.A + (size_t)i * n, sv, n, lane);
                if (lane == 0) {
                    const double zi = p.z[i];
                    const double rho_i = p.rho[ri] * (double)__ldg(p.rs + i);
                    const double f = p.rsz ? p.rsz[i] : 1.0;
                    p.Axf[i] = v;
                    p.lstd[i] = p.lam[i] + rho_i * (v - zi);
                    red_max(slot, RED_RP, (v - zi) * f);
                    red_max(slot, RED_AX, v * f);
                    red_max(slot, RED_Z, zi * f);
                }
            }
        }
        if (!grid_barrier(p, &s_ok)) return;
        if (m > 0) load_shared_cg(sv, p.lstd, m);
        __syncthreads();
        for (int j = r2_0 + warp; j < r2_1; j += kWarps) {
            const double v = (m > 0) ? row_dot(p.At + (size_t)j * m, sv, m, lane) : 0.0;
            if (lane == 0) {
                const double f = p.rsx ? p.rsx[j] : 1.0;
                red_max(slot, RED_RD, (__ldcg(p.Py + j) + __ldg(p.q + j) + v) * f);
                red_max(slot, RED_ATL, v * f);
            }
        }
        if (!grid_barrier(p, &s_ok)) return;

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
                p.out_i[OUT_STATUS] = numerical ? RELU_QP_NUMERICAL : (converged ? RELU_QP_SOLVED : RELU_QP_MAX_ITER);
                p.out_i[OUT_ITERS] = it;
                p.out_i[OUT_RHO] = ri;
                p.out_i[OUT_SWITCHES] = switches;
                p.out_f[0] = rp;
                p.out_f[1] = rd;
            }
            return;
        }
        // the directly computed Ax replaces the carried one
        for (int r = max(row0, n) + threadIdx.x; r < row1; r += blockDim.x) p.Ay[r - n] = p.Axf[r - n];
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
                    if (d < best) {
                        best = d;
                        nri = k;
                    }
                }
            }
        }
        if (nri == ri) continue;
        // switch: rebase lam' so that the next layer is standard ADMM with the new rho
        double* scur2 = cur ? p.s1 : p.s0;
        for (int r = max(row0, n) + threadIdx.x; r < row1; r += blockDim.x) {
            const int i = r - n;
            const double rho_i = p.rho[nri] * (double)__ldg(p.rs + i);
            const double zi = p.z[i];
            const double lnew = p.lstd[i] - rho_i * (p.Axf[i] - zi);
            p.lam[i] = lnew;
            scur2[r] = 2.0 * rho_i * zi - lnew;
        }
        ri = nri;
        ++switches;
        if (!grid_barrier(p, &s_ok)) return;
    }
}

// Start state: x given (or 0), z = A x, carried Ax = A x, lam' = lam (or 0),
// s0 = [x; 2 rho z - lam'] for the starting bank entry.
__global__ void init64_kernel(int n, int m, const double* __restrict__ A, const double* __restrict__ xin,
                              const double* __restrict__ lin, const float* __restrict__ rs, double rho, double* y,
                              double* z, double* lam, double* Ay, double* s0) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < n + m; r += nw) {
        if (r < n) {
            if (lane == 0) {
                const double v = xin ? xin[r] : 0.0;
                y[r] = v;
                s0[r] = v;
            }
        } else {
            const int i = r - n;
            double v = 0.0;
            if (xin) {
                for (int k = lane; k < n; k += 32) v = fma(A[(size_t)i * n + k], xin[k], v);
                v = warp_sum(v);
            }
            if (lane == 0) {
                const double li = lin ? lin[i] : 0.0;
                const double rho_i = rho * (double)rs[i];
                z[i] = v;
                Ay[i] = v;
                lam[i] = li;
                s0[r] = 2.0 * rho_i * v - li;
            }
        }
    }
}

// out[r] = sum_k M[r][k] x[k] (row-major, ld = cols), one warp per row.
__global__ void matvec64_kernel(const double* __restrict__ M, int rows, int cols, const double* __restrict__ x,
                                double* __restrict__ out) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < rows; r += nw) {
        double v = 0.0;
        for (int k = lane; k < cols; k += 32) v = fma(M[(size_t)r * cols + k], x[k], v);
        v = warp_sum(v);
        if (lane == 0) out[r] = v;
    }
}

void fill_params(relu_qp_t h, SP64& p, int grid) {
    p.n = h->n;
    p.m = h->m;
    p.R = h->R;
    p.nr = h->nr;
    p.ldw = h->ldw;
    p.anchor_every = h->opts.check_interval > 0 ? h->opts.check_interval : 25;
    p.c = h->sw64.c;
    p.sref = h->sw64.sref;
    p.d32 = h->sw64.d32;
    for (int r = 0; r < h->nr; ++r) {
        p.Wt32[r] = h->be[r].Wt;
        p.Wt[r] = h->be[r].Wt64;
        p.bias[r] = h->be[r].bias64;
        p.rho[r] = h->be[r].rho;
    }
    p.P = h->P64; p.A = h->A64; p.At = h->At64;
    p.q = h->q64; p.l = h->l64; p.u = h->u64; p.rs = h->rs32;
    p.rsx = h->sc64_rx;
    p.rsz = h->sc64_z;
    SingleWork64& w = h->sw64;
    p.y = w.y; p.z = w.z; p.lam = w.lam; p.Ay = w.Ay; p.s0 = w.s0; p.s1 = w.s1;
    p.Py = w.Py; p.Axf = w.Axf; p.lstd = w.lstd;
    p.red = w.red; p.bar = w.bar; p.out_i = w.out_i; p.out_f = w.out_f;
    p.rows_per_cta = ceil_div(h->R, grid);
    p.rows2_per_cta = ceil_div(h->n, grid);
    p.timeout_ns = 2000000000LL;
    p.qnorm = h->qnorm;
}

// the operand in shared memory: R doubles, or (refined layers) ldw floats of the increment
size_t smem64(relu_qp_t h) {
    return std::max(sizeof(double) * (size_t)h->R, sizeof(float) * (size_t)h->ldw);
}

bool refined(relu_qp_t h) { return h->opts.single_precision == RELU_QP_PREC_FP64R; }

const void* kernel_for(relu_qp_t h) {
    return refined(h) ? (const void*)single64_kernel<true> : (const void*)single64_kernel<false>;
}

int init_state(relu_qp_t h, const double* x, const double* lam, int rho_index) {
    SingleWork64& w = h->sw64;
    const int R = h->R;
    // s1 and the padding of s0 start at zero
    RQ_CUDA(h, cudaMemsetAsync(w.s1, 0, sizeof(double) * R, h->stream));
    const int blocks = std::max(1, std::min(1024, ceil_div(R * 32, 256)));
    init64_kernel<<<blocks, 256, 0, h->stream>>>(h->n, h->m, h->A64, x, lam, h->rs32, h->be[rho_index].rho, w.y, w.z,
                                                 w.lam, w.Ay, w.s0);
    RQ_CUDA(h, cudaGetLastError());
    return RELU_QP_OK;
}

int launch(relu_qp_t h, int grid, int rho_index, double eps_abs, double eps_rel, int max_iter, int check_interval,
           int adaptive) {
    SP64 p{};
    fill_params(h, p, grid);
    p.rho_index0 = rho_index;
    p.check_interval = check_interval;
    p.adaptive = adaptive;
    p.max_iter = max_iter;
    p.eps_abs = eps_abs;
    p.eps_rel = eps_rel;
    SingleWork64& w = h->sw64;
    RQ_CUDA(h, cudaMemsetAsync(w.red, 0, sizeof(unsigned long long) * 3 * RED_WORDS, h->stream));
    RQ_CUDA(h, cudaMemsetAsync(w.bar, 0, sizeof(unsigned) * 2, h->stream));
    RQ_CUDA(h, cudaMemsetAsync(w.out_i, 0, sizeof(int) * OUT_WORDS, h->stream));
    const size_t smem = smem64(h);
    RQ_CUDA(h, cudaFuncSetAttribute(kernel_for(h), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    void* args[] = {&p};
    RQ_CUDA(h, cudaLaunchCooperativeKernel(kernel_for(h), dim3(grid), dim3(kThreads), args, smem,
                                           h->stream));
    return RELU_QP_OK;
}

}  // namespace

int single64_alloc(relu_qp_t h, const double* P, const double* A) {
    const int n = h->n, m = h->m, R = h->R, mm = m > 0 ? m : 1;
    if (R > kMaxRows64)
        return fail(h, RELU_QP_ERR_INVALID,
                    "single_precision FP64 supports n + m <= " + std::to_string(kMaxRows64));
    RQ_TRY(alloc(h, &h->P64, (size_t)n * n));
    RQ_TRY(alloc(h, &h->A64, (size_t)mm * n));
    RQ_TRY(alloc(h, &h->At64, (size_t)n * mm));
    RQ_TRY(alloc(h, &h->q64, (size_t)n));
    RQ_TRY(alloc(h, &h->l64, (size_t)mm));
    RQ_TRY(alloc(h, &h->u64, (size_t)mm));
    for (int r = 0; r < h->nr; ++r) RQ_TRY(alloc(h, &h->be[r].bias64, (size_t)R));
    SingleWork64& w = h->sw64;
    for (double** v : {&w.y, &w.z, &w.lam, &w.Ay, &w.s0, &w.s1, &w.Py, &w.Axf, &w.lstd, &w.xin, &w.lin, &w.c, &w.sref})
        RQ_TRY(alloc(h, v, (size_t)R));
    RQ_TRY(alloc(h, &w.d32, (size_t)h->ldw));   // zero beyond R (set once here)
    RQ_TRY(alloc(h, &w.red, 3 * RED_WORDS));
    RQ_TRY(alloc(h, &w.bar, 2));
    RQ_TRY(alloc(h, &w.out_i, OUT_WORDS));
    RQ_TRY(alloc(h, &w.out_f, 8));
    RQ_CUDA(h, cudaMemcpy(h->P64, P, sizeof(double) * n * n, cudaMemcpyHostToDevice));
    if (m > 0) {
        std::vector<double> At((size_t)n * m);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) At[(size_t)j * m + i] = A[(size_t)i * n + j];
        RQ_CUDA(h, cudaMemcpy(h->A64, A, sizeof(double) * (size_t)m * n, cudaMemcpyHostToDevice));
        RQ_CUDA(h, cudaMemcpy(h->At64, At.data(), sizeof(double) * At.size(), cudaMemcpyHostToDevice));
    }
    if (h->scaled) {
        std::vector<double> fx(n), fz(mm, 1.0);
        for (int j = 0; j < n; ++j) fx[j] = 1.0 / (h->sC * h->sD[j]);
        for (int i = 0; i < m; ++i) fz[i] = 1.0 / h->sE[i];
        RQ_TRY(alloc(h, &h->sc64_rx, (size_t)n));
        RQ_TRY(alloc(h, &h->sc64_z, (size_t)mm));
        RQ_CUDA(h, cudaMemcpy(h->sc64_rx, fx.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        RQ_CUDA(h, cudaMemcpy(h->sc64_z, fz.data(), sizeof(double) * mm, cudaMemcpyHostToDevice));
    }
    return RELU_QP_OK;
}

int single64_upload(relu_qp_t h, const double* q, const double* l, const double* u) {
    const int n = h->n, m = h->m, R = h->R;
    RQ_CUDA(h, cudaMemcpyAsync(h->q64, q, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    if (m > 0) {
        RQ_CUDA(h, cudaMemcpyAsync(h->l64, l, sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
        RQ_CUDA(h, cudaMemcpyAsync(h->u64, u, sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
    }
    const int blocks = std::max(1, std::min(2048, ceil_div(R * 32, 256)));
    for (int r = 0; r < h->nr; ++r) {
        matvec64_kernel<<<blocks, 256, 0, h->stream>>>(h->be[r].Bop64, R, n, h->q64, h->be[r].bias64);
        RQ_CUDA(h, cudaGetLastError());
    }
    // the host arrays are the caller's temporaries: finish the copies before returning
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return RELU_QP_OK;
}

// CTA count of the cooperative launch: the fastest of the co-resident
// candidates over 50 fixed-rho layers (no checks).
int single64_prepare(relu_qp_t h) {
    int per_sm = 0;
    const size_t smem = smem64(h);
    RQ_CUDA(h, cudaFuncSetAttribute(kernel_for(h), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for(h), kThreads, smem));
    if (per_sm < 1) return fail(h, RELU_QP_ERR_UNSUPPORTED, "FP64 solve kernel does not fit on an SM");
    std::vector<int> cands;
    for (int g = 1; g <= h->num_sms; g *= 2) cands.push_back(g);
    cands.push_back(h->num_sms);
    int best_g = 1;
    float best_t = 1e30f;
    for (int g : cands) {
        if (g > h->R || g > per_sm * h->num_sms) continue;
        RQ_TRY(init_state(h, nullptr, nullptr, 0));
        RQ_TRY(launch(h, g, 0, 0.0, 0.0, 10, 0, 0));   // warm-up
        RQ_TRY(init_state(h, nullptr, nullptr, 0));
        RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
        RQ_TRY(launch(h, g, 0, 0.0, 0.0, 50, 0, 0));
        RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
        RQ_CUDA(h, cudaStreamSynchronize(h->stream));
        int err = 0;
        RQ_CUDA(h, cudaMemcpy(&err, h->sw64.out_i + OUT_ERR, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) return fail(h, RELU_QP_ERR_TIMEOUT, "grid barrier deadline passed while tuning the FP64 solve");
        float ms = 0.f;
        RQ_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        if (ms < best_t) {
            best_t = ms;
            best_g = g;
        }
    }
    h->sw64.grid = best_g;
    return RELU_QP_OK;
}

int single64_solve(relu_qp_t h, const double* x_warm, const double* lam_warm, int rho_index, double eps_abs,
                   double eps_rel, int max_iter, double* x_out, double* z_out, double* lam_out,
                   relu_qp_info* info) {
    SingleWork64& w = h->sw64;
    const int n = h->n, m = h->m;
    const double* xin = nullptr;
    const double* lin = nullptr;
    if (x_warm) {
        RQ_CUDA(h, cudaMemcpyAsync(w.xin, x_warm, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
        xin = w.xin;
        if (lam_warm && m > 0) {
            RQ_CUDA(h, cudaMemcpyAsync(w.lin, lam_warm, sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
            lin = w.lin;
        }
    }
    RQ_TRY(init_state(h, xin, lin, rho_index));
    RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
    RQ_TRY(launch(h, w.grid, rho_index, eps_abs, eps_rel, max_iter, h->opts.check_interval, h->opts.adaptive_rho));
    h->launches += 2;
    RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
    int oi[OUT_WORDS];
    double of[2];
    RQ_CUDA(h, cudaMemcpyAsync(oi, w.out_i, sizeof(oi), cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaMemcpyAsync(of, w.out_f, sizeof(of), cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaMemcpyAsync(x_out, w.y, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    if (z_out && m > 0) RQ_CUDA(h, cudaMemcpyAsync(z_out, w.z, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
    if (lam_out && m > 0)
        RQ_CUDA(h, cudaMemcpyAsync(lam_out, w.lstd, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    if (oi[OUT_ERR]) return fail(h, RELU_QP_ERR_TIMEOUT, "grid barrier deadline passed in the FP64 solve");
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
