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
// rest stream from L2), and each warp produces one row at a time (coalesced
// 128-bit loads, shuffle reduction).  A grid barrier separates layers; every
// barrier wait has a deadline after which the kernel records
// RELU_QP_ERR_TIMEOUT and returns.
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

__global__ void __launch_bounds__(kThreads, 1) single_solve_kernel(SP p) {
    extern __shared__ __align__(16) float smem[];
    __shared__ GridSyncState s_ok;
    grid_sync_init(&s_ok);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = p.n, m = p.m, R = p.R;
    const int row0 = blockIdx.x * p.rows_per_cta;
    const int row1 = min(row0 + p.rows_per_cta, R);
    const int ncache = max(0, min(p.cached_rows, row1 - row0));
    float* wcache = smem;
    float* sv = smem + (size_t)p.cached_rows * p.ldw;     // ldw floats
    const int r2_0 = blockIdx.x * p.rows2_per_cta;
    const int r2_1 = min(r2_0 + p.rows2_per_cta, n);

    int ri = p.rho_index0;
    int switches = 0, checks = 0, cur = 0;
    if (ncache > 0) load_w_cache(p, wcache, ri, row0, ncache);
    __syncthreads();

    for (int it = 1; it <= p.max_iter; ++it) {
        // ---------------- one layer: s[cur] -> s[cur^1] ----------------
        const float* scur = cur ? p.s1 : p.s0;
        float* snext = cur ? p.s0 : p.s1;
        load_shared_cg(sv, scur, p.ldw);
        __syncthreads();
        const float* Wg = p.Wt[ri];
        const float* bias = p.bias[ri];
        const double rho = p.rho[ri];
        for (int r = row0 + warp; r < row1; r += kWarps) {
            const int lr = r - row0;
            const float acc = (lr < ncache) ? row_dot(wcache + (size_t)lr * p.ldw, sv, p.ldw, lane)
                                            : row_dot_global(Wg + (size_t)r * p.ldw, sv, p.ldw, lane);
            if (lane == 0) {
                const float t = acc + __ldg(bias + r);
                if (r < n) {
                    p.y[r] = t;
                    snext[r] = t;
                } else {
                    const int i = r - n;
                    const float rho_i = (float)(rho * (double)__ldg(p.rs + i));
                    const float rr = p.Ay[i] - p.z[i] + p.lam[i] / rho_i;
                    const float zn = fminf(fmaxf(t + rr, __ldg(p.l + i)), __ldg(p.u + i));
                    const float ln = rho_i * rr;
                    p.Ay[i] = t;
                    p.z[i] = zn;
                    p.lam[i] = ln;
                    snext[r] = 2.0f * rho_i * zn - ln;
                }
            }
        }
        cur ^= 1;
        if (!grid_barrier(p, &s_ok)) return;

        const bool is_check = (p.check_interval > 0) && (it % p.check_interval == 0);
        const bool last = (it == p.max_iter);
        if (!is_check && !last) continue;

        // ---------------- residuals (Eqs. primal, dual) ----------------
        unsigned* slot = p.red + (checks % 3) * RED_WORDS;
        if (blockIdx.x == 0 && threadIdx.x < RED_WORDS)
            p.red[((checks + 1) % 3) * RED_WORDS + threadIdx.x] = 0u;
        ++checks;
        load_shared_cg(sv, p.y, p.ldp);
        __syncthreads();
        for (int r = row0 + warp; r < row1; r += kWarps) {
            if (r < n) {
                const float v = row_dot_global(p.P + (size_t)r * p.ldp, sv, p.ldp, lane);
                if (lane == 0) {
                    p.Py[r] = v;
                    red_max(slot, RED_PX, p.rsx ? v * p.rsx[r] : v);
                }
            } else {
                const int i = r - n;
                const float v = row_dot_global(p.A + (size_t)i * p.lda, sv, p.lda, lane);
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
        if (!grid_barrier(p, &s_ok)) return;
        if (m > 0) load_shared_cg(sv, p.lstd, p.ldt);
        __syncthreads();
        for (int j = r2_0 + warp; j < r2_1; j += kWarps) {
            const float v = (m > 0) ? row_dot_global(p.At + (size_t)j * p.ldt, sv, p.ldt, lane) : 0.f;
            if (lane == 0) {
                const float f = p.rsx ? p.rsx[j] : 1.f;
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
            scur2[r] = 2.0f * rho_i * zi - lnew;
        }
        ri = nri;
        ++switches;
        if (ncache > 0) load_w_cache(p, wcache, ri, row0, ncache);
        if (!grid_barrier(p, &s_ok)) return;
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

size_t smem_bytes(int cached_rows, int ldw) { return ((size_t)cached_rows + 1) * ldw * sizeof(float); }

// Largest dynamic shared memory the solve kernel may request: the opt-in
// per-block limit minus the kernel's static shared memory.
int max_shared(relu_qp_t h) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, single_solve_kernel) == cudaSuccess) v -= (int)fa.sharedSizeBytes;
    cudaGetLastError();
    return v - 256;
}

// Shared-memory rows a CTA of a `grid`-CTA launch can cache.
int cached_rows_for(relu_qp_t h, int grid) {
    const int rows = ceil_div(h->R, grid);
    const size_t budget = (size_t)max_shared(h);
    long cap = (long)(budget / ((size_t)h->ldw * sizeof(float))) - 1;
    if (cap < 0) cap = 0;
    return rows < cap ? rows : (int)cap;
}

int launch(relu_qp_t h, int grid, int cached, int rho_index, double eps_abs, double eps_rel,
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
    const size_t smem = smem_bytes(cached, h->ldw);
    RQ_CUDA(h, cudaFuncSetAttribute(single_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    void* args[] = {&p};
    RQ_CUDA(h, cudaLaunchCooperativeKernel((const void*)single_solve_kernel, dim3(grid), dim3(kThreads),
                                           args, smem, h->stream));
    return RELU_QP_OK;
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
    const int smem_max = max_shared(h);
    RQ_CUDA(h, cudaFuncSetAttribute(single_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    smem_max));
    std::vector<int> cands;
    for (int g = 1; g <= 4 * h->num_sms; g *= 2) cands.push_back(g);
    cands.push_back(h->num_sms);
    int best_g = 1, best_c = cached_rows_for(h, 1);
    float best_t = 1e30f;
    for (int g : cands) {
        if (g > h->R) continue;
        const int cached = cached_rows_for(h, g);
        RQ_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, single_solve_kernel, kThreads,
                                                                 smem_bytes(cached, h->ldw)));
        if (per_sm < 1 || g > per_sm * h->num_sms) continue;
        h->sw.grid = g;
        RQ_TRY(init_state(h, nullptr, nullptr, 0));
        RQ_TRY(launch(h, g, cached, 0, 0.0, 0.0, 10, 0, 0));   // warm-up
        RQ_TRY(init_state(h, nullptr, nullptr, 0));
        RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
        RQ_TRY(launch(h, g, cached, 0, 0.0, 0.0, 50, 0, 0));
        RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
        RQ_CUDA(h, cudaStreamSynchronize(h->stream));
        int err = 0;
        RQ_CUDA(h, cudaMemcpy(&err, h->sw.out_i + OUT_ERR, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) return fail(h, RELU_QP_ERR_TIMEOUT, "grid barrier deadline passed while tuning");
        float ms = 0.f;
        RQ_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
        if (ms < best_t) {
            best_t = ms;
            best_g = g;
            best_c = cached;
        }
    }
    h->sw.grid = best_g;
    h->sw.cached_rows = best_c;
    h->sw.rows_per_cta = ceil_div(h->R, best_g);
    return RELU_QP_OK;
}

int single_solve(relu_qp_t h, const float* x_warm, const float* lam_warm, int rho_index, double eps_abs,
                 double eps_rel, int max_iter, relu_qp_info* info) {
    SingleWork& w = h->sw;
    RQ_TRY(init_state(h, x_warm, lam_warm, rho_index));
    RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
    RQ_TRY(launch(h, w.grid, w.cached_rows, rho_index, eps_abs, eps_rel, max_iter, h->opts.check_interval,
                  h->opts.adaptive_rho));
    h->launches += 2;
    RQ_CUDA(h, cudaEventRecord(h->ev1, h->stream));
    int oi[OUT_WORDS];
    float of[2];
    RQ_CUDA(h, cudaMemcpyAsync(oi, w.out_i, sizeof(oi), cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaMemcpyAsync(of, w.out_f, sizeof(of), cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    if (oi[OUT_ERR]) return fail(h, RELU_QP_ERR_TIMEOUT, "grid barrier deadline passed in relu_qp_solve");
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
    const size_t smem = smem_bytes(p.cached_rows, ldw);
    RQ_CUDA(h, cudaFuncSetAttribute(single_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RQ_CUDA(h, cudaEventRecord(h->ev0, h->stream));
    void* args[] = {&p};
    RQ_CUDA(h, cudaLaunchCooperativeKernel((const void*)single_solve_kernel, dim3(h->sw.grid), dim3(kThreads),
                                           args, smem, h->stream));
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
    if (oi[OUT_ERR]) return fail(h, RELU_QP_ERR_TIMEOUT, "grid barrier deadline passed in relu_qp_solve_noalloc");
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
