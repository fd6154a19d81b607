// C ABI entry points of librelu_qp.so (declared in include/relu_qp.h).
#include "common.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

namespace {
thread_local std::string g_setup_error;

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// l <= u, no NaN, l != +inf, u != -inf.
bool bounds_ok(const double* l, const double* u, int m) {
    for (int i = 0; i < m; ++i) {
        if (std::isnan(l[i]) || std::isnan(u[i])) return false;
        if (l[i] > u[i]) return false;
        if (l[i] == INFINITY || u[i] == -INFINITY) return false;
    }
    return true;
}

std::vector<float> to_f32(const double* p, size_t n) {
    std::vector<float> v(n);
    for (size_t i = 0; i < n; ++i) v[i] = (float)p[i];
    return v;
}

// Algorithm 1 "Scale problem" (Sec. III-D "Preconditioning"): a modified Ruiz
// equilibration of the KKT matrix K = [[P, A^T], [A, 0]] in FP64.  Each iteration
// divides column j of K (and row j, K being symmetric) by the square root of its
// infinity norm (norms below 1e-4 count as 1, above 1e4 as 1e4) and then divides
// the cost by max(mean column infinity norm of P, |q|_inf) with the same limits.
// On return Ps = c D P D and As = E A D (row-major, in place).
void ruiz_equilibrate(int n, int m, std::vector<double>& Ps, std::vector<double>& As, const std::vector<double>& q,
                      int iters, std::vector<double>& D, std::vector<double>& E, double& c) {
    constexpr double kNormMin = 1e-4, kNormMax = 1e4;
    auto inv_sqrt = [&](double v) { return 1.0 / std::sqrt(v < kNormMin ? 1.0 : std::fmin(v, kNormMax)); };
    D.assign(n, 1.0);
    E.assign(m, 1.0);
    c = 1.0;
    std::vector<double> qs = q, cx(n), cz(m);
    for (int it = 0; it < iters; ++it) {
        std::fill(cx.begin(), cx.end(), 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) cx[j] = std::fmax(cx[j], std::fabs(Ps[(size_t)i * n + j]));
        for (int i = 0; i < m; ++i) {
            double r = 0.0;
            for (int j = 0; j < n; ++j) {
                const double a = std::fabs(As[(size_t)i * n + j]);
                cx[j] = std::fmax(cx[j], a);
                r = std::fmax(r, a);
            }
            cz[i] = r;
        }
        for (int j = 0; j < n; ++j) cx[j] = inv_sqrt(cx[j]);
        for (int i = 0; i < m; ++i) cz[i] = inv_sqrt(cz[i]);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) Ps[(size_t)i * n + j] *= cx[i] * cx[j];
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) As[(size_t)i * n + j] *= cz[i] * cx[j];
        for (int j = 0; j < n; ++j) {
            qs[j] *= cx[j];
            D[j] *= cx[j];
        }
        for (int i = 0; i < m; ++i) E[i] *= cz[i];
        // cost scale
        std::fill(cx.begin(), cx.end(), 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) cx[j] = std::fmax(cx[j], std::fabs(Ps[(size_t)i * n + j]));
        double mean = 0.0, qn = 0.0;
        for (int j = 0; j < n; ++j) {
            mean += cx[j];
            qn = std::fmax(qn, std::fabs(qs[j]));
        }
        mean /= n;
        double cost = std::fmax(mean, qn);
        cost = cost < kNormMin ? 1.0 : std::fmin(cost, kNormMax);
        const double gamma = 1.0 / cost;
        for (double& v : Ps) v *= gamma;
        for (double& v : qs) v *= gamma;
        c *= gamma;
    }
}

// Factor vectors of a scaled handle on the device (FP32).
int upload_scaling(relu_qp_t h) {
    const int n = h->n, m = h->m, mm = m > 0 ? m : 1;
    std::vector<float> f(n > mm ? n : mm);
    auto put = [&](float** dst, int len, auto fn) -> int {
        RQ_TRY(rq::alloc(h, dst, (size_t)len));
        for (int k = 0; k < len; ++k) f[k] = (float)fn(k);
        RQ_CUDA(h, cudaMemcpy(*dst, f.data(), sizeof(float) * len, cudaMemcpyHostToDevice));
        return RELU_QP_OK;
    };
    const std::vector<double>& D = h->sD;
    const std::vector<double>& E = h->sE;
    const double c = h->sC;
    RQ_TRY(put(&h->sc_q, n, [&](int k) { return c * D[k]; }));
    RQ_TRY(put(&h->sc_x, n, [&](int k) { return D[k]; }));
    RQ_TRY(put(&h->sc_xi, n, [&](int k) { return 1.0 / D[k]; }));
    RQ_TRY(put(&h->sc_rx, n, [&](int k) { return 1.0 / (c * D[k]); }));
    RQ_TRY(put(&h->sc_e, mm, [&](int i) { return i < m ? E[i] : 1.0; }));
    RQ_TRY(put(&h->sc_z, mm, [&](int i) { return i < m ? 1.0 / E[i] : 1.0; }));
    RQ_TRY(put(&h->sc_l, mm, [&](int i) { return i < m ? E[i] / c : 1.0; }));
    RQ_TRY(put(&h->sc_li, mm, [&](int i) { return i < m ? c / E[i] : 1.0; }));
    return RELU_QP_OK;
}

int upload_problem(relu_qp_t h) {
    const int n = h->n, m = h->m;
    std::vector<float> q(n);
    for (int j = 0; j < n; ++j) q[j] = (float)(h->scaled ? h->sC * h->sD[j] * h->h_q[j] : h->h_q[j]);
    RQ_CUDA(h, cudaMemcpyAsync(h->q32, q.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
    if (m > 0) {
        std::vector<float> l(m), u(m);
        for (int i = 0; i < m; ++i) {
            const double e = h->scaled ? h->sE[i] : 1.0;
            l[i] = (float)(e * h->h_l[i]);
            u[i] = (float)(e * h->h_u[i]);
        }
        RQ_CUDA(h, cudaMemcpyAsync(h->l32, l.data(), sizeof(float) * m, cudaMemcpyHostToDevice, h->stream));
        RQ_CUDA(h, cudaMemcpyAsync(h->u32, u.data(), sizeof(float) * m, cudaMemcpyHostToDevice, h->stream));
        RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    double qn = 0.0;
    for (int i = 0; i < n; ++i) qn = std::fmax(qn, std::fabs(h->h_q[i]));
    h->qnorm = qn;
    if (h->opts.single_precision != RELU_QP_PREC_FP32) {
        std::vector<double> q64(n), l64(m), u64(m);
        for (int j = 0; j < n; ++j) q64[j] = h->scaled ? h->sC * h->sD[j] * h->h_q[j] : h->h_q[j];
        for (int i = 0; i < m; ++i) {
            const double e = h->scaled ? h->sE[i] : 1.0;
            l64[i] = e * h->h_l[i];
            u64[i] = e * h->h_u[i];
        }
        RQ_TRY(rq::single64_upload(h, q64.data(), l64.data(), u64.data()));
    }
    RQ_TRY(rq::compute_bias(h));
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return RELU_QP_OK;
}

int setup_impl(relu_qp_t h, const double* P, const double* q, const double* A, const double* l,
               const double* u, const double* rho_bank) {
    const int n = h->n, m = h->m, R = h->R;
    RQ_CUDA(h, cudaGetDevice(&h->device));
    RQ_CUDA(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    RQ_CUDA(h, cudaEventCreate(&h->ev0));
    RQ_CUDA(h, cudaEventCreate(&h->ev1));
    h->h_q.assign(n, 0.0);
    if (q) std::memcpy(h->h_q.data(), q, sizeof(double) * n);
    h->h_l.assign(l, l + m);
    h->h_u.assign(u, u + m);
    h->eq.resize(m);
    std::vector<double> row_scale(m);
    std::vector<float> rs(m > 0 ? m : 1, 1.0f);
    for (int i = 0; i < m; ++i) {
        h->eq[i] = (l[i] == u[i]) ? 1 : 0;
        row_scale[i] = h->eq[i] ? h->opts.eq_scale : 1.0;
        rs[i] = (float)row_scale[i];
    }
    const int ldp = (int)rq::round_up(n, 4), ldt = (int)rq::round_up(m > 0 ? m : 1, 4);
    for (int r = 0; r < h->nr; ++r) {
        rq::BankEntry& be = h->be[r];
        be.rho = rho_bank[r];
        RQ_TRY(rq::alloc(h, &be.Wt, (size_t)R * h->ldw));
        RQ_TRY(rq::alloc(h, &be.Bop, (size_t)R * n));
        RQ_TRY(rq::alloc(h, &be.bias, (size_t)R));
        if (h->opts.keep_fp64) {
            RQ_TRY(rq::alloc(h, &be.Wt64, (size_t)R * R));
            RQ_TRY(rq::alloc(h, &be.Bop64, (size_t)R * n));
        }
    }
    RQ_TRY(rq::alloc(h, &h->P32, (size_t)n * ldp));
    RQ_TRY(rq::alloc(h, &h->A32, (size_t)(m > 0 ? m : 1) * ldp));
    RQ_TRY(rq::alloc(h, &h->At32, (size_t)n * ldt));
    RQ_TRY(rq::alloc(h, &h->q32, (size_t)n));
    RQ_TRY(rq::alloc(h, &h->l32, (size_t)(m > 0 ? m : 1)));
    RQ_TRY(rq::alloc(h, &h->u32, (size_t)(m > 0 ? m : 1)));
    RQ_TRY(rq::alloc(h, &h->rs32, (size_t)(m > 0 ? m : 1)));
    RQ_CUDA(h, cudaMemcpy(h->rs32, rs.data(), sizeof(float) * rs.size(), cudaMemcpyHostToDevice));
    rq::SingleWork& w = h->sw;
    RQ_TRY(rq::alloc(h, &w.y, (size_t)h->ldw));
    RQ_TRY(rq::alloc(h, &w.z, (size_t)ldt));
    RQ_TRY(rq::alloc(h, &w.lam, (size_t)ldt));
    RQ_TRY(rq::alloc(h, &w.Ay, (size_t)ldt));
    RQ_TRY(rq::alloc(h, &w.s0, (size_t)h->ldw));
    RQ_TRY(rq::alloc(h, &w.s1, (size_t)h->ldw));
    RQ_TRY(rq::alloc(h, &w.Py, (size_t)ldp));
    RQ_TRY(rq::alloc(h, &w.Axf, (size_t)ldt));
    RQ_TRY(rq::alloc(h, &w.lstd, (size_t)ldt));
    RQ_TRY(rq::alloc(h, &w.xin, (size_t)ldp));
    RQ_TRY(rq::alloc(h, &w.lin, (size_t)ldt));
    RQ_TRY(rq::alloc(h, &w.red, 3 * 8));
    RQ_TRY(rq::alloc(h, &w.bar, 2));
    RQ_TRY(rq::alloc(h, &w.out_i, 8));
    RQ_TRY(rq::alloc(h, &w.out_f, 8));
    if (h->opts.max_batch > 0) RQ_TRY(rq::batch_alloc(h));
    // problem scaling: the offline stage below sees the scaled P and A
    std::vector<double> Ps, As;
    if (h->opts.scaling_iters > 0) {
        Ps.assign(P, P + (size_t)n * n);
        if (m > 0) As.assign(A, A + (size_t)m * n);
        ruiz_equilibrate(n, m, Ps, As, h->h_q, h->opts.scaling_iters, h->sD, h->sE, h->sC);
        P = Ps.data();
        A = m > 0 ? As.data() : A;
        h->scaled = 1;
        RQ_TRY(upload_scaling(h));
    }
    // FP64 inputs for the offline stage (freed at the end of setup)
    double *dP = nullptr, *dA = nullptr;
    cudaError_t e1 = cudaMalloc(&dP, sizeof(double) * n * n);
    cudaError_t e2 = cudaMalloc(&dA, sizeof(double) * (size_t)(m > 0 ? m : 1) * n);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaFree(dP);
        cudaFree(dA);
        cudaGetLastError();
        return rq::fail(h, RELU_QP_ERR_OOM, "setup: FP64 input allocation failed");
    }
    int rc = RELU_QP_OK;
    if (cudaMemcpy(dP, P, sizeof(double) * n * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        (m > 0 && cudaMemcpy(dA, A, sizeof(double) * (size_t)m * n, cudaMemcpyHostToDevice) != cudaSuccess))
        rc = rq::fail(h, RELU_QP_ERR_CUDA, "setup: FP64 input upload failed");
    if (rc == RELU_QP_OK) rc = rq::make_check_matrices(h, dP, dA);
    if (rc == RELU_QP_OK) rc = rq::build_bank(h, dP, dA, row_scale);
    if (rc == RELU_QP_OK && h->bw.cap > 0 && h->bw.prec == RELU_QP_PREC_BF16X3)
        rc = rq::pack_bf16_check(h, dP, dA);
    if (rc == RELU_QP_OK && h->opts.single_precision != RELU_QP_PREC_FP32) rc = rq::single64_alloc(h, P, A);
    cudaStreamSynchronize(h->stream);
    cudaFree(dP);
    cudaFree(dA);
    if (rc != RELU_QP_OK) return rc;
    RQ_TRY(upload_problem(h));
    RQ_TRY(rq::single_prepare(h));
    if (h->opts.single_precision != RELU_QP_PREC_FP32) RQ_TRY(rq::single64_prepare(h));
    if (h->bw.cap > 0) RQ_TRY(rq::batch_finish_setup(h));
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return RELU_QP_OK;
}

int nearest_index(relu_qp_t h, double rho) {
    int best = 0;
    double bd = 1e300;
    for (int k = 0; k < h->nr; ++k) {
        const double d = std::fabs(std::log(rho) - std::log(h->bank[k]));
        if (d < bd) {
            bd = d;
            best = k;
        }
    }
    return best;
}

}  // namespace

namespace rq {

int fail(relu_qp_t h, int code, const std::string& msg) {
    if (h)
        h->err = msg;
    else
        g_setup_error = msg;
    return code;
}

int dev_alloc(relu_qp_t h, void** p, size_t bytes) {
    *p = nullptr;
    const long long cap = h->opts.device_budget;
    if (cap > 0 && h->dev_bytes + bytes > (size_t)cap)
        return fail(h, RELU_QP_ERR_OOM, "device-memory budget of " + std::to_string(cap) + " bytes exceeded (" +
                                             std::to_string(h->dev_bytes) + " held, " + std::to_string(bytes) +
                                             " more asked)");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(h, RELU_QP_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) +
                                            " bytes): " + cudaGetErrorString(e));
    }
    h->allocs.push_back(*p);
    h->dev_bytes += bytes;
    e = cudaMemset(*p, 0, bytes);
    if (e != cudaSuccess) return fail(h, RELU_QP_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
    return RELU_QP_OK;
}

}  // namespace rq

extern "C" {

void relu_qp_default_opts(relu_qp_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->check_interval = 25;
    o->adaptive_rho = 1;
    o->rho0 = 0.1;
    o->eq_scale = 1e3;
    o->keep_fp64 = 0;
    o->max_batch = 0;
    o->batch_precision = RELU_QP_PREC_FP32;
    o->stream = nullptr;
    o->scaling_iters = 0;
    o->single_precision = RELU_QP_PREC_FP32;
}

int relu_qp_setup(relu_qp_t* out, int n, int m, const double* P, const double* q, const double* A,
                  const double* l, const double* u, double sigma, const double* rho_bank, int n_rho,
                  const relu_qp_opts* opts) {
    if (out) *out = nullptr;
    if (!out) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "out is NULL");
    if (n < 1 || m < 0 || (long)n + m > 40000)
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "need 1 <= n and 0 <= m with n + m <= 40000");
    if (!P || (m > 0 && (!A || !l || !u)) || !rho_bank)
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "P, A, l, u and rho_bank are required");
    if (!(sigma > 0.0) || !std::isfinite(sigma))
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "sigma must be finite and > 0");
    if (n_rho < 1 || n_rho > RQ_MAX_RHO)
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "n_rho must be in [1, 16]");
    for (int r = 0; r < n_rho; ++r)
        if (!(rho_bank[r] > 0.0) || !std::isfinite(rho_bank[r]))
            return rq::fail(nullptr, RELU_QP_ERR_INVALID, "rho_bank entries must be finite and > 0");
    if (!finite_all(P, (size_t)n * n) || (m > 0 && !finite_all(A, (size_t)m * n)) ||
        (q && !finite_all(q, n)))
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "P, q and A must be finite");
    if (m > 0 && !bounds_ok(l, u, m))
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "bounds need l <= u, no NaN, l != +inf, u != -inf");
    relu_qp_opts o;
    relu_qp_default_opts(&o);
    if (opts) o = *opts;
    if (o.check_interval < 0 || !(o.rho0 > 0.0) || !(o.eq_scale > 0.0) || o.scaling_iters < 0 ||
        o.scaling_iters > 100)
        return rq::fail(nullptr, RELU_QP_ERR_INVALID,
                        "opts: check_interval >= 0, rho0 > 0, eq_scale > 0, 0 <= scaling_iters <= 100");
    if (o.max_batch < 0 || o.max_batch > (1 << 20) ||
        (o.batch_precision != RELU_QP_PREC_FP32 && o.batch_precision != RELU_QP_PREC_BF16X3))
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "opts: 0 <= max_batch <= 2^20, batch_precision FP32 or BF16X3");
    if (o.single_precision != RELU_QP_PREC_FP32 && o.single_precision != RELU_QP_PREC_FP64 &&
        o.single_precision != RELU_QP_PREC_FP64R)
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "opts: single_precision FP32, FP64 or FP64R");
    if (o.device_budget < 0) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "opts: device_budget >= 0");
    if (o.single_precision != RELU_QP_PREC_FP32) o.keep_fp64 = 1;   // the FP64 solves read the FP64 bank
    relu_qp_t h = new (std::nothrow) relu_qp_s;
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_OOM, "host allocation failed");
    h->n = n;
    h->m = m;
    h->R = n + m;
    h->ldw = (int)rq::round_up(h->R, 64);
    h->nr = n_rho;
    h->sigma = sigma;
    h->opts = o;
    h->stream = (cudaStream_t)o.stream;
    h->bank.assign(rho_bank, rho_bank + n_rho);
    static const double empty = 0.0;
    const int rc = setup_impl(h, P, q, A, m > 0 ? l : &empty, m > 0 ? u : &empty, rho_bank);
    if (rc != RELU_QP_OK) {
        g_setup_error = h->err;
        relu_qp_destroy(h);
        return rc;
    }
    *out = h;
    return RELU_QP_OK;
}

int relu_qp_update(relu_qp_t h, const double* q, const double* l, const double* u) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    const int n = h->n, m = h->m;
    if (q && !finite_all(q, n)) return rq::fail(h, RELU_QP_ERR_INVALID, "q must be finite");
    std::vector<double> nl = h->h_l, nu = h->h_u;
    if (l) nl.assign(l, l + m);
    if (u) nu.assign(u, u + m);
    if (m > 0 && !bounds_ok(nl.data(), nu.data(), m))
        return rq::fail(h, RELU_QP_ERR_INVALID, "bounds need l <= u, no NaN, l != +inf, u != -inf");
    for (int i = 0; i < m; ++i)
        if ((nl[i] == nu[i]) != (h->eq[i] != 0))
            return rq::fail(h, RELU_QP_ERR_INVALID, "the equality-row pattern (l_i == u_i) changed since setup");
    if (q) std::memcpy(h->h_q.data(), q, sizeof(double) * n);
    h->h_l = nl;
    h->h_u = nu;
    return upload_problem(h);
}

int relu_qp_solve(relu_qp_t h, const double* x_warm, const double* lam_warm, int rho_index_warm,
                  double eps_abs, double eps_rel, int max_iter, double* x_out, double* z_out,
                  double* lam_out, relu_qp_info* info) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    if (!x_out || max_iter < 1 || !(eps_abs >= 0.0) || !(eps_rel >= 0.0) || rho_index_warm < -1 ||
        rho_index_warm >= h->nr)
        return rq::fail(h, RELU_QP_ERR_INVALID, "solve: x_out required, max_iter >= 1, eps >= 0, "
                                                "rho_index_warm in [-1, n_rho)");
    const int n = h->n, m = h->m;
    if (x_warm && !finite_all(x_warm, n)) return rq::fail(h, RELU_QP_ERR_INVALID, "x_warm must be finite");
    if (lam_warm && !finite_all(lam_warm, m)) return rq::fail(h, RELU_QP_ERR_INVALID, "lam_warm must be finite");
    const int ri = rho_index_warm >= 0 ? rho_index_warm : nearest_index(h, h->opts.rho0);
    const bool sc = h->scaled != 0;
    if (h->opts.single_precision != RELU_QP_PREC_FP32) {
        // scaled handles: xb = x / D, lamb = c lam / E in; x = D xb, z = zb / E, lam = E lamb / c out
        std::vector<double> xw, lw, zb(m), lb(m);
        if (x_warm) {
            xw.assign(x_warm, x_warm + n);
            if (sc)
                for (int j = 0; j < n; ++j) xw[j] /= h->sD[j];
            if (lam_warm && m > 0) {
                lw.assign(lam_warm, lam_warm + m);
                if (sc)
                    for (int i = 0; i < m; ++i) lw[i] *= h->sC / h->sE[i];
            }
        }
        relu_qp_info inf{};
        RQ_TRY(rq::single64_solve(h, x_warm ? xw.data() : nullptr, lw.empty() ? nullptr : lw.data(), ri, eps_abs,
                                  eps_rel, max_iter, x_out, m > 0 ? zb.data() : nullptr,
                                  m > 0 ? lb.data() : nullptr, &inf));
        if (sc)
            for (int j = 0; j < n; ++j) x_out[j] *= h->sD[j];
        for (int i = 0; i < m; ++i) {
            if (z_out) z_out[i] = sc ? zb[i] / h->sE[i] : zb[i];
            if (lam_out) lam_out[i] = sc ? h->sE[i] * lb[i] / h->sC : lb[i];
        }
        if (info) *info = inf;
        return RELU_QP_OK;
    }
    const float* xin = nullptr;
    const float* lin = nullptr;
    if (x_warm) {
        // scaled handles: xb = x / D, lamb = c lam / E
        std::vector<float> xf(n);
        for (int j = 0; j < n; ++j) xf[j] = (float)(h->scaled ? x_warm[j] / h->sD[j] : x_warm[j]);
        RQ_CUDA(h, cudaMemcpyAsync(h->sw.xin, xf.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
        xin = h->sw.xin;
        if (lam_warm && m > 0) {
            std::vector<float> lf(m);
            for (int i = 0; i < m; ++i) lf[i] = (float)(h->scaled ? h->sC * lam_warm[i] / h->sE[i] : lam_warm[i]);
            RQ_CUDA(h, cudaMemcpyAsync(h->sw.lin, lf.data(), sizeof(float) * m, cudaMemcpyHostToDevice,
                                       h->stream));
            lin = h->sw.lin;
        }
        RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    relu_qp_info inf{};
    RQ_TRY(rq::single_solve(h, xin, lin, ri, eps_abs, eps_rel, max_iter, &inf));
    // scaled handles: x = D xb, z = zb / E, lam = E lamb / c
    std::vector<float> buf((size_t)(n > m ? n : m));
    RQ_CUDA(h, cudaMemcpy(buf.data(), h->sw.y, sizeof(float) * n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) x_out[i] = sc ? h->sD[i] * (double)buf[i] : buf[i];
    if (z_out && m > 0) {
        RQ_CUDA(h, cudaMemcpy(buf.data(), h->sw.z, sizeof(float) * m, cudaMemcpyDeviceToHost));
        for (int i = 0; i < m; ++i) z_out[i] = sc ? (double)buf[i] / h->sE[i] : buf[i];
    }
    if (lam_out && m > 0) {
        RQ_CUDA(h, cudaMemcpy(buf.data(), h->sw.lstd, sizeof(float) * m, cudaMemcpyDeviceToHost));
        for (int i = 0; i < m; ++i) lam_out[i] = sc ? h->sE[i] * (double)buf[i] / h->sC : buf[i];
    }
    if (info) *info = inf;
    return RELU_QP_OK;
}

int relu_qp_solve_noalloc(relu_qp_t h, const float* x_warm, const float* lam_warm, int rho_index_warm,
                          double eps_abs, double eps_rel, int max_iter, float* x_out, float* z_out, float* lam_out,
                          relu_qp_info* info) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    if (!x_out || max_iter < 1 || !(eps_abs >= 0.0) || !(eps_rel >= 0.0) || rho_index_warm < -1 ||
        rho_index_warm >= h->nr || (lam_warm && !x_warm))
        return rq::fail(h, RELU_QP_ERR_INVALID, "solve_noalloc: x_out required, max_iter >= 1, eps >= 0, "
                                                "rho_index_warm in [-1, n_rho), lam_warm needs x_warm");
    if (h->scaled)
        return rq::fail(h, RELU_QP_ERR_UNSUPPORTED, "solve_noalloc: the handle was set up with scaling_iters > 0");
    if (h->opts.single_precision != RELU_QP_PREC_FP32)
        return rq::fail(h, RELU_QP_ERR_UNSUPPORTED, "solve_noalloc: the handle was set up for FP64 solves");
    const int ri = rho_index_warm >= 0 ? rho_index_warm : nearest_index(h, h->opts.rho0);
    return rq::single_solve_noalloc(h, x_warm, lam_warm, ri, eps_abs, eps_rel, max_iter, x_out, z_out, lam_out,
                                    info);
}

int relu_qp_get_layer(relu_qp_t h, int rho_index, double* Wt, double* Bop) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    if (rho_index < 0 || rho_index >= h->nr) return rq::fail(h, RELU_QP_ERR_INVALID, "rho_index out of range");
    const int n = h->n, R = h->R;
    const rq::BankEntry& be = h->be[rho_index];
    if (Wt) {
        if (be.Wt64) {
            RQ_CUDA(h, cudaMemcpy(Wt, be.Wt64, sizeof(double) * R * R, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f((size_t)R * R);
            RQ_CUDA(h, cudaMemcpy2D(f.data(), sizeof(float) * R, be.Wt, sizeof(float) * h->ldw, sizeof(float) * R,
                                    R, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < f.size(); ++i) Wt[i] = f[i];
        }
    }
    if (Bop) {
        if (be.Bop64) {
            RQ_CUDA(h, cudaMemcpy(Bop, be.Bop64, sizeof(double) * R * n, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f((size_t)R * n);
            RQ_CUDA(h, cudaMemcpy(f.data(), be.Bop, sizeof(float) * R * n, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < f.size(); ++i) Bop[i] = f[i];
        }
    }
    return RELU_QP_OK;
}

int relu_qp_set_opts(relu_qp_t h, const relu_qp_opts* opts) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    if (!opts || opts->check_interval < 0 || !(opts->rho0 > 0.0))
        return rq::fail(h, RELU_QP_ERR_INVALID, "opts: check_interval >= 0, rho0 > 0");
    h->opts.check_interval = opts->check_interval;
    h->opts.adaptive_rho = opts->adaptive_rho;
    h->opts.rho0 = opts->rho0;
    return RELU_QP_OK;
}

int relu_qp_dims(relu_qp_t h, int* n, int* m, int* n_rho) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    if (n) *n = h->n;
    if (m) *m = h->m;
    if (n_rho) *n_rho = h->nr;
    return RELU_QP_OK;
}

long long relu_qp_device_bytes(relu_qp_t h) { return h ? (long long)h->dev_bytes : -1; }

int relu_qp_single_config(relu_qp_t h, int* ctas, int* cluster, int* cached_rows) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    return rq::single_get_config(h, ctas, cluster, cached_rows);
}

int relu_qp_single_set_config(relu_qp_t h, int ctas, int cluster) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    return rq::single_set_config(h, ctas, cluster);
}

void relu_qp_destroy(relu_qp_t h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    rq::batch_release(h);
    for (cudaEvent_t e : h->prof_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : h->gap_ev)
        if (e) cudaEventDestroy(e);
    for (void* p : h->allocs) cudaFree(p);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

int relu_qp_update_batch(relu_qp_t h, int B, const float* Q, const float* L, const float* U) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    if (h->bw.cap <= 0) return rq::fail(h, RELU_QP_ERR_UNSUPPORTED, "handle was set up with max_batch = 0");
    if (B < 1 || B > h->bw.cap || !Q || (h->m > 0 && (!L || !U)))
        return rq::fail(h, RELU_QP_ERR_INVALID, "update_batch: 1 <= B <= max_batch; Q, L, U required");
    return rq::batch_update(h, B, Q, L, U);
}

int relu_qp_set_parametric(relu_qp_t h, int nx, const double* F, const double* E, const double* l0,
                           const double* u0) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    if (h->bw.cap <= 0) return rq::fail(h, RELU_QP_ERR_UNSUPPORTED, "handle was set up with max_batch = 0");
    if (nx < 1 || nx > 4096 || !F || (h->m > 0 && (!E || !l0 || !u0)))
        return rq::fail(h, RELU_QP_ERR_INVALID, "set_parametric: 1 <= nx <= 4096; F, E, l0, u0 required");
    if (!finite_all(F, (size_t)h->n * nx) || (h->m > 0 && !finite_all(E, (size_t)h->m * nx)))
        return rq::fail(h, RELU_QP_ERR_INVALID, "F and E must be finite");
    if (h->m > 0 && !bounds_ok(l0, u0, h->m))
        return rq::fail(h, RELU_QP_ERR_INVALID, "bounds need l0 <= u0, no NaN, l0 != +inf, u0 != -inf");
    for (int i = 0; i < h->m; ++i)
        if ((l0[i] == u0[i]) != (h->eq[i] != 0))
            return rq::fail(h, RELU_QP_ERR_INVALID, "the equality-row pattern (l_i == u_i) differs from setup");
    return rq::batch_set_parametric(h, nx, F, E, l0, u0);
}

int relu_qp_update_batch_x0(relu_qp_t h, int B, const float* X0) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    if (h->bw.cap <= 0 || h->bw.nx <= 0)
        return rq::fail(h, RELU_QP_ERR_UNSUPPORTED, "needs max_batch > 0 and relu_qp_set_parametric first");
    if (B < 1 || B > h->bw.cap || !X0) return rq::fail(h, RELU_QP_ERR_INVALID, "update_batch_x0: 1 <= B <= max_batch");
    return rq::batch_update_x0(h, B, X0);
}

int relu_qp_condense_mpc(int nx, int nu, int N, const double* A, const double* B, const double* Q,
                         const double* R, const double* Q_N, const double* umin, const double* umax,
                         const double* xmin, const double* xmax, const double* K, int lqr_precondition,
                         void* stream, double* P, double* A_con, double* F, double* E, double* l0,
                         double* u0, double* K_out) {
    if (nx < 1 || nu < 1 || N < 1 || (long)N * nu > 40000 || (long)N * nx > 1000000)
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "condense: nx, nu, N >= 1 and N nu <= 40000");
    if (!A || !B || !Q || !R || !P || !A_con || !F || !E || !l0 || !u0)
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "condense: A, B, Q, R and every output but K_out are required");
    if (!finite_all(A, (size_t)nx * nx) || !finite_all(B, (size_t)nx * nu) || !finite_all(Q, (size_t)nx * nx) ||
        !finite_all(R, (size_t)nu * nu) || (Q_N && !finite_all(Q_N, (size_t)nx * nx)) ||
        (K && !finite_all(K, (size_t)nu * nx)))
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "condense: A, B, Q, R, Q_N and K must be finite");
    for (int i = 0; i < nu; ++i) {
        const double lo = umin ? umin[i] : -INFINITY, hi = umax ? umax[i] : INFINITY;
        if (std::isnan(lo) || std::isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY)
            return rq::fail(nullptr, RELU_QP_ERR_INVALID, "condense: need umin <= umax, no NaN");
    }
    for (int i = 0; (xmin || xmax) && i < nx; ++i) {
        const double lo = xmin ? xmin[i] : -INFINITY, hi = xmax ? xmax[i] : INFINITY;
        if (std::isnan(lo) || std::isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY)
            return rq::fail(nullptr, RELU_QP_ERR_INVALID, "condense: need xmin <= xmax, no NaN");
    }
    const bool state = xmin || xmax;
    std::string err;
    const int rc = rq::condense_mpc(nx, nu, N, A, B, Q, R, Q_N, state, K, lqr_precondition, stream, P, A_con, F,
                                    E, K_out, &err);
    if (rc != RELU_QP_OK) return rq::fail(nullptr, rc, err);
    // bounds of the constraint rows: the limits of every stage
    for (int k = 0; k < N; ++k)
        for (int i = 0; i < nu; ++i) {
            l0[(size_t)k * nu + i] = umin ? umin[i] : -INFINITY;
            u0[(size_t)k * nu + i] = umax ? umax[i] : INFINITY;
        }
    if (state)
        for (int k = 0; k < N; ++k)
            for (int i = 0; i < nx; ++i) {
                l0[(size_t)N * nu + (size_t)k * nx + i] = xmin ? xmin[i] : -INFINITY;
                u0[(size_t)N * nu + (size_t)k * nx + i] = xmax ? xmax[i] : INFINITY;
            }
    return RELU_QP_OK;
}

int relu_qp_solve_batch(relu_qp_t h, int B, const float* X_warm, const float* Lam_warm, const int* rho_warm,
                        double eps_abs, double eps_rel, int max_iter, float* X_out, float* Z_out, float* Lam_out,
                        relu_qp_info* infos) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    if (h->bw.cap <= 0) return rq::fail(h, RELU_QP_ERR_UNSUPPORTED, "handle was set up with max_batch = 0");
    if (B < 1 || B > h->bw.B || !X_out || max_iter < 1 || !(eps_abs >= 0.0) || !(eps_rel >= 0.0))
        return rq::fail(h, RELU_QP_ERR_INVALID,
                        "solve_batch: 1 <= B <= the last update's batch, X_out required, max_iter >= 1, eps >= 0");
    if (rho_warm && !X_warm) return rq::fail(h, RELU_QP_ERR_INVALID, "rho_warm needs X_warm");
    return rq::batch_solve(h, B, X_warm, Lam_warm, rho_warm, eps_abs, eps_rel, max_iter, X_out, Z_out, Lam_out,
                           infos);
}

int relu_qp_server_create(relu_qp_server_t* out, relu_qp_t const* families, int n_families, const int* clients,
                          double eps_abs, double eps_rel, int max_iter) {
    if (!out) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!families || n_families < 1 || n_families > 16 || max_iter < 1 || !(eps_abs >= 0.0) || !(eps_rel >= 0.0))
        return rq::fail(nullptr, RELU_QP_ERR_INVALID, "server: 1..16 families, max_iter >= 1, eps >= 0");
    for (int f = 0; f < n_families; ++f) {
        relu_qp_t h = families[f];
        if (!h || h->bw.cap <= 0 || h->bw.nx <= 0 || h->opts.check_interval <= 0)
            return rq::fail(nullptr, RELU_QP_ERR_INVALID,
                            "server: every family needs max_batch > 0, check_interval > 0 and relu_qp_set_parametric");
        if (clients && (clients[f] < 0 || clients[f] > (1 << 20)))
            return rq::fail(nullptr, RELU_QP_ERR_INVALID, "server: clients per family in [0, 2^20]");
        for (int g = 0; g < f; ++g)
            if (families[g] == h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "server: families must be distinct");
    }
    relu_qp_server_t s = nullptr;
    const int rc = rq::server_create(&s, families, n_families, clients, eps_abs, eps_rel, max_iter);
    if (rc != RELU_QP_OK) {
        const std::string msg = s ? rq::server_error(s) : "server: host allocation failed";
        if (s) rq::server_destroy(s);
        return rq::fail(nullptr, rc, msg);
    }
    *out = s;
    return RELU_QP_OK;
}

int relu_qp_server_submit(relu_qp_server_t s, int family, int client, const float* x0, long long tag) {
    if (!s || !x0 || family < 0 || family >= rq::server_families(s) || client < -1 ||
        client >= rq::server_clients(s, family))
        return RELU_QP_ERR_INVALID;
    for (int k = 0; k < rq::server_nx(s, family); ++k)
        if (!std::isfinite(x0[k])) return RELU_QP_ERR_INVALID;
    return rq::server_submit(s, family, client, x0, tag);
}

int relu_qp_server_step(relu_qp_server_t s, int* active, int* waiting) {
    if (!s) return RELU_QP_ERR_INVALID;
    return rq::server_step(s, active, waiting);
}

int relu_qp_server_poll(relu_qp_server_t s, int max_results, relu_qp_result* results, float* x_out, int x_stride) {
    if (!s || max_results < 0) return RELU_QP_ERR_INVALID;
    return rq::server_poll(s, max_results, results, x_out, x_stride);
}

double relu_qp_server_clock(relu_qp_server_t s) { return s ? rq::server_clock(s) : 0.0; }

int relu_qp_server_set_budget(relu_qp_server_t s, long long bytes) {
    if (!s || bytes < 0) return RELU_QP_ERR_INVALID;
    return rq::server_set_budget(s, bytes);
}

int relu_qp_server_family_bytes(relu_qp_server_t s, int family, long long* fixed_bytes, long long* slot_bytes) {
    if (!s || family < 0 || family >= rq::server_families(s)) return RELU_QP_ERR_INVALID;
    return rq::server_family_bytes(s, family, fixed_bytes, slot_bytes);
}

long long relu_qp_server_bytes_in_use(relu_qp_server_t s) { return s ? rq::server_bytes_in_use(s) : -1; }

void relu_qp_server_destroy(relu_qp_server_t s) {
    if (s) rq::server_destroy(s);
}

const char* relu_qp_server_error(relu_qp_server_t s) { return s ? rq::server_error(s) : relu_qp_last_error(nullptr); }

int relu_qp_profile(relu_qp_t h, int enable, int reset, relu_qp_prof* out) {
    if (!h) return rq::fail(nullptr, RELU_QP_ERR_INVALID, "handle is NULL");
    if (out) {
        out->launches = h->launches;
        out->layer_launches = h->layer_launches;
        out->layer_timed = h->layer_timed;
        out->layer_ms = h->layer_ms;
        out->layer_flops = h->layer_flops;
        out->host_checks = h->host_checks;
        out->host_gap_ms = h->host_gap_ms;
        out->resident_launches = h->resident_launches;
    }
    if (reset) {
        h->launches = h->layer_launches = h->layer_timed = 0;
        h->layer_ms = h->layer_flops = 0.0;
        h->host_checks = h->resident_launches = 0;
        h->host_gap_ms = 0.0;
    }
    if (enable >= 0) {
        if (enable && h->prof_ev.empty()) {
            h->prof_ev.resize(2 * 8192, nullptr);
            for (auto& e : h->prof_ev) RQ_CUDA(h, cudaEventCreate(&e));
            h->gap_ev.resize(2 * 256, nullptr);
            for (auto& e : h->gap_ev) RQ_CUDA(h, cudaEventCreate(&e));
        }
        h->prof_on = enable ? 1 : 0;
    }
    return RELU_QP_OK;
}

const char* relu_qp_last_error(relu_qp_t h) {
    return h ? h->err.c_str() : g_setup_error.c_str();
}

}  // extern "C"
