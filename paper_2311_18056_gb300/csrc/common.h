// Internal declarations shared by the translation units of librelu_qp.so.
// Nothing here is part of the public ABI (include/relu_qp.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/relu_qp.h"

#define RQ_MAX_RHO 16

namespace rq {

// ---------------------------------------------------------------------------
// error plumbing: every CUDA call on the host goes through RQ_CUDA, which
// records a message on the handle and returns RELU_QP_ERR_CUDA.
// ---------------------------------------------------------------------------
struct Status {
    int code = RELU_QP_OK;
    std::string msg;
};

#define RQ_CUDA(h, call)                                                              \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            cudaGetLastError();                                                       \
            return ::rq::fail((h), e_ == cudaErrorMemoryAllocation ? RELU_QP_ERR_OOM  \
                                                                  : RELU_QP_ERR_CUDA, \
                              std::string(#call) + ": " + cudaGetErrorString(e_));    \
        }                                                                             \
    } while (0)

#define RQ_TRY(expr)                    \
    do {                                \
        int rc_ = (expr);               \
        if (rc_ != RELU_QP_OK) return rc_; \
    } while (0)

// Device buffer owned by a handle.
template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
};

// Per-bank-entry device data.
struct BankEntry {
    double rho = 0.0;
    float* Wt = nullptr;      // R x ldw FP32, rows [x; Ax], cols [x; 2 rho z - lam'] (padded)
    float* Bop = nullptr;     // R x n FP32: [-D; -A D]
    float* bias = nullptr;    // R FP32 = Bop q (single-QP path)
    double* Wt64 = nullptr;   // R x R FP64 (keep_fp64 or the FP64 single solve)
    double* Bop64 = nullptr;  // R x n FP64 (same)
    double* bias64 = nullptr; // R FP64 = Bop64 q (FP64 single solve)
};

// Workspace of the single-QP cooperative solve.
struct SingleWork {
    float *y = nullptr, *z = nullptr, *lam = nullptr, *Ay = nullptr;
    float *s0 = nullptr, *s1 = nullptr;
    float *Py = nullptr, *Axf = nullptr, *lstd = nullptr;
    float* xin = nullptr;       // warm-start x (FP32)
    float* lin = nullptr;       // warm-start lam (FP32)
    unsigned* red = nullptr;    // 3 slots x 8 reduction words
    unsigned* bar = nullptr;    // grid barrier: arrival count of the launch (+ pad word)
    int* out_i = nullptr;       // status, iters, rho_index, switches, err
    float* out_f = nullptr;     // r_prim, r_dual
    int grid = 0;               // CTAs of the launch (autotuned)
    int cluster = 0;            // > 1: the launch is one cluster of `grid` CTAs (else a cooperative grid)
    int cached_rows = 0;        // rows of W each CTA keeps in shared memory
    int rows_per_cta = 0;
};

// Workspace of the FP64 single-QP solve (opts.single_precision = FP64 or FP64R).
struct SingleWork64 {
    double *y = nullptr, *z = nullptr, *lam = nullptr, *Ay = nullptr;
    double *s0 = nullptr, *s1 = nullptr;
    double *Py = nullptr, *Axf = nullptr, *lstd = nullptr;
    double *xin = nullptr, *lin = nullptr;
    double *c = nullptr, *sref = nullptr;   // refined form: anchor layer product and its operand
    float* d32 = nullptr;                   // refined form: FP32 increment of the next layer (ldw)
    unsigned long long* red = nullptr;   // 3 slots x 8 reduction words (bits of non-negative doubles)
    unsigned* bar = nullptr;             // grid barrier: arrival count of the launch (+ pad word)
    int* out_i = nullptr;                // status, iters, rho_index, switches, err
    double* out_f = nullptr;             // r_prim, r_dual
    int grid = 0;
};

// Workspace of batched solves (allocated when opts.max_batch > 0).
struct BatchWork {
    int cap = 0, slots = 0, prec = 0, B = 0;
    int rebase_tc = 1;   // BF16 form: 1 = accurate layer on the tensor cores (3-way split, every
                         // k-block's products drained into FP32 sums; default), 0 = on the CUDA
                         // cores in FP32
    int check_tc = 1;    // BF16 form: 1 = residual products on the tensor cores (3-way split,
                         // drained like the accurate layer; default), 0 = on the CUDA cores in FP32
    int ldn = 0, ldm = 0, ldR = 0, ldk = 0, n64 = 0, m64 = 0, ldkc = 0, Rpad = 0, npad = 0;
    // check matrix [[P, A^T], [A, 0]]: (n + m) rows (padded to npad), ldkc = n64 + m64 columns
    // per-QP state (QP-indexed rows)
    float *Y = nullptr, *Z = nullptr, *LAM = nullptr, *AY = nullptr, *LSTD = nullptr;
    float* RR = nullptr;                   // BF16 form: r = (Ax) - z + lam'/rho carried between layers
    float *L = nullptr, *U = nullptr, *Q = nullptr, *QN = nullptr, *C = nullptr, *SREF = nullptr, *PY = nullptr;
    float* BIAS = nullptr;                 // [nr][cap][ldR]
    float *XO = nullptr, *ZO = nullptr, *LO = nullptr;   // dense outputs [cap][n|m]
    unsigned* RED = nullptr;               // [cap][8] per-QP reduction words
    int *rho_idx = nullptr, *status = nullptr, *iters = nullptr, *nsw = nullptr;
    float *rp = nullptr, *rd = nullptr;
    // slot data
    int *perm = nullptr, *tile_rho = nullptr, *counters = nullptr;
    // FP32 backend
    float *S32 = nullptr, *CK32 = nullptr, *Wc32 = nullptr;
    // BF16 split backend (tcgen05); 2-byte elements
    void *OPND = nullptr, *CK = nullptr, *WB = nullptr, *WCB = nullptr;
    void* tc = nullptr;                    // backend state (tensor maps, tuned tiles)
    // parametric problem: q = F x0, l = l0 - E x0, u = u0 - E x0
    int nx = 0, ldx = 0;
    float *F32 = nullptr, *Ft32 = nullptr, *E32 = nullptr, *l0 = nullptr, *u0 = nullptr, *X0 = nullptr;
    float* G[RQ_MAX_RHO] = {};             // G_r = Bop_r F
    // convergence tail (batch_tail.cu): operands, check operand, reduction and barrier words, QP list
    float *TS = nullptr, *TCK = nullptr;
    unsigned *TRED = nullptr, *TBAR = nullptr;
    int* TLIST = nullptr;
    int tail_grid = 0;                     // CTAs of its cooperative launch (0: unavailable)
    int tail_rpc = 0, tail_cache = 0;      // rows per CTA; 1 = those rows of Wt cached in shared memory
    int tail_pr = 0;                       // rows of the layer product per pass of the tail kernel
    size_t tail_smem = 0;                  // its dynamic shared memory
    unsigned* chunk_sync = nullptr;        // per slot tile: layer counters of the persistent chunk kernel
    int* cnt_host = nullptr;               // pinned host copy of the counters read back after a check
    cudaEvent_t ev_cnt = nullptr;          // recorded after that copy
};

}  // namespace rq

struct relu_qp_s {
    int n = 0, m = 0, R = 0, ldw = 0, nr = 0;
    double sigma = 0.0;
    relu_qp_opts opts{};
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    std::vector<double> bank;
    std::vector<double> h_q, h_l, h_u;      // current problem data (host FP64)
    std::vector<unsigned char> eq;         // equality-row pattern fixed at setup
    rq::BankEntry be[RQ_MAX_RHO];
    float *P32 = nullptr, *A32 = nullptr, *At32 = nullptr;   // check matrices (FP32)
    float *q32 = nullptr, *l32 = nullptr, *u32 = nullptr, *rs32 = nullptr;
    double qnorm = 0.0;
    // problem scaling (opts.scaling_iters > 0): the device holds the scaled problem
    // (c D P D, c D q, E A D, E l, E u); x = D xb, z = zb / E, lam = E lamb / c.
    // Host FP64 D, E, c and device FP32 factor vectors, all nullptr without scaling:
    // sc_q = c D (q in), sc_x = D (x out), sc_xi = 1/D (x in), sc_e = E (l, u in),
    // sc_z = 1/E (z out; residual rows of constraints), sc_l = E/c (lam out),
    // sc_li = c/E (lam in), sc_rx = 1/(c D) (residual rows of x)
    int scaled = 0;
    std::vector<double> sD, sE;
    double sC = 1.0;
    float *sc_q = nullptr, *sc_x = nullptr, *sc_xi = nullptr, *sc_e = nullptr, *sc_z = nullptr, *sc_l = nullptr,
          *sc_li = nullptr, *sc_rx = nullptr;
    double *sc64_rx = nullptr, *sc64_z = nullptr;   // the residual factors in FP64 (FP64 single solve)
    // FP64 single solve: check matrices and problem data (scaled problem when scaled)
    double *P64 = nullptr, *A64 = nullptr, *At64 = nullptr, *q64 = nullptr, *l64 = nullptr, *u64 = nullptr;
    rq::SingleWork64 sw64;
    rq::SingleWork sw;
    rq::BatchWork bw;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // profiling (relu_qp_profile): launch counter and event pairs around the
    // batched layer kernel launches
    long long launches = 0, layer_launches = 0, layer_timed = 0;
    double layer_ms = 0.0, layer_flops = 0.0;
    int prof_on = 0;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_span_launches;     // launches covered by each recorded event pair
    // host round trips of a batched solve (profiling): event pairs around each read-back
    std::vector<cudaEvent_t> gap_ev;
    long long host_checks = 0, resident_launches = 0;
    double host_gap_ms = 0.0;
    std::string err;
    std::vector<void*> allocs;               // every cudaMalloc of the handle
    size_t dev_bytes = 0;                    // bytes of those allocations (opts.device_budget caps it)
};

namespace rq {

int fail(relu_qp_t h, int code, const std::string& msg);
int dev_alloc(relu_qp_t h, void** p, size_t bytes);

template <typename T>
int alloc(relu_qp_t h, T** p, size_t count) {
    return dev_alloc(h, reinterpret_cast<void**>(p), count * sizeof(T) + 16);
}

// FP64 building blocks of the offline stage (setup_fp64.cu), on h->stream:
// C = alpha op(A) op(B) + beta C (row-major); in-place blocked Cholesky K = L L^T
// (Linv: ceil(n / kCholNB) diagonal-block inverses of kCholNB^2, T: n x kCholNB
// scratch, *flag set on a pivot <= 0); Rhs (n x NR) <- K^{-1} Rhs (T2: kCholNB x NR).
constexpr int kCholNB = 64;
int dgemm(relu_qp_t h, bool ta, bool tb, int M, int N, int K, double alpha, const double* A, int lda,
          const double* B, int ldb, double beta, double* C, int ldc);
int cholesky(relu_qp_t h, double* Km, int n, double* Linv, double* T, int* flag);
int chol_solve(relu_qp_t h, const double* L, int n, const double* Linv, double* Rhs, int NR, double* T2);
// Condensing of a linear MPC problem (condense.cu); error text in *err.
int condense_mpc(int nx, int nu, int N, const double* A, const double* B, const double* Q, const double* R,
                 const double* QN, bool state_rows, const double* K, int precondition, void* stream, double* P,
                 double* Acon, double* F, double* E, double* K_out, std::string* err);
// FP64 setup (setup_fp64.cu): builds every bank entry of h from P, A (device FP64).
int build_bank(relu_qp_t h, const double* dP, const double* dA, const std::vector<double>& rho_rows_scale);
// FP32 copies of P, A, A^T from FP64 device arrays (setup_fp64.cu).
int make_check_matrices(relu_qp_t h, const double* dP, const double* dA);
// b_r = Bop_r q for every bank entry (single_solve.cu).
int compute_bias(relu_qp_t h);
// Cooperative single-QP solve (single_solve.cu).
int single_solve(relu_qp_t h, const float* x_warm_dev, const float* lam_warm_dev, int rho_index,
                 double eps_abs, double eps_rel, int max_iter, relu_qp_info* info);
int single_prepare(relu_qp_t h);
int single_get_config(relu_qp_t h, int* ctas, int* cluster, int* cached_rows);
int single_set_config(relu_qp_t h, int ctas, int cluster);
// Same solve with its scratch in a fixed device array (single_solve.cu).
int single_solve_noalloc(relu_qp_t h, const float* x_warm, const float* lam_warm, int rho_index, double eps_abs,
                         double eps_rel, int max_iter, float* x_out, float* z_out, float* lam_out,
                         relu_qp_info* info);
// FP64 single-QP solve (single_solve64.cu).
int single64_alloc(relu_qp_t h, const double* P, const double* A);
int single64_upload(relu_qp_t h, const double* q, const double* l, const double* u);
int single64_prepare(relu_qp_t h);
int single64_solve(relu_qp_t h, const double* x_warm, const double* lam_warm, int rho_index, double eps_abs,
                   double eps_rel, int max_iter, double* x_out, double* z_out, double* lam_out,
                   relu_qp_info* info);
// Batched solves (batch.cu).
int batch_alloc(relu_qp_t h);
int batch_update(relu_qp_t h, int B, const float* Q, const float* L, const float* U);
int batch_set_parametric(relu_qp_t h, int nx, const double* F, const double* E, const double* l0,
                         const double* u0);
int batch_update_x0(relu_qp_t h, int B, const float* X0);
int batch_solve(relu_qp_t h, int B, const float* Xw, const float* Lw, const int* rw, double eps_abs,
                double eps_rel, int max_iter, float* Xo, float* Zo, float* Lo, relu_qp_info* infos);
// BF16 hi/mid/lo parts of the FP64 layer for the tcgen05 backend (setup_fp64.cu).
int pack_bf16_layer(relu_qp_t h, int r, const double* X, const double* AX);
int pack_bf16_check(relu_qp_t h, const double* dP, const double* dA);
int batch_finish_setup(relu_qp_t h);
// Continuous batching (batch.cu).
int server_create(relu_qp_server_t* out, relu_qp_t const* families, int nf, const int* clients, double eps_abs,
                  double eps_rel, int max_iter);
int server_submit(relu_qp_server_t s, int family, int client, const float* x0, long long tag);
int server_step(relu_qp_server_t s, int* active, int* waiting);
int server_poll(relu_qp_server_t s, int max_results, relu_qp_result* results, float* x_out, int x_stride);
void server_destroy(relu_qp_server_t s);
const char* server_error(relu_qp_server_t s);
double server_clock(relu_qp_server_t s);
int server_families(relu_qp_server_t s);
int server_clients(relu_qp_server_t s, int family);
int server_nx(relu_qp_server_t s, int family);
int server_set_budget(relu_qp_server_t s, long long bytes);
int server_family_bytes(relu_qp_server_t s, int family, long long* fixed_bytes, long long* slot_bytes);
long long server_bytes_in_use(relu_qp_server_t s);
// device bytes of one QP slot of a batched handle (every array that scales with max_batch)
size_t batch_slot_bytes(relu_qp_t h);
void batch_release(relu_qp_t h);

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
inline size_t round_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

}  // namespace rq
