/*
 * relu_qp.h -- C ABI of the GB300 (sm_103a) ReLU-QP solver.
 *
 * Problem (paper Sec. II-A, Eq. qp_def, with H->P, g->q, G->A, c,d->l,u):
 *
 *     minimise 1/2 x^T P x + q^T x   subject to   l <= A x <= u,
 *
 * P (n x n) symmetric positive definite, A (m x n), l_i in [-inf, +inf),
 * u_i in (-inf, +inf], l <= u.  Rows with l_i == u_i are equality rows.
 *
 * Method (paper Sec. III, Algorithm 1): ADMM with a fixed penalty written as
 * the weight-tied layer v+ = clamp(W_rho v + b_rho) on v = [x; z; lam]
 * (Eq. gpu_update).  A bank of penalties rho_i is factored offline
 * (relu_qp_setup); online, the layer runs until the residuals of Eqs. primal
 * and dual meet the tolerance, checking every `check_interval` layers and
 * switching to the bank entry closest to the estimate of Eq. rho_update
 * (Sec. III-C).
 *
 * Conventions for every entry point:
 *  - Matrices are dense, row-major, contiguous.
 *  - Host arrays passed in are copied before the call returns; the caller
 *    keeps ownership.  Output arrays are caller-owned and written in full.
 *  - The handle owns all device memory it allocates; relu_qp_destroy frees it.
 *  - All GPU work is issued on opts.stream and the call synchronises that
 *    stream before returning (results are ready on return).
 *  - Return value: RELU_QP_OK (0) or a negative RELU_QP_ERR_* code;
 *    relu_qp_last_error(h) gives a one-line message.  Non-convergence is not
 *    an error: it is reported as info->status == RELU_QP_MAX_ITER.
 *  - No C++ exception crosses the ABI.  One handle must not be used from two
 *    host threads at the same time.
 */
#ifndef RELU_QP_H
#define RELU_QP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define RELU_QP_OK                0
#define RELU_QP_ERR_INVALID      -1   /* bad sizes, NULL where required, l > u, NaN input */
#define RELU_QP_ERR_NOT_PD       -2   /* Cholesky pivot <= 0: P + sigma I + A^T rho A not PD */
#define RELU_QP_ERR_OOM          -3   /* device allocation refused (or over the memory budget) */
#define RELU_QP_ERR_CUDA         -4   /* a CUDA runtime call failed */
#define RELU_QP_ERR_TIMEOUT      -5   /* a device-side wait gave up at its deadline */
#define RELU_QP_ERR_UNSUPPORTED  -6   /* feature not available for this handle / device */

/* ---- per-solve status (relu_qp_info.status) ------------------------------ */
#define RELU_QP_SOLVED            0   /* both residuals met the tolerance at a check */
#define RELU_QP_MAX_ITER          1   /* max_iter layers ran without meeting it */
#define RELU_QP_NUMERICAL         2   /* a residual became NaN or Inf */

typedef struct relu_qp_s* relu_qp_t;

typedef struct relu_qp_opts {
    int    check_interval;  /* layers between residual checks; paper default 25
                               (Sec. III-C "Convergence Checking"); 0 = never check
                               (runs exactly max_iter layers at a fixed rho) */
    int    adaptive_rho;    /* 1: apply Eq. rho_update + nearest bank entry at each
                               unconverged check; 0: keep the starting rho */
    double rho0;            /* starting penalty (paper default 0.1, Sec. III-C), mapped
                               to the nearest bank entry */
    double eq_scale;        /* penalty factor of equality rows (paper: 1000, Sec. II-B) */
    int    keep_fp64;       /* 1: keep the FP64 layer matrices for relu_qp_get_layer */
    int    max_batch;       /* capacity of batched solves (0: single-QP handle) */
    int    batch_precision; /* RELU_QP_PREC_FP32 or RELU_QP_PREC_BF16X3 */
    void*  stream;          /* cudaStream_t for all work; NULL = the legacy default stream */
    int    scaling_iters;   /* Algorithm 1 "Scale problem" (Sec. III-D "Preconditioning"):
                               iterations of the modified Ruiz equilibration done in
                               FP64 at setup (0 = off, the default; 10 is typical).
                               The layer bank is built for the scaled problem
                               min 1/2 xb' (c D P D) xb + (c D q)' xb, E l <= E A D xb <= E u
                               (D, E diagonal, c > 0: every column of the KKT matrix
                               [[P, A'], [A, 0]] divided by the square root of its
                               infinity norm each iteration, then the cost rescaled);
                               every entry point takes and returns the original
                               problem's data and iterates (x = D xb, z = zb / E,
                               lam = E lamb / c), and the stop test, the residuals in
                               relu_qp_info and the penalty rule use the original
                               problem's residuals and norms.  relu_qp_get_layer
                               returns the scaled problem's layer; relu_qp_solve_noalloc
                               refuses a scaled handle. */
    int    single_precision; /* arithmetic of relu_qp_solve: RELU_QP_PREC_FP32 (default:
                               FP32 layers and checks, the paper's GPU arithmetic),
                               RELU_QP_PREC_FP64 (FP64 layer bank, iterates, residuals
                               and outputs; for tolerances FP32 cannot resolve, e.g.
                               1e-6 with the 1000x penalty of equality rows, Sec. II-B
                               and Sec. V-A) or RELU_QP_PREC_FP64R (the same with FP32
                               products of the layer increments between FP64 anchor
                               layers: faster, iterates within rounding of FP64).  Both
                               keep the FP64 bank (as keep_fp64) and FP64 copies of P
                               and A; relu_qp_solve_noalloc refuses them. */
    long long device_budget; /* cap, in bytes, on the device memory the handle keeps
                               (layer bank, problem data, single-QP and batch state);
                               0 = no cap.  An allocation that would pass it fails
                               with RELU_QP_ERR_OOM before cudaMalloc is called.  The
                               FP64 inputs and scratch of the offline stage, freed
                               before relu_qp_setup returns, are not counted.  No
                               counterpart in the paper (deployment limit). */
} relu_qp_opts;

#define RELU_QP_PREC_FP32    0   /* batched layer product in FP32 on the CUDA cores */
#define RELU_QP_PREC_BF16X3  1   /* batched layer product on tcgen05 tensor cores,
                                    BF16 hi+lo split operands, FP32 accumulate */
#define RELU_QP_PREC_FP64    2   /* single-QP solve in FP64 (opts.single_precision) */
#define RELU_QP_PREC_FP64R   3   /* single-QP solve with FP64 state, residuals and one FP64 layer
                                    product per check interval (the anchor c = Wt s_ref + b); the
                                    other layers apply the FP32 bank to the increment only,
                                    t = c + Wt (s - s_ref) (opts.single_precision) */

typedef struct relu_qp_info {
    int    status;       /* RELU_QP_SOLVED / RELU_QP_MAX_ITER / RELU_QP_NUMERICAL */
    int    iters;        /* layers executed */
    int    rho_index;    /* bank index in use at return (feed back as a warm start) */
    int    rho_switches; /* number of bank switches during the solve */
    double r_prim;       /* ||A x - z||_inf at the last check (Eq. primal) */
    double r_dual;       /* ||P x + q + A^T lam||_inf at the last check (Eq. dual) */
    double solve_ms;     /* device time of the solve (CUDA events) */
} relu_qp_info;

/* Fill *opts with the defaults above (check 25, adaptive, rho0 0.1, eq 1000,
 * no FP64 copy, single-QP, FP32, default stream, no scaling). */
void relu_qp_default_opts(relu_qp_opts* opts);

/*
 * relu_qp_setup -- offline stage of Algorithm 1 ("compute KKT inverse, W and b
 * for each rho").  For every bank entry rho_r the library forms, in FP64 on
 * the GPU, K_r = P + sigma I + A^T diag(rho_r) A, factors it with a blocked
 * Cholesky, and solves K_r X = [sigma I - A^T rho_r A, A^T, -I] by blocked
 * triangular solves; the layer matrices follow (Eq. gpu_update) and are
 * stored in FP32 (and BF16 hi/lo when batched precision is BF16X3).
 *
 *   out       receives the handle (set to NULL on failure)
 *   n, m      decision variables (n >= 1) and constraint rows (m >= 0)
 *   P         n*n FP64, symmetric positive definite (only its values are read)
 *   q         n FP64 linear cost (may be NULL: zeros; relu_qp_update can set it)
 *   A         m*n FP64 (may be NULL when m == 0)
 *   l, u      m FP64 bounds, +-INFINITY allowed, l <= u elementwise
 *   sigma     > 0, the proximal weight of Eq. admm_al (typical 1e-6)
 *   rho_bank  n_rho > 0 strictly positive penalties (paper: log-spaced list)
 *   opts      NULL for defaults
 * Errors: INVALID (sizes, l > u, NaN/Inf in P, q, A, sigma <= 0, rho <= 0),
 * NOT_PD (a Cholesky pivot <= 0), OOM, CUDA.
 */
int relu_qp_setup(relu_qp_t* out, int n, int m, const double* P, const double* q,
                  const double* A, const double* l, const double* u, double sigma,
                  const double* rho_bank, int n_rho, const relu_qp_opts* opts);

/*
 * relu_qp_update -- online "update b, c~, d~" of Algorithm 1: replaces the
 * linear cost and/or the bounds of the problem (NULL keeps the old array).
 * b_r = [-D_r; -A D_r] q is recomputed for every bank entry.  Equality rows
 * must keep the same pattern (l_i == u_i) they had at setup.
 * Errors: INVALID (l > u, NaN, changed equality pattern), CUDA.
 */
int relu_qp_update(relu_qp_t h, const double* q, const double* l, const double* u);

/*
 * relu_qp_solve -- online stage of Algorithm 1 for the single QP held by h.
 *   x_warm, lam_warm  n / m FP64 warm start (Sec. II-B "Warm Starting":
 *                     z = A x_warm); NULL = cold start v = 0 (lam_warm NULL
 *                     with x_warm given means lam = 0)
 *   rho_index_warm    bank index to start from, or -1 for the entry nearest rho0
 *   eps_abs, eps_rel  tolerances: converged when ||Ax-z|| <= eps_abs + eps_rel
 *                     max(||Ax||,||z||) and ||Px+q+A^T lam|| <= eps_abs + eps_rel
 *                     max(||Px||,||A^T lam||,||q||) (inf-norms, Eqs. primal, dual)
 *   max_iter          >= 1 layers at most
 *   x_out             n FP64 (required); z_out, lam_out m FP64 (may be NULL).
 *                     lam_out is the standard ADMM multiplier lam' + rho (Ax - z).
 *   info              may be NULL
 * The whole loop runs in one cooperative kernel on the device (FP32, or FP64
 * when opts.single_precision = RELU_QP_PREC_FP64); the host waits only for
 * its end.  Errors: INVALID, CUDA, TIMEOUT.
 */
int relu_qp_solve(relu_qp_t h, const double* x_warm, const double* lam_warm, int rho_index_warm,
                  double eps_abs, double eps_rel, int max_iter, double* x_out, double* z_out,
                  double* lam_out, relu_qp_info* info);

/*
 * relu_qp_solve_noalloc -- relu_qp_solve for callers that cannot allocate
 * device memory when they solve, e.g. a real-time control loop whose cycle
 * must not stall on cudaMalloc (it can synchronise the device and take an
 * unbounded time) or an application whose own allocator owns device memory.
 * The paper has no counterpart; it is a deployment variant of the same solve.
 *
 * It allocates nothing: the solve's scratch (iterate, layer operands,
 * residual vectors, grid-barrier and reduction words) lives in one fixed
 * 192 KiB device array inside the library, which every GPU that loads the
 * library holds until the process exits.  The layer bank and problem data
 * come from relu_qp_setup / relu_qp_update on h as usual.
 *   x_warm, lam_warm  device FP32 (n / m) warm start, or NULL (lam_warm needs x_warm)
 *   rho_index_warm, eps_abs, eps_rel, max_iter, info: as relu_qp_solve
 *   x_out (n, required), z_out, lam_out (m, may be NULL): device FP32 outputs
 * Unlike relu_qp_solve (host FP64 arrays), every array here is device FP32
 * memory (or managed memory) of the handle's device; each non-NULL pointer is
 * checked before any GPU work and anything else returns RELU_QP_ERR_INVALID.
 * Limits and rules: n + m <= 4096 (larger problems return RELU_QP_ERR_INVALID
 * before any GPU work).  All calls share the one array, so calls whose GPU
 * work overlaps (other streams or threads) race; order them.  The array keeps
 * the last call's contents; each call clears what must start at zero.  The
 * call is synchronous: it returns once the outputs and info are written.  The
 * first call for each device looks the array's device address up
 * (cudaGetSymbolAddress) with the handle's device current; make that first
 * call before any stream capture.
 * Errors: INVALID, UNSUPPORTED (device ordinal >= 64, or a handle set up with
 * scaling_iters > 0), CUDA, TIMEOUT.
 */
int relu_qp_solve_noalloc(relu_qp_t h, const float* x_warm, const float* lam_warm, int rho_index_warm,
                          double eps_abs, double eps_rel, int max_iter, float* x_out, float* z_out,
                          float* lam_out, relu_qp_info* info);

/*
 * relu_qp_get_layer -- export the layer of bank entry rho_index for checking:
 *   Wt   (n+m)*(n+m) FP64: rows [x; Ax] of the layer in the factored form
 *        [x+; (A x)+] = Wt [x; 2 rho z - lam'] + Bop q.  With D the KKT inverse,
 *        Wt = [D(sigma I - A^T rho A), D A^T; A D(sigma I - A^T rho A), A D A^T];
 *        the paper's W (Eq. gpu_update) follows by splitting the second block
 *        column into its z (times 2 rho) and lam (times -1) columns, adding
 *        [A, -I, rho^{-1}] to the z row, and appending the row [rho A, -rho, I].
 *   Bop  (n+m)*n FP64: [-D; -A D]
 * FP64 values if the handle was set up with keep_fp64, else the FP32 copies
 * widened.  Either pointer may be NULL.  Errors: INVALID, CUDA.
 */
int relu_qp_get_layer(relu_qp_t h, int rho_index, double* Wt, double* Bop);

/*
 * ---- batched QPs --------------------------------------------------------
 * A handle set up with opts.max_batch = Bmax > 0 also solves up to Bmax QPs
 * at once that share P and A (hence every layer of the bank) but have their
 * own q, l, u, warm start and penalty index.  Each layer is then one GEMM
 * over the batch (tcgen05 tensor cores with BF16 hi+lo split operands and
 * FP32 accumulation when opts.batch_precision = RELU_QP_PREC_BF16X3, FP32
 * CUDA cores otherwise), checks run per QP, converged QPs leave the batch,
 * and the rest are regrouped by bank entry after every check.
 *
 * Array arguments of the batched calls are row-major FP32 (B rows) and may
 * be host memory (pageable or pinned) or device memory; the library copies
 * through cudaMemcpyDefault.  Rows with l_i == u_i at setup must stay
 * equality rows (and the others inequality rows) in every QP of a batch.
 */

/* Per-QP problem data: Q (B x n), L and U (B x m).  1 <= B <= max_batch.
 * Recomputes b_r = [-D_r; -A D_r] q for every bank entry and QP.
 * Errors: INVALID, UNSUPPORTED (max_batch = 0), CUDA. */
int relu_qp_update_batch(relu_qp_t h, int B, const float* Q, const float* L, const float* U);

/* Parametric form of the problem data for MPC (condensed form, paper Sec. IV):
 * q = F x0, l = l0 - E x0, u = u0 - E x0 with F (n x nx), E (m x nx) FP64 and
 * l0, u0 (m) FP64.  Precomputes [-D_r; -A D_r] F for every bank entry so that
 * a batch update costs O((n + m) nx) per QP.  Errors: INVALID, UNSUPPORTED. */
int relu_qp_set_parametric(relu_qp_t h, int nx, const double* F, const double* E, const double* l0,
                           const double* u0);

/* Per-QP initial states X0 (B x nx FP32) for the parametric form ("update b,
 * c~, d~ with initial conditions", Algorithm 1).  Errors: INVALID, UNSUPPORTED. */
int relu_qp_update_batch_x0(relu_qp_t h, int B, const float* X0);

/*
 * relu_qp_condense_mpc -- the dense, LQR-preconditioned condensing of a linear
 * MPC problem (Sec. IV "Dense Model-Predictive Control"), in FP64 on the GPU.
 * It produces the parametric QP that relu_qp_setup (P, A_con, l0, u0) and
 * relu_qp_set_parametric (F, E, l0, u0) take.
 *
 * Plant x_{k+1} = A x_k + B u_k (k = 0..N-1).  Controls are u_k = -K x_k +
 * du_k.  K is the infinite-horizon LQR gain, used as a preconditioner.  The
 * decision vector is du = [du_0; ..; du_{N-1}], so n = N nu.  The trajectory
 * is y = [u_0; x_1; ..; u_{N-1}; x_N] = S du + M x0, with S and M as printed
 * in Sec. IV.  With H = blkdiag(R, Q, .., R, Q_N) the QP is
 *   min 1/2 du' P du + (F x0)' du,  P = S' H S,  F = S' H M,
 *   l0 - E x0 <= A_con du <= u0 - E x0.
 * The constraint rows are, in this order:
 *   - the control limits umin <= u_k <= umax for every k (N nu rows);
 *   - the state limits xmin <= x_{k+1} <= xmax (N nx rows), present only when
 *     xmin or xmax is given.
 * A_con holds the matching rows of S and E the matching rows of M.
 *
 *   nx, nu, N     state and control sizes, horizon (>= 1; N nu <= 40000)
 *   A, B, Q, R    nx x nx, nx x nu, nx x nx, nu x nu, row-major FP64 (host).
 *                 Q_N: nx x nx terminal weight, NULL = Q.
 *   umin, umax    nu each; NULL = unbounded on that side; +-INFINITY allowed
 *   xmin, xmax    nx each; both NULL = no state rows; one NULL = unbounded side
 *   K             nu x nx gain to use.  NULL with lqr_precondition = 1: the
 *                 infinite-horizon LQR gain, computed by the fixed-point
 *                 Riccati iteration X <- Q + A'X(A - B K(X)) until
 *                 max|dX| <= 1e-13 max(1, max|X|).  NULL with
 *                 lqr_precondition = 0: K = 0, plain condensing.
 *   stream        cudaStream_t for the work (NULL = legacy default stream)
 * Outputs (host FP64, caller-allocated; m = N nu + (state rows ? N nx : 0)):
 *   P (n x n), A_con (m x n), F (n x nx), E (m x nx), l0, u0 (m),
 *   K_out (nu x nx, may be NULL): the gain used.
 * Errors (message in relu_qp_last_error(NULL)):
 *   INVALID  sizes, NULL inputs, non-finite matrices, umin > umax or
 *            xmin > xmax, a Riccati iteration that diverges or does not
 *            converge (e.g. (A, B) not stabilizable)
 *   NOT_PD   R + B'XB not positive definite
 *   OOM, CUDA
 */
int relu_qp_condense_mpc(int nx, int nu, int N, const double* A, const double* B, const double* Q,
                         const double* R, const double* Q_N, const double* umin, const double* umax,
                         const double* xmin, const double* xmax, const double* K, int lqr_precondition,
                         void* stream, double* P, double* A_con, double* F, double* E, double* l0,
                         double* u0, double* K_out);

/*
 * relu_qp_solve_batch -- Algorithm 1 for the first B QPs of the last batch update.
 *   X_warm (B x n), Lam_warm (B x m), rho_warm (B, bank indices): warm start
 *     (z = A x_warm); NULL = cold start (rho_warm needs X_warm)
 *   eps_abs, eps_rel, max_iter: as relu_qp_solve, applied per QP
 *   X_out (B x n, required), Z_out, Lam_out (B x m, may be NULL): the iterate
 *     of each QP at its stop (Lam_out is the standard multiplier)
 *   infos: B entries (may be NULL); solve_ms is the time of the whole batch
 * Errors: INVALID, UNSUPPORTED, CUDA, TIMEOUT (a device wait passed its deadline).
 */
int relu_qp_solve_batch(relu_qp_t h, int B, const float* X_warm, const float* Lam_warm, const int* rho_warm,
                        double eps_abs, double eps_rel, int max_iter, float* X_out, float* Z_out,
                        float* Lam_out, relu_qp_info* infos);

/*
 * ---- serving: continuous batching of MPC requests -------------------------
 * A server owns several problem families (handles set up with max_batch > 0,
 * check_interval > 0 and relu_qp_set_parametric), each with its layer bank
 * and max_batch QP slots resident on the device.  A request is a new initial
 * state x0 (nx floats) for one client of one family.  Requests wait in a host
 * queue until their family has a free slot: admission is by device memory,
 * since every slot's state is allocated once, up front.  Each
 * relu_qp_server_step admits waiting requests into free slots (the parametric
 * update of q, l, u and b, and a warm start from that client's previous
 * solution, which stays on the device: x, lam and the bank index, with
 * z = A x, paper Sec. II-B "Warm Starting"), runs one chunk of check_interval
 * layers and the residual check for every family with work, each family on
 * its own stream so that their chunks overlap on the GPU, and retires the
 * QPs that finished (solved, max_iter reached, or non-finite).  Families
 * advance independently: a family whose chunk has finished retires, admits
 * and launches its next chunk at once, without waiting for the chunks of the
 * other families.  Results keep the request's tag and its submit and
 * completion times on the server clock.
 * Admission by device memory (relu_qp_server_set_budget): each family's
 * layer bank and fixed buffers are charged when the budget is set; every
 * admitted request is charged its family's bytes per QP slot (the batch state
 * it occupies on the device) until it retires.  A request waits while its
 * family has no free slot or the budget has no room for it, and a request of
 * one family is not admitted ahead of an older waiting request of another
 * family whose room it would take.
 * While a server exists its families' handles run on the server's streams;
 * do not use them for other calls until relu_qp_server_destroy.
 */
typedef struct relu_qp_server_s* relu_qp_server_t;

typedef struct relu_qp_result {
    long long tag;       /* the caller's id from relu_qp_server_submit */
    int    family;       /* family index */
    int    client;       /* client index (-1: none) */
    int    status;       /* RELU_QP_SOLVED / RELU_QP_MAX_ITER / RELU_QP_NUMERICAL */
    int    iters;        /* layers run for this request */
    int    rho_index;    /* bank index at the end */
    int    rho_switches; /* bank switches during the request */
    double r_prim, r_dual;      /* residuals at the last check */
    double t_submit, t_done;    /* seconds on the server clock */
} relu_qp_result;

/* families: n_families (1..16) distinct handles; clients: per family the
 * number of clients whose warm starts are kept (NULL = none); eps_abs,
 * eps_rel, max_iter as relu_qp_solve.  Errors: INVALID, OOM, CUDA. */
int relu_qp_server_create(relu_qp_server_t* out, relu_qp_t const* families, int n_families, const int* clients,
                          double eps_abs, double eps_rel, int max_iter);
/* Queue one request: x0 host FP32 (nx of the family), client in [-1, clients). */
int relu_qp_server_submit(relu_qp_server_t s, int family, int client, const float* x0, long long tag);
/* One round: every family without a chunk in flight admits waiting requests and
 * launches its next chunk; every family whose chunk has finished retires its
 * finished requests, admits and launches again.  Returns as soon as at least
 * one family has finished a chunk in this call (or at once when no chunk is
 * in flight); it does not wait for the other families.  *active / *waiting
 * (may be NULL): requests in slots / queued. */
int relu_qp_server_step(relu_qp_server_t s, int* active, int* waiting);
/* Device-memory budget of the server in bytes (0 = slots only, the default).
 * Errors: OOM when the families' banks and fixed buffers alone exceed it (the
 * budget is then unchanged), INVALID for a negative value. */
int relu_qp_server_set_budget(relu_qp_server_t s, long long bytes);
/* Memory accounting of one family: fixed bytes (its handle's bank and problem
 * data plus the server's buffers for it) and bytes per QP slot.  Any pointer
 * may be NULL.  Errors: INVALID (family out of range). */
int relu_qp_server_family_bytes(relu_qp_server_t s, int family, long long* fixed_bytes, long long* slot_bytes);
/* Bytes charged by the requests now in slots, over every family. */
long long relu_qp_server_bytes_in_use(relu_qp_server_t s);
/* Pop up to max_results finished requests; x_out (may be NULL) receives each
 * result's x (FP32) at row stride x_stride floats.  Returns the number popped. */
int relu_qp_server_poll(relu_qp_server_t s, int max_results, relu_qp_result* results, float* x_out, int x_stride);
/* Seconds since the server was created (the clock of t_submit / t_done). */
double relu_qp_server_clock(relu_qp_server_t s);
void relu_qp_server_destroy(relu_qp_server_t s);
const char* relu_qp_server_error(relu_qp_server_t s);

/*
 * Kernel-level counters of a handle, for benchmarks.  `launches` counts every
 * kernel the solve and update paths launched; `layer_*` cover the dominant
 * kernel of a batched solve (the tensor-core refined layer in the BF16 form,
 * the FP32 layer otherwise): its launches, the algorithmic FLOPs they did
 * (2 x products x (n+m)^2 per active QP) and, while profiling is enabled,
 * their device time from CUDA events recorded on the handle's stream around
 * each chunk's run of consecutive layer launches (layer_timed counts the
 * launches those spans cover; up to 8192 spans per solve are timed).
 * `host_checks` / `host_gap_ms` (batched solves, while profiling): the checks
 * after which the host read the active-QP count back (one stream synchronise
 * each) and the summed device time between the last kernel before each of
 * those reads and the first event the host enqueued after it returned, i.e.
 * how long the GPU waited on the host round trip.  `resident_launches`: chunk
 * launches that ran the resident-weight kernel (one slot tile of few QPs).
 */
typedef struct relu_qp_prof {
    long long launches;
    long long layer_launches;
    long long layer_timed;
    double layer_ms;
    double layer_flops;
    long long host_checks;
    double host_gap_ms;
    long long resident_launches;
} relu_qp_prof;

/* Read the counters into *out (may be NULL), then reset them if `reset`, then
 * turn event timing on (enable = 1) or off (0) or leave it (-1). */
int relu_qp_profile(relu_qp_t h, int enable, int reset, relu_qp_prof* out);

/* Change check_interval / adaptive_rho / rho0 of an existing handle
 * (other fields of opts are ignored).  Errors: INVALID. */
int relu_qp_set_opts(relu_qp_t h, const relu_qp_opts* opts);

/* Sizes of a handle (any pointer may be NULL). */
int relu_qp_dims(relu_qp_t h, int* n, int* m, int* n_rho);

/* Device memory the handle keeps, in bytes (what opts.device_budget caps);
 * -1 for a NULL handle. */
long long relu_qp_device_bytes(relu_qp_t h);

/*
 * ---- launch shape of the single-QP FP32 solve --------------------------------
 * relu_qp_setup times candidate launch shapes of the solve kernel behind
 * relu_qp_solve (the online stage of Algorithm 1, Sec. III-B) and keeps the
 * fastest: a cooperative grid of `ctas` CTAs with a grid barrier between
 * layers, or one thread-block cluster of `ctas` CTAs (cluster = ctas) that keep
 * the layer's operand in distributed shared memory and synchronise through
 * cluster-scope mbarriers.  Each row's dot product and update is the same
 * arithmetic in every shape, so the results do not depend on the choice; these
 * calls exist for tests and tuning.
 *
 * relu_qp_single_config: the shape in use: *ctas, *cluster (0 = grid form),
 *   *cached_rows (rows of the layer each CTA keeps in shared memory); any
 *   pointer may be NULL.  Errors: INVALID (NULL handle, or no setup yet).
 * relu_qp_single_set_config: use ctas CTAs (1 <= ctas <= n + m) as a grid
 *   (cluster = 0) or as one cluster (cluster = ctas, one of 2, 4, 8, 16).
 *   Errors: INVALID (handle, no setup, arguments), UNSUPPORTED (the shape
 *   cannot be resident on this GPU); the previous shape stays on error.
 */
int relu_qp_single_config(relu_qp_t h, int* ctas, int* cluster, int* cached_rows);
int relu_qp_single_set_config(relu_qp_t h, int ctas, int cluster);

/*
 * ---- deadline diagnostics ---------------------------------------------------
 * No counterpart in the paper.  Every device-side wait of the library (the
 * grid barrier of the cooperative kernels, and the mbarrier and layer-counter
 * waits of the tensor-core kernels) gives up at a deadline and reports
 * RELU_QP_ERR_TIMEOUT instead of hanging the GPU.  These calls make one kind
 * of wait run out on purpose, on the current device and the legacy stream,
 * so that a test can see the status come back and the context stay usable.
 *
 * relu_qp_diag_device_wait -- kind 0: a cooperative launch of a few CTAs
 *   whose grid barrier expects one arrival more than there are CTAs (every
 *   CTA waits until timeout_ns); kind 1: the same barrier with the right
 *   arrival count (passes; the control case); kind 2: an mbarrier wait that
 *   nothing completes; kind 3: a layer-counter wait that nothing increments;
 *   kind 4: a cluster of 2 CTAs whose cluster barrier (the one the
 *   single-QP solve uses in its cluster form) expects one arrival more than
 *   there are CTAs; kind 5: the same barrier with the right count, three
 *   rounds (passes).  timeout_ns in [1e3, 1e9].  *status receives the
 *   kernel's error word (RELU_QP_ERR_TIMEOUT, or 0 when the wait completed),
 *   *ms (may be NULL) the device time of the launch.  Returns INVALID, OOM,
 *   CUDA, UNSUPPORTED (no cooperative or cluster launch) or OK.
 * relu_qp_diag_host_barrier -- the grid barrier's arrival and wait logic (the
 *   template the kernels use) run by `threads` host threads for `rounds`
 *   barriers, with an arrival count of threads + extra: extra = 0 passes
 *   every round, extra > 0 makes every thread give up after timeout_ns.
 *   *timeouts receives the number of threads that gave up, *ms (may be NULL)
 *   the wall time.  Needs no GPU.  Returns INVALID or OK.
 */
int relu_qp_diag_device_wait(int kind, long long timeout_ns, int* status, double* ms);
int relu_qp_diag_host_barrier(int threads, int extra, int rounds, long long timeout_ns, int* timeouts, double* ms);

/* Free every device and host resource of h (NULL is a no-op). */
void relu_qp_destroy(relu_qp_t h);

/* One-line description of the last error on h (or of the last failed setup
 * when h is NULL).  Valid until the next call on h. */
const char* relu_qp_last_error(relu_qp_t h);

#ifdef __cplusplus
}
#endif

#endif /* RELU_QP_H */
