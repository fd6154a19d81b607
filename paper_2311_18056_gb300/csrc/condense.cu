// Dense, LQR-preconditioned condensing of a linear MPC problem (Sec. IV,
// "Dense Model-Predictive Control") in FP64 on the GPU.
//
// Plant x_{k+1} = A x_k + B u_k, controls u_k = -K x_k + du_k with the
// infinite-horizon LQR gain K as preconditioner, Abar = A - B K.  The
// decision vector is ytilde = [du_0; ...; du_{N-1}] (n = N nu) and the
// trajectory y = [u_0; x_1; u_1; x_2; ...; u_{N-1}; x_N] = S ytilde + M x0 with
//   u_k rows of S:     -K Abar^{k-1-j} B (j < k),  I (j = k),  0 (j > k)
//   x_{k+1} rows of S:  Abar^{k-j} B (j <= k),  0 (j > k)
//   u_k rows of M:     -K Abar^k,     x_{k+1} rows of M:  Abar^{k+1}.
// With H = blkdiag(R, Q, ..., R, Q_N) the QP is Hbar = S^T H S, gbar = S^T H M x0
// (so q = F x0 with F = S^T H M), and limits on u_k (and optionally x_{k+1})
// become rows of S with bounds shifted by the matching rows of M x0
// (l = l0 - E x0, u = u0 - E x0 with E = the rows of M).
//
// GPU formulation: the blocks T_j = Abar^j B, -K T_j, Abar^{k+1} and -K Abar^k
// are computed by chained DGEMMs, S is filled as a block-Toeplitz matrix, and
// Hbar, F are two DGEMMs each over the u and x row blocks (H applied block by
// block).  K comes from the fixed-point Riccati iteration
//   X <- Q + A^T X (A - B K(X)),  K(X) = (R + B^T X B)^{-1} B^T X A,
// run until max|X+ - X| <= 1e-13 max(1, max|X+|).
#include "common.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace rq {
namespace {

constexpr int kRiccatiMaxIter = 100000;
constexpr int kRiccatiCheckEvery = 16;
constexpr double kRiccatiTol = 1e-13;

int grid_for(size_t total) { return (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, 16384)); }

// S blocks: row block k (rows of one stage, `rb` rows each), column block j
// (`cb` columns each); block (k, j) = Blk[k - j - off] for j <= k - off, the
// identity (of size cb = rb) for j == k when `ident`, else 0.  Blk holds rb x cb
// row-major blocks.
__global__ void toeplitz_fill_kernel(const double* __restrict__ Blk, int N, int rb, int cb, int off, int ident,
                                     double* __restrict__ S) {
    const size_t rows = (size_t)N * rb, cols = (size_t)N * cb;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < rows * cols; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const int k = r / rb, i = r % rb, j = c / cb, t = c % cb;
        double v = 0.0;
        if (j <= k - off) v = Blk[((size_t)(k - j - off) * rb + i) * cb + t];
        else if (ident && j == k) v = (i == t) ? 1.0 : 0.0;
        S[e] = v;
    }
}

// out (N rb x cols) = blkdiag(W, ..., W, Wlast) in: block k of rows times W
// (rb x rb, Wlast for the last block).
__global__ void blkdiag_mul_kernel(const double* __restrict__ W, const double* __restrict__ Wlast, int N, int rb,
                                   const double* __restrict__ in, int cols, double* __restrict__ out) {
    const size_t rows = (size_t)N * rb;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < rows * cols; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const int k = r / rb, i = r % rb;
        const double* w = (k == N - 1 ? Wlast : W) + (size_t)i * rb;
        const double* x = in + (size_t)k * rb * cols + c;
        double v = 0.0;
        for (int t = 0; t < rb; ++t) v = fma(w[t], x[(size_t)t * cols], v);
        out[e] = v;
    }
}

// X <- (X + X^T) / 2 (n x n) and the convergence measures of the Riccati step:
// red[0] = max |X_new - X_old|, red[1] = max |X_new| (bits of non-negative doubles).
__global__ void sym_diff_kernel(double* __restrict__ Xn, const double* __restrict__ X, int n,
                                unsigned long long* red) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int i = e / n, j = e % n;
        if (j < i) continue;
        const double v = 0.5 * (Xn[(size_t)i * n + j] + Xn[(size_t)j * n + i]);
        Xn[(size_t)i * n + j] = v;
        Xn[(size_t)j * n + i] = v;
        const double d = fmax(fabs(v - X[(size_t)i * n + j]), fabs(v - X[(size_t)j * n + i]));
        atomicMax(red, (unsigned long long)__double_as_longlong(d));
        atomicMax(red + 1, (unsigned long long)__double_as_longlong(fabs(v)));
    }
}

__global__ void scale_copy_kernel(const double* __restrict__ in, double alpha, size_t count, double* __restrict__ out) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        out[e] = alpha * in[e];
}

__global__ void symmetrize_kernel(double* X, int n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        if (j <= i) continue;
        const double v = 0.5 * (X[(size_t)i * n + j] + X[(size_t)j * n + i]);
        X[(size_t)i * n + j] = v;
        X[(size_t)j * n + i] = v;
    }
}

struct Ctx {
    relu_qp_s h;     // carries the stream, the error message and the allocations
    ~Ctx() {
        cudaStreamSynchronize(h.stream);
        for (void* p : h.allocs) cudaFree(p);
    }
    template <typename T>
    int buf(T** p, size_t count) { return alloc(&h, p, count); }
    int up(double** p, const double* src, size_t count) {
        RQ_TRY(alloc(&h, p, count));
        RQ_CUDA(&h, cudaMemcpyAsync(*p, src, sizeof(double) * count, cudaMemcpyHostToDevice, h.stream));
        return RELU_QP_OK;
    }
};

// K (nu x nx) = (R + B^T X B)^{-1} B^T X A for the current X.
int gain(Ctx& c, int nx, int nu, const double* A, const double* B, const double* R, const double* X, double* BtX,
         double* G, double* K, double* Linv, double* T, double* T2, int* flag) {
    relu_qp_t h = &c.h;
    RQ_TRY(dgemm(h, true, false, nu, nx, nx, 1.0, B, nu, X, nx, 0.0, BtX, nx));        // B^T X
    RQ_CUDA(h, cudaMemcpyAsync(G, R, sizeof(double) * nu * nu, cudaMemcpyDeviceToDevice, h->stream));
    RQ_TRY(dgemm(h, false, false, nu, nu, nx, 1.0, BtX, nx, B, nu, 1.0, G, nu));        // R + B^T X B
    RQ_TRY(dgemm(h, false, false, nu, nx, nx, 1.0, BtX, nx, A, nx, 0.0, K, nx));        // B^T X A
    RQ_TRY(cholesky(h, G, nu, Linv, T, flag));
    RQ_TRY(chol_solve(h, G, nu, Linv, K, nx, T2));
    return RELU_QP_OK;
}

int lqr_gain(Ctx& c, int nx, int nu, const double* A, const double* B, const double* Q, const double* R, double* K) {
    relu_qp_t h = &c.h;
    const int nblk = ceil_div(nu, kCholNB);
    double *X, *Xn, *BtX, *G, *AmBK, *XA, *Linv, *T, *T2;
    unsigned long long* red;
    int* flag;
    RQ_TRY(c.buf(&X, (size_t)nx * nx));
    RQ_TRY(c.buf(&Xn, (size_t)nx * nx));
    RQ_TRY(c.buf(&BtX, (size_t)nu * nx));
    RQ_TRY(c.buf(&G, (size_t)nu * nu));
    RQ_TRY(c.buf(&AmBK, (size_t)nx * nx));
    RQ_TRY(c.buf(&XA, (size_t)nx * nx));
    RQ_TRY(c.buf(&Linv, (size_t)nblk * kCholNB * kCholNB));
    RQ_TRY(c.buf(&T, (size_t)nu * kCholNB));
    RQ_TRY(c.buf(&T2, (size_t)kCholNB * nx));
    RQ_TRY(c.buf(&red, 2 * kRiccatiCheckEvery));
    RQ_TRY(c.buf(&flag, 1));
    RQ_CUDA(h, cudaMemcpyAsync(X, Q, sizeof(double) * nx * nx, cudaMemcpyDeviceToDevice, h->stream));
    bool converged = false;
    for (int it = 0; it < kRiccatiMaxIter && !converged; it += kRiccatiCheckEvery) {
        RQ_CUDA(h, cudaMemsetAsync(red, 0, sizeof(unsigned long long) * 2 * kRiccatiCheckEvery, h->stream));
        for (int s = 0; s < kRiccatiCheckEvery; ++s) {
            RQ_TRY(gain(c, nx, nu, A, B, R, X, BtX, G, K, Linv, T, T2, flag));
            RQ_CUDA(h, cudaMemcpyAsync(AmBK, A, sizeof(double) * nx * nx, cudaMemcpyDeviceToDevice, h->stream));
            RQ_TRY(dgemm(h, false, false, nx, nx, nu, -1.0, B, nu, K, nx, 1.0, AmBK, nx));    // A - B K
            RQ_TRY(dgemm(h, false, false, nx, nx, nx, 1.0, X, nx, AmBK, nx, 0.0, XA, nx));     // X (A - B K)
            RQ_CUDA(h, cudaMemcpyAsync(Xn, Q, sizeof(double) * nx * nx, cudaMemcpyDeviceToDevice, h->stream));
            RQ_TRY(dgemm(h, true, false, nx, nx, nx, 1.0, A, nx, XA, nx, 1.0, Xn, nx));        // Q + A^T X (A - B K)
            sym_diff_kernel<<<grid_for((size_t)nx * nx), 256, 0, h->stream>>>(Xn, X, nx, red + 2 * s);
            RQ_CUDA(h, cudaGetLastError());
            std::swap(X, Xn);
        }
        unsigned long long r[2 * kRiccatiCheckEvery];
        int fl = 0;
        RQ_CUDA(h, cudaMemcpyAsync(r, red, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
        RQ_CUDA(h, cudaMemcpyAsync(&fl, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        RQ_CUDA(h, cudaStreamSynchronize(h->stream));
        // a diverging X (unstabilizable plant) also breaks the Cholesky of R + B^T X B:
        // report the divergence first
        for (int s = 0; s < kRiccatiCheckEvery; ++s) {
            double d, mx;
            std::memcpy(&d, &r[2 * s], sizeof(double));
            std::memcpy(&mx, &r[2 * s + 1], sizeof(double));
            if (!std::isfinite(d) || !std::isfinite(mx))
                return fail(h, RELU_QP_ERR_INVALID, "condense: the Riccati iteration diverged ((A, B) not stabilizable?)");
            if (d <= kRiccatiTol * std::max(1.0, mx)) converged = true;
        }
        if (fl) return fail(h, RELU_QP_ERR_NOT_PD, "condense: R + B^T X B is not positive definite");
    }
    if (!converged)
        return fail(h, RELU_QP_ERR_INVALID, "condense: the Riccati iteration did not converge");
    return gain(c, nx, nu, A, B, R, X, BtX, G, K, Linv, T, T2, flag);
}

int condense(Ctx& c, int nx, int nu, int N, const double* hA, const double* hB, const double* hQ, const double* hR,
             const double* hQN, bool state, const double* hK, int precondition, double* oP, double* oA, double* oF,
             double* oE, double* oK) {
    relu_qp_t h = &c.h;
    const int n = N * nu, ru = N * nu, rx = N * nx;
    double *A, *B, *Q, *R, *QN, *K;
    RQ_TRY(c.up(&A, hA, (size_t)nx * nx));
    RQ_TRY(c.up(&B, hB, (size_t)nx * nu));
    RQ_TRY(c.up(&Q, hQ, (size_t)nx * nx));
    RQ_TRY(c.up(&R, hR, (size_t)nu * nu));
    RQ_TRY(c.up(&QN, hQN ? hQN : hQ, (size_t)nx * nx));
    RQ_TRY(c.buf(&K, (size_t)nu * nx));     // zero: no preconditioning
    if (hK) RQ_CUDA(h, cudaMemcpyAsync(K, hK, sizeof(double) * nu * nx, cudaMemcpyHostToDevice, h->stream));
    else if (precondition) RQ_TRY(lqr_gain(c, nx, nu, A, B, Q, R, K));
    // blocks: Abar, T_j = Abar^j B, -K T_j, Mx[k] = Abar^{k+1}, Mu[k] = -K Abar^k
    double *Ab, *Tb, *KT, *Mx, *Mu;
    RQ_TRY(c.buf(&Ab, (size_t)nx * nx));
    RQ_TRY(c.buf(&Tb, (size_t)N * nx * nu));
    RQ_TRY(c.buf(&KT, (size_t)N * nu * nu));
    RQ_TRY(c.buf(&Mx, (size_t)rx * nx));
    RQ_TRY(c.buf(&Mu, (size_t)ru * nx));
    RQ_CUDA(h, cudaMemcpyAsync(Ab, A, sizeof(double) * nx * nx, cudaMemcpyDeviceToDevice, h->stream));
    RQ_TRY(dgemm(h, false, false, nx, nx, nu, -1.0, B, nu, K, nx, 1.0, Ab, nx));
    RQ_CUDA(h, cudaMemcpyAsync(Tb, B, sizeof(double) * nx * nu, cudaMemcpyDeviceToDevice, h->stream));
    RQ_CUDA(h, cudaMemcpyAsync(Mx, Ab, sizeof(double) * nx * nx, cudaMemcpyDeviceToDevice, h->stream));
    for (int j = 1; j < N; ++j) {
        RQ_TRY(dgemm(h, false, false, nx, nu, nx, 1.0, Ab, nx, Tb + (size_t)(j - 1) * nx * nu, nu, 0.0,
                     Tb + (size_t)j * nx * nu, nu));
        RQ_TRY(dgemm(h, false, false, nx, nx, nx, 1.0, Ab, nx, Mx + (size_t)(j - 1) * nx * nx, nx, 0.0,
                     Mx + (size_t)j * nx * nx, nx));
    }
    for (int j = 0; j < N; ++j)
        RQ_TRY(dgemm(h, false, false, nu, nu, nx, -1.0, K, nx, Tb + (size_t)j * nx * nu, nu, 0.0,
                     KT + (size_t)j * nu * nu, nu));
    scale_copy_kernel<<<grid_for((size_t)nu * nx), 256, 0, h->stream>>>(K, -1.0, (size_t)nu * nx, Mu);
    RQ_CUDA(h, cudaGetLastError());
    for (int k = 1; k < N; ++k)
        RQ_TRY(dgemm(h, false, false, nu, nx, nx, -1.0, K, nx, Mx + (size_t)(k - 1) * nx * nx, nx, 0.0,
                     Mu + (size_t)k * nu * nx, nx));
    // S: u rows (block-Toeplitz in -K T_j with I on the diagonal) and x rows (T_j)
    double *Su, *Sx, *HSu, *HSx, *HMu, *HMx, *P, *F;
    RQ_TRY(c.buf(&Su, (size_t)ru * n));
    RQ_TRY(c.buf(&Sx, (size_t)rx * n));
    RQ_TRY(c.buf(&HSu, (size_t)ru * n));
    RQ_TRY(c.buf(&HSx, (size_t)rx * n));
    RQ_TRY(c.buf(&HMu, (size_t)ru * nx));
    RQ_TRY(c.buf(&HMx, (size_t)rx * nx));
    RQ_TRY(c.buf(&P, (size_t)n * n));
    RQ_TRY(c.buf(&F, (size_t)n * nx));
    toeplitz_fill_kernel<<<grid_for((size_t)ru * n), 256, 0, h->stream>>>(KT, N, nu, nu, 1, 1, Su);
    toeplitz_fill_kernel<<<grid_for((size_t)rx * n), 256, 0, h->stream>>>(Tb, N, nx, nu, 0, 0, Sx);
    // H applied block by block: R on the u rows, Q (Q_N for x_N) on the x rows
    blkdiag_mul_kernel<<<grid_for((size_t)ru * n), 256, 0, h->stream>>>(R, R, N, nu, Su, n, HSu);
    blkdiag_mul_kernel<<<grid_for((size_t)rx * n), 256, 0, h->stream>>>(Q, QN, N, nx, Sx, n, HSx);
    blkdiag_mul_kernel<<<grid_for((size_t)ru * nx), 256, 0, h->stream>>>(R, R, N, nu, Mu, nx, HMu);
    blkdiag_mul_kernel<<<grid_for((size_t)rx * nx), 256, 0, h->stream>>>(Q, QN, N, nx, Mx, nx, HMx);
    RQ_CUDA(h, cudaGetLastError());
    // Hbar = S^T H S and F = S^T H M over both row groups
    RQ_TRY(dgemm(h, true, false, n, n, ru, 1.0, Su, n, HSu, n, 0.0, P, n));
    RQ_TRY(dgemm(h, true, false, n, n, rx, 1.0, Sx, n, HSx, n, 1.0, P, n));
    symmetrize_kernel<<<grid_for((size_t)n * n), 256, 0, h->stream>>>(P, n);
    RQ_TRY(dgemm(h, true, false, n, nx, ru, 1.0, Su, n, HMu, nx, 0.0, F, nx));
    RQ_TRY(dgemm(h, true, false, n, nx, rx, 1.0, Sx, n, HMx, nx, 1.0, F, nx));
    RQ_CUDA(h, cudaGetLastError());
    // outputs: constraint rows [u rows; x rows], E = the matching rows of M
    RQ_CUDA(h, cudaMemcpyAsync(oP, P, sizeof(double) * n * n, cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaMemcpyAsync(oF, F, sizeof(double) * n * nx, cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaMemcpyAsync(oA, Su, sizeof(double) * ru * n, cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaMemcpyAsync(oE, Mu, sizeof(double) * ru * nx, cudaMemcpyDeviceToHost, h->stream));
    if (state) {
        RQ_CUDA(h, cudaMemcpyAsync(oA + (size_t)ru * n, Sx, sizeof(double) * rx * n, cudaMemcpyDeviceToHost,
                                   h->stream));
        RQ_CUDA(h, cudaMemcpyAsync(oE + (size_t)ru * nx, Mx, sizeof(double) * rx * nx, cudaMemcpyDeviceToHost,
                                   h->stream));
    }
    if (oK) RQ_CUDA(h, cudaMemcpyAsync(oK, K, sizeof(double) * nu * nx, cudaMemcpyDeviceToHost, h->stream));
    RQ_CUDA(h, cudaStreamSynchronize(h->stream));
    return RELU_QP_OK;
}

}  // namespace

int condense_mpc(int nx, int nu, int N, const double* A, const double* B, const double* Q, const double* R,
                 const double* QN, bool state_rows, const double* K, int precondition, void* stream, double* P,
                 double* Acon, double* F, double* E, double* K_out, std::string* err) {
    Ctx c;
    c.h.stream = (cudaStream_t)stream;
    const int rc = condense(c, nx, nu, N, A, B, Q, R, QN, state_rows, K, precondition, P, Acon, F, E, K_out);
    if (rc != RELU_QP_OK) *err = c.h.err;
    return rc;
}

}  // namespace rq
