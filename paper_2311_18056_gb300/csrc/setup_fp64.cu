// FP64 offline stage of Algorithm 1 ("compute KKT inverse, W and b for each
// rho", Sec. III-B) -- the only FP64 arithmetic on the GPU.
//
// For one bank entry with row penalties rho (rho_i = rho_r, or eq_scale*rho_r
// on equality rows, Sec. II-B):
//   C   = A^T diag(rho) A                        (tiled DGEMM)
//   K   = P + sigma I + C                        (the matrix of Eq. Xbar_update)
//   K   = L L^T                                  (blocked right-looking Cholesky)
//   X   = K^{-1} [sigma I - C, A^T, -I]          (blocked forward/back substitution)
//   AX  = A X
// X = [D(sigma I - A^T rho A) | D A^T | -D] and AX = A X hold the layer in the
// factored form used on the hot path:
//   [x+; (Ax)+] = [X_1 X_2; AX_1 AX_2] [x; 2 rho z - lam'] + [X_3; AX_3] q,
// which is Eq. gpu_update with its z and lam columns merged
// (2 D A^T rho z - D A^T lam = D A^T (2 rho z - lam)) and its z row written
// as A x+ + (A x - z + lam'/rho): the paper's z row is
// [A D(sI - A^T rho A) + A, 2 A D A^T rho - I, -A D A^T + rho^{-1}], i.e. A times
// the x row plus [A, -I, rho^{-1}], and [A, -I, rho^{-1}] v = A x - z + lam'/rho.
#include "common.h"

#include <cuda_bf16.h>

#include <cmath>

namespace rq {

namespace {

constexpr int NB = kCholNB;   // Cholesky / triangular-solve block size

// C = alpha * op(A) * op(B) + beta * C, row-major, 64x64 tiles, 4x4 per thread.
// FP64 on GB300 runs at a small fraction of the FP32 rate, so this kernel is
// bound by the DFMA pipe; the tiling only has to keep it fed.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, double alpha,
                                                    const double* __restrict__ A, int lda,
                                                    const double* __restrict__ B, int ldb,
                                                    double beta, double* __restrict__ C, int ldc) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int i, k;
            if (!TA) { i = e >> 4; k = e & 15; } else { k = e >> 6; i = e & 63; }
            const int gi = m0 + i, gk = k0 + k;
            double v = 0.0;
            if (gi < M && gk < K) v = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
            As[k][i] = v;
        }
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int j, k;
            if (!TB) { k = e >> 6; j = e & 63; } else { j = e >> 4; k = e & 15; }
            const int gj = n0 + j, gk = k0 + k;
            double v = 0.0;
            if (gj < N && gk < K) v = TB ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
            Bs[k][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gi = m0 + ty + 16 * i;
        if (gi >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gj = n0 + tx + 16 * j;
            if (gj >= N) continue;
            double* c = C + (size_t)gi * ldc + gj;
            *c = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
        }
    }
}

// Unblocked Cholesky of one jb x jb diagonal block (in shared memory) and the
// inverse of its lower factor, used to turn the panel and block solves into
// DGEMMs.  A pivot <= 0 (or NaN) sets *flag and is replaced by 1 so that the
// rest of the factorisation stays finite; the host then reports NOT_PD.
constexpr size_t kPotrfSmem = 2 * sizeof(double) * NB * (NB + 1);

__global__ void __launch_bounds__(256) potrf_diag_kernel(double* Km, int ld, int j0, int jb,
                                                         double* Linv, int* flag) {
    extern __shared__ double potrf_smem[];
    double (*a)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(potrf_smem);
    double (*inv)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(potrf_smem + NB * (NB + 1));
    const int tid = threadIdx.x;
    for (int e = tid; e < jb * jb; e += blockDim.x) {
        const int i = e / jb, k = e % jb;
        a[i][k] = (k <= i) ? Km[(size_t)(j0 + i) * ld + j0 + k] : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < jb; ++k) {
        if (tid == 0) {
            double d = a[k][k];
            if (!(d > 0.0)) {
                atomicExch(flag, 1);
                d = 1.0;
            }
            a[k][k] = sqrt(d);
        }
        __syncthreads();
        const double piv = a[k][k];
        for (int i = k + 1 + tid; i < jb; i += blockDim.x) a[i][k] /= piv;
        __syncthreads();
        const int rem = jb - k - 1;
        for (int e = tid; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e / rem, j = k + 1 + e % rem;
            if (j <= i) a[i][j] = fma(-a[i][k], a[j][k], a[i][j]);
        }
        __syncthreads();
    }
    if (tid < jb) {  // column c of L^{-1} by forward substitution
        const int c = tid;
        for (int i = 0; i < jb; ++i) {
            if (i < c) { inv[i][c] = 0.0; continue; }
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) s = fma(-a[i][k], inv[k][c], s);
            inv[i][c] = s / a[i][i];
        }
    }
    __syncthreads();
    for (int e = tid; e < jb * jb; e += blockDim.x) {
        const int i = e / jb, k = e % jb;
        Km[(size_t)(j0 + i) * ld + j0 + k] = (k <= i) ? a[i][k] : 0.0;
        Linv[i * NB + k] = inv[i][k];
    }
}

__global__ void scale_rows_kernel(const double* __restrict__ A, const double* __restrict__ rho,
                                  double* __restrict__ out, int m, int n) {
    const size_t total = (size_t)m * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x)
        out[e] = rho[e / n] * A[e];
}

// K = P + sigma I + C and the right-hand side [sigma I - C, A^T, -I].
__global__ void kkt_rhs_kernel(const double* __restrict__ P, const double* __restrict__ C,
                               const double* __restrict__ A, double sigma, int n, int m,
                               double* __restrict__ Km, double* __restrict__ Rhs) {
    const int NR = 2 * n + m;
    const size_t total = (size_t)n * NR;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / NR), j = (int)(e % NR);
        double v;
        if (j < n) {
            const double c = C[(size_t)i * n + j];
            const double d = (i == j) ? sigma : 0.0;
            Km[(size_t)i * n + j] = P[(size_t)i * n + j] + d + c;
            v = d - c;
        } else if (j < n + m) {
            v = A[(size_t)(j - n) * n + i];
        } else {
            v = (j - n - m == i) ? -1.0 : 0.0;
        }
        Rhs[e] = v;
    }
}

// Layer matrices from X (n x NR) and AX (m x NR): Wt (R x ldw, zero padded)
// and Bop (R x n), FP32 and optionally FP64.
__global__ void pack_layer_kernel(const double* __restrict__ X, const double* __restrict__ AX,
                                  int n, int m, int ldw, float* __restrict__ Wt,
                                  float* __restrict__ Bop, double* __restrict__ Wt64,
                                  double* __restrict__ Bop64) {
    const int R = n + m, NR = 2 * n + m;
    const size_t total = (size_t)R * (ldw + n);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / (ldw + n)), c = (int)(e % (ldw + n));
        const double* src = (r < n) ? X + (size_t)r * NR : AX + (size_t)(r - n) * NR;
        if (c < ldw) {
            const double v = (c < R) ? src[c] : 0.0;
            Wt[(size_t)r * ldw + c] = (float)v;
            if (Wt64 && c < R) Wt64[(size_t)r * R + c] = v;
        } else {
            const int k = c - ldw;
            const double v = src[R + k];
            Bop[(size_t)r * n + k] = (float)v;
            if (Bop64) Bop64[(size_t)r * n + k] = v;
        }
    }
}

// out (rows x ldo, FP32) <- in (rows x cols, FP64); the padding stays zero.
__global__ void to_f32_pad_kernel(const double* __restrict__ in, float* __restrict__ out, int rows,
                                  int cols, int ldo) {
    const size_t count = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
         e += (size_t)gridDim.x * blockDim.x)
        out[(e / cols) * ldo + e % cols] = (float)in[e];
}

// out (cols x ldo, FP32) <- in^T with in (rows x cols, FP64).
__global__ void transpose_f32_kernel(const double* __restrict__ in, float* __restrict__ out,
                                     int rows, int cols, int ldo) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = (float)in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * ldo + r] = tile[threadIdx.x][i];
    }
}

// v = a + b + c with each part the BF16 rounding of what is left (FP64 arithmetic).
__device__ __forceinline__ void split3_f64(double v, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __double2bfloat16(v);
    const double r1 = v - (double)__bfloat162float(a);
    b = __double2bfloat16(r1);
    c = __double2bfloat16(r1 - (double)__bfloat162float(b));
}

// The three BF16 parts of the factored layer (rows [x; Ax], K-major rows of ldk).
__global__ void pack_bf16_layer_kernel(const double* __restrict__ X, const double* __restrict__ AX, int n, int m,
                                       int ldk, size_t part, __nv_bfloat16* __restrict__ out) {
    const int R = n + m, NR = 2 * n + m;
    const size_t total = (size_t)R * ldk;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / ldk), k = (int)(e % ldk);
        double v = 0.0;
        if (k < R) v = (r < n) ? X[(size_t)r * NR + k] : AX[(size_t)(r - n) * NR + k];
        __nv_bfloat16 a, b, c;
        split3_f64(v, a, b, c);
        out[e] = a;
        out[e + part] = b;
        out[e + 2 * part] = c;
    }
}

// The three BF16 parts of the check matrix [[P, A^T], [A, 0]] (x columns
// [0, n64), multiplier columns [n64, n64 + m); rows [0, n) and [n, n + m)).
__global__ void pack_bf16_check_kernel(const double* __restrict__ P, const double* __restrict__ A, int n, int m,
                                       int n64, int ldkc, size_t part, __nv_bfloat16* __restrict__ out) {
    const size_t total = (size_t)(n + m) * ldkc;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / ldkc), k = (int)(e % ldkc);
        double v = 0.0;
        if (j < n) {
            if (k < n) v = P[(size_t)j * n + k];
            else if (k >= n64 && k < n64 + m) v = A[(size_t)(k - n64) * n + j];
        } else if (k < n) {
            v = A[(size_t)(j - n) * n + k];
        }
        __nv_bfloat16 a, b, c;
        split3_f64(v, a, b, c);
        out[e] = a;
        out[e + part] = b;
        out[e + 2 * part] = c;
    }
}

int grid1d(size_t total) {
    size_t g = (total + 255) / 256;
    if (g > 16384) g = 16384;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int dgemm(relu_qp_t h, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
          int lda, const double* B, int ldb, double beta, double* C, int ldc) {
    if (M <= 0 || N <= 0) return RELU_QP_OK;
    dim3 grid(ceil_div(N, 64), ceil_div(M, 64));
    if (!ta && !tb)
        dgemm_kernel<false, false><<<grid, 256, 0, h->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (!ta && tb)
        dgemm_kernel<false, true><<<grid, 256, 0, h->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (ta && !tb)
        dgemm_kernel<true, false><<<grid, 256, 0, h->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else
        dgemm_kernel<true, true><<<grid, 256, 0, h->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    RQ_CUDA(h, cudaGetLastError());
    return RELU_QP_OK;
}

// In-place blocked Cholesky of Km (n x n, ld n); Linv receives the inverse of
// every diagonal block (nblk x NB x NB), T is an n x NB scratch panel.
int cholesky(relu_qp_t h, double* Km, int n, double* Linv, double* T, int* flag) {
    RQ_CUDA(h, cudaFuncSetAttribute(potrf_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kPotrfSmem));
    for (int j = 0; j < n; j += NB) {
        const int jb = (n - j < NB) ? n - j : NB;
        double* Lj = Linv + (size_t)(j / NB) * NB * NB;
        potrf_diag_kernel<<<1, 256, kPotrfSmem, h->stream>>>(Km, n, j, jb, Lj, flag);
        RQ_CUDA(h, cudaGetLastError());
        const int rest = n - j - jb;
        if (rest > 0) {
            double* A21 = Km + (size_t)(j + jb) * n + j;
            RQ_TRY(dgemm(h, false, true, rest, jb, jb, 1.0, A21, n, Lj, NB, 0.0, T, NB));
            RQ_CUDA(h, cudaMemcpy2DAsync(A21, (size_t)n * 8, T, (size_t)NB * 8, (size_t)jb * 8, rest,
                                         cudaMemcpyDeviceToDevice, h->stream));
            RQ_TRY(dgemm(h, false, true, rest, rest, jb, -1.0, T, NB, T, NB, 1.0,
                         Km + (size_t)(j + jb) * n + j + jb, n));
        }
    }
    return RELU_QP_OK;
}

// Rhs (n x NR) <- K^{-1} Rhs with K = L L^T from cholesky().
int chol_solve(relu_qp_t h, const double* L, int n, const double* Linv, double* Rhs, int NR,
               double* T2) {
    for (int j = 0; j < n; j += NB) {  // L Y = R
        const int jb = (n - j < NB) ? n - j : NB;
        const double* Lj = Linv + (size_t)(j / NB) * NB * NB;
        RQ_TRY(dgemm(h, false, false, jb, NR, jb, 1.0, Lj, NB, Rhs + (size_t)j * NR, NR, 0.0, T2, NR));
        RQ_CUDA(h, cudaMemcpyAsync(Rhs + (size_t)j * NR, T2, (size_t)jb * NR * 8,
                                   cudaMemcpyDeviceToDevice, h->stream));
        const int rest = n - j - jb;
        if (rest > 0)
            RQ_TRY(dgemm(h, false, false, rest, NR, jb, -1.0, L + (size_t)(j + jb) * n + j, n,
                         Rhs + (size_t)j * NR, NR, 1.0, Rhs + (size_t)(j + jb) * NR, NR));
    }
    const int last = ((n - 1) / NB) * NB;
    for (int j = last; j >= 0; j -= NB) {  // L^T X = Y
        const int jb = (n - j < NB) ? n - j : NB;
        const double* Lj = Linv + (size_t)(j / NB) * NB * NB;
        RQ_TRY(dgemm(h, true, false, jb, NR, jb, 1.0, Lj, NB, Rhs + (size_t)j * NR, NR, 0.0, T2, NR));
        RQ_CUDA(h, cudaMemcpyAsync(Rhs + (size_t)j * NR, T2, (size_t)jb * NR * 8,
                                   cudaMemcpyDeviceToDevice, h->stream));
        if (j > 0)
            RQ_TRY(dgemm(h, true, false, j, NR, jb, -1.0, L + (size_t)j * n, n, Rhs + (size_t)j * NR,
                         NR, 1.0, Rhs, NR));
    }
    return RELU_QP_OK;
}

namespace {

struct Scratch {
    relu_qp_t h;
    std::vector<void*> ptrs;
    ~Scratch() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    int get(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
        if (e != cudaSuccess)
            return fail(h, RELU_QP_ERR_OOM, std::string("setup scratch: ") + cudaGetErrorString(e));
        ptrs.push_back(q);
        *p = static_cast<T*>(q);
        return RELU_QP_OK;
    }
};

}  // namespace

int make_check_matrices(relu_qp_t h, const double* dP, const double* dA) {
    const int n = h->n, m = h->m;
    const int ldp = (int)round_up(n, 4), ldt = (int)round_up(m > 0 ? m : 1, 4);
    to_f32_pad_kernel<<<grid1d((size_t)n * n), 256, 0, h->stream>>>(dP, h->P32, n, n, ldp);
    RQ_CUDA(h, cudaGetLastError());
    if (m > 0) {
        to_f32_pad_kernel<<<grid1d((size_t)m * n), 256, 0, h->stream>>>(dA, h->A32, m, n, ldp);
        RQ_CUDA(h, cudaGetLastError());
        dim3 g(ceil_div(n, 32), ceil_div(m, 32));
        transpose_f32_kernel<<<g, dim3(32, 8), 0, h->stream>>>(dA, h->At32, m, n, ldt);
        RQ_CUDA(h, cudaGetLastError());
    }
    return RELU_QP_OK;
}

int pack_bf16_layer(relu_qp_t h, int r, const double* X, const double* AX) {
    BatchWork& w = h->bw;
    const size_t part = (size_t)w.Rpad * w.ldk;
    __nv_bfloat16* out = static_cast<__nv_bfloat16*>(w.WB) + (size_t)r * 3 * part;
    pack_bf16_layer_kernel<<<grid1d((size_t)h->R * w.ldk), 256, 0, h->stream>>>(X, AX, h->n, h->m, w.ldk, part, out);
    RQ_CUDA(h, cudaGetLastError());
    return RELU_QP_OK;
}

int pack_bf16_check(relu_qp_t h, const double* dP, const double* dA) {
    BatchWork& w = h->bw;
    const size_t part = (size_t)w.npad * w.ldkc;
    pack_bf16_check_kernel<<<grid1d((size_t)(h->n + h->m) * w.ldkc), 256, 0, h->stream>>>(
        dP, dA, h->n, h->m, w.n64, w.ldkc, part, static_cast<__nv_bfloat16*>(w.WCB));
    RQ_CUDA(h, cudaGetLastError());
    return RELU_QP_OK;
}

int build_bank(relu_qp_t h, const double* dP, const double* dA, const std::vector<double>& row_scale) {
    const int n = h->n, m = h->m, R = h->R, NR = 2 * n + m;
    const int nblk = ceil_div(n, NB);
    Scratch s{h, {}};
    double *C, *Km, *Rhs, *AX = nullptr, *rA = nullptr, *Linv, *T, *T2, *rho_d = nullptr;
    int* flag;
    RQ_TRY(s.get(&C, (size_t)n * n));
    RQ_TRY(s.get(&Km, (size_t)n * n));
    RQ_TRY(s.get(&Rhs, (size_t)n * NR));
    RQ_TRY(s.get(&Linv, (size_t)nblk * NB * NB));
    RQ_TRY(s.get(&T, (size_t)n * NB));
    RQ_TRY(s.get(&T2, (size_t)NB * NR));
    RQ_TRY(s.get(&flag, 1));
    if (m > 0) {
        RQ_TRY(s.get(&AX, (size_t)m * NR));
        RQ_TRY(s.get(&rA, (size_t)m * n));
        RQ_TRY(s.get(&rho_d, (size_t)m));
    }
    std::vector<double> rho_h(m > 0 ? m : 1);
    for (int r = 0; r < h->nr; ++r) {
        const double rho = h->bank[r];
        RQ_CUDA(h, cudaMemsetAsync(flag, 0, sizeof(int), h->stream));
        if (m > 0) {
            for (int i = 0; i < m; ++i) rho_h[i] = rho * row_scale[i];
            RQ_CUDA(h, cudaMemcpyAsync(rho_d, rho_h.data(), sizeof(double) * m, cudaMemcpyHostToDevice,
                                       h->stream));
            scale_rows_kernel<<<grid1d((size_t)m * n), 256, 0, h->stream>>>(dA, rho_d, rA, m, n);
            RQ_CUDA(h, cudaGetLastError());
            RQ_TRY(dgemm(h, true, false, n, n, m, 1.0, dA, n, rA, n, 0.0, C, n));   // A^T (rho A)
        } else {
            RQ_CUDA(h, cudaMemsetAsync(C, 0, sizeof(double) * n * n, h->stream));
        }
        kkt_rhs_kernel<<<grid1d((size_t)n * NR), 256, 0, h->stream>>>(dP, C, dA, h->sigma, n, m, Km, Rhs);
        RQ_CUDA(h, cudaGetLastError());
        RQ_TRY(cholesky(h, Km, n, Linv, T, flag));
        RQ_TRY(chol_solve(h, Km, n, Linv, Rhs, NR, T2));
        if (m > 0) RQ_TRY(dgemm(h, false, false, m, NR, n, 1.0, dA, n, Rhs, NR, 0.0, AX, NR));
        rq::BankEntry& be = h->be[r];
        be.rho = rho;
        pack_layer_kernel<<<grid1d((size_t)R * (h->ldw + n)), 256, 0, h->stream>>>(
            Rhs, AX, n, m, h->ldw, be.Wt, be.Bop, be.Wt64, be.Bop64);
        RQ_CUDA(h, cudaGetLastError());
        if (h->bw.cap > 0 && h->bw.prec == RELU_QP_PREC_BF16X3) RQ_TRY(pack_bf16_layer(h, r, Rhs, AX));
        int hflag = 0;
        RQ_CUDA(h, cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        RQ_CUDA(h, cudaStreamSynchronize(h->stream));
        if (hflag)
            return fail(h, RELU_QP_ERR_NOT_PD,
                        "Cholesky pivot <= 0 for rho = " + std::to_string(rho) +
                            ": P + sigma I + A^T rho A is not positive definite");
    }
    return RELU_QP_OK;
}

}  // namespace rq
