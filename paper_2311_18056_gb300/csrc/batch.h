// Batched solves: many QPs that share P and A (hence every W_rho) but each
// have their own q, l, u and iterate.  Internal to librelu_qp.so.
//
// Layout.  Per-QP state is indexed by the QP id (rows of length n, m or
// R = n + m, padded).  The GEMM operand is indexed by *slot*: the slots of a
// tile of 128 consecutive slots all use the same bank entry, so after every
// check the active QPs are regrouped by their rho index (perm[slot] = QP id,
// -1 for padding) and converged QPs leave the batch.
//
// Each layer is one GEMM  T[slot, r] = sum_k S[slot, k] Wt_rho[r, k]  followed
// by the element-wise part of the layer (bias, clamp, multiplier step) in the
// epilogue; see layer_elem below.
#pragma once

#include "common.h"

#include <cuda_bf16.h>

#include <vector>

namespace rq {

constexpr int kSlotTile = 128;        // slots per GEMM tile (the tcgen05 M dimension)

enum : unsigned {
    EPI_REBASE = 1u,   // first layer of a chunk: accurate product of s, stores c and s_ref
    EPI_LAST = 2u,     // last layer of a chunk: the next operand is written by the fill kernel
    EPI_CHECK = 4u,    // last layer before a check: write x into the check operand
    EPI_REFINE = 8u,   // BF16 split form: t = c + Wt (s - s_ref)
};

enum { QP_ACTIVE = -1, QP_UNUSED = -2 };
enum { RW_RP = 0, RW_RD, RW_AX, RW_Z, RW_PX, RW_ATL, RW_WORDS = 8 };
enum { CNT_TILES = 0, CNT_ACTIVE = 1, CNT_ERR = 2, CNT_WORDS = 4 };

struct BatchParams {
    int n, m, R, ldn, ldm, ldR, ldk, n64, ldkc, cap, slots, nr;
    float rho[RQ_MAX_RHO];
    double rhod[RQ_MAX_RHO];
    double logrho[RQ_MAX_RHO];              // log of each bank entry (the penalty rule's distance)
    const float* rs;                         // per-row penalty scale (1 or eq_scale)
    // scaled problems: the residual and norm factors back to the original problem,
    // 1/(c D) for rows of x and 1/E for constraint rows (nullptr without scaling)
    const float *rsx, *rsz;
    float *Y, *Z, *LAM, *AY, *LSTD, *C, *SREF, *PY;
    float* RR;                               // refined layers: r = (Ax) - z + lam'/rho for the next layer
    const float *L, *U, *Q, *BIAS, *QN;
    const int* perm;
    const int* tile_rho;
    const int* counters;
    unsigned* RED;
    const float* Sin;                        // FP32 operand in  [slots][ldk]
    float* Sout;                             // FP32 operand out [slots][ldk]
    __nv_bfloat16 *Dhi, *Dlo;                // BF16 split operand out (refined form)
    float* CK32;                             // FP32 check operand [slots][ldkc]
    __nv_bfloat16* CK;                       // BF16 3-way check operand [3][slots][ldkc]
    unsigned flags;
};

// max that keeps a NaN (fmaxf would drop it)
__device__ __forceinline__ float nmax(float a, float b) { return (b > a || b != b) ? b : a; }

__device__ __forceinline__ void split2(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// v = a + b + c + O(2^-27 |v|); each difference is exact in FP32.
__device__ __forceinline__ void split3(float v, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(a);
    b = __float2bfloat16_rn(r1);
    c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

__device__ __forceinline__ void put_check(const BatchParams& p, int slot, int col, float v) {
    const size_t o = (size_t)slot * p.ldkc + col;
    if (p.CK) {
        __nv_bfloat16 a, b, c;
        split3(v, a, b, c);
        const size_t part = (size_t)p.slots * p.ldkc;
        p.CK[o] = a;
        p.CK[o + part] = b;
        p.CK[o + 2 * part] = c;
    } else {
        p.CK32[o] = v;
    }
}

// The element-wise part of one layer for output row r of the QP in `slot`
// (Eq. gpu_update in the factored form; see setup_fp64.cu):
//   t = acc + b (or + c in the refined form), x rows: x+ = t;
//   Ax rows i:  r_i = (Ax)_i - z_i + lam'_i/rho_i,  z+ = clamp(t + r_i, l_i, u_i),
//               lam'+ = rho_i r_i,  (Ax)+ = t,  operand entry 2 rho_i z+ - lam'+.
// The BF16 split form carries r itself between the layers of a chunk:
// r+ = (Ax)+ - z+ + lam'+/rho_i = t - z+ + r (array RR); the refined layers
// read r from RR and write x, Ax, z and lam' only at the last layer of the
// chunk.  With EPI_CHECK the new x also goes into the check operand.
// The z, lam' and operand update of one row of A x (FP32), given the layer's
// product t and the carried r = (Ax) - z + lam'/rho_i.  Every FP32 path calls
// this one function (tiled kernels and the convergence tail), so that a QP's
// iterates do not depend on which kernel runs its layer.
//
// The steps that combine a product with a sum are written with explicit
// roundings (fmaf, __fmul_rn) rather than left to the compiler's contraction
// choice, which can differ between kernels: every kernel then rounds them
// alike and produces the same bits.
// 2 rho_i z - lam': the operand entry of a row of A x
__device__ __forceinline__ float next_operand(float rho_i, float z, float lam) { return fmaf(2.f * rho_i, z, -lam); }
// lam' = rho_i r
__device__ __forceinline__ float lam_layer(float rho_i, float rr) { return __fmul_rn(rho_i, rr); }
// lam_std = lam' + rho_i (A x - z)
__device__ __forceinline__ float lam_standard(float lam, float rho_i, float d) { return fmaf(rho_i, d, lam); }

__device__ __forceinline__ void ax_row_update(float t, float rr, float lo, float up, float rho_i, float& zn,
                                              float& ln, float& s_new) {
    zn = fminf(fmaxf(t + rr, lo), up);
    ln = lam_layer(rho_i, rr);
    s_new = next_operand(rho_i, zn, ln);
}

__device__ __forceinline__ float ax_row_carry(float ay, float zi, float li, float rho_i) {
    return ay - zi + li / rho_i;
}

__device__ __forceinline__ void layer_elem(const BatchParams& p, int slot, int qp, int ri, int r, float acc) {
    const unsigned f = p.flags;
    const bool refine_only = (f & EPI_REFINE) && !(f & EPI_REBASE);
    // the split form writes x, Ax, z, lam' only at a chunk's last layer (its other layers,
    // the accurate first one included, keep chunk-local data: c, s_ref, r and the operand)
    const bool store_state = !(f & EPI_REFINE) || (f & EPI_LAST);
    const size_t oR = (size_t)qp * p.ldR + r;
    const float* bias = p.BIAS + (size_t)ri * p.cap * p.ldR;
    float t;
    if (f & EPI_REBASE) {
        t = acc + bias[oR];
        p.C[oR] = t;
    } else if (f & EPI_REFINE) {
        t = acc + p.C[oR];
    } else {
        t = acc + bias[oR];
    }
    float s_new;
    if (r < p.n) {
        const size_t o = (size_t)qp * p.ldn + r;
        if (f & EPI_REBASE) p.SREF[oR] = p.Y[o];
        if (store_state) p.Y[o] = t;
        s_new = t;
        if (f & EPI_CHECK) put_check(p, slot, r, t);
    } else {
        const int i = r - p.n;
        const size_t o = (size_t)qp * p.ldm + i;
        const float rho_i = p.rho[ri] * p.rs[i];
        float rr;
        if (refine_only) {
            rr = p.RR[o];
        } else {
            const float ay = p.AY[o], zi = p.Z[o], li = p.LAM[o];
            if (f & EPI_REBASE) p.SREF[oR] = next_operand(rho_i, zi, li);
            rr = ax_row_carry(ay, zi, li, rho_i);
        }
        float zn, ln;
        ax_row_update(t, rr, p.L[o], p.U[o], rho_i, zn, ln, s_new);
        if (f & EPI_REFINE) p.RR[o] = t - zn + rr;
        if (store_state) {
            p.AY[o] = t;
            p.Z[o] = zn;
            p.LAM[o] = ln;
        }
    }
    if (!(f & EPI_LAST)) {
        const size_t so = (size_t)slot * p.ldk + r;
        if (f & EPI_REFINE) {
            __nv_bfloat16 hi, lo;
            split2(s_new - p.SREF[oR], hi, lo);
            p.Dhi[so] = hi;
            p.Dlo[so] = lo;
        } else {
            p.Sout[so] = s_new;
        }
    }
}

__device__ __forceinline__ void ld4(const float* __restrict__ src, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(src);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}

__device__ __forceinline__ void st4(float* __restrict__ dst, const float (&v)[4]) {
    *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
}

// layer_elem for 4 consecutive rows r0..r0+3 of one QP, all x rows or all Ax
// rows, 16-byte aligned, in two halves: chunk4_load reads every input the
// layer needs (none of it depends on the product) and chunk4_apply combines it
// with the product and writes the new state.  The tensor-core epilogue issues
// the loads of all its 4-row pieces before the first apply, so one memory
// round trip covers 16 rows of 8 QPs; 4 lanes per QP make each warp-wide
// 128-bit access cover 8 QPs' contiguous 64-byte row segments.
struct Chunk4 {
    float t[4], sref[4], ay[4], zz[4], lm[4], lo[4], up[4];
};

__device__ __forceinline__ void chunk4_load(const BatchParams& p, int qp, int ri, int r0, Chunk4& c) {
    const unsigned f = p.flags;
    const size_t oR = (size_t)qp * p.ldR + r0;
    const bool refine_only = (f & EPI_REFINE) && !(f & EPI_REBASE);
    ld4(refine_only ? p.C + oR : p.BIAS + (size_t)ri * p.cap * p.ldR + oR, c.t);
    if (refine_only) ld4(p.SREF + oR, c.sref);
    if (r0 < p.n) {
        if (f & EPI_REBASE) ld4(p.Y + (size_t)qp * p.ldn + r0, c.sref);
    } else {
        const size_t o = (size_t)qp * p.ldm + (r0 - p.n);
        ld4(p.AY + o, c.ay);
        ld4(p.Z + o, c.zz);
        ld4(p.LAM + o, c.lm);
        ld4(p.L + o, c.lo);
        ld4(p.U + o, c.up);
    }
}

// rs = p.rs[r0 - n .. r0 - n + 3] for Ax rows (unused for x rows)
__device__ __forceinline__ void chunk4_apply(const BatchParams& p, int slot, int qp, int ri, int r0,
                                             const float (&acc)[4], Chunk4& c, const float (&rs)[4]) {
    const unsigned f = p.flags;
    const size_t oR = (size_t)qp * p.ldR + r0;
    const bool store_state = !(f & EPI_REFINE) || (f & EPI_LAST);   // as layer_elem
    float s_new[4];
    if (r0 < p.n) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            c.t[k] += acc[k];
            s_new[k] = c.t[k];
        }
        if (store_state) st4(p.Y + (size_t)qp * p.ldn + r0, c.t);
        if (f & EPI_CHECK)
            for (int k = 0; k < 4; ++k) put_check(p, slot, r0 + k, c.t[k]);
    } else {
        const size_t o = (size_t)qp * p.ldm + (r0 - p.n);
        float rn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            c.t[k] += acc[k];
            const float rho_i = p.rho[ri] * rs[k];
            if (f & EPI_REBASE) c.sref[k] = next_operand(rho_i, c.zz[k], c.lm[k]);
            const float rr = ax_row_carry(c.ay[k], c.zz[k], c.lm[k], rho_i);
            const float zn = fminf(fmaxf(c.t[k] + rr, c.lo[k]), c.up[k]);
            const float ln = lam_layer(rho_i, rr);
            rn[k] = c.t[k] - zn + rr;
            c.zz[k] = zn;
            c.lm[k] = ln;
            s_new[k] = next_operand(rho_i, zn, ln);
        }
        if (store_state) {
            st4(p.AY + o, c.t);
            st4(p.Z + o, c.zz);
            st4(p.LAM + o, c.lm);
        }
        if (f & EPI_REFINE) st4(p.RR + o, rn);
    }
    if (f & EPI_REBASE) {
        st4(p.C + oR, c.t);
        st4(p.SREF + oR, c.sref);
    }
    if (!(f & EPI_LAST)) {
        const size_t so = (size_t)slot * p.ldk + r0;
        if (f & EPI_REFINE) {
            __nv_bfloat16 hi[4], lo[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) split2(s_new[k] - c.sref[k], hi[k], lo[k]);
            uint2 vh, vl;
            vh.x = (uint32_t)__bfloat16_as_ushort(hi[0]) | ((uint32_t)__bfloat16_as_ushort(hi[1]) << 16);
            vh.y = (uint32_t)__bfloat16_as_ushort(hi[2]) | ((uint32_t)__bfloat16_as_ushort(hi[3]) << 16);
            vl.x = (uint32_t)__bfloat16_as_ushort(lo[0]) | ((uint32_t)__bfloat16_as_ushort(lo[1]) << 16);
            vl.y = (uint32_t)__bfloat16_as_ushort(lo[2]) | ((uint32_t)__bfloat16_as_ushort(lo[3]) << 16);
            *reinterpret_cast<uint2*>(p.Dhi + so) = vh;
            *reinterpret_cast<uint2*>(p.Dlo + so) = vl;
        } else {
            st4(p.Sout + so, s_new);
        }
    }
}

// The refined layers' 4-row piece (flags EPI_REFINE without EPI_REBASE): the
// inputs are c, s_ref and, for Ax rows, r, l, u.
struct Chunk4R {
    float t[4], sref[4], rr[4], lo[4], up[4];
};

__device__ __forceinline__ void chunk4_load(const BatchParams& p, int qp, int ri, int r0, Chunk4R& c) {
    const size_t oR = (size_t)qp * p.ldR + r0;
    ld4(p.C + oR, c.t);
    ld4(p.SREF + oR, c.sref);
    if (r0 >= p.n) {
        const size_t o = (size_t)qp * p.ldm + (r0 - p.n);
        ld4(p.RR + o, c.rr);
        ld4(p.L + o, c.lo);
        ld4(p.U + o, c.up);
    }
}

__device__ __forceinline__ void chunk4_apply(const BatchParams& p, int slot, int qp, int ri, int r0,
                                             const float (&acc)[4], Chunk4R& c, const float (&rs)[4]) {
    const unsigned f = p.flags;
    const bool last = (f & EPI_LAST) != 0;
    float s_new[4];
    if (r0 < p.n) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            c.t[k] += acc[k];
            s_new[k] = c.t[k];
        }
        if (last) st4(p.Y + (size_t)qp * p.ldn + r0, c.t);
        if (f & EPI_CHECK)
            for (int k = 0; k < 4; ++k) put_check(p, slot, r0 + k, c.t[k]);
    } else {
        const size_t o = (size_t)qp * p.ldm + (r0 - p.n);
        float zn[4], ln[4], rn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            c.t[k] += acc[k];
            const float rho_i = p.rho[ri] * rs[k];
            zn[k] = fminf(fmaxf(c.t[k] + c.rr[k], c.lo[k]), c.up[k]);
            ln[k] = lam_layer(rho_i, c.rr[k]);
            rn[k] = c.t[k] - zn[k] + c.rr[k];
            s_new[k] = next_operand(rho_i, zn[k], ln[k]);
        }
        st4(p.RR + o, rn);
        if (last) {
            st4(p.AY + o, c.t);
            st4(p.Z + o, zn);
            st4(p.LAM + o, ln);
        }
    }
    if (!last) {
        const size_t so = (size_t)slot * p.ldk + r0;
        __nv_bfloat16 hi[4], lo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) split2(s_new[k] - c.sref[k], hi[k], lo[k]);
        uint2 vh, vl;
        vh.x = (uint32_t)__bfloat16_as_ushort(hi[0]) | ((uint32_t)__bfloat16_as_ushort(hi[1]) << 16);
        vh.y = (uint32_t)__bfloat16_as_ushort(hi[2]) | ((uint32_t)__bfloat16_as_ushort(hi[3]) << 16);
        vl.x = (uint32_t)__bfloat16_as_ushort(lo[0]) | ((uint32_t)__bfloat16_as_ushort(lo[1]) << 16);
        vl.y = (uint32_t)__bfloat16_as_ushort(lo[2]) | ((uint32_t)__bfloat16_as_ushort(lo[3]) << 16);
        *reinterpret_cast<uint2*>(p.Dhi + so) = vh;
        *reinterpret_cast<uint2*>(p.Dlo + so) = vl;
    }
}

__device__ __forceinline__ void red_slot(unsigned* RED, int qp, int word, float v) {
    atomicMax(RED + (size_t)qp * RW_WORDS + word, __float_as_uint(fabsf(v)));
}

// First residual product, row r of [P; A] x (Eqs. primal, dual): P x is kept
// for the second product; A x refreshes the carried Ax, gives the primal
// residual A x - z and the multiplier lam_std = lam' + rho (A x - z), which
// goes into the check operand.
// (Scaled problems: the maxima are those of the original problem's quantities,
// each row's value times its factor rsx or rsz.)
__device__ __forceinline__ void check1_elem(const BatchParams& p, int slot, int qp, int ri, int r, float acc,
                                            float& rp, float& nax, float& nz, float& npx) {
    if (r < p.n) {
        p.PY[(size_t)qp * p.ldn + r] = acc;
        npx = nmax(npx, fabsf(p.rsx ? acc * p.rsx[r] : acc));
    } else {
        const int i = r - p.n;
        const size_t o = (size_t)qp * p.ldm + i;
        const float zi = p.Z[o];
        const float d = acc - zi;
        const float ls = lam_standard(p.LAM[o], p.rho[ri] * p.rs[i], d);
        p.AY[o] = acc;
        p.LSTD[o] = ls;
        put_check(p, slot, p.n64 + i, ls);
        const float f = p.rsz ? p.rsz[i] : 1.f;
        rp = nmax(rp, fabsf(p.rsz ? d * f : d));
        nax = nmax(nax, fabsf(p.rsz ? acc * f : acc));
        nz = nmax(nz, fabsf(p.rsz ? zi * f : zi));
    }
}

// check1_elem for 4 consecutive rows r0..r0+3 of one QP, all rows of x
// (r0 + 3 < n) or all of A x (r0 >= n, n a multiple of 4), 16-byte aligned:
// the same arithmetic with 128-bit loads and stores of the QP's rows.
__device__ __forceinline__ void check1_4(const BatchParams& p, int slot, int qp, int ri, int r0, const float (&a)[4],
                                         float& rp, float& nax, float& nz, float& npx) {
    if (r0 < p.n) {
        st4(p.PY + (size_t)qp * p.ldn + r0, a);
#pragma unroll
        for (int k = 0; k < 4; ++k) npx = nmax(npx, fabsf(p.rsx ? a[k] * p.rsx[r0 + k] : a[k]));
        return;
    }
    const int i0 = r0 - p.n;
    const size_t o = (size_t)qp * p.ldm + i0;
    float z[4], lm[4], rs[4], ls[4];
    ld4(p.Z + o, z);
    ld4(p.LAM + o, lm);
    ld4(p.rs + i0, rs);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float d = a[k] - z[k];
        ls[k] = lam_standard(lm[k], p.rho[ri] * rs[k], d);
        const float f = p.rsz ? p.rsz[i0 + k] : 1.f;
        rp = nmax(rp, fabsf(p.rsz ? d * f : d));
        nax = nmax(nax, fabsf(p.rsz ? a[k] * f : a[k]));
        nz = nmax(nz, fabsf(p.rsz ? z[k] * f : z[k]));
    }
    st4(p.AY + o, a);
    st4(p.LSTD + o, ls);
#pragma unroll
    for (int k = 0; k < 4; ++k) put_check(p, slot, p.n64 + i0 + k, ls[k]);
}

// check2_elem for 4 consecutive rows j0..j0+3 (< n) of one QP, 16-byte aligned.
__device__ __forceinline__ void check2_4(const BatchParams& p, int qp, int j0, const float (&a)[4], float& rd,
                                         float& natl) {
    float px[4], q[4];
    ld4(p.PY + (size_t)qp * p.ldn + j0, px);
    ld4(p.Q + (size_t)qp * p.ldn + j0, q);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float r = px[k] + q[k] + a[k];
        rd = nmax(rd, fabsf(p.rsx ? r * p.rsx[j0 + k] : r));
        natl = nmax(natl, fabsf(p.rsx ? a[k] * p.rsx[j0 + k] : a[k]));
    }
}

// Second residual product, row j of A^T lam_std: dual residual P x + q + A^T lam_std.
__device__ __forceinline__ void check2_elem(const BatchParams& p, int qp, int j, float acc, float& rd, float& natl) {
    const float r = p.PY[(size_t)qp * p.ldn + j] + p.Q[(size_t)qp * p.ldn + j] + acc;
    rd = nmax(rd, fabsf(p.rsx ? r * p.rsx[j] : r));
    natl = nmax(natl, fabsf(p.rsx ? acc * p.rsx[j] : acc));
}

struct DecideArgs {
    int B, it, final_iter, adaptive;
    double eps_abs, eps_rel;
    float *XO, *ZO, *LO;
    int *status, *iters, *rho_idx, *nsw;
    float *rpo, *rdo;
    // continuous batching: layers since the previous check of each QP (0 = whole-batch
    // solve, where `it` and `final_iter` hold for every QP), per-QP layer budget, and the
    // list the finished QPs are appended to
    int serve_len, max_iter;
    int *done_list, *done_count;
};

// Stop test (Eqs. primal, dual with eps_abs + eps_rel * norms) and penalty rule
// (Eq. rho_update, nearest bank entry in log distance) for one active QP from
// its reduction words w (|.|-maxima as float bits, RW_*), its bank index ri and
// (continuous batching) its layer count before this chunk.  Pure: act = 1 if
// the QP finished (status, it_qp, residuals filled in), 2 if it switches to
// bank entry nri, 0 otherwise.
struct Decision {
    int act, status, it_qp, nri;
    float rp, rd;
};

__device__ __forceinline__ Decision decide_eval(const BatchParams& p, const DecideArgs& d, int qp,
                                                const unsigned (&w)[RW_WORDS], int ri, int iters_before) {
    const double rp = __uint_as_float(w[RW_RP]), rd = __uint_as_float(w[RW_RD]);
    const double nax = __uint_as_float(w[RW_AX]), nz = __uint_as_float(w[RW_Z]);
    const double npx = __uint_as_float(w[RW_PX]), natl = __uint_as_float(w[RW_ATL]);
    const double qn = p.QN[qp];
    Decision x{0, 0, d.serve_len > 0 ? iters_before + d.serve_len : d.it, ri, (float)rp, (float)rd};
    const bool final_qp = d.serve_len > 0 ? x.it_qp >= d.max_iter : d.final_iter != 0;
    const bool numerical = !(isfinite(rp) && isfinite(rd) && isfinite(npx) && isfinite(natl));
    const double eps_p = d.eps_abs + d.eps_rel * fmax(nax, nz);
    const double eps_d = d.eps_abs + d.eps_rel * fmax(fmax(npx, natl), qn);
    const bool converged = !numerical && rp <= eps_p && rd <= eps_d;
    if (converged || numerical || final_qp) {
        x.act = 1;
        x.status = numerical ? RELU_QP_NUMERICAL : (converged ? RELU_QP_SOLVED : RELU_QP_MAX_ITER);
        return x;
    }
    if (d.adaptive) {
        const double num = rp * fmax(fmax(npx, natl), fmax(qn, 1e-4));
        const double den = rd * fmax(fmax(nax, nz), 1e-4);
        if (num > 0.0 && den > 0.0) {
            const double est = p.rhod[ri] * sqrt(num / den);
            if (isfinite(est) && est > 0.0) {
                const double le = log(est);
                double best = 1e300;
                for (int k = 0; k < p.nr; ++k) {
                    const double dd = fabs(le - p.logrho[k]);
                    if (dd < best) { best = dd; x.nri = k; }
                }
            }
        }
        if (x.nri != ri) x.act = 2;
    }
    return x;
}

// decide_eval for the QP's own records, which it then updates (status, iters,
// residuals, the done list; bank index and switch count).  Returns act; nri
// receives the bank index to continue with.
__device__ __forceinline__ int decide_qp(const BatchParams& p, const DecideArgs& d, int qp,
                                         const unsigned (&w)[RW_WORDS], int& nri) {
    const Decision x = decide_eval(p, d, qp, w, d.rho_idx[qp], d.iters[qp]);
    nri = x.nri;
    if (x.act == 1) {
        d.status[qp] = x.status;
        d.iters[qp] = x.it_qp;
        d.rpo[qp] = x.rp;
        d.rdo[qp] = x.rd;
        if (d.done_list) d.done_list[atomicAdd(d.done_count, 1)] = qp;
        return 1;
    }
    if (x.act == 2) {
        d.rho_idx[qp] = x.nri;
        d.nsw[qp] += 1;
    }
    if (d.serve_len > 0) d.iters[qp] = x.it_qp;
    return x.act;
}

// --- entry points of the tcgen05 backend (batch_tc.cu) ---------------------
int tc_prepare(relu_qp_t h);                     // BF16 splits of every W_rho and of [P | A^T]
// operand_set < 0: accurate (3-way) layer; pdl: programmatic dependent launch on the
// previous kernel of the stream (refined layers only)
int tc_layer(relu_qp_t h, const BatchParams& p, int operand_set, int tiles, int active_tiles, bool pdl = false);
// phase 1: [P; A] x, 2: A^T lam; active_tiles: slot tiles in use (an upper bound)
int tc_check(relu_qp_t h, const BatchParams& p, int phase, int tiles, int active_tiles);
// Refined layers 1 .. nl of a chunk in one persistent launch (flags of layer nl
// get last_flags); active_tiles = slot tiles in use (an upper bound).
// RELU_QP_ERR_UNSUPPORTED: not possible here (too many CTAs for one wave, or the
// launch was refused, which disables it for the handle); the caller launches the
// layers one by one.
int tc_chunk(relu_qp_t h, const BatchParams& p, int nl, unsigned last_flags, int active_tiles);
void tc_disable_chunk(relu_qp_t h);
// Resident-weight chunk kernel (one slot tile of at most 64 active QPs, the
// layer's rows of Wt kept in shared memory over a cluster of 8 CTAs that
// split k): refined layers 1 .. nl of a chunk, as tc_chunk.
// RELU_QP_ERR_UNSUPPORTED: not possible here (more tiles or QPs, too large a
// problem for one wave, or a refused launch, which disables it for the handle).
bool tc_small_eligible(relu_qp_t h, int active, int active_tiles);
int tc_small(relu_qp_t h, const BatchParams& p, int nl, unsigned last_flags, int active, int active_tiles);
void tc_small_set(relu_qp_t h, bool use);   // use it where eligible (set by the tuner)
bool tc_small_chosen(relu_qp_t h);
void tc_release(relu_qp_t h);
// refined-layer configuration: K split over a cluster of ks CTAs, tile width bn
struct LayerCfg {
    int ks, bn;
};
int tc_layer_cfgs(relu_qp_t h, std::vector<LayerCfg>& out);          // every configuration the problem allows
int tc_set_layer_cfg(relu_qp_t h, LayerCfg c);                        // one for every tile count
int tc_set_layer_table(relu_qp_t h, const std::vector<LayerCfg>& by_tiles);  // [t] = for t active slot tiles
// device error word of the backend (0 = none) and, for a deadline, which wait gave up
// (site); clears both
int tc_error(relu_qp_t h, int* site = nullptr);

// Deadline diagnostics of the tensor-core kernels' waits (kind 0: mbarrier,
// 1: layer counter); dev: >= 4 zeroed ints (error word, site, counter).
int tc_diag_wait(int kind, int* dev, long long ns, cudaStream_t stream);

// --- convergence tail (batch_tail.cu) --------------------------------------
constexpr int kTailMax = 8;      // QPs the tail kernel takes at most
int batch_tail_alloc(relu_qp_t h);
// Run every remaining chunk (layers it0 + 1 .. max_iter) of the nq <= kTailMax
// active QPs in one cooperative launch; d holds the decision records.
int batch_tail(relu_qp_t h, const BatchParams& p, const DecideArgs& d, int nq, int it0, int max_iter);
int batch_tail_error(relu_qp_t h);   // device error word of the last tail launch

}  // namespace rq
