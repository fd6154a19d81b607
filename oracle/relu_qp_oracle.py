"""FP64 CPU oracle for ReLU-QP (arXiv 2311.18056) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The GPU library never calls it and it
shares no code with the GPU library (no kernels, helpers, constants or
generators); it takes plain NumPy arrays and works in float64 throughout.

What it computes, in the paper's order and notation (paper letter -> here):
H -> P, g -> q, G -> A, c,d -> l,u, primal y -> x, dual lambda -> lam.

* Sec. II-B, Eqs. Xbar_update .. lambda_update_gen: one step of standard
  ADMM for the split problem (Eq. admm_qp_def), with the sigma prox term and
  the extra multiplier mu: ``admm_step_standard``.
* Sec. III-A, Eqs. basic_lambda_update, basic_y_update, clamp: the reordered
  ("modified") step that updates lam first: ``admm_step_modified``.
* Sec. III-A, Eq. gpu_update: the same step as one weight-tied layer
  v+ = clamp(W v + b) on v = [x; z; lam], with W and b written out as the
  3x3 block matrix of the paper: ``relu_layer_weights`` / ``relu_layer_step``.
* Sec. II-B "Convergence Criteria", Eqs. primal, dual: ``residuals``.
* Sec. II-B "Adaptive Penalty", Eq. rho_update and Sec. III-C "Penalty
  Scaling Heuristics" (nearest entry of a rho list): ``rho_estimate``,
  ``nearest_rho_index``.
* Sec. II-B "Warm Starting" and Algorithm 1: ``solve``.
* Algorithm 1 "Scale problem" and Sec. III-D "Preconditioning" (a modified
  Ruiz equilibration that, like OSQP, scales the variables and the cost):
  ``ruiz_scaling``, and ``solve_scaled`` = Algorithm 1 on the scaled problem
  with the solution mapped back.
* ``reference_solution``: an accurate optimum (ADMM to 1e-10 then an exact
  equality-constrained KKT solve on the identified active set), used as the
  "converged answer" that GPU results are compared to.
* ``brute_force_qp``: enumerates every active set of a small QP; it is an
  independent solver used only to pin the oracle.

Readings of points the paper leaves open:
  R1 the layer state after k layers is (x_k, z_k, lam'_k) where lam' is the
     multiplier *before* the lam-step of the next layer; the multiplier of
     standard ADMM is lam_std = lam' + rho (A x - z).
  R2 residuals, the rho rule and the returned dual use lam_std.
  R3 at a check the convergence test comes first; the rho rule runs only if
     the test fails.  When the rho index changes, lam' is rebased so that the
     next layer starts standard ADMM with the new rho from (x, z, lam_std):
     lam' <- lam_std - rho_new (A x - z).
  R4 rho-rule guards: if r_p or r_d is zero or the estimate is not finite the
     rho index is kept; nearest entry by |log rho - log rho_i|, ties to the
     lower index.
  R5 equality rows are rows with l_i == u_i; their rho is eq_scale (1000)
     times the inequality rho (Sec. II-B).
  R6 eps_prim = eps_abs + eps_rel max(|Ax|, |z|),
     eps_dual = eps_abs + eps_rel max(|Px|, |A^T lam|, |q|) (inf-norms).
  R7 checks at iterations i with i % check_interval == 0 (i counts from 1).
  R8 cold start v0 = 0; warm start x = x_w, lam = lam_w, z = A x_w.
  R9 the 1e-4 floors of Eq. rho_update are kept as printed.
  R10 scaling (details unstated in the paper): Ruiz iterations on the
     infinity norms of the columns of the KKT matrix [[P, A^T], [A, 0]]
     (norms below 1e-4 are left unscaled, above 1e4 clipped), each followed by
     a cost scale 1 / max(mean column norm of P, |q|_inf); the scaled problem
     is min 1/2 xb^T (c D P D) xb + (c D q)^T xb, E l <= (E A D) xb <= E u, with
     x = D xb, z = zb / E, lam = E lamb / c; the stop test and the penalty rule
     use the residuals and norms of the original problem at the mapped-back
     iterate (OSQP's default, unscaled termination).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "rho_vector", "kkt_matrix", "kkt_inverse", "relu_layer_weights", "relu_layer_step",
    "admm_step_standard", "admm_step_modified", "residuals", "rho_estimate",
    "nearest_rho_index", "solve", "SolveResult", "reference_solution", "brute_force_qp",
    "kkt_violation", "std_multiplier", "layer_iterates", "admm_iterates", "ruiz_scaling", "solve_scaled",
]


# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------

def rho_vector(l: np.ndarray, u: np.ndarray, rho: float, eq_scale: float = 1e3) -> np.ndarray:
    """Diagonal of the penalty matrix rho (Sec. II-B): equality rows get eq_scale * rho (R5)."""
    l = np.asarray(l, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    r = np.full(l.shape, float(rho))
    r[l == u] *= eq_scale
    return r


def kkt_matrix(P: np.ndarray, A: np.ndarray, sigma: float, rho_vec: np.ndarray) -> np.ndarray:
    """H + sigma I + G^T rho G, the matrix inverted in Eq. Xbar_update."""
    n = P.shape[0]
    return P + sigma * np.eye(n) + A.T @ (rho_vec[:, None] * A)


def kkt_inverse(P, A, sigma, rho_vec):
    """D = (H + sigma I + G^T rho G)^{-1} (Sec. III-A), via a Cholesky factor and two solves."""
    K = kkt_matrix(P, A, sigma, rho_vec)
    L = np.linalg.cholesky(K)
    n = K.shape[0]
    Y = np.linalg.solve(L, np.eye(n))
    D = np.linalg.solve(L.T, Y)
    return 0.5 * (D + D.T), L


def relu_layer_weights(P, A, sigma, rho_vec):
    """W (N_s x N_s) and the bias operator Bop (b = Bop q) of Eq. gpu_update.

    Block rows for [y; z; lam] exactly as printed in Sec. III-A:
      [ D(sI - G^T r G)       2 D G^T r       -D G^T            ]
      [ G D(sI - G^T r G)+G   2 G D G^T r - I  -G D G^T + r^{-1} ]
      [ r G                   -r               I                 ]
    and b = [-D; -G D; 0] g.
    """
    n = P.shape[0]
    m = A.shape[0]
    D, _ = kkt_inverse(P, A, sigma, rho_vec)
    R = np.diag(rho_vec)
    Rinv = np.diag(1.0 / rho_vec)
    In = np.eye(n)
    Im = np.eye(m)
    T = sigma * In - A.T @ R @ A
    W = np.zeros((n + 2 * m, n + 2 * m))
    W[:n, :n] = D @ T
    W[:n, n:n + m] = 2.0 * D @ A.T @ R
    W[:n, n + m:] = -D @ A.T
    W[n:n + m, :n] = A @ D @ T + A
    W[n:n + m, n:n + m] = 2.0 * A @ D @ A.T @ R - Im
    W[n:n + m, n + m:] = -A @ D @ A.T + Rinv
    W[n + m:, :n] = R @ A
    W[n + m:, n:n + m] = -R
    W[n + m:, n + m:] = Im
    Bop = np.zeros((n + 2 * m, n))
    Bop[:n] = -D
    Bop[n:n + m] = -A @ D
    return W, Bop


def relu_layer_step(W, b, v, n, m, l, u):
    """v+ = clamp(W v + b, c~, d~): only the z rows are clamped (Eq. gpu_update)."""
    w = W @ v + b
    w[n:n + m] = np.minimum(np.maximum(w[n:n + m], l), u)
    return w


def admm_step_standard(P, q, A, l, u, sigma, rho_vec, x, z, lam, mu):
    """One standard ADMM step, Eqs. Xbar_update, x_update, z_update, mu_update_gen,
    lambda_update_gen (Sec. II-B).  Returns (x+, z+, lam+, mu+, xbar+)."""
    K = kkt_matrix(P, A, sigma, rho_vec)
    rhs = -q + sigma * x - mu + A.T @ (rho_vec * z - lam)
    xbar = np.linalg.solve(K, rhs)
    x_new = xbar + mu / sigma
    z_new = np.minimum(np.maximum(A @ xbar + lam / rho_vec, l), u)
    mu_new = mu + sigma * (xbar - x_new)
    lam_new = lam + rho_vec * (A @ x_new - z_new)
    return x_new, z_new, lam_new, mu_new, xbar


def admm_step_modified(P, q, A, l, u, sigma, rho_vec, x, z, lam):
    """The reordered step of Sec. III-A: Eq. basic_lambda_update first, then
    Eq. basic_y_update, then Eq. clamp.  Returns (x+, z+, lam+)."""
    lam_new = lam + rho_vec * (A @ x - z)
    K = kkt_matrix(P, A, sigma, rho_vec)
    x_new = np.linalg.solve(K, -q + sigma * x + A.T @ (rho_vec * z - lam_new))
    z_new = np.minimum(np.maximum(A @ x_new + lam_new / rho_vec, l), u)
    return x_new, z_new, lam_new


def std_multiplier(A, x, z, lam_layer, rho_vec):
    """lam_std = lam' + rho (A x - z): the standard-ADMM multiplier of a layer state (R1)."""
    return lam_layer + rho_vec * (A @ x - z)


def residuals(P, q, A, x, z, lam):
    """Eqs. primal and dual (inf-norms) plus the norms Eq. rho_update needs.

    Returns dict(r_prim, r_dual, Ax, Px, Atl, q) with the last four as inf-norms.
    """
    Ax = A @ x
    Px = P @ x
    Atl = A.T @ lam
    r_prim = np.max(np.abs(Ax - z)) if A.shape[0] else 0.0
    r_dual = np.max(np.abs(Px + q + Atl))
    return dict(r_prim=float(r_prim), r_dual=float(r_dual),
                Ax=float(np.max(np.abs(Ax))) if A.shape[0] else 0.0,
                z=float(np.max(np.abs(z))) if A.shape[0] else 0.0,
                Px=float(np.max(np.abs(Px))), Atl=float(np.max(np.abs(Atl))),
                q=float(np.max(np.abs(q))))


def rho_estimate(rho: float, res: dict) -> float:
    """Nominal penalty of Eq. rho_update (inf-norms, 1e-4 floors as printed)."""
    num = res["r_prim"] * max(res["Px"], res["Atl"], res["q"], 1e-4)
    den = res["r_dual"] * max(res["Ax"], res["z"], 1e-4)
    if den == 0.0 or num == 0.0:
        return float("nan")
    return rho * math.sqrt(num / den)


def nearest_rho_index(bank, rho_nominal: float, current: int) -> int:
    """Closest bank entry in log distance (Sec. III-C); guards of reading R4."""
    if not (rho_nominal > 0.0) or not math.isfinite(rho_nominal):
        return current
    lr = math.log(rho_nominal)
    best, bestd = current, float("inf")
    for i, r in enumerate(bank):
        d = abs(lr - math.log(r))
        if d < bestd:
            best, bestd = i, d
    return best


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------

@dataclass
class SolveResult:
    x: np.ndarray
    z: np.ndarray
    lam: np.ndarray          # lam_std (R2)
    iters: int
    status: str              # "solved" | "max_iter"
    rho_index: int
    r_prim: float
    r_dual: float
    rho_history: list


def solve(P, q, A, l, u, sigma=1e-6, rho_bank=(0.1, 1.0, 10.0), rho0=0.1, eps_abs=1e-3,
          eps_rel=0.0, check_interval=25, max_iter=4000, x_warm=None, lam_warm=None,
          rho_index_warm=None, eq_scale=1e3, adaptive_rho=True, weights=None, residual_fn=None):
    """Algorithm 1 (Sec. III-B) in FP64 with the readings R1-R9.

    Offline: W and b operator for every rho in the bank (Eq. gpu_update).
    Online: v <- clamp(W v + b) each iteration; every check_interval
    iterations: residuals (Eqs. primal, dual), convergence test, then the
    penalty rule (Eq. rho_update) and the nearest bank entry.
    ``weights`` may pass a precomputed list of (W, Bop) per bank entry;
    ``residual_fn(x, z, lam)`` replaces the residuals of this problem (the
    scaled solve measures them on the original problem, R10).
    """
    P = np.asarray(P, np.float64)
    q = np.asarray(q, np.float64)
    A = np.asarray(A, np.float64)
    l = np.asarray(l, np.float64)
    u = np.asarray(u, np.float64)
    n = P.shape[0]
    m = A.shape[0]
    if weights is None:
        weights = [relu_layer_weights(P, A, sigma, rho_vector(l, u, r, eq_scale)) for r in rho_bank]
    rvecs = [rho_vector(l, u, r, eq_scale) for r in rho_bank]
    if rho_index_warm is not None:
        ri = int(rho_index_warm)
    else:
        ri = nearest_rho_index(rho_bank, rho0, 0)
    # initial state (R8)
    if x_warm is None:
        x = np.zeros(n)
        z = np.zeros(m)
        lam_l = np.zeros(m)
    else:
        x = np.asarray(x_warm, np.float64).copy()
        z = A @ x
        lam_std0 = np.zeros(m) if lam_warm is None else np.asarray(lam_warm, np.float64)
        lam_l = lam_std0 - rvecs[ri] * (A @ x - z)      # = lam_std0 since A x = z
    v = np.concatenate([x, z, lam_l])
    W, Bop = weights[ri]
    b = Bop @ q
    history = [ri]
    res = None
    for it in range(1, max_iter + 1):
        v = relu_layer_step(W, b, v, n, m, l, u)
        if check_interval > 0 and it % check_interval == 0:
            x, z, lam_l = v[:n], v[n:n + m], v[n + m:]
            lam = std_multiplier(A, x, z, lam_l, rvecs[ri])
            res = residuals(P, q, A, x, z, lam) if residual_fn is None else residual_fn(x, z, lam)
            eps_p = eps_abs + eps_rel * max(res["Ax"], res["z"])
            eps_d = eps_abs + eps_rel * max(res["Px"], res["Atl"], res["q"])
            if res["r_prim"] <= eps_p and res["r_dual"] <= eps_d:
                return SolveResult(x.copy(), z.copy(), lam, it, "solved", ri, res["r_prim"],
                                   res["r_dual"], history)
            if adaptive_rho:
                nri = nearest_rho_index(rho_bank, rho_estimate(rho_bank[ri], res), ri)
                if nri != ri:
                    ri = nri
                    W, Bop = weights[ri]
                    b = Bop @ q
                    lam_l = lam - rvecs[ri] * (A @ x - z)       # rebase (R3)
                    v = np.concatenate([x, z, lam_l])
                    history.append(ri)
    x, z, lam_l = v[:n], v[n:n + m], v[n + m:]
    lam = std_multiplier(A, x, z, lam_l, rvecs[ri])
    res = residuals(P, q, A, x, z, lam) if residual_fn is None else residual_fn(x, z, lam)
    return SolveResult(x.copy(), z.copy(), lam, max_iter, "max_iter", ri, res["r_prim"],
                       res["r_dual"], history)


def ruiz_scaling(P, A, q, iters=10, norm_min=1e-4, norm_max=1e4):
    """Modified Ruiz equilibration (Algorithm 1 "Scale problem", Sec. III-D), reading R10.

    Each iteration divides every column of the KKT matrix K = [[P, A^T], [A, 0]]
    (and, symmetrically, every row) by the square root of its infinity norm,
    which drives all those norms towards 1, and then rescales the cost so that
    max(mean column norm of P, |q|_inf) = 1.  Returns (D, E, c, Pb, Ab, qb) with
    Pb = c D P D, Ab = E A D, qb = c D q (D, E as vectors)."""
    P = np.asarray(P, np.float64)
    A = np.asarray(A, np.float64)
    q = np.asarray(q, np.float64)
    n, m = P.shape[0], A.shape[0]
    D, E, c = np.ones(n), np.ones(m), 1.0
    Pb, Ab, qb = P.copy(), A.copy(), q.copy()

    def inv_sqrt(norms):
        norms = np.where(norms < norm_min, 1.0, np.minimum(norms, norm_max))
        return 1.0 / np.sqrt(norms)

    for _ in range(iters):
        # column j < n of K: column j of P and of A; column n + i: row i of A
        col_x = np.abs(Pb).max(axis=0)
        if m:
            col_x = np.maximum(col_x, np.abs(Ab).max(axis=0))
        col_z = np.abs(Ab).max(axis=1) if m else np.zeros(0)
        dx, dz = inv_sqrt(col_x), inv_sqrt(col_z)
        Pb = dx[:, None] * Pb * dx[None, :]
        Ab = dz[:, None] * Ab * dx[None, :]
        qb = dx * qb
        D, E = D * dx, E * dz
        cost = max(np.abs(Pb).max(axis=0).mean(), np.abs(qb).max() if n else 0.0)
        cost = 1.0 if cost < norm_min else min(cost, norm_max)
        gamma = 1.0 / cost
        Pb, qb, c = gamma * Pb, gamma * qb, gamma * c
    return D, E, c, Pb, Ab, qb


def solve_scaled(P, q, A, l, u, scaling_iters=10, x_warm=None, lam_warm=None, scaling=None, **kw):
    """Algorithm 1 with its offline "Scale problem" step (reading R10): solve the
    equilibrated problem and map x, z, lam back.  The stop test and the penalty
    rule use the residuals of the original problem at the mapped-back iterate,
    which are also the ones returned.

    The scaling step is offline: a parametric problem keeps the (D, E, c) that
    ruiz_scaling found for the q it was set up with while q, l, u change
    online.  `scaling` = (D, E, c) applies such a fixed scaling; None computes it
    from this q."""
    P = np.asarray(P, np.float64)
    A = np.asarray(A, np.float64)
    q = np.asarray(q, np.float64)
    if scaling is None:
        D, E, c, Pb, Ab, qb = ruiz_scaling(P, A, q, scaling_iters)
    else:
        D, E, c = (np.asarray(scaling[0], np.float64), np.asarray(scaling[1], np.float64), float(scaling[2]))
        Pb = c * D[:, None] * P * D[None, :]
        Ab = E[:, None] * A * D[None, :]
        qb = c * D * q
    lb = E * np.asarray(l, np.float64)
    ub = E * np.asarray(u, np.float64)
    xw = None if x_warm is None else np.asarray(x_warm, np.float64) / D
    lw = None if lam_warm is None else c * np.asarray(lam_warm, np.float64) / E

    def original(xb, zb, lamb):
        return residuals(P, q, A, D * xb, zb / E, E * lamb / c)

    r = solve(Pb, qb, Ab, lb, ub, x_warm=xw, lam_warm=lw, residual_fn=original, **kw)
    return SolveResult(D * r.x, r.z / E, E * r.lam / c, r.iters, r.status, r.rho_index, r.r_prim, r.r_dual,
                       r.rho_history)


def layer_iterates(P, q, A, l, u, sigma, rho, iters, x0=None, z0=None, lam0=None, eq_scale=1e3):
    """Fixed-rho layer iterates v_k = clamp(W v_{k-1} + b), k = 1..iters (list of arrays)."""
    n = P.shape[0]
    m = A.shape[0]
    rv = rho_vector(l, u, rho, eq_scale)
    W, Bop = relu_layer_weights(P, A, sigma, rv)
    b = Bop @ q
    v = np.concatenate([np.zeros(n) if x0 is None else x0, np.zeros(m) if z0 is None else z0,
                        np.zeros(m) if lam0 is None else lam0])
    out = []
    for _ in range(iters):
        v = relu_layer_step(W, b, v, n, m, l, u)
        out.append(v.copy())
    return out


def admm_iterates(P, q, A, l, u, sigma, rho, iters, x0=None, z0=None, lam0=None, eq_scale=1e3):
    """Standard ADMM iterates (x_k, z_k, lam_k), k = 1..iters, with mu carried (Sec. II-B)."""
    n = P.shape[0]
    m = A.shape[0]
    rv = rho_vector(l, u, rho, eq_scale)
    x = np.zeros(n) if x0 is None else x0.copy()
    z = np.zeros(m) if z0 is None else z0.copy()
    lam = np.zeros(m) if lam0 is None else lam0.copy()
    mu = np.zeros(n)
    out = []
    for _ in range(iters):
        x, z, lam, mu, _ = admm_step_standard(P, q, A, l, u, sigma, rv, x, z, lam, mu)
        out.append((x.copy(), z.copy(), lam.copy()))
    return out


# ---------------------------------------------------------------------------
# accurate optimum and independent checks
# ---------------------------------------------------------------------------

def kkt_violation(P, q, A, l, u, x, lam):
    """Max of stationarity, primal infeasibility and complementarity/sign violations."""
    Ax = A @ x
    stat = np.max(np.abs(P @ x + q + A.T @ lam)) if x.size else 0.0
    if A.shape[0] == 0:
        return float(stat)
    feas = np.max(np.maximum(np.maximum(l - Ax, Ax - u), 0.0))
    # lam > 0 only where Ax = u, lam < 0 only where Ax = l
    pos = np.maximum(lam, 0.0)
    neg = np.minimum(lam, 0.0)
    # a finite bound: |lam| (capped at 1) times the distance to the bound; an
    # infinite bound can never be active, so there the multiplier itself must
    # vanish and its size is the violation
    fu, fl = np.isfinite(u), np.isfinite(l)
    up_gap = np.abs(np.where(fu, u, 0.0) - Ax)
    lo_gap = np.abs(Ax - np.where(fl, l, 0.0))
    comp_u = np.max(np.where(fu, np.minimum(pos, 1.0) * up_gap, pos))
    comp_l = np.max(np.where(fl, np.minimum(-neg, 1.0) * lo_gap, -neg))
    return float(max(stat, feas, comp_u, comp_l))


def _equality_kkt(P, q, A, l, u, up, lo):
    """Solve min 1/2 x'Px + q'x s.t. A_i x = u_i (i in up), A_i x = l_i (i in lo)."""
    n = P.shape[0]
    act = np.concatenate([np.nonzero(up)[0], np.nonzero(lo & ~up)[0]])
    rhs_b = np.concatenate([u[up], l[lo & ~up]])
    k = act.size
    M = np.zeros((n + k, n + k))
    M[:n, :n] = P
    M[:n, n:] = A[act].T
    M[n:, :n] = A[act]
    r = np.concatenate([-q, rhs_b])
    sol, *_ = np.linalg.lstsq(M, r, rcond=None)
    x = sol[:n]
    lam = np.zeros(A.shape[0])
    lam[act] = sol[n:]
    return x, lam


def reference_solution(P, q, A, l, u, sigma=1e-6, rho_bank=(0.1, 1.0, 10.0), tol=1e-10,
                       max_iter=200000, polish=True):
    """Accurate optimum: Algorithm 1 to tol, then an exact KKT solve on the active set.

    Rows whose multiplier sign or whose bound distance marks them active are
    held at their bound; the polished point is kept only if its KKT violation
    is smaller than the ADMM point's.
    """
    r = solve(P, q, A, l, u, sigma=sigma, rho_bank=rho_bank, eps_abs=tol, eps_rel=0.0,
              max_iter=max_iter)
    x, z, lam = r.x, r.z, r.lam
    best = (kkt_violation(P, q, A, l, u, x, lam), x, z, lam)
    if polish and A.shape[0]:
        Ax = A @ x
        scale = 1.0 + np.abs(Ax)
        up = np.isfinite(u) & ((lam > 0) | (np.abs(u - Ax) <= 1e-7 * scale)) & (lam >= 0)
        lo = np.isfinite(l) & ((lam < 0) | (np.abs(Ax - l) <= 1e-7 * scale)) & (lam <= 0) & ~up
        eq = (l == u) & np.isfinite(l)
        up = up | eq
        xp, lp = _equality_kkt(P, q, A, l, u, up, lo)
        vp = kkt_violation(P, q, A, l, u, xp, lp)
        if vp < best[0]:
            best = (vp, xp, np.minimum(np.maximum(A @ xp, l), u), lp)
    return dict(x=best[1], z=best[2], lam=best[3], kkt=best[0], admm=r)


def brute_force_qp(P, q, A, l, u, tol=1e-9):
    """Exact optimum of a small QP (m <= 10) by enumerating all 3^m active sets.

    Each row is free, held at l_i, or held at u_i; the equality-constrained
    KKT system is solved for every assignment and the assignment whose point
    is primal feasible with multipliers of the right sign is returned.  This
    is an independent route to the optimum (no ADMM involved).
    """
    n = P.shape[0]
    m = A.shape[0]
    if m > 10:
        raise ValueError("brute force is for m <= 10")
    best = None
    for code in range(3 ** m):
        c = code
        up = np.zeros(m, bool)
        lo = np.zeros(m, bool)
        ok = True
        for i in range(m):
            t = c % 3
            c //= 3
            if t == 1:
                if not np.isfinite(l[i]):
                    ok = False
                    break
                lo[i] = True
            elif t == 2:
                if not np.isfinite(u[i]) or l[i] == u[i]:
                    ok = False
                    break
                up[i] = True
        if not ok:
            continue
        if np.count_nonzero(up | lo) > n:
            continue
        x, lam = _equality_kkt(P, q, A, l, u, up, lo)
        Ax = A @ x
        if np.any(Ax < l - tol * (1 + np.abs(l))) or np.any(Ax > u + tol * (1 + np.abs(u))):
            continue
        if np.any(lam[up] < -tol) or np.any(lam[lo & (l != u)] > tol):
            continue
        if np.max(np.abs(P @ x + q + A.T @ lam)) > 1e-7 * (1 + np.max(np.abs(q))):
            continue
        obj = 0.5 * x @ P @ x + q @ x
        if best is None or obj < best[0] - 1e-12:
            best = (obj, x, lam)
    if best is None:
        raise RuntimeError("no feasible active set")
    return dict(x=best[1], lam=best[2], obj=best[0])
