"""FP64 CPU oracle of the dense MPC condensing (Sec. IV) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module; the GPU library never calls it and
shares no code with it.  It writes the paper's definitions out literally:

* the infinite-horizon LQR gain K from the discrete algebraic Riccati
  equation (SciPy's DARE solver as the library step), K = (R + B'XB)^{-1} B'XA;
* Abar = A - B K, and the stacked trajectory y = [u_0; x_1; u_1; ...; u_{N-1};
  x_N] = S ytilde + M x0 with S and M assembled block by block exactly as
  printed in Sec. IV (u_k rows: -K Abar^{k-1-j} B left of the diagonal
  identity; x_{k+1} rows: Abar^{k-j} B; M rows -K Abar^k and Abar^{k+1});
* H = blkdiag(R, Q, R, Q, ..., R, Q_N), Hbar = S'HS, gbar = S'HM x0 (F = S'HM),
  Gbar = G S and cbar, dbar = c, d - G M x0, with G selecting the limited
  rows of y (every u_k, then every x_{k+1} when state limits are given).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

__all__ = ["lqr_gain_dare", "prediction_matrices", "condense_mpc"]


def lqr_gain_dare(A, B, Q, R):
    """Infinite-horizon discrete LQR gain from the Riccati equation's stabilizing solution."""
    X = scipy.linalg.solve_discrete_are(A, B, Q, R)
    return np.linalg.solve(R + B.T @ X @ B, B.T @ X @ A)


def prediction_matrices(A, B, K, N):
    """S ((N (nu + nx)) x N nu) and M ((N (nu + nx)) x nx) of Sec. IV, rows ordered
    u_0, x_1, u_1, x_2, ..., u_{N-1}, x_N."""
    nx, nu = B.shape
    Abar = A - B @ K
    powers = [np.eye(nx)]
    for _ in range(N):
        powers.append(Abar @ powers[-1])
    stage = nu + nx
    S = np.zeros((N * stage, N * nu))
    M = np.zeros((N * stage, nx))
    for k in range(N):
        ru = k * stage          # rows of u_k
        rx = ru + nu            # rows of x_{k+1}
        for j in range(N):
            cols = slice(j * nu, (j + 1) * nu)
            if j < k:
                S[ru:ru + nu, cols] = -K @ powers[k - 1 - j] @ B
            elif j == k:
                S[ru:ru + nu, cols] = np.eye(nu)
            if j <= k:
                S[rx:rx + nx, cols] = powers[k - j] @ B
        M[ru:ru + nu] = -K @ powers[k]
        M[rx:rx + nx] = powers[k + 1]
    return S, M


def condense_mpc(A, B, Q, R, N, QN=None, umin=None, umax=None, xmin=None, xmax=None, K=None, precondition=True):
    """dict(P, A, F, E, l0, u0, K) of the condensed QP (rows: control limits of every
    stage, then state limits of every stage when xmin or xmax is given)."""
    A, B, Q, R = (np.asarray(v, np.float64) for v in (A, B, Q, R))
    nx, nu = B.shape
    QN = Q if QN is None else np.asarray(QN, np.float64)
    if K is None:
        K = lqr_gain_dare(A, B, Q, R) if precondition else np.zeros((nu, nx))
    K = np.asarray(K, np.float64)
    S, M = prediction_matrices(A, B, K, N)
    # H = blkdiag(R, Q, ..., R, Q_N) applied to S and M one diagonal block at a time
    stage = nu + nx
    HS, HM = np.empty_like(S), np.empty_like(M)
    for k in range(N):
        ru, rx = k * stage, k * stage + nu
        W = QN if k == N - 1 else Q
        HS[ru:rx], HM[ru:rx] = R @ S[ru:rx], R @ M[ru:rx]
        HS[rx:ru + stage], HM[rx:ru + stage] = W @ S[rx:ru + stage], W @ M[rx:ru + stage]
    P = S.T @ HS
    P = 0.5 * (P + P.T)
    F = S.T @ HM
    rows_u = np.concatenate([np.arange(k * stage, k * stage + nu) for k in range(N)])
    rows = [rows_u]
    lo = [np.tile(-np.inf * np.ones(nu) if umin is None else np.asarray(umin, np.float64), N)]
    hi = [np.tile(np.inf * np.ones(nu) if umax is None else np.asarray(umax, np.float64), N)]
    if xmin is not None or xmax is not None:
        rows.append(np.concatenate([np.arange(k * stage + nu, (k + 1) * stage) for k in range(N)]))
        lo.append(np.tile(-np.inf * np.ones(nx) if xmin is None else np.asarray(xmin, np.float64), N))
        hi.append(np.tile(np.inf * np.ones(nx) if xmax is None else np.asarray(xmax, np.float64), N))
    rows = np.concatenate(rows)
    return {"P": P, "A": S[rows], "F": F, "E": M[rows], "l0": np.concatenate(lo), "u0": np.concatenate(hi),
            "K": K}
