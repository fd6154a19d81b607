"""Pins of the condensing oracle (Sec. IV), independent of the GPU path.

* the literal S, M of Sec. IV reproduce the trajectory of a direct simulation
  of x+ = A x + B u with u_k = -K x_k + du_k (random du, x0): brute force;
* the unconstrained optimum of the condensed QP gives the controls of the
  finite-horizon Riccati recursion (textbook closed form);
* the DARE gain satisfies the Riccati equation and stabilises A - B K;
* the oracle agrees with the workload generator's recurrence-based condensing
  (a third, independently written construction).
"""
import numpy as np
import pytest

from oracle import condense_oracle as C
from workloads import mpc


def plant(seed, nx, nu):
    rng = mpc.rng_for(seed, 0)
    A, B = mpc.random_dynamics(rng, nx, nu, 1.05)
    return A, B, np.eye(nx), 0.1 * np.eye(nu)


def simulate(A, B, K, x0, du):
    nx, nu = B.shape
    y = []
    x = x0
    for k in range(len(du) // nu):
        u = -K @ x + du[k * nu:(k + 1) * nu]
        x = A @ x + B @ u
        y += [u, x]
    return np.concatenate(y)


@pytest.mark.parametrize("nx,nu,N,seed,pre", [(6, 2, 10, 0, True), (9, 3, 7, 4, False), (5, 5, 12, 9, True)])
def test_prediction_matrices_match_simulation(nx, nu, N, seed, pre):
    A, B, Q, R = plant(seed, nx, nu)
    K = C.lqr_gain_dare(A, B, Q, R) if pre else np.zeros((nu, nx))
    S, M = C.prediction_matrices(A, B, K, N)
    rng = mpc.rng_for(seed, 7)
    x0, du = rng.standard_normal(nx), rng.standard_normal(N * nu)
    y = simulate(A, B, K, x0, du)
    assert np.max(np.abs(S @ du + M @ x0 - y)) <= 1e-11 * (1 + np.max(np.abs(y)))


def riccati_controls(A, B, Q, R, QN, N, x0):
    """Finite-horizon LQR by the backward Riccati recursion, applied forward from x0."""
    X = QN
    gains = []
    for _ in range(N):
        Kk = np.linalg.solve(R + B.T @ X @ B, B.T @ X @ A)
        X = Q + A.T @ X @ (A - B @ Kk)
        gains.append(Kk)
    gains.reverse()
    us, x = [], x0
    for Kk in gains:
        u = -Kk @ x
        us.append(u)
        x = A @ x + B @ u
    return np.concatenate(us)


@pytest.mark.parametrize("nx,nu,N,seed", [(6, 2, 10, 0), (12, 4, 20, 40)])
def test_unconstrained_optimum_is_finite_horizon_lqr(nx, nu, N, seed):
    A, B, Q, R = plant(seed, nx, nu)
    QN = 2.0 * Q
    c = C.condense_mpc(A, B, Q, R, N, QN=QN)
    x0 = mpc.rng_for(seed, 5).standard_normal(nx)
    du = -np.linalg.solve(c["P"], c["F"] @ x0)
    u = c["A"] @ du + c["E"] @ x0          # the control rows are u_k
    u_ric = riccati_controls(A, B, Q, R, QN, N, x0)
    assert np.max(np.abs(u - u_ric)) <= 1e-9 * (1 + np.max(np.abs(u_ric)))


def test_dare_gain_is_the_stabilising_fixed_point():
    A, B, Q, R = plant(3, 10, 3)
    K = C.lqr_gain_dare(A, B, Q, R)
    assert np.max(np.abs(np.linalg.eigvals(A - B @ K))) < 1.0
    # X from the gain: X = Q + K'RK + (A-BK)' X (A-BK) solved as a Lyapunov equation
    import scipy.linalg
    Ab = A - B @ K
    X = scipy.linalg.solve_discrete_lyapunov(Ab.T, Q + K.T @ R @ K)
    assert np.max(np.abs(K - np.linalg.solve(R + B.T @ X @ B, B.T @ X @ A))) <= 1e-9


@pytest.mark.parametrize("nx,nu,N,seed", [(6, 2, 10, 0), (12, 4, 40, 2)])
def test_oracle_matches_generator_recurrence(nx, nu, N, seed):
    A, B, Q, R = plant(seed, nx, nu)
    P, Acon, F, E, l0, u0, K = mpc.condensed_mpc(A, B, Q, R, Q, N, 1.5)
    c = C.condense_mpc(A, B, Q, R, N, umin=-1.5 * np.ones(nu), umax=1.5 * np.ones(nu))
    assert np.max(np.abs(c["K"] - K)) <= 1e-8 * (1 + np.max(np.abs(K)))
    for a, b in ((c["P"], P), (c["A"], Acon), (c["F"], F), (c["E"], E)):
        assert np.max(np.abs(a - b)) <= 1e-8 * (1 + np.max(np.abs(b)))
    assert np.array_equal(c["l0"], l0) and np.array_equal(c["u0"], u0)


def test_state_limit_rows_are_the_predicted_states():
    A, B, Q, R = plant(1, 6, 2)
    N = 8
    c = C.condense_mpc(A, B, Q, R, N, umin=-np.ones(2), umax=np.ones(2), xmin=-5 * np.ones(6), xmax=None)
    assert c["A"].shape == (N * 8, N * 2) and np.all(np.isposinf(c["u0"][N * 2:]))
    rng = mpc.rng_for(1, 3)
    x0, du = rng.standard_normal(6), rng.standard_normal(N * 2)
    y = simulate(A, B, c["K"], x0, du)
    xs = np.concatenate([y[k * 8 + 2:(k + 1) * 8] for k in range(N)])
    assert np.max(np.abs(c["A"][N * 2:] @ du + c["E"][N * 2:] @ x0 - xs)) <= 1e-11 * (1 + np.max(np.abs(xs)))
