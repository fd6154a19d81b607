"""Pins for the seeded MPC workload generator (shared by the solver and the oracle).

Without extra constraints the MPC problem of Sec. II-C (Eq. mpc_def) is an LQR
problem solved by a Riccati recursion; the condensed, LQR-preconditioned QP of
Sec. IV must give the same controls.  Condensing with and without the
preconditioner must also agree, since u_k = -K x_k + du_k is only a change of
variables.
"""
import numpy as np
import pytest

from workloads import mpc


def riccati_controls(A, B, Q, R, QN, N, x0):
    X = QN.copy()
    gains = []
    for _ in range(N):
        Kk = np.linalg.solve(R + B.T @ X @ B, B.T @ X @ A)
        X = Q + A.T @ X @ (A - B @ Kk)
        gains.append(Kk)
    gains = gains[::-1]
    x = x0.copy()
    us = []
    for k in range(N):
        u = -gains[k] @ x
        us.append(u)
        x = A @ x + B @ u
    return np.concatenate(us)


def condensed_controls(A, B, K, N, F, P, x0):
    yt = -np.linalg.solve(P, F @ x0)
    nu = B.shape[1]
    Abar = A - B @ K
    x = x0.copy()
    us = []
    for k in range(N):
        du = yt[k * nu:(k + 1) * nu]
        us.append(-K @ x + du)
        x = Abar @ x + B @ du
    return np.concatenate(us)


@pytest.mark.parametrize("nx,nu,N,seed", [(6, 2, 10, 0), (9, 3, 25, 7), (12, 4, 20, 40)])
def test_unconstrained_condensed_equals_riccati(nx, nu, N, seed):
    rng = mpc.rng_for(seed, 0)
    A, B = mpc.random_dynamics(rng, nx, nu, 1.05)
    Q, R = np.eye(nx), 0.1 * np.eye(nu)
    P, Acon, F, E, l0, u0, K = mpc.condensed_mpc(A, B, Q, R, Q, N, 1.0)
    x0 = mpc.rng_for(seed, 5).standard_normal(nx)
    u_ric = riccati_controls(A, B, Q, R, Q, N, x0)
    u_con = condensed_controls(A, B, K, N, F, P, x0)
    assert np.max(np.abs(u_con - u_ric)) <= 1e-10 * (1 + np.max(np.abs(u_ric)))
    # the constraint rows are exactly the applied controls: A_con yt + E x0 = u
    yt = -np.linalg.solve(P, F @ x0)
    assert np.max(np.abs(Acon @ yt + E @ x0 - u_con)) <= 1e-12 * (1 + np.max(np.abs(u_con)))


def test_preconditioning_is_a_change_of_variables():
    rng = mpc.rng_for(3, 0)
    A, B = mpc.random_dynamics(rng, 8, 3, 1.05)
    Q, R = np.eye(8), 0.1 * np.eye(3)
    x0 = mpc.rng_for(3, 1).standard_normal(8)
    P1, A1, F1, E1, *_ , K1 = mpc.condensed_mpc(A, B, Q, R, Q, 12, 1.0, precondition=True)
    P0, A0, F0, E0, *_ , K0 = mpc.condensed_mpc(A, B, Q, R, Q, 12, 1.0, precondition=False)
    assert np.all(K0 == 0)
    u1 = condensed_controls(A, B, K1, 12, F1, P1, x0)
    u0 = condensed_controls(A, B, K0, 12, F0, P0, x0)
    assert np.max(np.abs(u1 - u0)) <= 1e-9 * (1 + np.max(np.abs(u0)))
    # the preconditioner improves conditioning (the reason Sec. IV gives for it)
    assert np.linalg.cond(P1) < np.linalg.cond(P0)


def test_lqr_gain_solves_dare():
    rng = mpc.rng_for(9, 0)
    A, B = mpc.random_dynamics(rng, 10, 4, 1.05)
    Q, R = np.eye(10), 0.1 * np.eye(4)
    K = mpc.lqr_gain(A, B, Q, R)
    assert np.max(np.abs(np.linalg.eigvals(A - B @ K))) < 1.0


@pytest.mark.parametrize("name,n,m", [("small", 20, 20), ("sweep4", 160, 160), ("family0", 80, 80)])
def test_workload_shapes_and_pd(name, n, m):
    pq, X0, s = mpc.workload(name, 4)
    assert pq.P.shape == (n, n) and pq.A.shape == (m, n)
    assert np.allclose(pq.P, pq.P.T)
    assert np.min(np.linalg.eigvalsh(pq.P)) > 0
    assert X0.shape == (4, pq.nx)
    # seeded: a second call draws the same data
    pq2, X02, s2 = mpc.workload(name, 4)
    assert np.array_equal(pq.P, pq2.P) and np.array_equal(X0, X02) and s == s2


def test_x0_scale_rule_hits_its_ratio():
    pq = mpc.small_mpc()
    s = mpc.x0_scale(pq, 4.0)
    X = mpc.rng_for(pq.meta["workload_id"], 9).standard_normal((64, pq.nx))
    r = np.max(np.abs(s * X @ pq.E.T) / pq.u0[None, :], axis=1)
    assert np.median(r) == pytest.approx(4.0)


def test_humanoid_workload_structure():
    pq = mpc.humanoid_mpc()
    assert (pq.n, pq.m) == (600, 1000)
    assert np.all(np.isinf(pq.l0[600:])) and np.all((pq.u0[600:] >= 1) & (pq.u0[600:] <= 2))
    assert np.all(pq.E[600:] == 0)
    # block-diagonal dynamics with unit spectral radius per 10x10 block
    A = pq.Ad
    off = A.copy()
    for s in range(0, 70, 10):
        assert np.max(np.abs(np.linalg.eigvals(A[s:s + 10, s:s + 10]))) == pytest.approx(1.0)
        off[s:s + 10, s:s + 10] = 0
    assert np.all(off == 0)


def test_random_qp_sizes_and_structure():
    """Sec. V-A: ten sizes log-spaced 10..2000, n/4 equality and n/4 inequality rows."""
    from workloads import random_qp as R
    assert R.SIZES[0] == 10 and R.SIZES[-1] == 2000 and len(R.SIZES) == 10
    assert all(b > a for a, b in zip(R.SIZES, R.SIZES[1:]))
    for n in (10, 105, 342):
        P, q, A, l, u = R.random_dense_qp(0, n)
        me = n // 4
        assert A.shape == (2 * me, n) and P.shape == (n, n) and q.shape == (n,)
        assert np.all(l[:me] == u[:me]) and np.all(np.isneginf(l[me:])) and np.all(np.isfinite(u))
        assert np.all(np.linalg.eigvalsh(P) > 5e-3)
        assert np.allclose(P, P.T)
    # reproducible and distinct per seed
    a = R.random_dense_qp(3, 58)
    b = R.random_dense_qp(3, 58)
    c = R.random_dense_qp(4, 58)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])


def test_random_qp_oracle_meets_1e6_and_kkt():
    """The FP64 oracle reaches residuals of 1e-6 on the small sizes, and its
    point agrees with the accurate KKT solution (active set + exact solve)."""
    from oracle import relu_qp_oracle as O
    from workloads import random_qp as R
    for n in (10, 32, 105):
        P, q, A, l, u = R.random_dense_qp(1, n)
        r = O.solve(P, q, A, l, u, eps_abs=1e-6, max_iter=4000)
        res = O.residuals(P, q, A, r.x, r.z, r.lam)
        assert r.status == "solved", n
        assert res["r_prim"] <= 1e-6 and res["r_dual"] <= 1e-6
        ref = O.reference_solution(P, q, A, l, u)
        assert O.kkt_violation(P, q, A, l, u, ref["x"], ref["lam"]) <= 1e-9
        assert np.max(np.abs(r.x - ref["x"])) <= 1e-4
        me = n // 4
        assert np.max(np.abs(A[:me] @ r.x - l[:me])) <= 1e-6   # equalities hold to the tolerance
