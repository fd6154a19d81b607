"""GPU parity of relu_qp_condense_mpc (Sec. IV, FP64 on the GPU) against the
condensing oracle, through the C ABI.

* P, A_con, F, E match the oracle's literal S'HS, G S, S'HM, G M to 1e-10
  relative (LQR gain by the GPU's Riccati iteration vs the oracle's DARE
  solve: 1e-9), l0 and u0 exactly, for the workload plants (n from 20 to 800),
  with state limits, a given gain and no preconditioning;
* an unstabilizable plant is reported, not returned;
* end to end: a handle set up from the GPU's condensed problem solves the
  same MPC QPs as the oracle (x within 1e-3).
"""
import numpy as np
import pytest

from oracle import condense_oracle as C
from oracle import relu_qp_oracle as O
from workloads import mpc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build
    build.build()
    return rq


def close(a, b, tol):
    return np.max(np.abs(a - b)) <= tol * (1 + np.max(np.abs(b)))


def plant(seed, nx, nu):
    A, B = mpc.random_dynamics(mpc.rng_for(seed, 0), nx, nu, 1.05)
    return A, B, np.eye(nx), 0.1 * np.eye(nu)


@pytest.mark.parametrize("nx,nu,N", [(6, 2, 10), (12, 4, 40), (60, 20, 40), (7, 3, 5)])
def test_condense_matches_oracle(rq, nx, nu, N):
    A, B, Q, R = plant(nx * 100 + nu, nx, nu)
    QN = 3.0 * Q
    umin, umax = -np.linspace(0.5, 1.5, nu), np.linspace(1.0, 2.0, nu)
    g = rq.condense_mpc(A, B, Q, R, N, QN=QN, umin=umin, umax=umax)
    o = C.condense_mpc(A, B, Q, R, N, QN=QN, umin=umin, umax=umax)
    assert close(g["K"], o["K"], 1e-9)
    for k in ("P", "A", "F", "E"):
        assert g[k].shape == o[k].shape and close(g[k], o[k], 1e-9), k
    assert np.array_equal(g["l0"], o["l0"]) and np.array_equal(g["u0"], o["u0"])
    # with the oracle's gain given, the rest is the same arithmetic to rounding
    g2 = rq.condense_mpc(A, B, Q, R, N, QN=QN, umin=umin, umax=umax, K=o["K"])
    for k in ("P", "A", "F", "E"):
        assert close(g2[k], o[k], 1e-10), k


def test_condense_state_limits_and_no_preconditioning(rq):
    A, B, Q, R = plant(5, 8, 3)
    N = 12
    xmin, xmax = -4 * np.ones(8), 4 * np.ones(8)
    g = rq.condense_mpc(A, B, Q, R, N, umin=-np.ones(3), umax=np.ones(3), xmin=xmin, xmax=xmax,
                        lqr_precondition=False)
    o = C.condense_mpc(A, B, Q, R, N, umin=-np.ones(3), umax=np.ones(3), xmin=xmin, xmax=xmax,
                       precondition=False)
    assert np.all(g["K"] == 0)
    assert g["A"].shape == (N * (3 + 8), N * 3)
    for k in ("P", "A", "F", "E"):
        assert close(g[k], o[k], 1e-10), k
    assert np.array_equal(g["l0"], o["l0"]) and np.array_equal(g["u0"], o["u0"])
    # one-sided limits: the missing side is infinite
    g1 = rq.condense_mpc(A, B, Q, R, N, umax=np.ones(3), xmin=xmin)
    assert np.all(np.isneginf(g1["l0"][:N * 3])) and np.all(np.isposinf(g1["u0"][N * 3:]))


def test_condense_rejects_unstabilizable_plant(rq):
    A = 1.5 * np.eye(4)
    B = np.zeros((4, 2))
    with pytest.raises(rq.ReluQPError) as e:
        rq.condense_mpc(A, B, np.eye(4), np.eye(2), 10, umin=-np.ones(2), umax=np.ones(2))
    assert e.value.kind == "INVALID"
    with pytest.raises(rq.ReluQPError):
        rq.condense_mpc(A, B, np.eye(4), np.eye(2), 10, umin=np.ones(2), umax=-np.ones(2))


def test_condensed_problem_solves_like_oracle(rq):
    """Setup from the GPU-condensed problem, batched parametric solves vs the
    oracle on the oracle-condensed problem (Algorithm 1, eps 1e-3)."""
    A, B, Q, R = plant(11, 12, 4)
    N = 20
    g = rq.condense_mpc(A, B, Q, R, N, umin=-np.ones(4), umax=np.ones(4))
    o = C.condense_mpc(A, B, Q, R, N, umin=-np.ones(4), umax=np.ones(4))
    X0 = 6.0 * mpc.rng_for(11, 9).standard_normal((6, 12))
    q0 = g["F"] @ X0[0]
    h = rq.ReluQP(g["P"], g["A"], g["l0"] - g["E"] @ X0[0], g["u0"] - g["E"] @ X0[0], q=q0, max_batch=8)
    h.set_parametric(g["F"], g["E"], g["l0"], g["u0"])
    h.update_batch_x0(X0.astype(np.float32))
    out = h.solve_batch(eps_abs=1e-3)
    h.close()
    for b, x0 in enumerate(X0.astype(np.float32).astype(np.float64)):
        q, l, u = o["F"] @ x0, o["l0"] - o["E"] @ x0, o["u0"] - o["E"] @ x0
        r = O.solve(o["P"], q, o["A"], l, u, eps_abs=1e-3)
        assert out["status"][b] == rq.SOLVED and r.status == "solved"
        assert np.max(np.abs(out["x"][b] - r.x)) <= 1e-3, b


def test_condense_smallest_shapes(rq):
    """A scalar plant (nx = nu = 1) over one stage, and a single-input plant with N = 1."""
    for (A, B) in ((np.array([[1.2]]), np.array([[0.5]])), (np.array([[1.0, 0.1], [0.0, 1.0]]), np.array([[0.0], [0.1]]))):
        nx, nu = B.shape
        Q, R = np.eye(nx), 0.1 * np.eye(nu)
        for N in (1, 3):
            g = rq.condense_mpc(A, B, Q, R, N, umin=-np.ones(nu), umax=np.ones(nu))
            o = C.condense_mpc(A, B, Q, R, N, umin=-np.ones(nu), umax=np.ones(nu))
            for k in ("P", "A", "F", "E", "K"):
                assert close(g[k], o[k], 1e-9), (nx, N, k)
