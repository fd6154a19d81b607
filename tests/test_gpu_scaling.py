"""GPU parity of the problem scaling (Algorithm 1 "Scale problem", Sec. III-D)
against the FP64 oracle's modified Ruiz equilibration, through the C ABI.

* setup: a scaled handle's layer bank is the oracle's layer of the
  equilibrated problem (c D P D, E A D) to 1e-9 relative, so D, E and c agree;
* iterates: 50 fixed-rho FP32 layers of the equilibrated problem match the
  oracle's to 1e-5 (returned x, z, lam mapped into the scaled problem with
  xb = x / D, zb = E z, lamb = c lam / E);
* converged solves (single, batched FP32 and BF16 split, server): status
  SOLVED on QPs that do not converge unscaled, FP64-recomputed residuals of
  the ORIGINAL problem within eps_abs (the stop test runs on them), x within
  1e-3 of the oracle's solve with the same fixed scaling and, in FP32, the
  same iteration count;
* warm starts are mapped into the scaled problem (a warm start at the
  solution stops at the first check) and the no-alloc entry refuses a
  scaled handle.
"""
import ctypes

import numpy as np
import pytest

from oracle import relu_qp_oracle as O
from workloads import mpc

pytestmark = pytest.mark.gpu

SIGMA = 1e-6
BANK = (0.1, 1.0, 10.0)
ITERS = 10
EPS = 1e-3
RES_SLACK = 1.05


@pytest.fixture(scope="module")
def rq():
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build
    build.build()
    return rq


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30)


def expand_layer(Wt, Bop, A, rho_vec, n, m):
    """Paper's W (Eq. gpu_update) and Bop from the factored [x; Ax] = Wt [x; 2 rho z - lam] + Bop q."""
    Wy, WAy = Wt[:n], Wt[n:]
    W = np.zeros((n + 2 * m, n + 2 * m))
    W[:n, :n] = Wy[:, :n]
    W[:n, n:n + m] = Wy[:, n:] * (2 * rho_vec)[None, :]
    W[:n, n + m:] = -Wy[:, n:]
    W[n:n + m, :n] = WAy[:, :n] + A
    W[n:n + m, n:n + m] = WAy[:, n:] * (2 * rho_vec)[None, :] - np.eye(m)
    W[n:n + m, n + m:] = -WAy[:, n:] + np.diag(1.0 / rho_vec)
    W[n + m:, :n] = rho_vec[:, None] * A
    W[n + m:, n:n + m] = -np.diag(rho_vec)
    W[n + m:, n + m:] = np.eye(m)
    B = np.zeros((n + 2 * m, n))
    B[:n + m] = Bop
    return W, B


def check_solution(rq, P, q, A, l, u, x, z, lam, status, ref_x, eps=EPS):
    res = O.residuals(P, q, A, np.asarray(x, np.float64), np.asarray(z, np.float64), np.asarray(lam, np.float64))
    assert status == rq.SOLVED
    assert res["r_prim"] <= RES_SLACK * eps and res["r_dual"] <= RES_SLACK * eps, res
    assert np.max(np.abs(np.asarray(x, np.float64) - ref_x)) <= 1e-3


@pytest.mark.parametrize("seed,dims", [(0, (40, 30)), (1, (203, 77)), (2, (130, 250))])
def test_scaled_bank_is_the_oracles_equilibrated_layer(rq, seed, dims):
    P, q, A, l, u = mpc.badly_scaled_qp(seed, *dims)
    n, m = dims
    D, E, c, Pb, Ab, qb = O.ruiz_scaling(P, A, q, ITERS)
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, keep_fp64=True, scaling_iters=ITERS)
    for r, rho in enumerate(BANK):
        rv = O.rho_vector(E * l, E * u, rho)
        W_o, B_o = O.relu_layer_weights(Pb, Ab, SIGMA, rv)
        Wt, Bop = s.get_layer(r)
        W_g, B_g = expand_layer(Wt, Bop, Ab, rv, n, m)
        assert rel(W_g, W_o) <= 1e-9, rho
        assert rel(B_g, B_o) <= 1e-9, rho
    s.close()


@pytest.mark.parametrize("seed,dims", [(0, (40, 30)), (1, (203, 77))])
def test_scaled_iterates_map_back(rq, seed, dims):
    P, q, A, l, u = mpc.badly_scaled_qp(seed, *dims)
    n, m = dims
    D, E, c, Pb, Ab, qb = O.ruiz_scaling(P, A, q, ITERS)
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, check_interval=0, scaling_iters=ITERS)
    out = s.solve(rho_index=1, max_iter=50)
    s.close()
    lb, ub = E * l, E * u
    v = O.layer_iterates(Pb, qb, Ab, lb, ub, SIGMA, BANK[1], 50)[-1]
    xb, zb, lam_l = v[:n], v[n:n + m], v[n + m:]
    lamb = O.std_multiplier(Ab, xb, zb, lam_l, O.rho_vector(lb, ub, BANK[1]))
    # compared in the scaled problem, where the FP32 layers run (the map back
    # multiplies each component by a factor between 1e-2 and 1e2)
    assert out["iters"] == 50
    assert rel(out["x"] / D, xb) <= 1e-5
    assert rel(out["z"] * E, zb) <= 1e-5
    assert rel(c * out["lam"] / E, lamb) <= 1e-5


@pytest.mark.parametrize("seed,dims", [(0, (40, 30)), (1, (203, 77)), (2, (130, 250))])
def test_scaled_single_solve_matches_oracle(rq, seed, dims):
    P, q, A, l, u = mpc.badly_scaled_qp(seed, *dims)
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, scaling_iters=ITERS)
    out = s.solve(eps_abs=EPS, max_iter=4000)
    orc = O.solve_scaled(P, q, A, l, u, scaling_iters=ITERS, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS,
                         max_iter=4000)
    check_solution(rq, P, q, A, l, u, out["x"], out["z"], out["lam"], out["status"], orc.x)
    assert abs(out["iters"] - orc.iters) <= 25
    # the reported residuals are the original problem's
    res = O.residuals(P, q, A, out["x"], out["z"], out["lam"])
    assert abs(out["r_prim"] - res["r_prim"]) <= 0.05 * EPS + 1e-3 * res["r_prim"]
    assert abs(out["r_dual"] - res["r_dual"]) <= 0.05 * EPS + 1e-3 * res["r_dual"]
    # a warm start at the solution is mapped into the scaled problem: it stops at the first check
    warm = s.solve(x_warm=out["x"], lam_warm=out["lam"], rho_index=out["rho_index"], eps_abs=EPS)
    assert warm["status"] == rq.SOLVED and warm["iters"] == 25
    s.close()


def test_unscaled_solve_does_not_converge(rq):
    """The workload is one where scaling matters: 4000 unscaled layers do not reach eps."""
    P, q, A, l, u = mpc.badly_scaled_qp(0, 40, 30)
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    out = s.solve(eps_abs=EPS, max_iter=4000)
    s.close()
    assert out["status"] == rq.MAX_ITER


def test_scaled_update_keeps_setup_scaling(rq):
    """relu_qp_update: new q, l, u go through the scaling found at setup."""
    P, q, A, l, u = mpc.badly_scaled_qp(1, 203, 77)
    D, E, c, *_ = O.ruiz_scaling(P, A, q, ITERS)
    rng = np.random.default_rng(5)
    q2 = q * (1 + 0.3 * rng.standard_normal(q.shape))
    w = u - l
    l2, u2 = l - 0.1 * w, u + 0.05 * w
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, scaling_iters=ITERS)
    s.update(q2, l2, u2)
    out = s.solve(eps_abs=EPS, max_iter=4000)
    s.close()
    orc = O.solve_scaled(P, q2, A, l2, u2, scaling=(D, E, c), sigma=SIGMA, rho_bank=BANK, eps_abs=EPS,
                         max_iter=4000)
    check_solution(rq, P, q2, A, l2, u2, out["x"], out["z"], out["lam"], out["status"], orc.x)
    assert abs(out["iters"] - orc.iters) <= 25


@pytest.mark.parametrize("prec", [0, 1])
def test_scaled_batched_solves(rq, prec):
    P, q, A, l, u = mpc.badly_scaled_qp(1, 203, 77)
    n, m = P.shape[0], A.shape[0]
    D, E, c, *_ = O.ruiz_scaling(P, A, q, ITERS)
    B = 6
    rng = np.random.default_rng(11)
    Q = np.stack([q] + [q * (1 + 0.3 * rng.standard_normal(n)) for _ in range(B - 1)])
    w = u - l
    L = np.stack([l] + [l - 0.2 * rng.uniform(0, 1, m) * w for _ in range(B - 1)])
    U = np.stack([u] + [u + 0.2 * rng.uniform(0, 1, m) * w for _ in range(B - 1)])
    Qf, Lf, Uf = (a.astype(np.float32) for a in (Q, L, U))
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, max_batch=8, precision=prec, scaling_iters=ITERS)
    s.update_batch(Qf, Lf, Uf)
    out = s.solve_batch(eps_abs=EPS, max_iter=4000)
    same = 0
    for b in range(B):
        qb, lb, ub = (np.asarray(a[b], np.float64) for a in (Qf, Lf, Uf))
        orc = O.solve_scaled(P, qb, A, lb, ub, scaling=(D, E, c), sigma=SIGMA, rho_bank=BANK, eps_abs=EPS,
                             max_iter=4000)
        check_solution(rq, P, qb, A, lb, ub, out["x"][b], out["z"][b], out["lam"][b], out["status"][b], orc.x)
        same += int(out["iters"][b] == orc.iters)
    if prec == 0:
        assert same >= B - 1
    # warm starts at the solutions, mapped into the scaled problem: every QP stops at the first check
    warm = s.solve_batch(X_warm=out["x"], Lam_warm=out["lam"], rho_warm=out["rho_index"].astype(np.int32),
                         eps_abs=EPS, max_iter=4000)
    assert np.all(warm["status"] == rq.SOLVED) and np.all(warm["iters"] == 25)
    s.close()


def test_scaled_server_family(rq):
    pq, X0, sx = mpc.workload("small", 12)
    q, l, u = pq.instance(X0[0])
    D, E, c, *_ = O.ruiz_scaling(pq.P, pq.A, q, ITERS)
    h = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, max_batch=16, precision=0,
                  scaling_iters=ITERS)
    h.set_parametric(pq.F, pq.E, pq.l0, pq.u0)
    srv = rq.Server([h], eps_abs=EPS)
    for t, x0 in enumerate(X0):
        srv.submit(0, x0.astype(np.float32), tag=t)
    res = {}
    for _ in range(2000):
        active, waiting = srv.step()
        for r in srv.poll():
            res[r["tag"]] = r
        if active == 0 and waiting == 0:
            break
    srv.close()
    h.close()
    assert sorted(res) == list(range(len(X0)))
    for t, x0 in enumerate(X0):
        qi, li, ui = pq.instance(x0.astype(np.float32).astype(np.float64))
        orc = O.solve_scaled(pq.P, qi, pq.A, li, ui, scaling=(D, E, c), sigma=SIGMA, rho_bank=BANK, eps_abs=EPS,
                             max_iter=4000)
        assert res[t]["status"] == rq.SOLVED
        assert np.max(np.abs(res[t]["x"] - orc.x)) <= 1e-3, t


def test_noalloc_refuses_a_scaled_handle(rq):
    P, q, A, l, u = mpc.badly_scaled_qp(0, 40, 30)
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, scaling_iters=ITERS)
    x = np.zeros(40, np.float32)
    info = rq.Info()
    rc = rq.lib().relu_qp_solve_noalloc(s.handle, None, None, -1, EPS, 0.0, 100,
                                        x.ctypes.data_as(ctypes.c_void_p), None, None, ctypes.byref(info))
    assert rq.ERRORS[rc] == "UNSUPPORTED"
    s.close()


def test_scaled_equality_and_infinite_rows(rq):
    """Equality rows (1000x penalty, Sec. II-B) and one-sided rows in a badly scaled QP:
    the scaled problem keeps the row pattern (E l = E u exactly where l = u).  In FP32
    the equality rows' multiplier noise, mapped back by 1/(c D), stays above 1e-3 here
    (the floor the FP64 solve exists for), so this runs the FP64 arithmetic, which
    follows the oracle layer for layer."""
    P, q, A, l, u = mpc.badly_scaled_qp(3, 120, 60)
    x_f = np.linalg.lstsq(A, 0.5 * (l + u), rcond=None)[0]
    l, u = l.copy(), u.copy()
    l[:6] = u[:6] = (A @ x_f)[:6]          # equalities at a point inside the other bounds' range
    l[6:20] = -np.inf
    u[20:30] = np.inf
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, scaling_iters=ITERS, single_precision=rq.PREC_FP64)
    out = s.solve(eps_abs=EPS, max_iter=4000)
    s.close()
    orc = O.solve_scaled(P, q, A, l, u, scaling_iters=ITERS, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS, max_iter=4000)
    assert orc.status == "solved"
    check_solution(rq, P, q, A, l, u, out["x"], out["z"], out["lam"], out["status"], orc.x)
    assert out["iters"] == orc.iters
    assert np.all(np.isfinite(out["z"]))      # z is finite where a bound is infinite


def test_scaled_unconstrained(rq):
    P, q, A, l, u = mpc.badly_scaled_qp(4, 50, 10)
    s = rq.ReluQP(P, None, None, None, q=q, sigma=SIGMA, rho_bank=BANK, scaling_iters=ITERS)
    out = s.solve(eps_abs=1e-4, max_iter=4000)
    s.close()
    assert out["status"] == rq.SOLVED
    x = -np.linalg.solve(P, q)
    assert np.max(np.abs(out["x"] - x)) <= 1e-3 * (1 + np.max(np.abs(x)))
