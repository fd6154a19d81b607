"""GPU parity of the FP64 single-QP solve on the random dense QPs of Sec. V-A
(n/4 equality and n/4 inequality rows, residuals below 1e-6), against the
FP64 oracle, through the C ABI.

* iterates: 50 fixed-rho FP64 layers match the oracle's to 1e-11 relative
  (x, z) and 1e-9 (lam, whose equality rows carry 1000 rho);
* converged solves at eps_abs = 1e-6 for all ten sizes 10..2000: status
  SOLVED, the oracle's iteration count (FP64 on both sides), x within 1e-6 of
  the oracle's, residuals recomputed in FP64 from the returned vectors within
  1e-6 and the reported ones equal to them;
* with the scaling step, warm starts, and the equality-row accuracy that FP32
  cannot reach (the FP32 path stalls above 1e-6 on the same problem);
* the FP64-anchored form (FP32 products of the layer increments between FP64
  anchor layers) reaches the same 1e-6 at every size, within one check of the
  oracle's layer count and 1e-5 of its x.
"""
import numpy as np
import pytest

from oracle import relu_qp_oracle as O
from workloads import random_qp as R

pytestmark = pytest.mark.gpu

SIGMA = 1e-6
BANK = (0.1, 1.0, 10.0)
EPS = 1e-6


@pytest.fixture(scope="module")
def rq():
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build
    build.build()
    return rq


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30)


def handle(rq, P, q, A, l, u, **kw):
    return rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, single_precision=rq.PREC_FP64, **kw)


@pytest.mark.parametrize("n", [10, 105, 342])
def test_fp64_iterates_match_oracle(rq, n):
    P, q, A, l, u = R.random_dense_qp(0, n)
    m = A.shape[0]
    s = handle(rq, P, q, A, l, u, check_interval=0)
    out = s.solve(rho_index=1, max_iter=50)
    s.close()
    v = O.layer_iterates(P, q, A, l, u, SIGMA, BANK[1], 50)[-1]
    x, z, lam_l = v[:n], v[n:n + m], v[n + m:]
    lam = O.std_multiplier(A, x, z, lam_l, O.rho_vector(l, u, BANK[1]))
    # lam_std = lam' + rho_eq (Ax - z) on the equality rows multiplies the FP64
    # rounding of Ax - z (~1e-16 |Ax| per layer, different summation order
    # on both sides) by 1000 rho = 1e3: the bound is 100x that of x and z.
    assert out["iters"] == 50
    assert rel(out["x"], x) <= 1e-11
    assert rel(out["z"], z) <= 1e-11
    assert rel(out["lam"], lam) <= 1e-9


@pytest.mark.parametrize("n", R.SIZES)
def test_fp64_converges_at_1e6_like_oracle(rq, n):
    seeds = (0, 1) if n <= 342 else (0,)
    for seed in seeds:
        P, q, A, l, u = R.random_dense_qp(seed, n)
        s = handle(rq, P, q, A, l, u)
        out = s.solve(eps_abs=EPS, max_iter=4000)
        s.close()
        orc = O.solve(P, q, A, l, u, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS, max_iter=4000)
        res = O.residuals(P, q, A, out["x"], out["z"], out["lam"])
        assert out["status"] == rq.SOLVED, (n, seed)
        assert out["iters"] == orc.iters and out["rho_index"] == orc.rho_index, (n, seed)
        assert res["r_prim"] <= EPS and res["r_dual"] <= EPS, (n, seed, res)
        assert abs(out["r_prim"] - res["r_prim"]) <= 1e-9 and abs(out["r_dual"] - res["r_dual"]) <= 1e-9
        assert np.max(np.abs(out["x"] - orc.x)) <= 1e-6, (n, seed)
        me = n // 4
        assert np.max(np.abs(A[:me] @ out["x"] - l[:me])) <= EPS


def test_fp64_with_scaling_matches_oracle(rq):
    P, q, A, l, u = R.random_dense_qp(0, 105)
    s = handle(rq, P, q, A, l, u, scaling_iters=10)
    out = s.solve(eps_abs=EPS, max_iter=4000)
    s.close()
    orc = O.solve_scaled(P, q, A, l, u, scaling_iters=10, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS, max_iter=4000)
    res = O.residuals(P, q, A, out["x"], out["z"], out["lam"])
    assert out["status"] == rq.SOLVED
    assert out["iters"] == orc.iters
    assert res["r_prim"] <= EPS * (1 + 1e-6) and res["r_dual"] <= EPS * (1 + 1e-6)
    assert np.max(np.abs(out["x"] - orc.x)) <= 1e-6


def test_fp64_warm_start_and_update(rq):
    P, q, A, l, u = R.random_dense_qp(2, 190)
    s = handle(rq, P, q, A, l, u)
    cold = s.solve(eps_abs=EPS)
    warm = s.solve(x_warm=cold["x"], lam_warm=cold["lam"], rho_index=cold["rho_index"], eps_abs=EPS)
    assert warm["status"] == rq.SOLVED and warm["iters"] == 25
    # a new cost through relu_qp_update: the FP64 bias is recomputed
    q2 = np.random.default_rng(7).standard_normal(q.shape)
    s.update(q2)
    out = s.solve(eps_abs=EPS)
    s.close()
    orc = O.solve(P, q2, A, l, u, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS, max_iter=4000)
    assert out["status"] == rq.SOLVED and out["iters"] == orc.iters
    assert np.max(np.abs(out["x"] - orc.x)) <= 1e-6


def test_fp32_cannot_resolve_1e6_with_equality_rows(rq):
    """Why the FP64 solve exists: the same problem in FP32 stalls above 1e-6
    (equality rows multiply the FP32 rounding of Ax - z by 1000 rho)."""
    P, q, A, l, u = R.random_dense_qp(0, 342)
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    out = s.solve(eps_abs=EPS, max_iter=1000)
    s.close()
    assert out["status"] == rq.MAX_ITER
    assert out["r_dual"] > EPS
    s64 = handle(rq, P, q, A, l, u)
    out64 = s64.solve(eps_abs=EPS, max_iter=1000)
    s64.close()
    assert out64["status"] == rq.SOLVED


def test_fp64_noalloc_is_refused(rq):
    import ctypes
    P, q, A, l, u = R.random_dense_qp(0, 10)
    s = handle(rq, P, q, A, l, u)
    x = np.zeros(10, np.float32)
    info = rq.Info()
    rc = rq.lib().relu_qp_solve_noalloc(s.handle, None, None, -1, EPS, 0.0, 100,
                                        x.ctypes.data_as(ctypes.c_void_p), None, None, ctypes.byref(info))
    s.close()
    assert rq.ERRORS[rc] == "UNSUPPORTED"


def test_fp64_degenerate_shapes(rq):
    """m = 0 (the solve is x = -P^-1 q), n = m = 1, and max_iter = 1."""
    P, q, A, l, u = R.random_dense_qp(5, 58)
    s = rq.ReluQP(P, None, None, None, q=q, sigma=SIGMA, rho_bank=BANK, single_precision=rq.PREC_FP64)
    out = s.solve(eps_abs=1e-9, max_iter=4000)
    s.close()
    assert out["status"] == rq.SOLVED
    assert np.max(np.abs(out["x"] + np.linalg.solve(P, q))) <= 1e-7
    s = rq.ReluQP([[2.0]], [[1.0]], [0.5], [0.5], q=[1.0], sigma=SIGMA, rho_bank=BANK,
                  single_precision=rq.PREC_FP64)
    out = s.solve(eps_abs=EPS, max_iter=4000)
    assert out["status"] == rq.SOLVED and abs(out["x"][0] - 0.5) <= 1e-6
    one = s.solve(eps_abs=EPS, max_iter=1)
    s.close()
    assert one["iters"] == 1 and one["status"] == rq.MAX_ITER


@pytest.mark.parametrize("n", R.SIZES)
def test_fp64_anchored_converges_at_1e6(rq, n):
    P, q, A, l, u = R.random_dense_qp(0, n)
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, single_precision=rq.PREC_FP64R)
    out = s.solve(eps_abs=EPS, max_iter=4000)
    warm = s.solve(x_warm=out["x"], lam_warm=out["lam"], rho_index=out["rho_index"], eps_abs=EPS)
    s.close()
    orc = O.solve(P, q, A, l, u, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS, max_iter=4000)
    res = O.residuals(P, q, A, out["x"], out["z"], out["lam"])
    assert out["status"] == rq.SOLVED, n
    assert res["r_prim"] <= EPS and res["r_dual"] <= EPS, (n, res)
    assert abs(out["iters"] - orc.iters) <= 25, (n, out["iters"], orc.iters)
    assert np.max(np.abs(out["x"] - orc.x)) <= 1e-5, n
    assert warm["status"] == rq.SOLVED and warm["iters"] == 25


def test_fp64_anchored_first_layers_match_fp64(rq):
    """Within one anchor period the anchored layers are the FP64 layers up to the FP32
    rounding of the increment products (1e-6 relative over 24 layers)."""
    P, q, A, l, u = R.random_dense_qp(1, 342)
    outs = []
    for prec in (rq.PREC_FP64, rq.PREC_FP64R):
        s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, check_interval=25, single_precision=prec)
        outs.append(s.solve(rho_index=1, max_iter=24, eps_abs=0.0))
        s.close()
    assert rel(outs[1]["x"], outs[0]["x"]) <= 1e-6
    assert rel(outs[1]["z"], outs[0]["z"]) <= 1e-6


def test_fp64_anchored_with_scaling(rq):
    """The anchored form on a scaled problem: residuals of the original problem within 1e-6."""
    P, q, A, l, u = R.random_dense_qp(0, 105)
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, scaling_iters=10, single_precision=rq.PREC_FP64R)
    out = s.solve(eps_abs=EPS, max_iter=4000)
    s.close()
    orc = O.solve_scaled(P, q, A, l, u, scaling_iters=10, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS, max_iter=4000)
    res = O.residuals(P, q, A, out["x"], out["z"], out["lam"])
    assert out["status"] == rq.SOLVED
    assert res["r_prim"] <= EPS * (1 + 1e-6) and res["r_dual"] <= EPS * (1 + 1e-6)
    assert abs(out["iters"] - orc.iters) <= 25
    assert np.max(np.abs(out["x"] - orc.x)) <= 1e-5
