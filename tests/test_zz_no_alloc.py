"""relu_qp_solve_noalloc (the solve that allocates no device memory) against
relu_qp_solve, through the C ABI, on two calls in a row.

Callers that cannot allocate when they solve (a real-time loop that must not
stall on cudaMalloc, an application that owns all device memory) use the
variant whose scratch is a fixed array inside the library.  Its answers must
be those of the ordinary solve; the second call also shows that what the first
call left in the shared array does not leak into the next one.  This file is
collected last so that a failure here stops a -x run only after every other
test has run.
"""
import ctypes

import numpy as np
import pytest

from workloads import mpc

pytestmark = pytest.mark.gpu

SIGMA = 1e-6
BANK = (0.1, 1.0, 10.0)
CHECK_INTERVAL = 25          # the handles below use the default check interval


@pytest.fixture(scope="module")
def rq():
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build
    build.build()
    return rq


def noalloc(rq, s, x_warm=None, lam_warm=None, rho_index=-1, eps=1e-3, max_iter=4000):
    import torch
    dev = torch.device("cuda:0")
    x = torch.full((s.n,), float("nan"), dtype=torch.float32, device=dev)
    z = torch.full((s.m,), float("nan"), dtype=torch.float32, device=dev)
    lam = torch.full((s.m,), float("nan"), dtype=torch.float32, device=dev)
    xw = None if x_warm is None else torch.tensor(x_warm, dtype=torch.float32, device=dev)
    lw = None if lam_warm is None else torch.tensor(lam_warm, dtype=torch.float32, device=dev)
    info = rq.Info()
    rc = rq.lib().relu_qp_solve_noalloc(s.handle, None if xw is None else xw.data_ptr(),
                                        None if lw is None else lw.data_ptr(), int(rho_index), float(eps), 0.0,
                                        int(max_iter), x.data_ptr(), z.data_ptr(), lam.data_ptr(),
                                        ctypes.byref(info))
    if rc != 0:
        raise rq.ReluQPError(rc, rq.lib().relu_qp_last_error(s.handle).decode())
    out = info.as_dict()
    out.update(x=x.cpu().numpy().astype(np.float64), z=z.cpu().numpy().astype(np.float64),
               lam=lam.cpu().numpy().astype(np.float64))
    return out


@pytest.mark.parametrize("name", ["small", "sweep4", "humanoid"])
def test_noalloc_matches_solve_twice(rq, name):
    pq, X0, _ = mpc.workload(name, 2)
    q, l, u = pq.instance(X0[0])
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    for k in range(2):                      # two calls in a row, different problems
        q, l, u = pq.instance(X0[k])
        s.update(q, l, u)
        ref = s.solve(eps_abs=1e-3)
        got = noalloc(rq, s)
        assert got["status"] == ref["status"] == rq.SOLVED
        assert got["iters"] == ref["iters"]
        tol = 1e-5 * (1 + np.max(np.abs(ref["x"])))
        assert np.max(np.abs(got["x"] - ref["x"])) <= tol
        assert np.max(np.abs(got["z"] - ref["z"])) <= 1e-5 * (1 + np.max(np.abs(ref["z"])))
        assert np.max(np.abs(got["lam"] - ref["lam"])) <= 1e-5 * (1 + np.max(np.abs(ref["lam"])))
    s.close()


def test_noalloc_in_cluster_shape(rq):
    """The allocation-free solve launches the same shape as relu_qp_solve; as
    one cluster of 8 CTAs (operand in distributed shared memory) it returns the
    ordinary solve's bits."""
    pq, X0, _ = mpc.workload("sweep4", 2)
    q, l, u = pq.instance(X0[0])
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    try:
        s.set_single_config(8, 8)
    except rq.ReluQPError as e:
        s.close()
        pytest.skip(f"a cluster of 8 CTAs is not resident here: {e}")
    for x0 in X0:
        q, l, u = pq.instance(x0)
        s.update(q, l, u)
        ref = s.solve(eps_abs=1e-3)
        got = noalloc(rq, s)
        assert got["status"] == ref["status"] == rq.SOLVED and got["iters"] == ref["iters"]
        for k in ("x", "z", "lam"):
            assert np.array_equal(got[k], ref[k]), k
    s.close()


def test_noalloc_warm_start_and_fixed_layers(rq):
    pq, X0, _ = mpc.workload("sweep4", 1)
    q, l, u = pq.instance(X0[0])
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    cold = s.solve(eps_abs=1e-3)
    for _ in range(2):
        ref = s.solve(x_warm=cold["x"], lam_warm=cold["lam"], rho_index=cold["rho_index"], eps_abs=1e-3)
        got = noalloc(rq, s, x_warm=cold["x"], lam_warm=cold["lam"], rho_index=cold["rho_index"])
        assert got["iters"] == ref["iters"]
        # warm-started at the optimum: both stop at the first check
        assert ref["iters"] == CHECK_INTERVAL
        assert np.max(np.abs(got["x"] - ref["x"])) <= 1e-5 * (1 + np.max(np.abs(ref["x"])))
    s.close()


def test_noalloc_after_a_larger_problem(rq):
    """A small problem solved right after a larger one: the larger call leaves
    values in the shared array beyond the small problem's vectors (padding of
    x, lam_std, the operands), which must not leak into its answer."""
    big, Xb, _ = mpc.workload("humanoid", 1)
    q, l, u = big.instance(Xb[0])
    sb = rq.ReluQP(big.P, big.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    small, Xs, _ = mpc.workload("small", 2)
    q, l, u = small.instance(Xs[1])
    ss = rq.ReluQP(small.P, small.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    for _ in range(2):
        noalloc(rq, sb)
        ref = ss.solve(eps_abs=1e-3)
        got = noalloc(rq, ss)
        assert got["status"] == ref["status"] == rq.SOLVED
        assert got["iters"] == ref["iters"]
        assert np.max(np.abs(got["x"] - ref["x"])) <= 1e-5 * (1 + np.max(np.abs(ref["x"])))
        assert np.max(np.abs(got["lam"] - ref["lam"])) <= 1e-5 * (1 + np.max(np.abs(ref["lam"])))
    sb.close()
    ss.close()


def test_noalloc_rejects_host_pointers(rq):
    """The outputs of this entry point are device arrays; a host array is
    refused before any GPU work."""
    pq, X0, _ = mpc.workload("small", 1)
    q, l, u = pq.instance(X0[0])
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    host = np.zeros(s.n, dtype=np.float32)
    info = rq.Info()
    rc = rq.lib().relu_qp_solve_noalloc(s.handle, None, None, -1, 1e-3, 0.0, 4000,
                                        host.ctypes.data, None, None, ctypes.byref(info))
    assert rc != 0
    assert "x_out" in rq.lib().relu_qp_last_error(s.handle).decode()
    s.close()


def test_noalloc_rejects_problems_over_the_limit(rq):
    n, m = 3000, 1200                        # n + m = 4200 > 4096
    rng = np.random.default_rng(0)
    P = np.eye(n) * 2.0
    A = rng.standard_normal((m, n)) / np.sqrt(n)
    s = rq.ReluQP(P, A, -np.ones(m), np.ones(m), q=rng.standard_normal(n), sigma=SIGMA, rho_bank=(1.0,))
    with pytest.raises(rq.ReluQPError) as e:
        noalloc(rq, s)
    assert e.value.kind == "INVALID" and "4096" in str(e.value)
    s.close()
