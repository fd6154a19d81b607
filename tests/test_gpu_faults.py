"""Failure detection on the GPU without a GPU fault.

* Every kind of device-side wait in the library (the cooperative kernels'
  grid barrier, the tensor-core kernels' mbarrier and layer-counter waits) is
  made to run out on purpose with a 1 ms deadline: the wait gives up, the
  kernel returns RELU_QP_ERR_TIMEOUT to the host within milliseconds, and the
  CUDA context still solves afterwards.  No kernel faults, traps or spins
  without a bound.
* Allocation refusal is injected on the host: a handle whose device-memory
  budget is too small for its bank fails with RELU_QP_ERR_OOM before any
  cudaMalloc beyond the budget, and the same problem sets up within a budget
  equal to what it needs.
"""
import ctypes

import numpy as np
import pytest

from oracle import relu_qp_oracle as O
from workloads import mpc

pytestmark = pytest.mark.gpu

SIGMA = 1e-6
BANK = (0.1, 1.0, 10.0)
TIMEOUT = -5


@pytest.fixture(scope="module")
def rq():
    import torch
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return rq


def device_wait(rq, kind, ns):
    st, ms = ctypes.c_int(99), ctypes.c_double(-1.0)
    rc = rq.lib().relu_qp_diag_device_wait(kind, ns, ctypes.byref(st), ctypes.byref(ms))
    return rc, st.value, ms.value


def solve_small(rq):
    pq, X0, _ = mpc.workload("small", 2)
    q, l, u = pq.instance(X0[1])
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    out = s.solve(eps_abs=1e-3)
    s.close()
    ref = O.solve(pq.P, q, pq.A, l, u, sigma=SIGMA, rho_bank=BANK, eps_abs=1e-3)
    return out, ref


@pytest.mark.parametrize("kind,what", [(0, "grid barrier"), (2, "mbarrier"), (3, "layer counter"),
                                       (4, "cluster barrier")])
def test_device_wait_gives_up_at_its_deadline(rq, kind, what):
    rc, status, ms = device_wait(rq, kind, 1_000_000)          # 1 ms deadline
    assert rc == 0, what
    assert status == TIMEOUT, what
    assert 0.9 <= ms < 100.0, (what, ms)                        # gave up after ~1 ms, not at some later point
    out, ref = solve_small(rq)                                  # the context is still usable
    assert out["status"] == rq.SOLVED and out["iters"] == ref.iters
    assert np.max(np.abs(out["x"] - ref.x)) <= 1e-3


@pytest.mark.parametrize("kind", [1, 5], ids=["grid barrier", "cluster barrier"])
def test_barrier_with_every_arrival_passes(rq, kind):
    rc, status, ms = device_wait(rq, kind, 1_000_000)
    assert rc == 0 and status == 0 and ms < 100.0


def test_device_budget_refuses_then_admits(rq):
    pq, X0, _ = mpc.workload("humanoid", 1)
    q, l, u = pq.instance(X0[0])
    kw = dict(q=q, sigma=SIGMA, rho_bank=BANK, max_batch=64, precision=rq.PREC_BF16X3)
    full = rq.ReluQP(pq.P, pq.A, l, u, **kw)
    full.set_parametric(pq.F, pq.E, pq.l0, pq.u0)            # allocates the parametric maps too
    need = full.device_bytes()
    full.close()
    assert need > 10 * 2**20                                    # three FP32 layers of 1600^2 alone are 30 MB
    with pytest.raises(rq.ReluQPError) as e:
        rq.ReluQP(pq.P, pq.A, l, u, device_budget=need // 2, **kw)
    assert e.value.kind == "OOM" and "budget" in str(e.value)
    ok = rq.ReluQP(pq.P, pq.A, l, u, device_budget=need, **kw)
    ok.set_parametric(pq.F, pq.E, pq.l0, pq.u0)
    assert ok.device_bytes() == need
    ok.update_batch_x0(X0[:4].astype(np.float32))
    out = ok.solve_batch(eps_abs=1e-3)
    ok.close()
    assert np.all(out["status"] == rq.SOLVED)
