"""GPU parity of batched solves (many QPs sharing P and A) against the FP64 oracle.

FP32 backend (CUDA cores) and BF16 hi+lo split backend (tcgen05 tensor cores):
* iterates of 50 fixed-rho layers vs the oracle's, per QP (1e-5 FP32, 1e-4 BF16);
* converged solves: every QP within 1e-3 of the oracle, FP64-recomputed
  residuals within eps_abs (plus FP32 rounding of the returned vectors);
* batch invariance: a QP alone and inside a batch give the same answer;
* ragged sizes (B not a multiple of 128, n + m not a multiple of the tile),
  m = 0, the parametric x0 update, warm starts, host and device buffers.
"""
import numpy as np
import pytest

from oracle import relu_qp_oracle as O
from workloads import mpc

pytestmark = pytest.mark.gpu

SIGMA = 1e-6
BANK = (0.1, 1.0, 10.0)
RES_SLACK = 1.05
TOL_ITER = {0: 1e-5, 1: 1e-4}


@pytest.fixture(scope="module")
def rq():
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build
    build.build()
    return rq


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30)


def mpc_batch(name, B, x0_std=None):
    pq, X0, _ = mpc.workload(name, B, x0_std=x0_std)
    Q, L, U = pq.instance(X0)
    return pq, X0, Q, L, U


def iterate_batch(rq, prec, pq, Q, L, U, iters=50):
    B = Q.shape[0]
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, check_interval=0,
                  max_batch=B, precision=prec)
    s.update_batch(Q, L, U)
    out = s.solve_batch(max_iter=iters)
    s.close()
    n, m = pq.n, pq.m
    worst = 0.0
    for b in range(B):
        v = O.layer_iterates(pq.P, Q[b], pq.A, L[b], U[b], SIGMA, BANK[0], iters)[-1]
        x, z, lam_l = v[:n], v[n:n + m], v[n + m:]
        lam = O.std_multiplier(pq.A, x, z, lam_l, O.rho_vector(L[b], U[b], BANK[0]))
        ref = np.concatenate([x, z, lam])
        got = np.concatenate([out["x"][b], out["z"][b], out["lam"][b]]).astype(np.float64)
        worst = max(worst, rel(got, ref))
    assert np.all(out["iters"] == iters)
    return worst


def check_converged(rq, pq, Q, L, U, out, idx, eps=1e-3):
    for b in idx:
        x = out["x"][b].astype(np.float64)
        z = out["z"][b].astype(np.float64)
        lam = out["lam"][b].astype(np.float64)
        assert out["status"][b] == rq.SOLVED, (b, out["status"][b], out["iters"][b])
        res = O.residuals(pq.P, Q[b], pq.A, x, z, lam)
        assert res["r_prim"] <= RES_SLACK * eps and res["r_dual"] <= RES_SLACK * eps, (b, res)
        orc = O.solve(pq.P, Q[b], pq.A, L[b], U[b], sigma=SIGMA, rho_bank=BANK, eps_abs=eps, max_iter=4000)
        assert np.max(np.abs(x - orc.x)) <= 1e-3, b


# ---------------------------------------------------------------------------
# FP32 batched backend first, then the tensor-core backend from the smallest case
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_iterates_small_batch(rq, prec):
    pq, X0, Q, L, U = mpc_batch("small", 5)
    assert iterate_batch(rq, prec, pq, Q, L, U) <= TOL_ITER[prec]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_iterates_ragged_batch(rq, prec):
    """n + m = 280 (not a multiple of the row tile), B = 130 (two slot tiles, ragged)."""
    pq, X0, Q, L, U = mpc_batch("family0", 130)
    pick = [0, 77, 129]
    assert iterate_batch(rq, prec, pq, Q[pick], L[pick], U[pick]) <= TOL_ITER[prec]
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, check_interval=0,
                  max_batch=130, precision=prec)
    s.update_batch(Q, L, U)
    full = s.solve_batch(max_iter=50)
    s.close()
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, check_interval=0,
                  max_batch=3, precision=prec)
    s.update_batch(Q[pick], L[pick], U[pick])
    part = s.solve_batch(max_iter=50)
    s.close()
    # batch invariance of the raw layers
    assert np.max(np.abs(full["x"][pick] - part["x"])) <= 1e-6 * (1 + np.max(np.abs(part["x"])))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_iterates_batched_mpc_shape(rq, prec):
    pq, X0, Q, L, U = mpc_batch("batched", 3)
    assert iterate_batch(rq, prec, pq, Q, L, U) <= TOL_ITER[prec]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_converged_small_batch_all(rq, prec):
    pq, X0, Q, L, U = mpc_batch("small", 100)
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, max_batch=100, precision=prec)
    s.update_batch(Q, L, U)
    out = s.solve_batch(eps_abs=1e-3)
    s.close()
    check_converged(rq, pq, Q, L, U, out, range(100))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_converged_batched_workload_sampled(rq, prec):
    """n = m = 800, B = 1024: every QP solved with FP64 residuals <= eps; 6 sampled vs the oracle."""
    pq, X0, Q, L, U = mpc_batch("batched", 1024)
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, max_batch=1024, precision=prec)
    s.update_batch(Q, L, U)
    out = s.solve_batch(eps_abs=1e-3)
    s.close()
    assert np.all(out["status"] == rq.SOLVED)
    X = out["x"].astype(np.float64)
    Z = out["z"].astype(np.float64)
    LM = out["lam"].astype(np.float64)
    rp = np.max(np.abs(X @ pq.A.T - Z), axis=1)
    rd = np.max(np.abs(X @ pq.P + Q + LM @ pq.A), axis=1)
    assert np.max(rp) <= RES_SLACK * 1e-3 and np.max(rd) <= RES_SLACK * 1e-3, (np.max(rp), np.max(rd))
    check_converged(rq, pq, Q, L, U, out, [0, 1, 333, 512, 800, 1023])


def test_converged_batched_workload_4096_sampled(rq):
    """The largest bench configuration (n = m = 800, B = 4096, BF16 split, the
    launch configuration bench.py times): every QP solved with FP64-recomputed
    residuals <= eps; 4 sampled QPs within 1e-3 of the oracle."""
    B = 4096
    pq, X0, Q, L, U = mpc_batch("batched", B)
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, max_batch=B,
                  precision=rq.PREC_BF16X3)
    s.update_batch(Q, L, U)
    out = s.solve_batch(eps_abs=1e-3)
    s.close()
    assert np.all(out["status"] == rq.SOLVED)
    X = out["x"].astype(np.float64)
    Z = out["z"].astype(np.float64)
    LM = out["lam"].astype(np.float64)
    rp = np.max(np.abs(X @ pq.A.T - Z), axis=1)
    rd = np.max(np.abs(X @ pq.P + Q + LM @ pq.A), axis=1)
    assert np.max(rp) <= RES_SLACK * 1e-3 and np.max(rd) <= RES_SLACK * 1e-3, (np.max(rp), np.max(rd))
    check_converged(rq, pq, Q, L, U, out, [0, 1777, 2048, 4095])


def test_batch_sizes_are_validated(rq):
    """An empty batch and a batch over the handle's capacity are refused with
    INVALID before any GPU work; the handle then still solves."""
    pq, X0, Q, L, U = mpc_batch("family0", 8)
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, max_batch=8)
    for bad in (0, 9):
        with pytest.raises(rq.ReluQPError) as e:
            s.solve_batch(B=bad, eps_abs=1e-3)
        assert e.value.kind == "INVALID", bad
    s.update_batch(Q, L, U)
    out = s.solve_batch(eps_abs=1e-3)
    s.close()
    assert np.all(out["status"] == rq.SOLVED)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_converged_humanoid_sampled(rq, prec):
    pq, X0, Q, L, U = mpc_batch("humanoid", 256)
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, max_batch=256, precision=prec)
    s.update_batch(Q, L, U)
    out = s.solve_batch(eps_abs=1e-3)
    s.close()
    check_converged(rq, pq, Q, L, U, out, [0, 100, 255])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_alone_equals_in_batch(rq, prec):
    """Batch invariance of full solves (checks, rho switches, regrouping, the
    convergence tail).  FP32: the same layers and the same iterates to rounding
    (the tail kernel repeats the tiled kernels' arithmetic).  BF16 split: a QP
    alone reaches the FP32 tail kernel after its first check, inside the batch
    only once at most 8 QPs are left, so the two solves agree to the stated
    tolerance of converged solutions: both solved, x within 1e-3 of each other."""
    pq, X0, Q, L, U = mpc_batch("family0", 300)
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, max_batch=300, precision=prec)
    s.update_batch(Q, L, U)
    full = s.solve_batch(eps_abs=1e-3)
    for b in [0, 150, 299]:
        s.update_batch(Q[b:b + 1], L[b:b + 1], U[b:b + 1])
        one = s.solve_batch(eps_abs=1e-3)
        if prec == 0:
            assert one["iters"][0] == full["iters"][b]
            assert np.max(np.abs(one["x"][0] - full["x"][b])) <= 1e-6 * (1 + np.max(np.abs(one["x"][0])))
        else:
            assert one["status"][0] == full["status"][b] == rq.SOLVED
            assert np.max(np.abs(one["x"][0] - full["x"][b])) <= 1e-3
    s.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_parametric_update_matches_explicit(rq, prec):
    pq, X0, Q, L, U = mpc_batch("family0", 64)
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, max_batch=64, precision=prec)
    s.set_parametric(pq.F, pq.E, pq.l0, pq.u0)
    s.update_batch_x0(X0.astype(np.float32))
    a = s.solve_batch(eps_abs=1e-3)
    s.update_batch(Q, L, U)
    b = s.solve_batch(eps_abs=1e-3)
    s.close()
    assert np.all(a["status"] == rq.SOLVED) and np.all(b["status"] == rq.SOLVED)
    assert np.max(np.abs(a["x"] - b["x"])) <= 1e-3
    check_converged(rq, pq, Q, L, U, a, [0, 31, 63])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_warm_start_batch_and_device_buffers(rq, prec):
    import torch
    pq, X0, Q, L, U = mpc_batch("sweep4", 40)
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, max_batch=40, precision=prec)
    dev = torch.device("cuda:0")
    Qd, Ld, Ud = (torch.tensor(a, dtype=torch.float32, device=dev) for a in (Q, L, U))
    s.update_batch(Qd, Ld, Ud)
    outd = tuple(torch.empty((40, k), dtype=torch.float32, device=dev) for k in (pq.n, pq.m, pq.m))
    cold = s.solve_batch(eps_abs=1e-3, out=outd)
    x_cold = outd[0].cpu().numpy()
    warm = s.solve_batch(X_warm=outd[0].clone(), Lam_warm=outd[2].clone(),
                         rho_warm=torch.tensor(cold["rho_index"], dtype=torch.int32, device=dev), eps_abs=1e-3)
    s.close()
    assert np.all(warm["status"] == rq.SOLVED) and np.all(warm["iters"] == 25)
    # both solves stop within eps of the optimum; 25 more layers may move x by about eps
    assert np.max(np.abs(warm["x"] - x_cold)) <= 2e-3
    check_converged(rq, pq, Q, L, U, {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in cold.items()},
                    [0, 39])
    check_converged(rq, pq, Q, L, U, warm, [0, 17, 39])


def test_batch_unconstrained_m0(rq):
    rng = np.random.default_rng(5)
    n = 70
    M = rng.standard_normal((n, n))
    P = M @ M.T / n + np.eye(n)
    Q = rng.standard_normal((9, n))
    for prec in (0, 1):
        s = rq.ReluQP(P, np.zeros((0, n)), None, None, q=Q[0], sigma=SIGMA, rho_bank=BANK, max_batch=9,
                      precision=prec)
        s.update_batch(Q)
        out = s.solve_batch(eps_abs=1e-4)
        s.close()
        X = -np.linalg.solve(P, Q.T).T
        assert np.all(out["status"] == rq.SOLVED)
        assert np.max(np.abs(out["x"] - X)) <= 1e-4


@pytest.mark.parametrize("B", [20, 48])
def test_one_tile_resident_weight_kernel(rq, B):
    """One slot tile of few QPs (n = m = 800): the tuner times the
    resident-weight chunk kernel (rows of the layer kept in shared memory over a
    cluster of 8 CTAs) against the tiled one and uses it where faster.  The
    iterates after 50 fixed-rho layers match the oracle's within the split
    form's 1e-4, and a converged solve matches the oracle within 1e-3 with
    FP64-recomputed residuals within eps."""
    pq, X0, Q, L, U = mpc_batch("batched", B)
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, check_interval=0,
                  max_batch=B, precision=rq.PREC_BF16X3)
    s.update_batch(Q, L, U)
    s.profile(enable=1, reset=True)
    out = s.solve_batch(max_iter=50)
    used = s.profile(enable=0)["resident_launches"]
    s.close()
    n, m = pq.n, pq.m
    worst = 0.0
    for b in range(0, B, 7):
        v = O.layer_iterates(pq.P, Q[b], pq.A, L[b], U[b], SIGMA, BANK[0], 50)[-1]
        x, z, lam_l = v[:n], v[n:n + m], v[n + m:]
        lam = O.std_multiplier(pq.A, x, z, lam_l, O.rho_vector(L[b], U[b], BANK[0]))
        ref = np.concatenate([x, z, lam])
        got = np.concatenate([out["x"][b], out["z"][b], out["lam"][b]]).astype(np.float64)
        worst = max(worst, rel(got, ref))
    assert worst <= TOL_ITER[1], worst
    # converged, adaptive rho, checks every 25 layers
    s = rq.ReluQP(pq.P, pq.A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, max_batch=B,
                  precision=rq.PREC_BF16X3)
    s.update_batch(Q, L, U)
    s.profile(enable=1, reset=True)
    conv = s.solve_batch(eps_abs=1e-3, max_iter=4000)
    used += s.profile(enable=0)["resident_launches"]
    s.close()
    assert np.all(conv["status"] == rq.SOLVED)
    check_converged(rq, pq, Q, L, U, conv, range(0, B, 9))
    print(f"B={B}: resident-weight chunk launches {used}, iterate error {worst:.2e}")


@pytest.mark.parametrize("B", [2, 5])
@pytest.mark.parametrize("case", ["mpc_n800", "random_n2000"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_tail_kernel_iterates(rq, prec, case, B):
    """Fixed-rho layers through the convergence-tail kernel.  Five QPs, a check
    every 25 layers with an eps no iterate reaches and adaptive rho off: after
    the first check at most 8 QPs are left, so layers 26..100 run in the tail
    kernel.  The same five QPs inside a batch of nine (more than 8 stay active,
    so the tail never starts) run all 100 layers in the tiled kernels.  FP32:
    the tail repeats the tiled kernels' arithmetic (products in the same
    summation order, the element-wise steps with explicit roundings), so the
    two give the same bits.  Both match the oracle's fixed-rho iterates: 1e-5
    FP32 and 1e-4 BF16 split on the MPC problem; on the random QP the equality
    rows (rho scaled by 1e3) amplify rounding over 100 layers, and the bound
    there is 2e-4.
    n = m = 800 runs the tail's one-pass form (all step partials of a CTA's rows
    at once, every output's state in registers); the random QP with n = 2000
    and m = 1000 (3000 rows, 20 per CTA) adds up the step partials in two
    passes of 10 rows, and its Wt rows do not fit shared memory.  Two and five
    QPs: the step partials specialised on groups of 2 and 5 QPs."""
    from workloads import random_qp
    B_tiled = 9
    if case == "mpc_n800":
        pq, X0, Q, L, U = mpc_batch("batched", B_tiled)
        P, A = pq.P, pq.A
        tol = TOL_ITER[prec]
    else:
        P, q, A, l, u = random_qp.random_dense_qp(0, 2000)
        rng = np.random.default_rng(11)
        Q = q[None, :] + rng.standard_normal((B_tiled, q.size))
        L = np.repeat(l[None, :], B_tiled, axis=0)
        U = np.repeat(u[None, :], B_tiled, axis=0)
        tol = 2e-4
    n, m = P.shape[0], A.shape[0]
    outs = []
    for nb in (B, B_tiled):
        s = rq.ReluQP(P, A, L[0], U[0], q=Q[0], sigma=SIGMA, rho_bank=BANK, check_interval=25,
                      adaptive_rho=False, rho0=BANK[0], max_batch=nb, precision=prec)
        s.update_batch(Q[:nb], L[:nb], U[:nb])
        outs.append(s.solve_batch(eps_abs=1e-12, eps_rel=0.0, max_iter=100))
        s.close()
    tail, tiled = outs
    for out in outs:
        assert np.all(out["iters"] == 100) and np.all(out["status"] == rq.MAX_ITER)
    if prec == 0:
        for k in ("x", "z", "lam"):
            assert np.array_equal(tail[k], tiled[k][:B]), k
    worst = {"tail": 0.0, "tiled": 0.0}
    for b in (0, B - 1):
        v = O.layer_iterates(P, Q[b], A, L[b], U[b], SIGMA, BANK[0], 100)[-1]
        x, z, lam_l = v[:n], v[n:n + m], v[n + m:]
        lam = O.std_multiplier(A, x, z, lam_l, O.rho_vector(L[b], U[b], BANK[0]))
        ref = np.concatenate([x, z, lam])
        for name, out in (("tail", tail), ("tiled", tiled)):
            got = np.concatenate([out["x"][b], out["z"][b], out["lam"][b]]).astype(np.float64)
            worst[name] = max(worst[name], rel(got, ref))
    print(f"{case} prec={prec} B={B}: error vs oracle {worst}")
    assert worst["tail"] <= tol and worst["tiled"] <= tol, worst
