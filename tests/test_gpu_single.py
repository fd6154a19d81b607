"""GPU parity of the single-QP path against the FP64 oracle (through the C ABI).

* setup: the GPU's FP64 bank reproduces the oracle's W and b of Eq. gpu_update
  (rel 1e-10) once the factored form is expanded back to the paper's blocks;
* iterates: 50 fixed-rho layers in FP32 match the oracle's to 1e-5 relative;
* converged solves: x within 1e-3 of the oracle's and the residuals of Eqs.
  primal and dual, recomputed in FP64 from the returned (x, z, lam), within
  eps_abs (plus the FP32 rounding of the returned vectors);
* sizes that span several CTAs with ragged tails, and the degenerate cases
  (m = 0, n = 1, equality rows, infinite bounds, warm start at the optimum,
  a matrix that is not positive definite).
"""
import numpy as np
import pytest

from oracle import relu_qp_oracle as O
from workloads import mpc

pytestmark = pytest.mark.gpu

SIGMA = 1e-6
BANK = (0.1, 1.0, 10.0)
# FP32 rounding of the returned x, z, lam moves the FP64-recomputed residual a
# little off the FP32 value the kernel tested against eps_abs.
RES_SLACK = 1.05


@pytest.fixture(scope="module")
def rq():
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build
    build.build()
    return rq


def expand_factored(Wt, Bop, A, rho_vec, n, m):
    """Paper's W (Eq. gpu_update) and Bop from the factored layer [x; Ax] = Wt [x; 2 rho z - lam] + Bop q."""
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


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30)


def random_qp(seed, n, m, eq=0, inf_rows=0):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    P = M @ M.T / n + 0.5 * np.eye(n)
    A = rng.standard_normal((m, n)) / np.sqrt(n)
    q = rng.standard_normal(n) * 2.0
    l = -rng.uniform(0.1, 1.0, m)
    u = rng.uniform(0.1, 1.0, m)
    if eq:
        l[:eq] = u[:eq] = rng.uniform(-0.2, 0.2, eq)
    if inf_rows:
        l[eq:eq + inf_rows] = -np.inf
        u[eq + inf_rows:eq + 2 * inf_rows] = np.inf
    return P, q, A, l, u


# ---------------------------------------------------------------------------
# offline stage
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [("small", None), ("random", (203, 77, 3, 5)), ("sweep4", None)])
def test_setup_bank_matches_oracle_weights(rq, shape):
    name, dims = shape
    if name == "random":
        P, q, A, l, u = random_qp(1, *dims)
    else:
        pq, X0, _ = mpc.workload(name, 1)
        P, A = pq.P, pq.A
        q, l, u = pq.instance(X0[0])
    n, m = P.shape[0], A.shape[0]
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, keep_fp64=True)
    for r, rho in enumerate(BANK):
        rv = O.rho_vector(l, u, rho)
        W_o, B_o = O.relu_layer_weights(P, A, SIGMA, rv)
        Wt, Bop = s.get_layer(r)
        W_g, B_g = expand_factored(Wt, Bop, A, rv, n, m)
        assert rel(W_g, W_o) <= 1e-10, (name, rho)
        assert rel(B_g, B_o) <= 1e-10, (name, rho)
    s.close()


def test_not_positive_definite_is_reported(rq):
    P = np.diag([1.0, -2.0, 1.0])
    A = np.zeros((1, 3))
    with pytest.raises(rq.ReluQPError) as e:
        rq.ReluQP(P, A, [-1.0], [1.0], sigma=SIGMA, rho_bank=BANK)
    assert e.value.kind == "NOT_PD"


# ---------------------------------------------------------------------------
# iterates
# ---------------------------------------------------------------------------

def iterate_case(rq, P, q, A, l, u, rho_index, iters=50):
    n, m = P.shape[0], A.shape[0]
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, check_interval=0)
    out = s.solve(rho_index=rho_index, max_iter=iters)
    s.close()
    v = O.layer_iterates(P, q, A, l, u, SIGMA, BANK[rho_index], iters)[-1]
    x, z, lam_l = v[:n], v[n:n + m], v[n + m:]
    lam = O.std_multiplier(A, x, z, lam_l, O.rho_vector(l, u, BANK[rho_index]))
    ref = np.concatenate([x, z, lam])
    got = np.concatenate([out["x"], out["z"], out["lam"]])
    assert out["iters"] == iters
    return rel(got, ref)


@pytest.mark.parametrize("rho_index", [0, 1, 2])
def test_fp32_iterates_small_mpc(rq, rho_index):
    pq, X0, _ = mpc.workload("small", 3)
    for x0 in X0:
        q, l, u = pq.instance(x0)
        assert iterate_case(rq, pq.P, q, pq.A, l, u, rho_index) <= 1e-5


@pytest.mark.parametrize("dims", [(203, 77, 0, 5), (1, 1, 0, 0), (37, 0, 0, 0), (130, 250, 0, 20),
                                  (517, 300, 0, 10)])
def test_fp32_iterates_ragged_shapes(rq, dims):
    P, q, A, l, u = random_qp(7, *dims)
    assert iterate_case(rq, P, q, A, l, u, 1) <= 1e-5


@pytest.mark.parametrize("dims", [(203, 77, 3, 5), (517, 300, 4, 10)])
def test_fp32_iterates_with_equality_rows(rq, dims):
    # An equality row carries 1000x the penalty (Sec. II-B), so the FP32
    # rounding of A x (~2^-24 |A||x|) enters its multiplier step multiplied by
    # 1000 every layer; the bound is 10x the inequality-only one.
    P, q, A, l, u = random_qp(7, *dims)
    assert iterate_case(rq, P, q, A, l, u, 1) <= 1e-4


def test_fp32_iterates_batched_mpc_shape(rq):
    pq, X0, _ = mpc.workload("batched", 1)
    q, l, u = pq.instance(X0[0])
    assert iterate_case(rq, pq.P, q, pq.A, l, u, 0) <= 1e-5


# ---------------------------------------------------------------------------
# converged solves (Algorithm 1)
# ---------------------------------------------------------------------------

def converged_case(rq, s, P, q, A, l, u, eps=1e-3, **kw):
    out = s.solve(eps_abs=eps, max_iter=4000, **kw)
    orc = O.solve(P, q, A, l, u, sigma=SIGMA, rho_bank=BANK, eps_abs=eps, max_iter=4000)
    res = O.residuals(P, q, A, out["x"], out["z"], out["lam"])
    assert out["status"] == rq.SOLVED
    assert res["r_prim"] <= RES_SLACK * eps and res["r_dual"] <= RES_SLACK * eps, res
    assert np.max(np.abs(out["x"] - orc.x)) <= 1e-3
    return out, orc


def test_converged_small_mpc_all_initial_states(rq):
    """Config of 100 seeded initial states, n = m = 20 (FP32 GPU vs FP64 oracle)."""
    pq, X0, _ = mpc.workload("small", 100)
    q, l, u = pq.instance(X0[0])
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    same_iters = 0
    for x0 in X0:
        q, l, u = pq.instance(x0)
        s.update(q, l, u)
        out, orc = converged_case(rq, s, pq.P, q, pq.A, l, u)
        same_iters += out["iters"] == orc.iters
    s.close()
    assert same_iters >= 90


@pytest.mark.parametrize("name,count", [("sweep4", 5), ("family0", 5), ("batched", 2), ("humanoid", 2)])
def test_converged_mpc_workloads(rq, name, count):
    pq, X0, _ = mpc.workload(name, count)
    q, l, u = pq.instance(X0[0])
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    for x0 in X0:
        q, l, u = pq.instance(x0)
        s.update(q, l, u)
        converged_case(rq, s, pq.P, q, pq.A, l, u)
    s.close()


def test_converged_largest_sweep_sampled(rq):
    """n = m = 1600 (horizon 40, nu = 40): one sampled initial state."""
    pq, X0, _ = mpc.workload("sweep40", 1)
    q, l, u = pq.instance(X0[0])
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    converged_case(rq, s, pq.P, q, pq.A, l, u)
    s.close()


@pytest.mark.parametrize("dims", [(203, 77, 3, 5), (64, 0, 0, 0), (1, 1, 0, 0), (90, 180, 10, 30)])
def test_converged_ragged_and_degenerate(rq, dims):
    P, q, A, l, u = random_qp(11, *dims)
    s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    out, orc = converged_case(rq, s, P, q, A, l, u)
    if dims[1] == 0:
        assert np.max(np.abs(out["x"] + np.linalg.solve(P, q))) <= 1e-4
    s.close()


@pytest.mark.parametrize("name", ["sweep4", "sweep8", "sweep16"])
def test_launch_shapes_give_the_same_bits(rq, name):
    """The single-QP solve as a cooperative grid (1, 4 and one CTA per SM) and
    as one thread-block cluster (2, 4, 8 and 16 CTAs that keep the layer's
    operand in distributed shared memory and meet at cluster-scope mbarriers):
    each row's dot product and update is the same arithmetic in every shape, so
    every shape returns the same bits (x, z, lam, iterations, bank index) on two
    warm-started converged solves, and the result matches the oracle.
    n = m = 160, 320, 640 (closed-loop random MPC at nu = 4, 8, 16)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    pq, X0, _ = mpc.workload(name, 2)
    q, l, u = pq.instance(X0[0])
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    tuned = s.single_config()
    ref, shapes_run = None, []
    for ctas, cluster in [(1, 0), (4, 0), (sms, 0), (2, 2), (4, 4), (8, 8), (16, 16)]:
        try:
            s.set_single_config(ctas, cluster)
        except rq.ReluQPError as e:
            assert e.code == -6, e          # UNSUPPORTED: the shape cannot be resident
            continue
        assert s.single_config()[:2] == (ctas, cluster)
        outs = []
        x_w, lam_w, ri = None, None, -1
        for x0 in X0:
            qq, ll, uu = pq.instance(x0)
            s.update(qq, ll, uu)
            o = s.solve(x_warm=x_w, lam_warm=lam_w, rho_index=ri, eps_abs=1e-3)
            assert o["status"] == rq.SOLVED
            x_w, lam_w, ri = o["x"], o["lam"], o["rho_index"]
            outs.append(o)
        if ref is None:
            ref = outs
            qq, ll, uu = pq.instance(X0[-1])
            orc = O.solve(pq.P, qq, pq.A, ll, uu, sigma=SIGMA, rho_bank=BANK, eps_abs=1e-3, max_iter=4000)
            assert np.max(np.abs(outs[-1]["x"] - orc.x)) <= 1e-3
        else:
            for a, b in zip(outs, ref):
                assert (a["iters"], a["rho_index"]) == (b["iters"], b["rho_index"]), (ctas, cluster)
                for k in ("x", "z", "lam"):
                    assert np.array_equal(a[k], b[k]), (ctas, cluster, k)
        shapes_run.append((ctas, cluster))
    s.close()
    assert any(c > 0 for _, c in shapes_run), shapes_run
    print(f"{name}: tuned shape {tuned}; shapes run {shapes_run}")


def test_warm_start_at_optimum_stops_at_first_check(rq):
    pq, X0, _ = mpc.workload("sweep4", 1)
    q, l, u = pq.instance(X0[0])
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    cold = s.solve(eps_abs=1e-3)
    warm = s.solve(x_warm=cold["x"], lam_warm=cold["lam"], rho_index=cold["rho_index"], eps_abs=1e-3)
    assert warm["status"] == rq.SOLVED and warm["iters"] == 25
    assert np.max(np.abs(warm["x"] - cold["x"])) <= 1e-3
    s.close()


def test_update_rejects_changed_equality_pattern(rq):
    P, q, A, l, u = random_qp(3, 10, 6, eq=2)
    s = rq.ReluQP(P, A, l, u, q=q)
    l2 = l.copy()
    l2[0] -= 0.5
    with pytest.raises(rq.ReluQPError) as e:
        s.update(l=l2)
    assert e.value.kind == "INVALID"
    s.close()
