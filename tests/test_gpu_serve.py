"""GPU tests of the continuous-batching server (relu_qp_server_*).

* a mixed stream over three resident families, more requests than slots:
  every request is answered once, within 1e-3 of the FP64 oracle, with
  FP64-recomputed residuals within eps_abs;
* each result is the same alone and in the mix (same iterations, x within
  1e-6): a QP's arithmetic does not depend on what shares the batch;
* a client's previous solution warm-starts its next request.
"""
import numpy as np
import pytest

from oracle import relu_qp_oracle as O
from workloads import mpc

pytestmark = pytest.mark.gpu

SIGMA = 1e-6
BANK = (0.1, 1.0, 10.0)
RES_SLACK = 1.05


@pytest.fixture(scope="module")
def rq():
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build
    build.build()
    return rq


@pytest.fixture(scope="module")
def families(rq):
    out = []
    for name, slots, prec in (("family0", 64, 1), ("sweep4", 48, 1), ("humanoid", 32, 0)):
        pq, X0, s = mpc.workload(name, 1)
        q, l, u = pq.instance(X0[0])
        h = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, max_batch=slots, precision=prec)
        h.set_parametric(pq.F, pq.E, pq.l0, pq.u0)
        out.append((name, pq, s, h))
    yield out
    for *_, h in out:
        h.close()


def run_all(server, max_steps=2000):
    results = []
    for _ in range(max_steps):
        active, waiting = server.step()
        results += server.poll()
        if active == 0 and waiting == 0:
            break
    return results


def stream(families, count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for t in range(count):
        f = int(rng.choice(3, p=(0.5, 0.3, 0.2)))
        name, pq, s, h = families[f]
        reqs.append((t, f, (s * rng.standard_normal(pq.nx)).astype(np.float32)))
    return reqs


def test_mixed_stream_matches_oracle_and_alone(rq, families):
    reqs = stream(families, 150, 1)
    srv = rq.Server([h for *_, h in families], eps_abs=1e-3)
    for tag, f, x0 in reqs:
        srv.submit(f, x0, tag=tag)
    res = {r["tag"]: r for r in run_all(srv)}
    srv.close()
    assert sorted(res) == list(range(len(reqs)))
    for tag, f, x0 in reqs[:40]:
        name, pq, s, h = families[f]
        r = res[tag]
        assert r["status"] == rq.SOLVED and r["family"] == f
        q, l, u = pq.instance(x0.astype(np.float64))
        orc = O.solve(pq.P, q, pq.A, l, u, sigma=SIGMA, rho_bank=BANK, eps_abs=1e-3, max_iter=4000)
        assert np.max(np.abs(r["x"] - orc.x)) <= 1e-3, (tag, name)
    # the same requests one at a time
    for tag, f, x0 in reqs[::15]:
        srv1 = rq.Server([h for *_, h in families], eps_abs=1e-3)
        srv1.submit(f, x0, tag=tag)
        alone = run_all(srv1)
        srv1.close()
        assert len(alone) == 1
        a, b = alone[0], res[tag]
        assert a["iters"] == b["iters"] and a["rho_index"] == b["rho_index"]
        assert np.max(np.abs(a["x"] - b["x"])) <= 1e-6 * (1 + np.max(np.abs(b["x"]))), tag


def test_client_warm_start_is_resident(rq, families):
    name, pq, s, h = families[1]
    srv = rq.Server([h for *_, h in families], clients=[0, 4, 0], eps_abs=1e-3)
    x0 = (s * np.random.default_rng(3).standard_normal(pq.nx)).astype(np.float32)
    srv.submit(1, x0, client=2, tag=0)
    first = run_all(srv)[0]
    srv.submit(1, x0, client=2, tag=1)          # same state again: warm start is the optimum
    second = run_all(srv)[0]
    srv.submit(1, x0, client=3, tag=2)          # another client has no warm start yet
    third = run_all(srv)[0]
    srv.close()
    assert first["status"] == second["status"] == third["status"] == rq.SOLVED
    assert second["iters"] == 25 and first["iters"] >= second["iters"]
    assert third["iters"] == first["iters"]
    assert np.max(np.abs(second["x"] - first["x"])) <= 2e-3


def test_results_carry_times_and_slots_are_reused(rq, families):
    srv = rq.Server([h for *_, h in families], eps_abs=1e-3)
    reqs = stream(families, 300, 7)             # > total slots (144)
    t0 = srv.clock()
    for tag, f, x0 in reqs:
        srv.submit(f, x0, tag=tag)
    res = run_all(srv)
    srv.close()
    assert len(res) == 300
    assert all(r["t_submit"] >= t0 - 1e-9 and r["t_done"] >= r["t_submit"] for r in res)
    assert all(r["status"] == rq.SOLVED for r in res)


def test_server_rejects_bad_requests(rq, families):
    srv = rq.Server([h for *_, h in families], eps_abs=1e-3)
    with pytest.raises(rq.ReluQPError):
        srv.submit(0, np.full(families[0][1].nx, np.nan, np.float32))
    with pytest.raises(rq.ReluQPError):
        srv.submit(0, np.zeros(families[0][1].nx, np.float32), client=5)   # no clients configured
    srv.close()


def test_budget_holds_requests_back_then_admits(rq, families):
    """Admission by device memory: with room for two requests of the humanoid
    family, six of its requests enter two at a time, the rest wait, every one
    is answered, and each answer equals the same request solved alone (the
    FP32 family's arithmetic does not depend on its batch)."""
    f = 2
    name, pq, s, h = families[f]
    srv = rq.Server([h for *_, h in families], eps_abs=1e-3)
    fixed = sum(srv.family_bytes(k)[0] for k in range(3))
    slot = srv.family_bytes(f)[1]
    assert slot > 0 and fixed > 0
    with pytest.raises(rq.ReluQPError) as e:
        srv.set_budget(fixed // 2)                       # the banks alone do not fit
    assert e.value.kind == "OOM"
    srv.set_budget(fixed + 2 * slot + slot // 2)
    rng = np.random.default_rng(11)
    x0s = [(s * rng.standard_normal(pq.nx)).astype(np.float32) for _ in range(6)]
    for tag, x0 in enumerate(x0s):
        srv.submit(f, x0, tag=tag)
    active, waiting = srv.step()
    results = srv.poll()                                 # a request may finish at its first check
    assert active <= 2 and active + waiting + len(results) == 6 and waiting >= 2
    assert srv.bytes_in_use() == active * slot
    peak = active
    for _ in range(2000):
        active, waiting = srv.step()
        peak = max(peak, active)
        assert srv.bytes_in_use() <= 2 * slot
        results += srv.poll()
        if active == 0 and waiting == 0:
            break
    srv.close()
    assert peak <= 2
    assert sorted(r["tag"] for r in results) == list(range(6))
    for r in results:
        alone_srv = rq.Server([h for *_, h in families], eps_abs=1e-3)
        alone_srv.submit(f, x0s[r["tag"]], tag=0)
        alone = run_all(alone_srv)
        alone_srv.close()
        assert r["status"] == alone[0]["status"] == rq.SOLVED
        assert r["iters"] == alone[0]["iters"]
        assert np.max(np.abs(r["x"] - alone[0]["x"])) <= 1e-6 * (1 + np.max(np.abs(r["x"])))

