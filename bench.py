#!/usr/bin/env python
"""QP solves/s at eps_abs = 1e-3 for batched condensed-MPC QPs on GB300.

Workload (one step): a batch of B = 1024 QPs of the condensed, LQR-
preconditioned MPC problem with nx = 60, nu = 20, N = 40 (n = m = 800) that
share P and A (one bank of layers, rho in {0.1, 1, 10}) and each have their
own initial state x0 (hence q, l, u).  A step is the whole online path:
x0 -> (q, l, u, b) update, Algorithm 1 to eps_abs = 1e-3 for every QP
(layers, checks every 25 layers, penalty rule, regrouping) and the outputs.
The offline stage (FP64 factorisation and layer bank) runs once before
timing.  Inputs are synthetic and seeded (workloads/mpc.py).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the same workload instead.  `--serve` measures the served stream and
`--random-qp` the random dense QPs of Sec. V-A (their own JSON lines).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "QP solves/s at eps=1e-3 (batched BF16-split, one GB300)"
UNIT = "QP solves/s"
SIGMA = 1e-6
BANK = (0.1, 1.0, 10.0)
EPS = 1e-3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp32"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--skip-extras", action="store_true", help="skip the FP32 comparison arms")
    ap.add_argument("--serve", action="store_true",
                    help="run the served stream (Poisson arrivals over three resident families) instead")
    ap.add_argument("--rate", type=float, default=2000.0, help="served stream: requests per second")
    ap.add_argument("--duration", type=float, default=10.0, help="served stream: measured seconds")
    ap.add_argument("--random-qp", action="store_true",
                    help="random dense QPs of Sec. V-A: FP64 single solves to 1e-6 per size")
    ap.add_argument("--rqp-count", type=int, default=10, help="random QPs per size")
    ap.add_argument("--rqp-sizes", type=str, default="", help="comma-separated subset of the ten sizes")
    ap.add_argument("--closed-loop", action="store_true",
                    help="random-MPC closed loop (Sec. V-B): single-QP FP32 solves, warm-started, per nu")
    ap.add_argument("--cl-nus", type=str, default="4,8,16,32,40", help="closed loop: comma-separated nu values")
    ap.add_argument("--cl-steps", type=int, default=100, help="closed loop: MPC steps per nu")
    ap.add_argument("--humanoid", action="store_true",
                    help="humanoid-sized QP (n=600, m=1000): single FP32 solves and a BF16-split batch of 256")
    ap.add_argument("--serve-rates", type=str, default="",
                    help="served stream: comma-separated request rates to sweep (max sustainable rate)")
    ap.add_argument("--profile-window", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


def workload_config(B, x0_std, precision):
    return {
        "workload": (f"batched condensed MPC nx=60 nu=20 N=40 (n=m=800), {B} QPs per step sharing one layer "
                     f"bank, own x0 ~ N(0, {x0_std:.3g}^2), eps_abs=1e-3, rho bank {list(BANK)}, sigma 1e-6"),
        "batch": B, "n": 800, "m": 800, "precision": precision, "check_interval": 25,
        "l2": "flushed (256 MiB write) before every timed step",
    }


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on a bounded sample
# ---------------------------------------------------------------------------

def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_oracle(pq, X0, seconds):
    from oracle import relu_qp_oracle as O
    l0, u0 = pq.l0, pq.u0
    weights = [O.relu_layer_weights(pq.P, pq.A, SIGMA, O.rho_vector(l0, u0, r)) for r in BANK]
    done = 0
    t0 = time.perf_counter()
    iters = []
    for x0 in X0:
        q, l, u = pq.instance(x0)
        r = O.solve(pq.P, q, pq.A, l, u, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS, weights=weights)
        iters.append(r.iters)
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return done, dt, iters


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows), "samples": len(rows),
                "reasons": reasons}


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d.get("bf16_tflops_sustained", 1700.0)), float(d.get("bf16_tflops", 1900.0)), "measured"
    return 1700.0, 1900.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("batch_tc.cu", "batch.h"):
        h.update(open(os.path.join(ROOT, "paper_2311_18056_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per refined layer and the QP slots that layer covered, from the
    committed ncu summary of the persistent chunk kernel, if it was taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "tc_chunk_refined_batched_n800.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_layer"]), float(vals["qp_slots_per_layer"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; weak scaling, no data collective)
# ---------------------------------------------------------------------------

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args):
    """The oracle (FP64 NumPy, as it stands) on the host cores, same metric."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from workloads import mpc
    pq, _, x0_std = mpc.workload("batched", 1)
    per_step = 2
    X0 = mpc.initial_states(pq.nx, per_step * (args.steps + args.warmup), 2, sub_id=7, std=x0_std)
    from oracle import relu_qp_oracle as O
    weights = [O.relu_layer_weights(pq.P, pq.A, SIGMA, O.rho_vector(pq.l0, pq.u0, r)) for r in BANK]
    times = []
    k = 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            q, l, u = pq.instance(X0[k])
            k += 1
            O.solve(pq.P, q, pq.A, l, u, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS, weights=weights)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * len(times) / total
    cores = blas_threads()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "value_is": f"the FP64 oracle's QP solves/s on the host ({per_step} QPs of the batched workload per step)",
            "config": workload_config(per_step, x0_std, "fp64 oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} QPs per step of the batched workload (n=m=800), FP64 NumPy"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build as _build
    _build.build()
    from workloads import mpc

    pq, _, x0_std = mpc.workload("batched", 1)
    B, K, W = args.batch, args.steps, args.warmup
    prec = rq.PREC_BF16X3 if args.precision == "bf16x3" else rq.PREC_FP32
    # per-step initial states: distinct seeded batches per rank and step
    X0_host = [mpc.initial_states(pq.nx, B, 2, sub_id=1000 + 97 * rank + k, std=x0_std).astype(np.float32)
               for k in range(W + K)]
    X0_dev = [torch.from_numpy(x).to(dev) for x in X0_host]
    q0, l0, u0 = pq.instance(X0_host[0][0].astype(np.float64))
    solver = rq.ReluQP(pq.P, pq.A, l0, u0, q=q0, sigma=SIGMA, rho_bank=BANK, max_batch=B, precision=prec)
    solver.set_parametric(pq.F, pq.E, pq.l0, pq.u0)
    Xo = torch.empty((B, pq.n), dtype=torch.float32, device=dev)
    Zo = torch.empty((B, pq.m), dtype=torch.float32, device=dev)
    Lo = torch.empty((B, pq.m), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2

    def step(X0):
        solver.update_batch_x0(X0)
        return solver.solve_batch(eps_abs=EPS, max_iter=4000, out=(Xo, Zo, Lo))

    for k in range(W):
        step(X0_dev[k])
    torch.cuda.synchronize()
    solver.profile(enable=1, reset=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    unsolved, iters = 0, []
    if args.profile_window:
        torch.cuda.profiler.start()
    for k in range(K):
        flush.fill_(float(k))
        ev[k][0].record()
        out = step(X0_dev[W + k])
        ev[k][1].record()
        unsolved += int(np.sum(out["status"] != rq.SOLVED))
        iters.append(out["iters"])
    torch.cuda.synchronize()
    if args.profile_window:
        torch.cuda.profiler.stop()
    barrier(world)
    clk = clocks.stop()
    prof = solver.profile(enable=0)
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    t_total = max_over_ranks(world, float(step_ms.sum()) / 1e3)
    solves = sum_over_ranks(world, B * K)
    value = solves / t_total

    # ---- end to end through the C ABI with host (pinned) buffers ----
    X0_pin = [torch.from_numpy(x).pin_memory() for x in X0_host[W:W + K]]
    Xh = torch.empty((B, pq.n), dtype=torch.float32).pin_memory()
    Zh = torch.empty((B, pq.m), dtype=torch.float32).pin_memory()
    Lh = torch.empty((B, pq.m), dtype=torch.float32).pin_memory()
    solver.update_batch_x0(X0_pin[0])
    solver.solve_batch(eps_abs=EPS, out=(Xh, Zh, Lh))
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        solver.update_batch_x0(X0_pin[k])
        solver.solve_batch(eps_abs=EPS, out=(Xh, Zh, Lh))
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(world, time.perf_counter() - t0)
    e2e = {"value": solves / t_e2e, "unit": UNIT, "h2d_bytes_per_step": B * pq.nx * 4,
           "d2h_bytes_per_step": B * (pq.n + 2 * pq.m) * 4 + B * 40}

    # ---- roofline of the dominant kernel: the tensor-core refined layer (one unit =
    # one layer over the active QPs; the persistent chunk kernel runs 24 per launch) ----
    peak_sus, peak_burst, peak_kind = measured_peaks()
    roof = None
    if prof["layer_timed"] > 0 and prof["layer_ms"] > 0:
        flops_per_layer = prof["layer_flops"] / max(prof["layer_launches"], 1)
        achieved = prof["layer_flops"] / (prof["layer_ms"] / 1e3) / 1e12
        qps_per_layer = flops_per_layer / (2.0 * 3.0 * (pq.n + pq.m) ** 2)
        tr = profiled_traffic()
        # the capture covered a known number of QP slots: scale its bytes to the average layer's QPs
        traffic = None if tr is None else tr[0] * qps_per_layer / tr[1]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak_sus, "unit": "TFLOP/s",
                "frac": achieved / peak_sus, "traffic": traffic,
                "traffic_basis": "ncu DRAM bytes per layer of a chunk-kernel launch "
                                 "(profiles/tc_chunk_refined_batched_n800.md), scaled by QPs",
                "kernel": "refined tensor-core layer (tc_chunk_kernel / tc_gemm_kernel): 3 BF16 products, "
                          "FP32 accumulate in TMEM, epilogue fused",
                "unit_of_work": "one refined layer over the active QPs",
                "peak_kind": f"bf16 sustained, {peak_kind}",
                "layers_timed": prof["layer_timed"], "avg_layer_us": 1e3 * prof["layer_ms"] / prof["layer_timed"],
                "flops_per_layer": flops_per_layer, "avg_qps_per_layer": qps_per_layer}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": float(step_ms.mean()), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if prec == rq.PREC_BF16X3 else "f32", "data": "synthetic",
            "config": workload_config(B, x0_std, args.precision),
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "unsolved": unsolved, "mean_iters": float(np.mean(np.concatenate(iters))),
            "e2e": e2e, "roofline": roof, "clocks": clk, "gpu_launches": int(prof["launches"]),
            "host_round_trips": {"per_step": prof["host_checks"] / K,
                                 "gpu_wait_ms_per_step": prof["host_gap_ms"] / K,
                                 "note": "device time between the last kernel before each check's read-back of "
                                         "the active count and the first event enqueued after it returned"}}

    # ---- comparison arms on the same GPU (rank 0, N = 1): plain FP32 ----
    if rank == 0 and world == 1 and not args.skip_extras:
        extras = {}
        s32 = rq.ReluQP(pq.P, pq.A, l0, u0, q=q0, sigma=SIGMA, rho_bank=BANK, max_batch=B, precision=rq.PREC_FP32)
        s32.set_parametric(pq.F, pq.E, pq.l0, pq.u0)
        s32.update_batch_x0(X0_dev[0])
        s32.solve_batch(eps_abs=EPS, out=(Xo, Zo, Lo))
        tt = []
        for k in range(2):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            s32.update_batch_x0(X0_dev[W + k])
            s32.solve_batch(eps_abs=EPS, out=(Xo, Zo, Lo))
            b.record()
            torch.cuda.synchronize()
            tt.append(a.elapsed_time(b))
        s32.close()
        extras["fp32_batched_solves_per_s"] = B / (np.mean(tt) / 1e3)
        single = rq.ReluQP(pq.P, pq.A, l0, u0, q=q0, sigma=SIGMA, rho_bank=BANK)
        Xs = X0_host[W][:48].astype(np.float64)
        single.update(*pq.instance(Xs[0]))
        single.solve(eps_abs=EPS)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat = []
        for x0 in Xs:
            single.update(*pq.instance(x0))
            r = single.solve(eps_abs=EPS)
            lat.append(r["solve_ms"])
        t_single = time.perf_counter() - t0
        single.close()
        extras["fp32_single_solves_per_s"] = len(Xs) / t_single
        extras["fp32_single_p50_ms"] = float(np.percentile(lat, 50))
        extras["fp32_single_p99_ms"] = float(np.percentile(lat, 99))
        extras["speedup_vs_fp32_single"] = value / extras["fp32_single_solves_per_s"]
        extras["speedup_vs_fp32_batched"] = value / extras["fp32_batched_solves_per_s"]
        line["comparison"] = extras
    solver.close()

    if rank == 0 and world == 1:
        X0c = mpc.initial_states(pq.nx, 200, 2, sub_id=5000, std=x0_std)
        done, dt, it = cpu_oracle(pq, X0c, args.cpu_seconds)
        line["cpu_baseline"] = {"value": done / dt, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                                "sample": f"{done} QPs of the batched workload solved one by one by the FP64 "
                                          f"NumPy oracle in {dt:.1f} s (mean {np.mean(it):.0f} layers)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args):
    """Served stream: Poisson arrivals at `rate` req/s from three resident families
    (n = 80, 600, 1600; 60/30/10 %), each request a new x0 for one of 64 clients
    per family, warm-started from that client's previous solution."""
    import torch
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build as _build
    from workloads import mpc
    _build.build()
    torch.cuda.set_device(0)
    names, slots, clients = ("family0", "family1", "family2"), (512, 256, 128), 64
    fams = []
    for name, sl in zip(names, slots):
        pq, X0, std = mpc.workload(name, 1)
        q, l, u = pq.instance(X0[0])
        h = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, max_batch=sl, precision=rq.PREC_BF16X3)
        h.set_parametric(pq.F, pq.E, pq.l0, pq.u0)
        fams.append((pq, std, h))
    warm_s = 1.0
    times, fam = mpc.poisson_arrivals(args.rate, warm_s + args.duration, mix=(0.6, 0.3, 0.1))
    rng = mpc.rng_for(4, 6)
    x0s = [(fams[f][1] * rng.standard_normal(fams[f][0].nx)).astype(np.float32) for f in fam]
    cl = rng.integers(0, clients, len(times))
    srv = rq.Server([h for _, _, h in fams], clients=[clients] * 3, eps_abs=EPS)
    t_base = srv.clock()
    i, done, lat, lat_f, status = 0, 0, [], [[], [], []], []
    while done < len(times):
        now = srv.clock() - t_base
        while i < len(times) and times[i] <= now:
            srv.submit(int(fam[i]), x0s[i], client=int(cl[i]), tag=i)
            i += 1
        active, waiting = srv.step()
        for r in srv.poll():
            done += 1
            k = r["tag"]
            if times[k] >= warm_s:
                ms = 1e3 * (r["t_done"] - t_base - times[k])
                lat.append(ms)
                lat_f[r["family"]].append(ms)
                status.append(r["status"])
        if active == 0 and waiting == 0 and i < len(times):
            time.sleep(max(0.0, min(0.001, times[i] - (srv.clock() - t_base))))
    t_end = srv.clock() - t_base
    srv.close()
    measured = sum(1 for t in times if t >= warm_s)
    value = measured / max(t_end - warm_s, 1e-9)
    # one-at-a-time plain FP32 single-QP solves of the same families
    single_ms = []
    for (pq, std, h), name in zip(fams, names):
        h.close()
        q, l, u = pq.instance(std * mpc.initial_states(pq.nx, 1, pq.meta["workload_id"], sub_id=11)[0])
        sq = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
        X = std * mpc.initial_states(pq.nx, 12, pq.meta["workload_id"], sub_id=12)
        t = []
        for x0 in X:
            sq.update(*pq.instance(x0))
            t0 = time.perf_counter()
            sq.solve(eps_abs=EPS)
            t.append(1e3 * (time.perf_counter() - t0))
        sq.close()
        single_ms.append(float(np.mean(t)))
    mix = np.array([0.6, 0.3, 0.1])
    util = float(args.rate * np.sum(mix * np.array(single_ms)) / 1e3)
    line = {"metric": "served MPC stream: solves/s and arrival-to-result latency (BF16-split, one GB300)",
            "value": value, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "bf16",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": f"Poisson {args.rate:g} req/s for {args.duration:g} s after {warm_s:g} s warm-up; "
                                   "families n=80 (nx12 nu4 N20), 600/1000 (humanoid), 1600 (nx120 nu40 N40) at "
                                   "60/30/10 %, 64 clients per family, warm start = the client's previous solution",
                       "slots": list(slots), "eps_abs": EPS},
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p50_ms_by_family": [float(np.percentile(v, 50)) if v else None for v in lat_f],
            "p99_ms_by_family": [float(np.percentile(v, 99)) if v else None for v in lat_f],
            "unsolved": int(sum(1 for s_ in status if s_ != 0)), "requests": measured,
            "offered_rate": args.rate, "sustained": bool(value >= 0.97 * args.rate),
            "fp32_one_at_a_time": {"mean_solve_ms_by_family": single_ms, "utilization_at_rate": util,
                                   "max_rate_req_per_s": float(1e3 / np.sum(mix * np.array(single_ms))),
                                   "stable": util < 1.0}}
    print(json.dumps(line), flush=True)


def run_random_qp(args):
    """Random dense QPs (Sec. V-A): for each of the ten sizes n = 10..2000 with
    n/4 equality and n/4 inequality rows, `rqp_count` seeded problems, each set
    up (FP64 bank, not timed) and solved cold to residuals below 1e-6 by the
    FP64 single-QP kernel and by its FP64-anchored form (FP32 increments).  Reports per size the device time of the solve
    (CUDA events around the cooperative launch), its p50 and max, the layers,
    and the FP64 NumPy oracle's time on the first problem of the size."""
    import paper_2311_18056_gb300 as rq
    from workloads import random_qp as R
    eps = 1e-6
    per_size = []
    cores = blas_threads()
    sizes = [int(v) for v in args.rqp_sizes.split(",")] if args.rqp_sizes else list(R.SIZES)
    for n in sizes:
        ms, iters, solved, wall = [], [], 0, []
        ms_r, iters_r, solved_r = [], [], 0
        for seed in range(args.rqp_count):
            P, q, A, l, u = R.random_dense_qp(seed, n)
            for prec in (rq.PREC_FP64, rq.PREC_FP64R):
                s = rq.ReluQP(P, A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, single_precision=prec)
                s.solve(eps_abs=eps, max_iter=50)            # first launch of this handle (not timed)
                t0 = time.perf_counter()
                r = s.solve(eps_abs=eps, max_iter=4000)
                dt = (time.perf_counter() - t0) * 1e3
                s.close()
                if prec == rq.PREC_FP64:
                    wall.append(dt)
                    ms.append(r["solve_ms"])
                    iters.append(r["iters"])
                    solved += int(r["status"] == rq.SOLVED)
                else:
                    ms_r.append(r["solve_ms"])
                    iters_r.append(r["iters"])
                    solved_r += int(r["status"] == rq.SOLVED)
        from oracle import relu_qp_oracle as O
        P, q, A, l, u = R.random_dense_qp(0, n)
        t0 = time.perf_counter()
        O.solve(P, q, A, l, u, sigma=SIGMA, rho_bank=BANK, eps_abs=eps, max_iter=4000)
        oracle_ms = (time.perf_counter() - t0) * 1e3
        per_size.append({"n": n, "m": 2 * (n // 4), "problems": args.rqp_count, "solved": solved,
                         "p50_ms": float(np.percentile(ms, 50)), "max_ms": float(np.max(ms)),
                         "p50_call_ms": float(np.percentile(wall, 50)), "mean_layers": float(np.mean(iters)),
                         "us_per_layer": float(np.sum(ms) * 1e3 / np.sum(iters)),
                         "refined": {"p50_ms": float(np.percentile(ms_r, 50)), "max_ms": float(np.max(ms_r)),
                                     "mean_layers": float(np.mean(iters_r)), "solved": solved_r,
                                     "us_per_layer": float(np.sum(ms_r) * 1e3 / np.sum(iters_r))},
                         "oracle_ms_first_problem": oracle_ms})
        print(f"n={n}: FP64 p50 {per_size[-1]['p50_ms']:.3f} ms, layers {np.mean(iters):.0f}, solved {solved}/"
              f"{args.rqp_count}; FP64R p50 {per_size[-1]['refined']['p50_ms']:.3f} ms, layers "
              f"{np.mean(iters_r):.0f}, solved {solved_r}", file=sys.stderr, flush=True)
    big = per_size[-1]
    line = {"metric": "random dense QP solve time at eps=1e-6 (FP64-anchored single QP, n=2000, one GB300)",
            "value": big["refined"]["p50_ms"], "unit": "ms", "n_gpus": 1, "higher_is_better": False, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "random dense QPs, n/4 equality + n/4 inequality rows, sizes 10..2000 "
                                   "log-spaced, seeded, eps_abs=1e-6, rho bank [0.1, 1.0, 10.0], sigma 1e-6, "
                                   "cold starts"},
            "per_size": per_size, "vs_baseline": None,
            "cpu_baseline": {"value": big["oracle_ms_first_problem"], "unit": "ms", "cores": cores,
                             "kind": "oracle", "sample": "first problem of n = 2000 solved by the FP64 oracle"}}
    print(json.dumps(line), flush=True)


def single_roofline(n, m, layers, ms):
    """Achieved bandwidth of the single-QP FP32 layer: one layer reads the FP32
    bank entry Wt ((n+m) x (n+m), 4 bytes each); bytes x layers / device time."""
    bytes_per_layer = 4.0 * (n + m) ** 2
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    gbs = bytes_per_layer * layers / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
            "bytes_per_layer": bytes_per_layer, "peak_kind": "measured copy bandwidth",
            "note": "algorithmic bytes of the bank entry per layer; the entry is served from L2 and shared memory "
                    "when it fits, so frac > 1 would mean on-chip reuse"}


def run_closed_loop(args):
    """Random linear MPC in closed loop (config 1; Sec. V-B): per nu, 100 MPC
    steps x+ = A x + B u0 + w, each QP solved to eps=1e-3 by the single-QP FP32
    path, warm-started from the previous step's (x, lam, rho); reports the
    device solve time p50/p99, layers, active-limit fraction, the layer's
    achieved bytes/s and the FP64 oracle on the first steps."""
    import torch
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build as _build
    from workloads import mpc
    from oracle import relu_qp_oracle as O
    _build.build()
    torch.cuda.set_device(0)
    per_nu = []
    for nu in [int(v) for v in args.cl_nus.split(",")]:
        pq, X0, x0_std = mpc.workload(f"sweep{nu}", 1)
        W = mpc.disturbances(pq, args.cl_steps, 0.1)
        x = X0[0].copy()
        q, l, u = pq.instance(x)
        s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
        s.solve(eps_abs=EPS)                  # first launch of the handle (not timed)
        # the oracle's layer bank is offline, like the GPU setup
        weights = [O.relu_layer_weights(pq.P, pq.A, SIGMA, O.rho_vector(pq.l0, pq.u0, r)) for r in BANK]
        warm = None
        ms, call_ms, layers, active, status, oracle_ms, oracle_err = [], [], [], [], [], [], []
        for k in range(args.cl_steps):
            q, l, u = pq.instance(x)
            if args.profile_window and k == 1:
                torch.cuda.profiler.start()
            t0 = time.perf_counter()
            s.update(q, l, u)
            if warm is None:
                r = s.solve(eps_abs=EPS)
            else:
                r = s.solve(x_warm=warm["x"], lam_warm=warm["lam"], rho_index=warm["rho_index"], eps_abs=EPS)
            call_ms.append(1e3 * (time.perf_counter() - t0))
            if args.profile_window and k == 1:
                torch.cuda.profiler.stop()
            ms.append(r["solve_ms"])
            layers.append(r["iters"])
            status.append(r["status"])
            Ax = pq.A @ r["x"]
            active.append(float(np.mean((Ax <= l + 1e-3) | (Ax >= u - 1e-3))))
            if k < 3:
                # the oracle takes the same warm start as the GPU solve
                wk = {} if warm is None else {"x_warm": warm["x"], "lam_warm": warm["lam"],
                                              "rho_index_warm": warm["rho_index"]}
                t1 = time.perf_counter()
                o = O.solve(pq.P, q, pq.A, l, u, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS, weights=weights, **wk)
                oracle_ms.append(1e3 * (time.perf_counter() - t1))
                oracle_err.append(float(np.max(np.abs(o.x - r["x"]))))
            warm = r
            x = pq.Ad @ x + pq.Bd @ pq.first_control(x, r["x"]) + W[k]
        s.close()
        roof = single_roofline(pq.n, pq.m, float(np.sum(layers)), float(np.sum(ms)))
        per_nu.append({"nu": nu, "n": pq.n, "m": pq.m, "steps": args.cl_steps, "x0_std": x0_std,
                       "solved": int(sum(1 for v in status if v == rq.SOLVED)),
                       "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                       "p50_call_ms": float(np.percentile(call_ms, 50)),
                       "solves_per_s": 1e3 / float(np.mean(ms)), "mean_layers": float(np.mean(layers)),
                       "us_per_layer": 1e3 * float(np.sum(ms)) / float(np.sum(layers)),
                       "active_fraction": float(np.mean(active)), "roofline": roof,
                       "oracle_ms_first3": oracle_ms, "max_abs_err_vs_oracle_first3": oracle_err})
        print(f"nu={nu}: p50 {per_nu[-1]['p50_ms']:.3f} ms p99 {per_nu[-1]['p99_ms']:.3f} ms, layers "
              f"{np.mean(layers):.0f}, {roof['achieved']:.0f} GB/s", file=sys.stderr, flush=True)
    big = per_nu[-1]
    line = {"metric": "closed-loop random MPC: single-QP FP32 solve time at eps=1e-3 (one GB300)",
            "value": big["p50_ms"], "unit": "ms", "n_gpus": 1, "higher_is_better": False, "dtype": "f32",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": "random linear MPC, horizon 40, nx = 3 nu, |u| <= 1, LQR-preconditioned "
                                   "condensing (n = m = 40 nu); x0 scaled so the limits bind, w ~ N(0, 0.1^2); "
                                   "each step warm-started from the previous solve", "nus": [p["nu"] for p in per_nu]},
            "per_nu": per_nu,
            "cpu_baseline": {"value": float(np.mean(big["oracle_ms_first3"])), "unit": "ms",
                             "cores": blas_threads(), "kind": "oracle",
                             "sample": f"first 3 closed-loop steps at nu={big['nu']} solved by the FP64 oracle "
                                       "(same warm starts, layer bank built beforehand)"}}
    print(json.dumps(line), flush=True)


def run_humanoid(args):
    """Humanoid-sized QP (config 3: n = 600, m = 1000 with 400 dense
    inequalities): single-QP FP32 solves one at a time and one BF16-split batch
    of 256 QPs, both to eps = 1e-3, with the oracle on a bounded sample."""
    import torch
    import paper_2311_18056_gb300 as rq
    from paper_2311_18056_gb300 import build as _build
    from workloads import mpc
    from oracle import relu_qp_oracle as O
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    pq, X0, x0_std = mpc.workload("humanoid", 256 + 32)
    q, l, u = pq.instance(X0[0])
    # single FP32, one at a time
    s = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK)
    s.solve(eps_abs=EPS)
    ms, layers, solved = [], [], 0
    for x0 in X0[256:256 + 32]:
        s.update(*pq.instance(x0))
        r = s.solve(eps_abs=EPS)
        ms.append(r["solve_ms"])
        layers.append(r["iters"])
        solved += int(r["status"] == rq.SOLVED)
    s.close()
    single = {"solves": len(ms), "solved": solved, "p50_ms": float(np.percentile(ms, 50)),
              "p99_ms": float(np.percentile(ms, 99)), "solves_per_s": 1e3 / float(np.mean(ms)),
              "mean_layers": float(np.mean(layers)),
              "roofline": single_roofline(pq.n, pq.m, float(np.sum(layers)), float(np.sum(ms)))}
    # batched BF16 split x 256
    B = 256
    sb = rq.ReluQP(pq.P, pq.A, l, u, q=q, sigma=SIGMA, rho_bank=BANK, max_batch=B, precision=rq.PREC_BF16X3)
    sb.set_parametric(pq.F, pq.E, pq.l0, pq.u0)
    X = torch.from_numpy(X0[:B].astype(np.float32)).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(3):
        sb.update_batch_x0(X)
        sb.solve_batch(eps_abs=EPS)
    sb.profile(enable=1, reset=True)
    tt, unsolved = [], 0
    for _ in range(args.steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        sb.update_batch_x0(X)
        out = sb.solve_batch(eps_abs=EPS)
        b.record()
        torch.cuda.synchronize()
        tt.append(a.elapsed_time(b))
        unsolved += int(np.sum(out["status"] != rq.SOLVED))
    prof = sb.profile(enable=0)
    sb.close()
    peak_sus, _, peak_kind = measured_peaks()
    roof = None
    if prof["layer_timed"] > 0:
        achieved = prof["layer_flops"] / (prof["layer_ms"] / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak_sus, "unit": "TFLOP/s",
                "frac": achieved / peak_sus, "peak_kind": f"bf16 sustained, {peak_kind}",
                "avg_layer_us": 1e3 * prof["layer_ms"] / prof["layer_timed"]}
    # oracle on a bounded sample
    t0 = time.perf_counter()
    worst = 0.0
    for b in range(2):
        qb, lb, ub = pq.instance(X0[b].astype(np.float32).astype(np.float64))
        o = O.solve(pq.P, qb, pq.A, lb, ub, sigma=SIGMA, rho_bank=BANK, eps_abs=EPS)
        worst = max(worst, float(np.max(np.abs(o.x - out["x"][b]))))
    oracle_ms = 1e3 * (time.perf_counter() - t0) / 2
    batched = {"batch": B, "ms_per_batch": float(np.mean(tt)), "solves_per_s": B / (float(np.mean(tt)) / 1e3),
               "unsolved": unsolved, "mean_layers": float(np.mean(out["iters"])), "roofline": roof,
               "max_abs_err_vs_oracle_2": worst}
    line = {"metric": "humanoid-sized QP (n=600, m=1000): QP solves/s at eps=1e-3, batched BF16-split x256 "
                      "and single FP32 (one GB300)",
            "value": batched["solves_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "bf16",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": "humanoid-sized MPC nx=70 nu=30 N=20, block dynamics, |u|<=50 + 400 dense rows "
                                   f"(n=600, m=1000), x0 ~ N(0, {x0_std:.3g}^2)", "batch": B},
            "batched": batched, "single_fp32": single,
            "speedup_batched_vs_single": batched["solves_per_s"] / single["solves_per_s"],
            "cpu_baseline": {"value": 1e3 / oracle_ms, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                             "sample": "2 humanoid QPs solved by the FP64 oracle"}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.closed_loop:
        run_closed_loop(args)
        return
    if args.humanoid:
        run_humanoid(args)
        return
    if args.serve and args.serve_rates:
        for r in args.serve_rates.split(","):
            args.rate = float(r)
            run_serve(args)
        return
    if args.serve:
        run_serve(args)
    elif args.random_qp:
        run_random_qp(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
