#!/usr/bin/env python3
"""Benchmark of the exact fast Matérn product and the GP solve on GB300.

One step = one pass of the whole hot path on the d=2 workload
(N = 200000 points x ~ U[0,1]^2, nu = 3/2, ell = (0.1, 0.3), product
kernel): build the cached sort and dominance structure and the rank-350
pivoted-Cholesky preconditioner (the paper uses rank 100; 350 is the
fastest whole step measured on this workload), then solve
(K + 0.01 I) alpha = y by preconditioned CG to an FP64 true relative
residual <= 1e-8 (FP32 scans, FP64 vectors, FP64 residual replacement).
``value`` is solves per second over all ranks (each rank solves its own
replica).  ``--precond-rank 0`` runs the unpreconditioned solve.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the CPU oracle (FP64 brute-force product, all host
cores) on a bounded sample of the same workload instead.  Prints one JSON
line (rank 0).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact Matérn MVM N·nrhs/sec & CG solves/sec at resid≤1e-8; p50/p99 latency"
UNIT = "solves/s"
TOL = 1e-8
WORKLOAD = ("d=2 N=200000 nu=3/2 ell=(0.1,0.3) x~U[0,1]^2 product kernel; "
            "CG (K+0.01I)alpha=y to FP64 true resid 1e-8; step = build + preconditioner + solve")
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# per-iteration kernels on this workload, by preconditioner rank, from the
# committed ncu captures of the kernels as built
# (profiles/pc_apply_and_scan_traffic_d2_N200k_rank350.txt; a kernel or rank
# missing here has no capture of its current version)
TRAFFIC_BYTES = {
    350: {
        "k_level_scan<float,P=2,NOFF=1,product,OUT>": 44105344 + 5504,
        "k_pc_apply (z = r/s2 - L c)": 281716992 + 631936,
    },
}
FALLBACK_HBM_GBS = 6800.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """The largest x over the ranks of the process group (x itself at one rank)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws: int, steps: int, slowest_total_ms: float) -> float:
    """Whole-job throughput of weak-scaled replicas: every rank does `steps`
    units, the job lasts as long as the slowest rank."""
    return ws * steps / (slowest_total_ms / 1e3)


def flush_l2(buf):
    buf.add_(1.0)  # writes 256 MiB, twice the 129 MB L2


def run_reference(args, ws, rank):
    """The oracle timed on the host cores on a bounded sample of the workload."""
    if rank != 0:
        return 0
    import oracle
    import workloads

    p = workloads.c2()
    y = p.V[:, 0]
    cores = oracle.max_threads()
    iters_est = args.ref_iters
    rng = np.random.default_rng(0)
    per_step = []
    n_rows = 0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < args.ref_seconds:
            rows = rng.choice(p.N, 1024, replace=False)
            oracle.mvm_brute(p.X, y, p.nu, p.ell, kind=oracle.PRODUCT, rows=rows)
            done += rows.size
        dt = time.perf_counter() - t0
        t_mvm = dt / done * p.N  # seconds for one full product
        if s >= args.warmup:
            per_step.append(t_mvm * iters_est)
            n_rows += done
    t_solve = statistics.mean(per_step)
    val = 1.0 / t_solve
    sample = (f"{n_rows} output rows of the FP64 brute-force product (O(N) each) timed over {args.steps} steps, "
              f"scaled to a full product x {iters_est} CG iterations (the iteration count of the preconditioned "
              f"GPU solve; the preconditioner's own CPU cost, under 0.1% of that, is left out)")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_solve, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(p, iters, seconds):
    import oracle

    rng = np.random.default_rng(1)
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < seconds:
        rows = rng.choice(p.N, 1024, replace=False)
        oracle.mvm_brute(p.X, p.V[:, 0], p.nu, p.ell, kind=oracle.PRODUCT, rows=rows)
        done += rows.size
    dt = time.perf_counter() - t0
    t_mvm = dt / done * p.N
    return {"value": 1.0 / (t_mvm * iters), "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": (f"{done} output rows of the FP64 brute-force product in {dt:.1f} s, scaled to a full product "
                       f"({t_mvm:.1f} s) x {iters} CG iterations (the GPU solve's count; the preconditioner's "
                       f"CPU cost, under 0.1% of that, is left out)"),
            "mvm_nrhs_per_s": p.N / t_mvm, "paper_dc": paper_dc_timing(p, iters)}


def paper_dc_timing(p, iters):
    """The oracle's literal divide and conquer (the paper's algorithm, one
    thread, sorts redone at every node) on one full product of the same
    workload: context for the GPU product, not the baseline above."""
    import oracle

    try:
        t0 = time.perf_counter()
        oracle.mvm_dc(p.X, p.V[:, 0], p.nu, p.ell, kind=oracle.PRODUCT)
        t = time.perf_counter() - t0
    except Exception as e:  # context only: never lose the benchmark line for it
        return {"error": f"{type(e).__name__}: {e}"}
    return {"mvm_s": t, "mvm_nrhs_per_s": p.N / t, "solves_per_s": 1.0 / (t * iters), "threads": 1,
            "note": f"one full FP64 product by the literal divide and conquer, x {iters} CG iterations"}


def run_batched(args, local):
    """The batched workload: K problems (N log-uniform 1k-100k, d in {1,2},
    nu mixed, 16 N(0,1) right-hand sides each) solved in one batch (mixed
    precision, rank --batched-rank preconditioners), against the same solves
    one problem at a time: plain FP64, FP64 preconditioned, mixed
    preconditioned, on every problem."""
    import torch

    import workloads
    from paper_2508_01864_gb300 import batch, fgk

    torch.cuda.set_device(local)
    probs = workloads.c4(n_problems=args.batched)
    nrhs = probs[0].V.shape[1]
    t0 = time.perf_counter()
    eng = batch.BatchEngine(probs, nrhs, kind="product", precond_rank=args.batched_rank)
    t_setup = time.perf_counter() - t0
    ys = [torch.as_tensor(p.V, device="cuda") for p in probs]
    sig = [p.sigma2 for p in probs]
    rows = sum(p.N for p in probs)
    V = torch.randn(rows, nrhs, dtype=torch.float32, device="cuda")
    Y = torch.empty_like(V)
    for _ in range(3):
        eng.matvec(V, out=Y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        eng.matvec(V, out=Y)
    e1.record()
    torch.cuda.synchronize()
    mvm_ms = e0.elapsed_time(e1) / 10
    times = []
    for _ in range(max(args.steps, 1)):
        eng._free_precs()  # each timed solve builds its preconditioners
        torch.cuda.synchronize()
        e0.record()
        alphas, infos, rc = eng.solve(ys, sig, tol=TOL, maxit=200000)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        assert rc == 0, infos
    t_batch = statistics.median(times)
    # The same 64 x 16 solves one problem at a time on the same GPU, every
    # problem (no sample, no extrapolation), three ways: the plain FP64 solve
    # (no preconditioner: the baseline the batched form is set against), the
    # FP64 solve with the same rank preconditioner, and the mixed solve with
    # it; plans are built before timing (as the batch's are, in its setup) and
    # preconditioner builds are timed (as the batch's are, inside its solve).
    per = {"f64_plain": 0.0, "f64_precond": 0.0, "mixed_precond": 0.0}
    iters = {k: 0 for k in per}
    worst = {k: 0.0 for k in per}
    for i, p in enumerate(probs):
        h = fgk.fgk_build(torch.as_tensor(p.X, device="cuda"), p.nu, p.ell, kind="product")
        k = min(args.batched_rank, p.N)
        for key, mode, rk in (("f64_plain", "f64", 0), ("f64_precond", "f64", k), ("mixed_precond", "mixed", k)):
            if args.f64_plain_max and key == "f64_plain" and i >= args.f64_plain_max:
                continue
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            pc = fgk.fgk_precond_build(h, rk, p.sigma2) if rk > 0 else None
            a, _, info, rc = fgk.fgk_cg_solve(h, ys[i], p.sigma2, tol=TOL, maxit=200000, mode=mode, precond=pc)
            torch.cuda.synchronize()
            per[key] += time.perf_counter() - t1
            if pc is not None:
                fgk.fgk_precond_destroy(pc)
            assert rc == 0, (key, i, info)
            iters[key] = max(iters[key], info["iterations"])
            worst[key] = max(worst[key], info["max_true_resid"])
        fgk.fgk_destroy(h)
    n_plain = len(probs) if not args.f64_plain_max else min(args.f64_plain_max, len(probs))
    solves = len(probs) * nrhs
    out = {"metric": "batched: CG solves/sec at resid<=1e-8 (problems x rhs) and MVM N*nrhs/sec",
           "unit": "solves/s", "value": solves / t_batch, "problems": len(probs), "nrhs": nrhs,
           "rows": rows, "rhs_per_cta": eng.rpc, "autotune_ms": eng.timings, "setup_s": t_setup,
           "precond_rank": args.batched_rank,
           "batch_solve_s": t_batch, "max_iterations": max(i["iterations"] for i in infos),
           "max_true_resid": max(i["max_true_resid"] for i in infos),
           "mvm_ms": mvm_ms, "mvm_nrhs_per_s": rows * nrhs / (mvm_ms * 1e-3),
           "per_problem": {key: {"problems": (n_plain if key == "f64_plain" else len(probs)), "seconds": per[key],
                                 "solves_per_s": (n_plain if key == "f64_plain" else len(probs)) * nrhs / per[key],
                                 "max_iterations": iters[key], "max_true_resid": worst[key]}
                           for key in per},
           "workload": "first %d problems of the seeded batched workload (N log-uniform 1k-100k, d in {1,2}, "
                       "nu in {1/2,3/2,5/2}, ell log-uniform 0.05-0.5, 16 N(0,1) rhs, sigma^2=0.01, product kernel)"
                       % len(probs)}
    eng.close()
    print(json.dumps(out), flush=True)
    return 0


def run_serving(args, local):
    """Continuous-batching replay of the serving stream's first K requests:
    first as a burst (all arriving at once) to measure the sustained capacity,
    then with Poisson arrivals at 0.8x that capacity for the latencies, then at
    1.5x (an overload: the queue grows and admission holds requests back)."""
    import torch

    import workloads
    from paper_2508_01864_gb300 import serving

    torch.cuda.set_device(local)
    reqs, gaps = workloads.c5(n_requests=args.serving)
    requests = serving.to_requests(reqs, tol=TOL)
    out = {"metric": "serving: GP solves/sec at resid<=1e-8 with p50/p99 latency", "unit": "solves/s",
           "requests": len(requests), "slots": args.slots, "budget_bytes": 150e9,
           "workload": (f"first {len(requests)} requests of the seeded serving stream: N log-uniform 2k-300k, "
                        "d in 1..3, nu in {1/2,3/2,5/2}, x~U[0,1]^d, product kernel, sigma^2=0.01, mixed CG")}
    mk = lambda: serving.Server(budget_bytes=150e9, slots=args.slots, batch_max=args.serve_batch)  # noqa: E731
    out["serve_batch"] = args.serve_batch
    srv = mk()
    burst = serving.replay(srv, requests, np.zeros(len(requests)), rate=1.0)
    srv.close()
    sb = serving.summarize(burst, requests)
    out["burst"] = sb
    print(json.dumps({"phase": "burst", **sb}), file=sys.stderr, flush=True)  # progress, in case of a limit
    cap = sb.get("solves_per_s", 0.0)
    if cap > 0:
        for name, f in (("steady_0.8x", 0.8), ("overload_1.5x", 1.5)):
            srv = mk()
            res = serving.replay(srv, requests, gaps[:len(requests)], rate=f * cap)
            srv.close()
            out[name] = serving.summarize(res, requests)
            out[name]["arrival_rate_per_s"] = f * cap
            out[name]["peak_concurrency"] = srv.stats.peak_concurrency
            out[name]["peak_bytes"] = srv.stats.peak_bytes
            out[name]["batches"] = srv.stats.batches
            out[name]["batched_requests"] = srv.stats.batched
            print(json.dumps({"phase": name, **out[name]}), file=sys.stderr, flush=True)
        out["value"] = out["steady_0.8x"].get("solves_per_s")
    print(json.dumps(out), flush=True)
    return 0


def run_pcg_probe(args, local):
    """A short preconditioned mixed solve of the d=2 workload (--pcg-probe
    RANK, --pcg-maxit iterations): the launch sequence of the benchmark's
    step, small enough for ncu captures."""
    import torch

    import workloads
    from paper_2508_01864_gb300 import fgk

    torch.cuda.set_device(local)
    p = workloads.c2()
    h = fgk.fgk_build(torch.as_tensor(p.X, device="cuda"), p.nu, p.ell, kind="product")
    pc = fgk.fgk_precond_build(h, args.pcg_probe, p.sigma2)
    y = torch.as_tensor(p.V, device="cuda")
    _, _, info, rc = fgk.fgk_cg_solve(h, y, p.sigma2, tol=TOL, maxit=args.pcg_maxit, mode="mixed", precond=pc)
    torch.cuda.synchronize()
    print(json.dumps({"pcg_probe_rank": args.pcg_probe, "iterations": info["iterations"], "status": rc}), flush=True)
    fgk.fgk_precond_destroy(pc)
    fgk.fgk_destroy(h)
    return 0


def run_mvm_only(args, local):
    """W + K products in the internal order on the d=2 workload drawn with
    --mvm-only points and --mvm-nrhs columns (structure above L2 from
    N ~ 1M; used for the roofline of the whole product and for the ncu
    captures of the scan kernels): FP32 and FP64 products, the output pass
    timed alone by the library's events, and the whole FP32 product against
    the measured HBM peak with the algorithmic bytes
    B_alg = E (12 + 8 nrhs) + 8 N nrhs (structure read once, each entry's
    operand read and its contribution written once, V read and Y written)."""
    import torch

    import workloads
    from paper_2508_01864_gb300 import fgk

    torch.cuda.set_device(local)
    p = workloads.c2(N=args.mvm_only)
    nrhs = args.mvm_nrhs
    X = torch.as_tensor(p.X, device="cuda")
    h = fgk.fgk_build(X, p.nu, p.ell, kind="product")
    gen = torch.Generator(device="cuda").manual_seed(7)
    out = {"metric": "exact Matérn MVM N·nrhs/sec", "unit": "N·nrhs/s", "N": p.N, "nrhs": nrhs,
           "workload": f"d=2 N={p.N} nu=3/2 ell=(0.1,0.3) x~U[0,1]^2 product kernel, nrhs={nrhs}"}
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MiB, above L2
    for prec, dt in (("f32", torch.float32), ("f64", torch.float64)):
        Vq = torch.randn(p.N, nrhs, dtype=dt, device="cuda", generator=gen)
        Yq = torch.empty_like(Vq)
        for _ in range(args.warmup):
            fgk.fgk_matvec_q(h, Vq, prec, out=Yq)
        torch.cuda.synchronize()
        if prec == "f32":
            fgk.fgk_scan_timing(1)
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fgk.fgk_matvec_q(h, Vq, prec, out=Yq)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        out[f"{prec}_ms"] = ms
        out[f"{prec}_value"] = p.N * nrhs / (ms * 1e-3)
        if prec == "f32":
            scan_ms, scan_n = fgk.fgk_scan_timing(0)
            out["scan_out_f32_ms"] = scan_ms / max(scan_n, 1)
    info = fgk.fgk_get_info(h)
    fgk.fgk_destroy(h)
    pk, src = peaks()
    E = info["n_levels"] * p.N
    b_alg = E * (12 + 8 * nrhs) + 8 * p.N * nrhs
    b_out = E * (12 + 8 * nrhs)
    gbs = b_alg / (out["f32_ms"] * 1e-3) / 1e9
    gbs_out = b_out / (out["scan_out_f32_ms"] * 1e-3) / 1e9
    out.update({"value": out["f32_value"], "levels": info["n_levels"], "entries": E, "l2_flushed": True,
                "roofline": {"bound": "hbm", "kernel": "whole FP32 product (all launches)", "achieved": gbs,
                             "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
                             "algorithmic_bytes": b_alg, "peak_source": src},
                "scan_out_roofline": {"bound": "hbm", "achieved": gbs_out, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                      "frac": gbs_out / pk["hbm_gbs"], "algorithmic_bytes": b_out}})
    print(json.dumps(out), flush=True)
    return 0


def run_latency(args, local):
    """The d=1 workload (N = 4096, nu = 1/2, ell = 0.2, one right-hand side):
    one product K v per replay of a CUDA graph holding it (the product in the
    plan's internal order, captured once after a warm-up), each replay timed
    on its own by events; p50 / p99 over --latency replays, FP64 and FP32.
    At this size the product is launch latency, not bandwidth."""
    import torch

    import workloads
    from paper_2508_01864_gb300 import fgk

    torch.cuda.set_device(local)
    p = workloads.c1()
    h = fgk.fgk_build(torch.as_tensor(p.X, device="cuda"), p.nu, p.ell, kind="l1")
    out = {"metric": "exact Matérn MVM latency (graph replay)", "unit": "us", "workload":
           "d=1 N=4096 nu=1/2 ell=0.2 x~U[0,1], one K v", "replays": args.latency}
    side = torch.cuda.Stream()
    for prec, dt in (("f64", torch.float64), ("f32", torch.float32)):
        Vq = torch.as_tensor(p.V, dtype=dt, device="cuda").contiguous()
        Yq = torch.empty_like(Vq)
        with torch.cuda.stream(side):
            for _ in range(3):
                fgk.fgk_matvec_q(h, Vq, prec, out=Yq, stream=side)
        side.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            fgk.fgk_matvec_q(h, Vq, prec, out=Yq, stream=side)
        for _ in range(max(args.warmup, 3)):
            g.replay()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.latency):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        ts.sort()
        out[f"{prec}_p50_us"] = ts[len(ts) // 2]
        out[f"{prec}_p99_us"] = ts[min(len(ts) - 1, int(0.99 * len(ts)))]
        out[f"{prec}_min_us"] = ts[0]
        del g
    out["kernels_per_product"] = 4
    fgk.fgk_destroy(h)
    print(json.dumps(out), flush=True)
    return 0


def run_peaks(args, local):
    """Measured FP32 and FP64 FMA throughput of this GPU (fgk_fma_rate), the
    ALU roofline denominators, beside the copy bandwidth of MEASURED_PEAKS."""
    import torch

    from paper_2508_01864_gb300 import fgk

    torch.cuda.set_device(local)
    pk, src = peaks()
    out = {"metric": "measured FMA throughput", "unit": "TFLOP/s",
           "fp32_tflops": fgk.fgk_fma_rate("f32", 10) / 1e12, "fp64_tflops": fgk.fgk_fma_rate("f64", 5) / 1e12,
           "hbm_gbs": pk.get("hbm_gbs"), "hbm_source": src,
           "how": "16 independent FMA chains per thread, 8 CTAs x 256 threads per SM, best of the timed launches"}
    print(json.dumps(out), flush=True)
    return 0


def run_likelihood(args, local):
    """The likelihood pieces on the d=2 workload (N = 200000): the gradient
    products (dK/d log ell_m) V with FP32 and FP64 scans (every lengthscale),
    and the log-determinant by stochastic Lanczos quadrature with 16 probes and
    the rank-200 preconditioner, with the Hutchinson trace of the gradient from
    its solves.  Medians of --steps runs after --warmup."""
    import torch

    import workloads
    from paper_2508_01864_gb300 import fgk

    torch.cuda.set_device(local)
    p = workloads.c2()
    X = torch.as_tensor(p.X, device="cuda")
    h = fgk.fgk_build(X, p.nu, p.ell, kind="product")
    gen = torch.Generator(device="cuda").manual_seed(11)
    out = {"metric": "likelihood pieces on the d=2 workload", "workload": WORKLOAD.split(";")[0]}

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    for prec, dt in (("f32", torch.float32), ("f64", torch.float64)):
        V = torch.randn(p.N, 1, dtype=dt, device="cuda", generator=gen)
        for dim in (0, 1):
            ms = timed(lambda: fgk.fgk_matvec_dlogell(h, V, dim, prec))
            out[f"dlogell_{prec}_dim{dim}_ms"] = ms
            out[f"dlogell_{prec}_dim{dim}_nrhs_per_s"] = p.N / (ms * 1e-3)
    nprobe, rank = 16, 200
    pc = fgk.fgk_precond_build(h, rank, p.sigma2)
    k = fgk.fgk_precond_info(pc)["rank"]
    Er = torch.randn(k, nprobe, dtype=torch.float64, device="cuda", generator=gen)
    En = torch.randn(p.N, nprobe, dtype=torch.float64, device="cuda", generator=gen)
    B = fgk.fgk_precond_sample(pc, Er, En)
    res = {}

    def slq():
        res["r"] = fgk.fgk_slq_logdet(h, B, p.sigma2, 2000, tol=1e-8, pc=pc, want_solves=True)

    out["slq_ms"] = timed(slq)
    r = res["r"]
    out.update({"slq_nprobe": nprobe, "slq_precond_rank": k, "slq_logdet": r["logdet"],
                "slq_logdet_precond": r["logdet_precond"], "slq_steps_max": r["steps_max"],
                "slq_std_error": float(np.std(r["quad"]) / np.sqrt(nprobe)), "slq_max_true_resid": r["max_true_resid"]})
    # Hutchinson trace tr(A^-1 dK/d log ell_m) with N(0, P) probes: (A^-1 b)^T dK (P^-1 b)
    Z = fgk.fgk_precond_apply(pc, B)
    for dim in (0, 1):
        D = fgk.fgk_matvec_dlogell(h, Z, dim, "f64")
        sm = (r["X"] * D).sum(0).cpu().numpy()
        out[f"trace_dim{dim}"] = float(sm.mean())
        out[f"trace_dim{dim}_std_error"] = float(sm.std() / np.sqrt(nprobe))
    fgk.fgk_precond_destroy(pc)
    fgk.fgk_destroy(h)
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--precond-rank", type=int, default=350,
                    help="rank of the pivoted-Cholesky preconditioner (0: none)")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--ref-iters", type=int, default=184,
                    help="reference arm: CG iterations to scale the timed product by (the preconditioned GPU "
                         "solve's count at rank 350)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", type=int, default=0,
                    help="replay the first K requests of the serving stream (burst, then 0.8x its capacity)")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serve-batch", type=int, default=0,
                    help="--serving: solve up to this many small requests queued together as one batch (0: off)")
    ap.add_argument("--batched", type=int, default=0,
                    help="solve the first K problems of the batched workload (16 rhs each) in one batch")
    ap.add_argument("--batched-rank", type=int, default=100,
                    help="batched mode: preconditioner rank per problem (min with N/8; 0: none)")
    ap.add_argument("--f64-plain-max", type=int, default=0,
                    help="--batched: solve only the first this-many problems with the plain FP64 solve (0: all)")
    ap.add_argument("--pcg-probe", type=int, default=0,
                    help="run only a short preconditioned solve with this rank (for ncu captures)")
    ap.add_argument("--pcg-maxit", type=int, default=40)
    ap.add_argument("--likelihood", action="store_true",
                    help="time the gradient products and the log-determinant on the d=2 workload")
    ap.add_argument("--mvm-nrhs", type=int, default=1, help="columns of the --mvm-only products")
    ap.add_argument("--latency", type=int, default=0,
                    help="d=1 workload: p50/p99 of this many CUDA-graph replays of one product")
    ap.add_argument("--peaks", action="store_true", help="measured FP32/FP64 FMA throughput")
    ap.add_argument("--mvm-only", type=int, default=0,
                    help="time only the FP32 product on the d=2 workload drawn with this many points")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.likelihood:
        return run_likelihood(args, local)
    if args.latency:
        return run_latency(args, local)
    if args.peaks:
        return run_peaks(args, local)
    if args.mvm_only:
        return run_mvm_only(args, local)
    if args.pcg_probe:
        return run_pcg_probe(args, local)
    if args.serving:
        return run_serving(args, local)
    if args.batched:
        return run_batched(args, local)

    import torch
    import torch.distributed as dist

    import workloads
    from paper_2508_01864_gb300 import fgk

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            dist.barrier()

    fgk.load()
    p = workloads.c2()
    y_host = np.ascontiguousarray(p.V[:, :1])
    X = torch.as_tensor(p.X, device="cuda")
    y = torch.as_tensor(y_host, device="cuda")
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    rank_pc = args.precond_rank

    def step(Xd=X, yd=y):
        h = fgk.fgk_build(Xd, p.nu, p.ell, kind="product")
        pc = fgk.fgk_precond_build(h, rank_pc, p.sigma2) if rank_pc > 0 else None
        alpha, _, info, rc = fgk.fgk_cg_solve(h, yd, p.sigma2, tol=TOL, maxit=100000, mode=args.mode, precond=pc)
        return h, pc, alpha, info, rc

    def release(h, pc):
        if pc is not None:
            fgk.fgk_precond_destroy(pc)
        fgk.fgk_destroy(h)

    infos = []
    pc_info = None
    for _ in range(args.warmup):
        h, pc, alpha, info, rc = step()
        if pc is not None:
            pc_info = {k: v for k, v in fgk.fgk_precond_info(pc).items() if k != "pivots"}
        release(h, pc)
        assert rc == 0 and info["max_true_resid"] <= TOL, info
    torch.cuda.synchronize()

    # ---------------- timed region: device-resident inputs
    clocks = Clocks(local)
    times = []
    barrier()
    torch.cuda.synchronize()
    launches0 = fgk.fgk_kernel_launches()
    clocks.start()
    for _ in range(args.steps):
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h, pc, alpha, info, rc = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        infos.append(info)
        assert rc == 0 and info["max_true_resid"] <= TOL, info
        release(h, pc)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = fgk.fgk_kernel_launches() - launches0
    barrier()
    total_ms = max_over_ranks(sum(times), ws)
    value = job_rate(ws, args.steps, total_ms)

    # ---------------- one more step, outside the timed region, split into its phases
    # (each library call synchronises the stream, so events between the calls bound them)
    try:
        flush_l2(flush)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        h = fgk.fgk_build(X, p.nu, p.ell, kind="product")
        ev[1].record(stream)
        pc = fgk.fgk_precond_build(h, rank_pc, p.sigma2) if rank_pc > 0 else None
        ev[2].record(stream)
        _, _, info_ph, _ = fgk.fgk_cg_solve(h, y, p.sigma2, tol=TOL, maxit=100000, mode=args.mode, precond=pc)
        ev[3].record(stream)
        ev[3].synchronize()
        release(h, pc)
        phases = {"build_ms": ev[0].elapsed_time(ev[1]), "precond_ms": ev[1].elapsed_time(ev[2]),
                  "solve_ms": ev[2].elapsed_time(ev[3]), "iterations": info_ph["iterations"]}
    except Exception as e:  # a breakdown is context: never lose the benchmark line for it
        phases = {"error": f"{type(e).__name__}: {e}"}

    # ---------------- end to end through the ABI with host buffers
    Xh = torch.as_tensor(p.X).pin_memory()
    yh = torch.as_tensor(y_host).pin_memory()
    ah = torch.empty_like(yh).pin_memory()
    e2e_times = []
    for _ in range(args.steps):
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Xd = Xh.to("cuda", non_blocking=True)
        yd = yh.to("cuda", non_blocking=True)
        h, pc, alpha, info, rc = step(Xd, yd)
        ah.copy_(alpha.reshape(ah.shape), non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
        assert rc == 0
        release(h, pc)
    e2e_ms = max_over_ranks(sum(e2e_times), ws)
    e2e_val = job_rate(ws, args.steps, e2e_ms)
    h2d = Xh.numel() * 8 + yh.numel() * 8
    d2h = ah.numel() * 8

    # ---------------- the dominant kernel: FP32 output scan of the product, timed by events
    h = fgk.fgk_build(X, p.nu, p.ell, kind="product")
    info_p = fgk.fgk_get_info(h)
    Vq = torch.randn(p.N, 1, dtype=torch.float32, device="cuda")
    Yq = torch.empty_like(Vq)
    for _ in range(5):
        fgk.fgk_matvec_q(h, Vq, "f32", out=Yq)
    torch.cuda.synchronize()
    fgk.fgk_scan_timing(1)
    reps = 50
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fgk.fgk_matvec_q(h, Vq, "f32", out=Yq)
    e1.record(stream)
    torch.cuda.synchronize()
    scan_ms, scan_n = fgk.fgk_scan_timing(0)
    mvm_ms = e0.elapsed_time(e1) / reps
    V64 = Vq.double()
    Y64 = torch.empty_like(V64)
    fgk.fgk_matvec_q(h, V64, "f64", out=Y64)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(5):
        fgk.fgk_matvec_q(h, V64, "f64", out=Y64)
    e1.record(stream)
    torch.cuda.synchronize()
    mvm64_ms = e0.elapsed_time(e1) / 5
    # the preconditioner's two passes over L (t = L^T R, Z = R/s2 - L c), timed by events
    pc_kernels = {}
    if rank_pc > 0:
        pc = fgk.fgk_precond_build(h, rank_pc, p.sigma2)
        r_eff = fgk.fgk_precond_info(pc)["rank"]
        R = torch.randn(p.N, 1, dtype=torch.float64, device="cuda")
        Z = torch.empty_like(R)
        for _ in range(3):
            fgk.fgk_precond_apply(pc, R, out=Z)
        torch.cuda.synchronize()
        fgk.fgk_kernel_timing(fgk.FGK_TIMED_PC_LTR, 1)
        fgk.fgk_kernel_timing(fgk.FGK_TIMED_PC_APPLY, 1)
        for _ in range(20):
            fgk.fgk_precond_apply(pc, R, out=Z)
        torch.cuda.synchronize()
        for key, kid, bytes_per in (("k_pc_ltr (t = L^T r)", fgk.FGK_TIMED_PC_LTR, p.N * (4 * r_eff + 8)),
                                    ("k_pc_apply (z = r/s2 - L c)", fgk.FGK_TIMED_PC_APPLY,
                                     p.N * (4 * r_eff + 16))):
            ms, n = fgk.fgk_kernel_timing(kid, 0)
            avg = ms / max(n, 1)
            pc_kernels[key] = {"avg_launch_ms": avg, "algorithmic_bytes_per_launch": bytes_per,
                               "achieved_gbs": bytes_per / (avg * 1e-3) / 1e9}
        fgk.fgk_precond_destroy(pc)
    fgk.fgk_destroy(h)
    # context: the same solve without the preconditioner (one run)
    plain_ms = None
    if rank_pc > 0:
        torch.cuda.synchronize()
        e0.record(stream)
        h = fgk.fgk_build(X, p.nu, p.ell, kind="product")
        _, _, plain_info, _ = fgk.fgk_cg_solve(h, y, p.sigma2, tol=TOL, maxit=100000, mode=args.mode)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms = e0.elapsed_time(e1)
        fgk.fgk_destroy(h)
    E = info_p["n_levels"] * p.N
    bytes_per_launch = E * (4 + 4 + 4 * (p.d - 1) + 2 * 4)  # q, gap, offsets, V gather, Y update
    pk, src = peaks()
    scan_avg_ms = scan_ms / max(scan_n, 1)
    kernels = {"k_level_scan<float,P=2,NOFF=1,product,OUT>": {
        "avg_launch_ms": scan_avg_ms, "algorithmic_bytes_per_launch": bytes_per_launch,
        "achieved_gbs": bytes_per_launch / (scan_avg_ms * 1e-3) / 1e9}}
    kernels.update(pc_kernels)
    for name, k in kernels.items():
        k["frac"] = k["achieved_gbs"] / pk["hbm_gbs"]
        k["traffic"] = TRAFFIC_BYTES.get(args.precond_rank, {}).get(name)  # DRAM bytes per launch (ncu)
    # each kernel launches once per CG iteration: the dominant one takes the longest
    dom = max(kernels, key=lambda k: kernels[k]["avg_launch_ms"])
    kd = kernels[dom]
    roofline = {"bound": "hbm", "achieved": kd["achieved_gbs"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": kd["frac"], "traffic": TRAFFIC_BYTES.get(args.precond_rank, {}).get(dom), "kernel": dom,
                "peak_source": f"{src} (hbm_gbs, copy burst)", "avg_launch_ms": kd["avg_launch_ms"],
                "algorithmic_bytes_per_launch": kd["algorithmic_bytes_per_launch"], "per_iteration_kernels": kernels}

    if rank != 0:
        return 0
    iters = int(statistics.median(i["iterations"] for i in infos))
    cpu = None if args.no_cpu_baseline else cpu_baseline(p, iters, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.mode == "mixed" else "f64",
        "data": "synthetic (seeded; stands in for the paper's uniform [0,1]^d simulations)",
        "config": {"workload": WORKLOAD, "mode": args.mode, "precond_rank": rank_pc, "parallelism": f"replicas x{ws}",
                   "l2": "flushed between timed steps (256 MiB write)", "global_batch": ws, "seq_len": None},
        "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clk,
        "mvm": {"f32_nrhs_per_s": p.N / (mvm_ms * 1e-3), "f32_ms": mvm_ms, "f64_nrhs_per_s": p.N / (mvm64_ms * 1e-3),
                "f64_ms": mvm64_ms, "structure_entries": E},
        "cg": {"iterations": iters, "refinements": infos[-1]["refinements"],
               "true_resid": infos[-1]["max_true_resid"]},
        "precond": pc_info,
        "unpreconditioned_step_ms": plain_ms,
        "phases_ms": phases,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
