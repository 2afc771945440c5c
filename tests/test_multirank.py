"""The benchmark's multi-rank path on the CPU: two gloo ranks of weak-scaled
replicas agree on the slowest rank's time (max over ranks, no data-path
collective besides it) and report the whole-job rate from it; the
reference arm runs on rank 0 only; the CPU context timing of the paper's
divide and conquer reports one full product.  No GPU."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = 100.0 + 37.5 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(local_ms, ws, device="cpu")
        out_q.put((rank, slowest, bench.job_rate(ws, 5, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [137.5, 137.5]
    # 2 ranks x 5 steps in 137.5 ms
    assert res[0][2] == pytest.approx(2 * 5 / 0.1375)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(1, 4, 500.0) == pytest.approx(8.0)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        ref_iters, warmup, steps, ref_seconds = 1, 0, 1, 0.0

    assert bench.run_reference(A(), 2, 1) == 0  # rank 1: no work, exit code 0


def test_paper_dc_timing_reports_one_full_product():
    sys.path.insert(0, ROOT)
    import bench
    import workloads

    p = workloads.c2(N=3000)
    r = bench.paper_dc_timing(p, 100)
    assert set(r) >= {"mvm_s", "mvm_nrhs_per_s", "solves_per_s", "threads"} and r["threads"] == 1
    assert r["solves_per_s"] == pytest.approx(1.0 / (100 * r["mvm_s"]))
    assert r["mvm_nrhs_per_s"] == pytest.approx(3000 / r["mvm_s"])


def test_cpu_baseline_reports_the_contract_fields():
    sys.path.insert(0, ROOT)
    import bench
    import workloads

    p = workloads.c2(N=3000)
    cb = bench.cpu_baseline(p, 50, 0.2)
    assert cb["kind"] == "oracle" and cb["unit"] == bench.UNIT and cb["cores"] >= 1
    assert cb["value"] > 0 and "output rows" in cb["sample"]
    # the rate is one full product per iteration: value = mvm rate / (N x iterations)
    assert cb["value"] == pytest.approx(cb["mvm_nrhs_per_s"] / (p.N * 50), rel=1e-12)
    assert cb["paper_dc"]["threads"] == 1 and cb["paper_dc"]["solves_per_s"] > 0
