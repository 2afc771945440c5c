"""The continuous-batching server on the GPU: requests admitted while others
run, overlapping on the device, each result the same alone and in the mix:
bit for bit (every reduction of a solve, the level sum of each product
included, runs in a fixed order, and the solver's path does not depend on
timing), and both meeting the solve tolerance, checked with the oracle's
product."""

import numpy as np
import pytest

import workloads
from paper_2508_01864_gb300 import serving

pytestmark = pytest.mark.gpu


def test_results_alone_and_in_the_mix(fgk_mod, orc):
    reqs, gaps = workloads.c5(n_requests=10, n_min=2000, n_max=12000)
    requests = serving.to_requests(reqs, tol=1e-8)
    run = serving.gpu_executor(mode="mixed")
    alone = [run(r) for r in requests]
    est = serving.gpu_estimator()
    budget = 2.5 * max(est(r) for r in requests)
    srv = serving.Server(budget_bytes=budget, slots=4, executor=run, estimator=est)
    mixed = serving.replay(srv, requests, gaps, rate=200.0)
    srv.close()
    assert srv.stats.completed == len(requests)
    assert srv.stats.peak_bytes <= budget
    assert srv.stats.peak_concurrency >= 2  # the solves overlapped
    for r, (a_alone, info_alone, rc_alone), res in zip(requests, alone, mixed):
        assert res.error is None and res.status == 0 and rc_alone == 0
        for a in (a_alone, res.alpha):
            Ka = orc.mvm_brute(r.X, a, r.nu, r.ell, kind=orc.PRODUCT if r.d > 1 else orc.L1)
            resid = np.linalg.norm(r.y - Ka - r.sigma2 * a) / np.linalg.norm(r.y)
            assert resid <= 1e-8, (r.rid, resid)
        assert np.array_equal(np.asarray(res.alpha).view(np.uint64), np.asarray(a_alone).view(np.uint64)), r.rid
    s = serving.summarize(mixed)
    assert s["completed"] == len(requests) and s["p99_s"] >= s["p50_s"]


def test_small_requests_solved_in_shared_batches(fgk_mod, orc):
    """batch_max > 1: the small requests queued together are solved as one
    libfgk batch (one launch per product phase for all of them, each with its
    own preconditioner); every one meets the tolerance by the oracle's
    product, and the large ones still run alone."""
    reqs, gaps = workloads.c5(seed=11, n_requests=16, n_min=2000, n_max=30000)
    requests = serving.to_requests(reqs, tol=1e-8)
    srv = serving.Server(budget_bytes=150e9, slots=1, batch_max=6, batch_max_n=12000)
    results = serving.replay(srv, requests, np.zeros(len(requests)), rate=1.0)  # a burst: they queue
    srv.close()
    assert srv.stats.completed == len(requests) and srv.stats.batches >= 1
    for r, res in zip(requests, results):
        assert res.error is None and res.status == 0, (r.rid, res.error, res.info)
        Ka = orc.mvm_brute(r.X, res.alpha, r.nu, r.ell, kind=orc.PRODUCT if r.d > 1 else orc.L1)
        resid = np.linalg.norm(r.y - Ka - r.sigma2 * res.alpha) / np.linalg.norm(r.y)
        assert resid <= 1e-8, (r.rid, resid)
