"""Scheduling logic of the continuous-batching server, without a GPU: a fake
executor stands in for the device work."""

import threading
import time

import numpy as np

from paper_2508_01864_gb300 import serving


def make_requests(n, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        N = int(rng.integers(50, 400))
        X = rng.uniform(size=(N, 2))
        reqs.append(serving.Request(i, X, rng.standard_normal(N), 1.5, np.array([0.2, 0.2]), 0.01))
    return reqs


class FakeDevice:
    """Sleeps in proportion to N and records the memory in use."""

    def __init__(self, per_point=2e-5):
        self.per_point = per_point
        self.lock = threading.Lock()
        self.in_use = 0
        self.peak = 0
        self.concurrent = 0
        self.peak_concurrent = 0
        self.order = []

    def estimate(self, req):
        return req.N * 1000

    def run(self, req):
        with self.lock:
            self.in_use += self.estimate(req)
            self.concurrent += 1
            self.peak = max(self.peak, self.in_use)
            self.peak_concurrent = max(self.peak_concurrent, self.concurrent)
            self.order.append(req.rid)
        time.sleep(req.N * self.per_point)
        if req.rid == 5:
            raise RuntimeError("injected failure")
        with self.lock:
            self.in_use -= self.estimate(req)
            self.concurrent -= 1
        return req.y.copy(), {"iterations": 1}, 0


def test_budget_slots_and_fifo():
    dev = FakeDevice()
    budget = 700 * 1000  # at most ~2-3 requests at once
    srv = serving.Server(budget_bytes=budget, slots=3, executor=dev.run, estimator=dev.estimate)
    reqs = make_requests(20)
    futs = [srv.submit(r) for r in reqs]
    res = [f.result(timeout=60) for f in futs]
    srv.close()
    assert srv.stats.completed == 20 and srv.stats.admitted == 20
    assert srv.stats.peak_bytes <= budget
    assert srv.stats.peak_concurrency <= 3
    assert dev.order == sorted(dev.order)  # admitted in arrival order
    failed = [r for r in res if r.error]
    assert [r.rid for r in failed] == [5]  # the failure is reported, the rest are served
    for r in res:
        if not r.error:
            assert np.array_equal(r.alpha, reqs[r.rid].y)
            assert r.finished >= r.admitted >= r.arrival


def test_oversized_request_rejected_and_summary():
    dev = FakeDevice(per_point=1e-6)
    srv = serving.Server(budget_bytes=500 * 1000, slots=2, executor=dev.run, estimator=dev.estimate)
    reqs = make_requests(6, seed=3)
    reqs[2].X = np.random.default_rng(1).uniform(size=(1000, 2))
    reqs[2].y = np.zeros(1000)
    out = serving.replay(srv, reqs, np.ones(6), rate=1000.0)
    srv.close()
    assert out[2].error and "budget" in out[2].error and srv.stats.rejected == 1
    s = serving.summarize(out)
    assert s["completed"] == 4  # 2 rejected/failed (rid 2 oversized, rid 5 raises)
    assert s["p99_s"] >= s["p50_s"] > 0


def test_cancelled_requests_never_reach_the_device_and_free_nothing_twice():
    dev = FakeDevice(per_point=2e-4)
    srv = serving.Server(budget_bytes=10**9, slots=1, executor=dev.run, estimator=dev.estimate)
    reqs = make_requests(6, seed=3)
    for r in reqs:
        r.rid += 100  # no injected failure (rid 5) here
    futs = [srv.submit(r) for r in reqs]
    time.sleep(0.01)  # the first is admitted; the others wait for the single slot
    assert srv.cancel(reqs[3].rid) and srv.cancel(reqs[5].rid)
    assert not srv.cancel(reqs[3].rid)  # already cancelled
    assert not srv.cancel(12345)        # unknown
    res = [f.result(timeout=30) for f in futs]
    srv.close()
    assert [r.error for r in res].count("cancelled") == 2
    assert res[3].error == "cancelled" and res[5].error == "cancelled"
    assert reqs[3].rid not in dev.order and reqs[5].rid not in dev.order
    assert all(r.error is None for i, r in enumerate(res) if i not in (3, 5))
    assert srv.stats.cancelled == 2 and srv.stats.completed == 4 and srv._used == 0 and srv._running == 0


def test_a_running_request_cannot_be_cancelled():
    gate = threading.Event()

    def slow(req):
        gate.wait(10)
        return req.y.copy(), {}, 0

    srv = serving.Server(budget_bytes=10**9, slots=2, executor=slow, estimator=lambda r: 1)
    r = make_requests(1)[0]
    fut = srv.submit(r)
    time.sleep(0.05)
    assert not srv.cancel(r.rid)
    gate.set()
    assert fut.result(timeout=10).error is None
    srv.close()


def test_an_out_of_memory_failure_releases_its_budget():
    """An executor failing as the library does when its allocator runs dry
    (FGK_ERR_OOM): the request is reported failed, its bytes return to the
    budget and later requests are admitted."""
    from paper_2508_01864_gb300 import fgk

    calls = []

    def oom_once(req):
        calls.append(req.rid)
        if req.rid == 0:
            raise fgk.FgkError(-3, "fgk_cg_solve: workspace allocation failed")
        return req.y.copy(), {}, 0

    srv = serving.Server(budget_bytes=1000, slots=4, executor=oom_once, estimator=lambda r: 600)
    reqs = make_requests(4, seed=5)
    res = [srv.submit(r).result(timeout=30) for r in reqs]
    srv.close()
    assert res[0].error is not None and "allocation failed" in res[0].error
    assert all(r.error is None for r in res[1:])
    assert calls == [0, 1, 2, 3] and srv._used == 0


def test_close_runs_what_was_queued_and_refuses_what_comes_after():
    dev = FakeDevice(per_point=1e-5)
    srv = serving.Server(budget_bytes=10**9, slots=2, executor=dev.run, estimator=dev.estimate)
    reqs = [r for r in make_requests(8, seed=3) if r.rid != 5]
    futs = [srv.submit(r) for r in reqs]
    srv.close()
    assert all(f.done() and f.result(timeout=0).error is None for f in futs)
    try:
        srv.submit(make_requests(1, seed=4)[0])
        raise AssertionError("a closed server took a request")
    except RuntimeError as e:
        assert "closed" in str(e)


def test_submissions_racing_close_either_run_or_are_refused():
    """Four threads submit while the server closes: every request that was
    taken resolves (none is left behind the end marker), the rest raise."""
    dev = FakeDevice(per_point=0.0)
    srv = serving.Server(budget_bytes=10**9, slots=3, executor=dev.run, estimator=dev.estimate)
    reqs = [r for r in make_requests(400, seed=5) if r.rid != 5]
    taken, refused, lock = [], [], threading.Lock()

    def client(part):
        for r in part:
            try:
                f = srv.submit(r)
                with lock:
                    taken.append(f)
            except RuntimeError:
                with lock:
                    refused.append(r.rid)

    threads = [threading.Thread(target=client, args=(reqs[i::4],)) for i in range(4)]
    for t in threads:
        t.start()
    time.sleep(0.002)
    srv.close()
    for t in threads:
        t.join(timeout=30)
    assert len(taken) + len(refused) == len(reqs)
    assert all(f.result(timeout=30).error is None for f in taken)
    assert srv.stats.completed == len(taken)


class FakeBatchDevice(FakeDevice):
    """Records the groups the server hands to the batch executor."""

    def __init__(self, per_point=2e-5):
        super().__init__(per_point)
        self.groups = []

    def run_group(self, reqs):
        with self.lock:
            self.groups.append([r.rid for r in reqs])
        time.sleep(sum(r.N for r in reqs) * self.per_point * 0.3)
        return [(r.y.copy(), {"iterations": 1}, 0) for r in reqs]


def test_small_requests_queued_together_share_a_batch_in_fifo_order():
    dev = FakeBatchDevice()
    reqs = make_requests(40, seed=3)
    big = {4, 17, 30}  # not batchable: above batch_max_n
    for r in reqs:
        if r.rid in big:
            r.X = np.random.default_rng(r.rid).uniform(size=(900, 2))
            r.y = np.zeros(900)
    srv = serving.Server(budget_bytes=1e12, slots=1, executor=dev.run, estimator=dev.estimate,
                         batch_max=5, batch_max_n=500, batch_executor=dev.run_group)
    futs = [srv.submit(r) for r in reqs]
    res = [f.result(timeout=60) for f in futs]
    srv.close()
    assert [r.rid for r in res] == list(range(40))
    assert all(r.error is None or r.rid == 5 for r in res)  # rid 5 fails only when it runs alone
    # every request ran exactly once, singles and groups together
    ran = [rid for rid in dev.order] + [rid for g in dev.groups for rid in g]
    assert sorted(ran) == list(range(40))
    # groups: at most batch_max, only batchable requests, consecutive and in submission order
    assert dev.groups and all(2 <= len(g) <= 5 for g in dev.groups)
    for g in dev.groups:
        assert not set(g) & big
        assert g == list(range(g[0], g[0] + len(g)))
    # with one slot, work starts in submission order
    starts = sorted(dev.groups + [[rid] for rid in dev.order], key=lambda g: g[0])
    assert [rid for g in starts for rid in g] == list(range(40))
    assert srv.stats.batches == len(dev.groups) and srv.stats.batched == sum(map(len, dev.groups))


def test_batched_groups_respect_the_budget_and_close_cleanly():
    dev = FakeBatchDevice()
    reqs = make_requests(30, seed=4)
    budget = 1200 * 1000  # a group's summed estimate must fit
    srv = serving.Server(budget_bytes=budget, slots=2, executor=dev.run, estimator=dev.estimate,
                         batch_max=8, batch_max_n=1000, batch_executor=dev.run_group)
    futs = [srv.submit(r) for r in reqs]
    srv.close()  # the end marker may be drawn while a group forms
    res = [f.result(timeout=60) for f in futs]
    assert len(res) == 30 and srv.stats.completed == 30
    for g in dev.groups:
        assert sum(reqs[i].N * 1000 for i in g) <= budget
    assert srv.stats.peak_bytes <= budget
