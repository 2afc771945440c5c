"""Continuous-batching server for GP solves on one GPU.

Requests (a point set, a right-hand side and kernel parameters) arrive over
time.  The dispatcher admits them in arrival order as soon as a slot is free
and the device-memory budget has room for the request's estimated footprint
(``fgk_bytes_estimate`` plus the preconditioner's factor).  Each admitted
request runs on a worker thread with its own CUDA stream: host->device
copies, ``fgk_build`` (its sort and dominance structure stay on the device
for the request's lifetime), the pivoted-Cholesky preconditioner
(``fgk_precond_build``, rank min(precond_rank, N / 8); 0 turns it off),
the preconditioned solve (its CG state stays on the device), the
device->host copy of alpha, ``fgk_destroy``.  The solves of all admitted requests overlap on the
device; a request leaves as soon as its own solve converges, freeing its slot
and memory for the next arrival.  Latency is measured from arrival to the
result being on the host.

With ``batch_max`` > 1 the server also shares launches between small
requests: when the request at the head of the queue is batchable (d <= 2,
nu <= 5/2, N <= ``batch_max_n``), the dispatcher admits it together with the
batchable requests queued right behind it (up to ``batch_max``, within the
budget; FIFO order is kept), and one worker solves the group as one libfgk
batch -- one launch per phase of the product for all of them, one captured
CG iteration -- each with its own preconditioner.  A batched request's
product sums its levels with atomics, so its alpha can differ in the last
bits from the same request solved alone; it meets the same tolerance.

All GPU work happens inside libfgk's kernels; this module only schedules.  The
executors are injectable so the scheduling logic can be exercised without a GPU.
"""

from __future__ import annotations

import queue
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    X: np.ndarray  # N x d float64
    y: np.ndarray  # N float64
    nu: float
    ell: np.ndarray
    sigma2: float
    kind: str = "product"
    tol: float = 1e-8
    arrival: float = 0.0  # set by the server when submitted

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]


@dataclass
class Result:
    rid: int
    alpha: np.ndarray | None
    info: dict
    status: int
    arrival: float
    admitted: float
    finished: float
    error: str | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class Stats:
    submitted: int = 0
    admitted: int = 0
    completed: int = 0
    rejected: int = 0
    cancelled: int = 0
    peak_bytes: int = 0
    peak_concurrency: int = 0
    batches: int = 0   # groups solved as one batch
    batched: int = 0   # requests in those groups
    results: list = field(default_factory=list)


def precond_rank_for(N: int, precond_rank: int) -> int:
    return max(0, min(int(precond_rank), int(N) // 8))


def gpu_executor(mode: str = "mixed", maxit: int = 200000, precond_rank: int = 100):
    """The real executor: one request, start to end, on a private stream."""
    import torch

    from . import fgk

    def run(req: Request):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            X = torch.as_tensor(np.ascontiguousarray(req.X)).pin_memory().to("cuda", non_blocking=True)
            y = torch.as_tensor(np.ascontiguousarray(req.y).reshape(-1, 1)).pin_memory().to("cuda",
                                                                                           non_blocking=True)
            h = fgk.fgk_build(X, req.nu, req.ell, kind=req.kind, stream=stream)
            pc = None
            try:
                k = precond_rank_for(req.N, precond_rank)
                if k > 0 and req.sigma2 > 0:
                    pc = fgk.fgk_precond_build(h, k, req.sigma2, stream=stream)
                alpha, _, info, rc = fgk.fgk_cg_solve(h, y, req.sigma2, tol=req.tol, maxit=maxit, mode=mode,
                                                      stream=stream, precond=pc)
                a = alpha.cpu().numpy().reshape(-1)
            finally:
                if pc is not None:
                    fgk.fgk_precond_destroy(pc)
                fgk.fgk_destroy(h)
        return a, info, rc

    return run


def batchable(req: Request, max_n: int) -> bool:
    """Whether the batched engine takes the request (d <= 2, nu <= 5/2)."""
    return req.d <= 2 and req.nu <= 2.5 and req.N <= max_n and req.sigma2 > 0


def gpu_batch_executor(maxit: int = 200000, precond_rank: int = 100):
    """Several small requests at once: one plan and one preconditioner each,
    one libfgk batch for their products, one mixed batched CG solve; returns
    one (alpha, info, status) per request, in order."""
    import torch

    from . import fgk

    def run(reqs: list):
        stream = torch.cuda.Stream()
        handles, pcs, b = [], [], None
        with torch.cuda.stream(stream):
            try:
                ys = []
                for req in reqs:
                    X = torch.as_tensor(np.ascontiguousarray(req.X)).pin_memory().to("cuda", non_blocking=True)
                    ys.append(torch.as_tensor(np.ascontiguousarray(req.y).reshape(-1, 1)).pin_memory().to(
                        "cuda", non_blocking=True))
                    handles.append(fgk.fgk_build(X, req.nu, req.ell, kind=req.kind, stream=stream))
                b = fgk.fgk_batch_create(handles, 1, 1, stream=stream)
                for h, req in zip(handles, reqs):
                    pcs.append(fgk.fgk_precond_build(h, precond_rank_for(req.N, precond_rank), req.sigma2,
                                                     stream=stream))
                tol = min(req.tol for req in reqs)
                alphas, infos, _ = fgk.fgk_batch_cg_solve(b, ys, [req.sigma2 for req in reqs], tol=tol, maxit=maxit,
                                                           stream=stream, precs=pcs)
                out = []
                for a, info, req in zip(alphas, infos, reqs):
                    ok = max(info["true_resid"]) <= req.tol
                    out.append((a.cpu().numpy().reshape(-1), info, 0 if ok else 1))
            finally:
                for q in pcs:
                    fgk.fgk_precond_destroy(q)
                if b is not None:
                    fgk.fgk_batch_destroy(b)
                for h in handles:
                    fgk.fgk_destroy(h)
        return out

    return run


def gpu_estimator(nrhs_cols: int = 1, precond_rank: int = 100):
    from . import fgk

    def est(req: Request) -> int:
        k = precond_rank_for(req.N, precond_rank)
        # factor (FP32), residual diagonal, the build's exponential tables and Gram partials
        # (<= 64 x k x k), apply scratch (the float pairs of R's rows and the per-CTA partials)
        pc_bytes = (req.N * k * 4 + req.N * 8 + 16 * req.d * req.N + 66 * k * k * 8 + 304 * k * 8
                    + req.N * 8 * nrhs_cols + (1 << 20) if k > 0 else 0)
        return (int(fgk.fgk_bytes_estimate(req.N, req.d, req.nu, req.kind, nrhs_cols)) + req.N * (req.d + 3) * 8
                + pc_bytes)

    return est


class Server:
    """FIFO admission by slots and a device-memory budget; workers overlap."""

    def __init__(self, budget_bytes: float = 150e9, slots: int = 8, executor=None, estimator=None,
                 batch_max: int = 0, batch_max_n: int = 20000, batch_executor=None):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.executor = executor or gpu_executor()
        self.estimator = estimator or gpu_estimator()
        # batch_max > 1: small requests queued together share one batched solve
        self.batch_max = int(batch_max)
        self.batch_max_n = int(batch_max_n)
        self.batch_executor = batch_executor or (gpu_batch_executor() if self.batch_max > 1 else None)
        self._carry = None  # an item taken from the queue while forming a group, next in line
        self._has_carry = False  # (the item may be the end marker None)
        self.stats = Stats()
        self._pending: queue.Queue = queue.Queue()
        self._lock = threading.Condition()
        self._used = 0
        self._running = 0
        self._pool = ThreadPoolExecutor(max_workers=self.slots)
        self._stop = False
        self._futures: dict[int, Future] = {}
        self._cancelled: set[int] = set()
        self._admitted: set[int] = set()
        self._dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self._dispatcher.start()

    # ------------------------------------------------------------ client side
    def submit(self, req: Request) -> Future:
        """Queue a request; its future resolves with a Result.  Raises
        RuntimeError once the server is closed (nothing would run it)."""
        fut: Future = Future()
        need = self.estimator(req)
        req.arrival = time.perf_counter()
        with self._lock:
            if self._stop:
                raise RuntimeError("the server is closed")
            self.stats.submitted += 1
            if need > self.budget:
                self.stats.rejected += 1
                fut.set_result(Result(req.rid, None, {}, -1, req.arrival, req.arrival, req.arrival,
                                      error=f"needs {need} bytes, more than the {self.budget}-byte budget"))
                return fut
            self._futures[req.rid] = fut
            # queued under the lock, so that it cannot land behind close()'s end marker
            self._pending.put((req, need))
        return fut

    def cancel(self, rid: int) -> bool:
        """Withdraw a request that has not been admitted yet: its future
        resolves at once with the error "cancelled" and it never reaches the
        device.  A request already admitted runs to completion (its device
        work is in flight); returns False then, or for an unknown rid."""
        with self._lock:
            if rid in self._admitted or rid not in self._futures or rid in self._cancelled:
                return False
            self._cancelled.add(rid)
            fut = self._futures.pop(rid)
            self.stats.cancelled += 1
            self._lock.notify_all()  # the dispatcher may be holding it at the head of the queue
        now = time.perf_counter()
        fut.set_result(Result(rid, None, {}, -1, now, now, now, error="cancelled"))
        return True

    def close(self, wait: bool = True):
        """Stop taking requests; those already queued are still admitted and
        run, then the dispatcher and the workers end."""
        with self._lock:
            self._stop = True
            self._pending.put(None)
        self._dispatcher.join()
        self._pool.shutdown(wait=wait)

    # ------------------------------------------------------------ scheduling
    def _next_item(self):
        if self._has_carry:
            item, self._carry, self._has_carry = self._carry, None, False
            return item
        return self._pending.get()

    def _dispatch(self):
        while True:
            item = self._next_item()
            if item is None:
                return
            req, need = item
            with self._lock:
                while (req.rid not in self._cancelled
                       and (self._running >= self.slots or self._used + need > self.budget)):
                    self._lock.wait()
                if req.rid in self._cancelled:
                    self._cancelled.discard(req.rid)
                    continue
                group = [(req, need)]
                if self.batch_max > 1 and batchable(req, self.batch_max_n):
                    # the batchable requests already queued right behind it, in order
                    total = need
                    while len(group) < self.batch_max:
                        try:
                            nxt = self._pending.get_nowait()
                        except queue.Empty:
                            break
                        if nxt is None or not batchable(nxt[0], self.batch_max_n) or \
                                self._used + total + nxt[1] > self.budget:
                            self._carry, self._has_carry = nxt, True  # next in line, in its turn
                            break
                        if nxt[0].rid in self._cancelled:
                            self._cancelled.discard(nxt[0].rid)
                            continue
                        group.append(nxt)
                        total += nxt[1]
                for r, n in group:
                    self._admitted.add(r.rid)
                    self._used += n
                    self.stats.admitted += 1
                self._running += 1
                self.stats.peak_bytes = max(self.stats.peak_bytes, self._used)
                self.stats.peak_concurrency = max(self.stats.peak_concurrency, self._running)
                if len(group) > 1:
                    self.stats.batches += 1
                    self.stats.batched += len(group)
            admitted = time.perf_counter()
            if len(group) == 1:
                self._pool.submit(self._work, req, need, admitted)
            else:
                self._pool.submit(self._work_group, group, admitted)

    def _work(self, req: Request, need: int, admitted: float):
        err = None
        alpha, info, rc = None, {}, -1
        try:
            alpha, info, rc = self.executor(req)
        except Exception as e:  # a failed request is reported, the server keeps going
            err = f"{type(e).__name__}: {e}"
        finished = time.perf_counter()
        res = Result(req.rid, alpha, info, rc, req.arrival, admitted, finished, err)
        with self._lock:
            self._used -= need
            self._running -= 1
            self._admitted.discard(req.rid)
            self.stats.completed += 1
            self.stats.results.append(res)
            fut = self._futures.pop(req.rid, None)
            self._lock.notify_all()
        if fut is not None:
            fut.set_result(res)

    def _work_group(self, group: list, admitted: float):
        reqs = [r for r, _ in group]
        outs, err = None, None
        try:
            outs = self.batch_executor(reqs)
        except Exception as e:  # the whole group is reported failed, the server keeps going
            err = f"{type(e).__name__}: {e}"
        finished = time.perf_counter()
        results = []
        for i, req in enumerate(reqs):
            alpha, info, rc = outs[i] if outs is not None else (None, {}, -1)
            results.append(Result(req.rid, alpha, info, rc, req.arrival, admitted, finished, err))
        futs = []
        with self._lock:
            self._running -= 1
            for (req, need), res in zip(group, results):
                self._used -= need
                self._admitted.discard(req.rid)
                self.stats.completed += 1
                self.stats.results.append(res)
                futs.append(self._futures.pop(req.rid, None))
            self._lock.notify_all()
        for fut, res in zip(futs, results):
            if fut is not None:
                fut.set_result(res)


def replay(server: Server, requests: list[Request], gaps: np.ndarray, rate: float) -> list[Result]:
    """Submit requests at the arrival times given by unit-mean gaps scaled to
    ``rate`` requests per second; return the results in request order."""
    t0 = time.perf_counter()
    arrivals = np.cumsum(np.asarray(gaps, dtype=np.float64) / rate)
    futs = []
    for req, at in zip(requests, arrivals):
        delay = t0 + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        futs.append(server.submit(req))
    return [f.result() for f in futs]


def summarize(results: list[Result], requests: list[Request] | None = None) -> dict:
    """Latency percentiles (arrival to result on the host), the time spent
    queued (arrival to admission) and solving (admission to result), the
    throughput over the replay's span; with the requests, the same per
    variant (d, nu) and the variants of the requests at or above the p99."""
    ok = [r for r in results if r.error is None and r.status in (0, 1)]
    if not ok:
        return {"completed": 0}
    lat = np.array([r.latency for r in ok])
    wait = np.array([r.admitted - r.arrival for r in ok])
    serve = np.array([r.finished - r.admitted for r in ok])
    span = max(r.finished for r in ok) - min(r.arrival for r in ok)
    out = {"completed": len(ok), "failed": len(results) - len(ok),
           "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "mean_s": float(lat.mean()), "queued_p50_s": float(np.percentile(wait, 50)),
           "queued_p99_s": float(np.percentile(wait, 99)), "solve_p50_s": float(np.percentile(serve, 50)),
           "solve_p99_s": float(np.percentile(serve, 99)), "makespan_s": float(span), "solves_per_s": len(ok) / span}
    if requests is not None:
        by_id = {q.rid: q for q in requests}
        groups: dict[str, list[float]] = {}
        for r in ok:
            q = by_id[r.rid]
            groups.setdefault(f"d={q.d} nu={q.nu:g}", []).append(r.latency)
        out["by_variant"] = {k: {"n": len(v), "p50_s": float(np.percentile(v, 50)),
                                 "p99_s": float(np.percentile(v, 99))} for k, v in sorted(groups.items())}
        p99 = out["p99_s"]
        tail: dict[str, int] = {}
        for r in ok:
            if r.latency >= p99:
                q = by_id[r.rid]
                key = f"d={q.d} nu={q.nu:g}"
                tail[key] = tail.get(key, 0) + 1
        out["at_or_above_p99"] = tail
    return out


def to_requests(problems, tol: float = 1e-8, kind: str = "product") -> list[Request]:
    out = []
    for i, p in enumerate(problems):
        out.append(Request(i, p.X, p.V[:, 0], p.nu, p.ell, p.sigma2, kind=kind, tol=tol))
    return out


__all__ = ["Request", "Result", "Server", "Stats", "batchable", "gpu_batch_executor", "gpu_executor", "gpu_estimator",
           "replay", "summarize", "to_requests"]
