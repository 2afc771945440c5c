"""Batched solves of many GP problems with an autotuned launch shape.

``BatchEngine`` builds one plan per problem, groups them into one libfgk batch
(one launch per phase of the product for the whole batch, the CG iteration a
captured CUDA graph) and solves all problems and right-hand sides together,
optionally with one pivoted-Cholesky preconditioner per problem (rank
min(precond_rank, N / 8), built for the sigma^2 of the solve and kept for
later solves with the same sigma^2).

The autotuner chooses how many right-hand sides one CTA scans (more per CTA
reuses each tile's loaded structure; fewer gives more CTAs): it times the
batched FP32 product for each candidate with CUDA events and keeps the
fastest.  Results are cached in a JSON file keyed by the GPU, nrhs, the mix
of kernel variants and the size bucket of the batch
(``FGK_AUTOTUNE_CACHE``, default ``_lib/autotune.json`` in this package).
"""

from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("FGK_AUTOTUNE_CACHE", os.path.join(_HERE, "_lib", "autotune.json"))


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(entries: dict, path: str | None = None) -> None:
    path = path or cache_path()
    with _lock:
        cur = load_cache(path)
        cur.update(entries)
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cur, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def tune_key(gpu: str, nrhs: int, variants: list, total_rows: int) -> str:
    mix = ",".join(f"{k}x{v}" for k, v in sorted(_count(variants).items()))
    bucket = int(math.log2(max(total_rows, 1)))
    return f"{gpu}|nrhs={nrhs}|mix={mix}|rows=2^{bucket}"


def _count(xs):
    out = {}
    for x in xs:
        out[x] = out.get(x, 0) + 1
    return out


def candidates(nrhs: int) -> list:
    c, k = [], nrhs
    while k >= 1:
        c.append(k)
        k //= 2
    return c


def pick(timings: dict) -> int:
    """The candidate with the smallest time (ties: more rhs per CTA)."""
    return min(timings, key=lambda k: (timings[k], -k))


class BatchEngine:
    def __init__(self, problems, nrhs: int, kind: str = "product", autotune: bool = True, reps: int = 5,
                 stream=None, precond_rank: int = 0):
        import torch

        from . import fgk

        self.fgk = fgk
        self.problems = problems
        self.nrhs = int(nrhs)
        self.precond_rank = int(precond_rank)
        self.precs = None
        self.precs_sigma2 = None
        self.stream = stream
        self.batch = None
        self.handles = []
        try:
            for p in problems:
                self.handles.append(fgk.fgk_build(torch.as_tensor(p.X, device="cuda"), p.nu, p.ell, kind=kind,
                                                  stream=stream))
            self._setup(problems, autotune, reps, stream)
        except BaseException:
            self.close()  # a failed build, tuning or batch: free what was made
            raise

    def _setup(self, problems, autotune, reps, stream):
        import torch

        fgk = self.fgk
        variants = [f"d{p.d}nu{p.nu}" for p in problems]
        rows = sum(p.N for p in problems)
        gpu = torch.cuda.get_device_name()
        self.key = tune_key(gpu, self.nrhs, variants, rows)
        self.timings = {}
        cached = load_cache().get(self.key)
        if cached is not None and not autotune:
            self.rpc = int(cached["rhs_per_cta"])
        elif cached is not None:
            self.rpc = int(cached["rhs_per_cta"])
            self.timings = cached.get("timings_ms", {})
        else:
            self.rpc = self._tune(reps, stream) if autotune else self.nrhs
        self.batch = fgk.fgk_batch_create(self.handles, self.nrhs, self.rpc, stream=stream)

    def _tune(self, reps, stream) -> int:
        import torch

        fgk = self.fgk
        rows = sum(p.N for p in self.problems)
        V = torch.randn(rows, self.nrhs, dtype=torch.float32, device="cuda")
        Y = torch.empty_like(V)
        for rpc in candidates(self.nrhs):
            b = fgk.fgk_batch_create(self.handles, self.nrhs, rpc, stream=stream)
            try:
                fgk.fgk_batch_matvec_q(b, V, out=Y)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    fgk.fgk_batch_matvec_q(b, V, out=Y)
                e1.record()
                torch.cuda.synchronize()
                self.timings[str(rpc)] = e0.elapsed_time(e1) / reps
            finally:
                fgk.fgk_batch_destroy(b)
        best = pick({int(k): v for k, v in self.timings.items()})
        store_cache({self.key: {"rhs_per_cta": best, "timings_ms": self.timings}})
        return best

    def matvec(self, Vq, out=None):
        return self.fgk.fgk_batch_matvec_q(self.batch, Vq, out=out)

    def preconditioners(self, sigma2s):
        """One rank-min(precond_rank, N/8) preconditioner per problem for these sigma^2."""
        key = [float(x) for x in sigma2s]
        if self.precs is not None and self.precs_sigma2 == key:
            return self.precs
        self._free_precs()
        precs = []
        try:
            for h, p, s2 in zip(self.handles, self.problems, key):
                precs.append(self.fgk.fgk_precond_build(h, max(0, min(self.precond_rank, p.N // 8)), s2,
                                                        stream=self.stream))
        except BaseException:
            for q in precs:
                self.fgk.fgk_precond_destroy(q)
            raise
        self.precs = precs
        self.precs_sigma2 = key
        return self.precs

    def solve(self, ys, sigma2s, tol: float = 1e-8, maxit: int = 100000):
        precs = self.preconditioners(sigma2s) if self.precond_rank > 0 else None
        return self.fgk.fgk_batch_cg_solve(self.batch, ys, sigma2s, tol=tol, maxit=maxit, precs=precs)

    def _free_precs(self):
        if self.precs:
            for q in self.precs:
                self.fgk.fgk_precond_destroy(q)
        self.precs = None
        self.precs_sigma2 = None

    def close(self):
        """Free the preconditioners, the batch and the plans (idempotent)."""
        self._free_precs()
        self.fgk.fgk_batch_destroy(self.batch)
        self.batch = None
        for h in self.handles:
            self.fgk.fgk_destroy(h)
        self.handles = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def pack(engine: BatchEngine, per_problem: list) -> np.ndarray:
    """Concatenate per-problem (N_i x nrhs) arrays already in each problem's internal order."""
    return np.concatenate([np.asarray(a).reshape(-1, engine.nrhs) for a in per_problem], axis=0)
