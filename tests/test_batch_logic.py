"""The batch engine's resource handling without a GPU: a fake binding stands
in for libfgk, and every plan, batch and preconditioner it hands out must be
freed exactly once, also when a build, the batch or a preconditioner fails
part way."""

import numpy as np
import pytest
import torch

import paper_2508_01864_gb300 as pkg
from paper_2508_01864_gb300 import batch


class FakeFgk:
    def __init__(self, fail_build_at=None, fail_batch=False, fail_precond_at=None):
        self.live = set()
        self.freed = []
        self.n = 0
        self.fail_build_at = fail_build_at
        self.fail_batch = fail_batch
        self.fail_precond_at = fail_precond_at
        self.precond_calls = 0

    class Obj:
        def __init__(self, ptr):
            self.ptr = ptr

    def _new(self, tag):
        self.n += 1
        o = self.Obj((tag, self.n))
        self.live.add(o.ptr)
        return o

    def _free(self, o):
        if o is not None and o.ptr:
            assert o.ptr in self.live, "freed twice"
            self.live.remove(o.ptr)
            self.freed.append(o.ptr)
            o.ptr = 0

    def fgk_build(self, X, nu, ell, kind="product", stream=None):
        if self.fail_build_at is not None and self.n == self.fail_build_at:
            raise RuntimeError("FGK_ERR_OOM: injected")
        return self._new("plan")

    def fgk_batch_create(self, handles, nrhs, rpc, stream=None):
        if self.fail_batch:
            raise RuntimeError("FGK_ERR_INVALID: injected")
        return self._new("batch")

    def fgk_precond_build(self, h, rank, s2, stream=None):
        self.precond_calls += 1
        if self.precond_calls == self.fail_precond_at:
            raise RuntimeError("FGK_ERR_OOM: injected")
        return self._new("pc")

    fgk_destroy = _free
    fgk_batch_destroy = _free
    fgk_precond_destroy = _free


class P:
    def __init__(self, N, d=2, nu=1.5):
        self.X = np.zeros((N, d))
        self.N, self.d, self.nu, self.ell = N, d, nu, [0.2] * d


@pytest.fixture
def fake(monkeypatch, tmp_path):
    monkeypatch.setenv("FGK_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(torch, "as_tensor", lambda a, **kw: a)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "fake")

    def use(f):
        monkeypatch.setattr(pkg, "fgk", f, raising=False)
        return f

    return use


def test_close_frees_everything_once(fake):
    f = fake(FakeFgk())
    eng = batch.BatchEngine([P(100), P(200), P(300)], 4, autotune=False, precond_rank=10)
    eng.preconditioners([0.01, 0.01, 0.01])
    eng.preconditioners([0.02, 0.02, 0.02])  # another sigma^2: the first set is freed
    assert len([p for p in f.live if p[0] == "pc"]) == 3
    eng.close()
    eng.close()
    assert not f.live and len(f.freed) == len(set(f.freed)) == 3 + 1 + 6


@pytest.mark.parametrize("at", [0, 1, 2])
def test_a_failed_build_frees_the_plans_already_made(fake, at):
    f = fake(FakeFgk(fail_build_at=at))
    with pytest.raises(RuntimeError, match="injected"):
        batch.BatchEngine([P(100), P(200), P(300)], 4, autotune=False)
    assert not f.live and len(f.freed) == at


def test_a_failed_batch_frees_the_plans(fake):
    f = fake(FakeFgk(fail_batch=True))
    with pytest.raises(RuntimeError, match="injected"):
        batch.BatchEngine([P(100), P(200)], 4, autotune=False)
    assert not f.live and len(f.freed) == 2


def test_a_failed_preconditioner_frees_the_others_of_its_set(fake):
    f = fake(FakeFgk(fail_precond_at=3))
    eng = batch.BatchEngine([P(100), P(200), P(300)], 4, autotune=False, precond_rank=10)
    with pytest.raises(RuntimeError, match="injected"):
        eng.preconditioners([0.01] * 3)
    assert not [p for p in f.live if p[0] == "pc"] and eng.precs is None
    eng.close()
    assert not f.live
