"""A bounded device-side wait that runs out: the radix sort's look-back waits
on earlier tiles with a spin limit; FGK_SORT_SPIN_LIMIT (read by fgk_build)
shortens it to one spin so that, with thousands of tiles running at once,
some tile finds its predecessor unfinished.  The build then returns
FGK_ERR_TIMEOUT, without hanging and without touching memory outside its
buffers (the expired tile's offsets are at most the true ones, later tiles
and passes stop, the host abandons the sort before using it), and the
context stays usable: a normal build and product afterwards match the
oracle.  No kernel faults, traps or spins without a bound here."""

import os

import numpy as np
import pytest
import torch

import workloads
from gpu_util import colwise_relerr, to_dev

pytestmark = pytest.mark.gpu


def test_expired_lookback_returns_timeout_and_leaves_the_context_usable(fgk_mod, orc):
    fgk = fgk_mod
    p = workloads.c2(N=4_000_000)
    X = to_dev(p.X)
    codes = []
    os.environ["FGK_SORT_SPIN_LIMIT"] = "1"
    try:
        for _ in range(3):
            try:
                h = fgk.fgk_build(X, p.nu, p.ell, kind="product")
                fgk.fgk_destroy(h)
                codes.append(0)
            except fgk.FgkError as e:
                codes.append(e.code)
                assert "wait expired" in str(e), str(e)
    finally:
        del os.environ["FGK_SORT_SPIN_LIMIT"]
    assert set(codes) <= {0, -6} and -6 in codes, codes  # FGK_ERR_TIMEOUT at least once
    # the context is intact: an ordinary build and product are correct
    small = workloads.small(12, 3000, 2, nu=1.5, ell=[0.1, 0.3], nrhs=1)
    with fgk.fgk_build(to_dev(small.X), small.nu, small.ell, kind="product") as h:
        y = fgk.fgk_matvec(h, to_dev(small.V), "f64").cpu().numpy()
    ref = orc.mvm_brute(small.X, small.V, small.nu, small.ell, kind=orc.PRODUCT)
    assert (colwise_relerr(y, ref) <= 1e-12).all()
    torch.cuda.synchronize()
