"""The oracle reproduces its frozen values in tests/golden/oracle_values.txt
(written by tests/golden/make_golden.py from the oracle alone): a change to
the oracle's arithmetic fails here until the values are rewritten on purpose."""

import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_values.txt")


def _records(tag):
    with open(GOLDEN) as f:
        return [ln.split() for ln in f if ln.startswith(tag + " ")]


def test_kernel_values(orc):
    recs = _records("kernel")
    assert len(recs) == 25
    for _, two_nu, u, k in recs:
        assert float(orc.kernel(int(two_nu) / 2, float(u))) == pytest.approx(float(k), rel=1e-15, abs=0)


def test_product_values(orc):
    recs = _records("mvm")
    assert len(recs) == 25
    for rec in recs:
        seed, N, d, nu = int(rec[1]), int(rec[2]), int(rec[3]), float(rec[4])
        ell = [float(e) for e in rec[5:5 + d]]
        kind, row, val = int(rec[5 + d]), int(rec[6 + d]), float(rec[7 + d])
        p = workloads.small(seed, N, d, nu=nu, ell=ell)
        y = orc.mvm_brute(p.X, p.V[:, 0], nu, ell, kind=kind, rows=np.array([row]), nthreads=1)[0]
        assert y == pytest.approx(val, rel=1e-14, abs=1e-300)
