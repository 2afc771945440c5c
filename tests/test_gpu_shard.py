"""The sharded d = 1 product on the GPU, through the C ABI: three shards
(contiguous ranges of the sorted points, one plan each) in one process, the
moments of fgk_shard_moments exchanged by hand, composed by the host code
that the ranks run, and added by fgk_shard_fixup: every shard's rows equal
the brute-force oracle (O1) within 1e-12; the moments equal their definition.
Multi-GPU runs are not tested on hardware (one GPU here); the CPU test runs
the same composition across two gloo ranks."""

import numpy as np
import pytest
import torch

import workloads
from gpu_util import to_dev
from paper_2508_01864_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nu,N,nshards,pattern", [(0.5, 4096, 3, "uniform"), (1.5, 20000, 4, "dups"),
                                                  (2.5, 9000, 2, "lattice"), (3.5, 6000, 3, "uniform"),
                                                  (4.5, 5000, 3, "uniform")])
def test_sharded_product_matches_the_oracle(fgk_mod, orc, nu, N, nshards, pattern):
    fgk = fgk_mod
    ell = 0.2 if pattern != "lattice" else 0.5
    p = workloads.small(77 + N, N, 1, nu=nu, ell=ell, nrhs=2, pattern=pattern, s2=1.4)
    order = np.argsort(p.X[:, 0], kind="stable")
    parts = np.array_split(order, nshards)
    ref = orc.mvm_brute(p.X, p.V, nu, [ell], s2=p.s2)
    hs = [fgk.fgk_build(to_dev(p.X[m]), nu, [ell], outscale2=p.s2) for m in parts]
    try:
        shs = [shard.GpuShard(h) for h in hs]
        Vs = [to_dev(p.V[m]) for m in parts]
        mom = [s.moments(V) for s, V in zip(shs, Vs)]
        a = np.sqrt(2 * nu) / ell
        for m, (xf, xl, M) in zip(parts, mom):  # the moments against their definition
            xs = a * p.X[m, 0]
            assert xf == xs.min() and xl == xs.max()
            for dirn, dl in ((0, xl - xs), (1, xs - xf)):
                for q in range(M.shape[2]):
                    want = (p.V[m] * (dl ** q * np.exp(-dl))[:, None]).sum(axis=0)
                    assert np.allclose(M[:, dirn, q], want, rtol=1e-12, atol=1e-12 * np.abs(p.V[m]).sum())
        for r, (s, V, m) in enumerate(zip(shs, Vs, parts)):
            Y = s.local_product(V)
            s.fixup(shard.compose_carries(mom, r), Y)
            got = Y.cpu().numpy()
            err = np.linalg.norm(got - ref[m], axis=0) / np.linalg.norm(ref[m], axis=0)
            assert (err <= 1e-12).all(), (r, err)
    finally:
        for h in hs:
            fgk.fgk_destroy(h)


def test_shard_calls_refuse_d2(fgk_mod):
    fgk = fgk_mod
    p = workloads.small(3, 200, 2, nu=1.5, ell=[0.2, 0.2])
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell) as h:
        with pytest.raises(fgk.FgkError):
            fgk.fgk_shard_moments(h, to_dev(p.V))
