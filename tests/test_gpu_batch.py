"""Batches: one launch per phase of the product for many problems, and the
batched mixed-precision CG, against the single-plan product (itself pinned
to the oracle) and the oracle's product."""

import numpy as np
import pytest
import torch

import workloads
from gpu_util import colwise_relerr, to_dev

pytestmark = pytest.mark.gpu

MIX = [(1, 0.5, 1500, "l1"), (1, 2.5, 5000, "l1"), (2, 1.5, 3000, "product"), (2, 2.5, 4500, "product"),
       (2, 0.5, 700, "l1"), (2, 1.5, 2500, "l1"), (2, 2.5, 2200, "l1"), (1, 1.5, 9000, "l1")]


def build_mix(fgk, nrhs, seed=0):
    probs, handles = [], []
    for i, (d, nu, N, kind) in enumerate(MIX):
        p = workloads.small(seed + 31 * i, N, d, nu=nu, ell=[0.12, 0.3][:d], nrhs=nrhs, s2=1.3)
        probs.append((p, kind))
        handles.append(fgk.fgk_build(to_dev(p.X), p.nu, p.ell, outscale2=p.s2, kind=kind))
    return probs, handles


@pytest.mark.parametrize("rpc", [0, 1, 2])
def test_batch_product_matches_single_plans(fgk_mod, orc, rpc):
    fgk = fgk_mod
    nrhs = 3
    probs, handles = build_mix(fgk, nrhs)
    b = fgk.fgk_batch_create(handles, nrhs, rpc)
    try:
        offs = b.rows
        rng = np.random.default_rng(7)
        V = rng.standard_normal((offs[-1], nrhs)).astype(np.float32)
        Y = fgk.fgk_batch_matvec_q(b, to_dev(V, torch.float32)).cpu().numpy()
        for i, ((p, kind), h) in enumerate(zip(probs, handles)):
            Vi = V[offs[i]:offs[i + 1]]
            Yi = Y[offs[i]:offs[i + 1]]
            ref64 = fgk.fgk_matvec_q(h, to_dev(Vi, torch.float64), "f64").cpu().numpy()
            assert (colwise_relerr(Yi, ref64) <= 1e-5).all(), i
            if i in (2, 5):  # straight against the oracle (inputs in the plan's order)
                perm = fgk.fgk_get_permutation(h, 0)
                ref = orc.mvm_brute(p.X[perm], Vi.astype(np.float64), p.nu, p.ell, s2=p.s2,
                                    kind=0 if kind == "l1" else 1)
                assert (colwise_relerr(Yi, ref) <= 1e-5).all(), i
    finally:
        fgk.fgk_batch_destroy(b)
        for h in handles:
            fgk.fgk_destroy(h)


def test_batch_cg_meets_tolerance(fgk_mod, orc):
    fgk = fgk_mod
    nrhs = 2
    probs, handles = [], []
    for i, (d, nu, N) in enumerate([(1, 0.5, 1200), (2, 1.5, 2500), (1, 2.5, 3000), (2, 2.5, 1800), (2, 0.5, 900)]):
        p = workloads.small(900 + i, N, d, nu=nu, ell=[0.1, 0.25][:d], nrhs=nrhs)
        probs.append(p)
        handles.append(fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product"))
    b = fgk.fgk_batch_create(handles, nrhs, 0)
    try:
        ys = [to_dev(p.V) for p in probs]
        sig = [0.01, 0.05, 0.01, 0.02, 0.1]
        alphas, infos, rc = fgk.fgk_batch_cg_solve(b, ys, sig, tol=1e-8, maxit=50000)
        assert rc == 0
        for p, a, s, info in zip(probs, alphas, sig, infos):
            a = a.cpu().numpy()
            Ka = orc.mvm_brute(p.X, a, p.nu, p.ell, kind=1)
            res = np.linalg.norm(p.V - Ka - s * a, axis=0) / np.linalg.norm(p.V, axis=0)
            assert (res <= 1e-8).all(), res
            assert info["max_true_resid"] <= 1e-8 and info["iterations"] > 0
    finally:
        fgk.fgk_batch_destroy(b)
        for h in handles:
            fgk.fgk_destroy(h)


def test_batch_rejects_d3(fgk_mod):
    fgk = fgk_mod
    p = workloads.small(5, 200, 3)
    with fgk.fgk_build(to_dev(p.X), 1.5, [0.2] * 3) as h:
        with pytest.raises(fgk.FgkError):
            fgk.fgk_batch_create([h], 2)


@pytest.mark.parametrize("rpc", [0, 1])
def test_batch_cg_iterations_track_single_solver(fgk_mod, rpc):
    """Badly conditioned small problems (smooth kernels, long length scales):
    the FP32 recursion drifts fast there, so the batched solve has to replace
    its residual as promptly as the single-problem solve; its iteration count
    stays close to the single solve's for every launch shape."""
    fgk = fgk_mod
    probs = workloads.c4(n_problems=18)
    sel = [probs[i] for i in (14, 17, 3)]  # d=1: nu 5/2 (N 1746, 1513), nu 3/2 (N 10165)
    handles = [fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") for p in sel]
    b = fgk.fgk_batch_create(handles, 16, rpc)
    try:
        ys = [to_dev(p.V) for p in sel]
        _, infos, rc = fgk.fgk_batch_cg_solve(b, ys, [p.sigma2 for p in sel], tol=1e-8, maxit=20000)
        assert rc == 0
        for p, h, y, info in zip(sel, handles, ys, infos):
            _, _, one, rc1 = fgk.fgk_cg_solve(h, y, p.sigma2, tol=1e-8, maxit=20000, mode="mixed")
            assert rc1 == 0
            assert info["max_true_resid"] <= 1e-8
            assert info["iterations"] <= 1.5 * one["iterations"] + 50, (p.name, info, one)
    finally:
        fgk.fgk_batch_destroy(b)
        for h in handles:
            fgk.fgk_destroy(h)


def test_batch_pcg_meets_tolerance_in_fewer_iterations(fgk_mod, orc):
    """Per-problem pivoted-Cholesky preconditioners (App. A.3) in the batched
    solve: every problem and column meets the tolerance on the oracle's
    residual, in fewer iterations than the unpreconditioned batch."""
    from paper_2508_01864_gb300 import batch as batchmod

    probs = [workloads.small(950 + i, N, d, nu=nu, ell=[0.12, 0.3][:d], nrhs=4)
             for i, (d, nu, N) in enumerate([(1, 0.5, 1500), (2, 1.5, 3000), (1, 2.5, 2500), (2, 2.5, 2000),
                                             (2, 0.5, 1200)])]
    sig = [0.01, 0.02, 0.01, 0.01, 0.05]
    ys = [to_dev(p.V) for p in probs]
    plain = batchmod.BatchEngine(probs, 4, kind="product", autotune=False)
    _, inf0, rc0 = plain.solve(ys, sig, tol=1e-8, maxit=50000)
    plain.close()
    eng = batchmod.BatchEngine(probs, 4, kind="product", autotune=False, precond_rank=100)
    try:
        alphas, infos, rc = eng.solve(ys, sig, tol=1e-8, maxit=50000)
        assert rc == 0 and rc0 == 0
        for p, a, s, info, i0 in zip(probs, alphas, sig, infos, inf0):
            a = a.cpu().numpy()
            Ka = orc.mvm_brute(p.X, a, p.nu, p.ell, kind=1)
            res = np.linalg.norm(p.V - Ka - s * a, axis=0) / np.linalg.norm(p.V, axis=0)
            assert (res <= 1e-8).all(), res
            assert info["iterations"] < i0["iterations"], (info, i0)
        # a second solve with the same sigma^2 reuses the preconditioners
        first = eng.precs
        eng.solve(ys, sig, tol=1e-8, maxit=50000)
        assert eng.precs is first
    finally:
        eng.close()


def test_full_batched_workload(fgk_mod, orc):
    """The batched workload at its full size: 64 problems (N log-uniform 1k-100k,
    d in {1, 2}, nu in {1/2, 3/2, 5/2}), 16 right-hand sides each, solved in one
    batch with rank-100 preconditioners to 1e-8.  For every problem the
    residual y - (K + sigma^2 I) alpha on 40 sampled rows, with K alpha from the
    brute-force oracle, has norm at most 1e-8 ||y|| per column (a subset of the
    rows cannot carry more than the whole residual), and the library's own
    FP64 true residual is at most 1e-8."""
    from paper_2508_01864_gb300 import batch as batchmod

    probs = workloads.c4()
    assert len(probs) == 64 and probs[0].V.shape[1] == 16
    ys = [to_dev(p.V) for p in probs]
    sig = [p.sigma2 for p in probs]
    eng = batchmod.BatchEngine(probs, 16, kind="product", precond_rank=100)
    try:
        alphas, infos, rc = eng.solve(ys, sig, tol=1e-8, maxit=200000)
        assert rc == 0
        rng = np.random.default_rng(64)
        for p, a, s, info in zip(probs, alphas, sig, infos):
            assert info["max_true_resid"] <= 1e-8, info
            a = a.cpu().numpy()
            rows = np.sort(rng.choice(p.N, size=min(40, p.N), replace=False))
            Ka = orc.mvm_brute(p.X, a, p.nu, p.ell, kind=1, rows=rows)
            r = p.V[rows] - Ka - s * a[rows]
            assert (np.linalg.norm(r, axis=0) <= 1e-8 * np.linalg.norm(p.V, axis=0)).all(), p.name
    finally:
        eng.close()
