"""GPU parity of the solve (K + sigma^2 I) alpha = y and of the GLS fixed
effects against the oracle (dense LAPACK solves at small N, the brute-force
product on sampled rows at full size), through the C ABI."""

import numpy as np
import pytest
import torch

import workloads
from gpu_util import to_dev
from oracle import solve as osolve

pytestmark = pytest.mark.gpu


def dense_A(orc, p, kind, sigma2):
    K = orc.kmat(p.X, p.nu, p.ell, s2=p.s2, kind=kind)
    return K + sigma2 * np.eye(p.N)


@pytest.mark.parametrize("d,nu", [(1, 0.5), (1, 2.5), (2, 1.5), (2, 2.5), (3, 1.5), (1, 3.5), (2, 3.5), (2, 4.5),
                                  (3, 3.5)])
@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_cg_matches_dense_solve(fgk_mod, orc, d, nu, mode):
    fgk = fgk_mod
    p = workloads.small(500 + d, 1500, d, nu=nu, ell=[0.15, 0.3, 0.45][:d], nrhs=3)
    sigma2, tol = 0.05, 1e-10
    A = dense_A(orc, p, 1, sigma2)
    ref = np.linalg.solve(A, p.V)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        alpha, beta, info, rc = fgk.fgk_cg_solve(h, to_dev(p.V), sigma2, tol=tol, mode=mode)
    a = alpha.cpu().numpy()
    assert rc == 0 and beta is None
    res = np.linalg.norm(p.V - A @ a, axis=0) / np.linalg.norm(p.V, axis=0)
    assert (res <= tol).all(), res
    assert info["max_true_resid"] <= tol
    assert np.allclose(info["true_resid"], res, rtol=1e-3, atol=1e-13)
    cond = np.linalg.cond(A)
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) <= cond * tol
    if mode == "mixed":
        assert info["mvm_f32"] > 0 and info["refinements"] >= 1
    else:
        assert info["mvm_f32"] == 0


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_gls_default_covariates(fgk_mod, orc, mode):
    """H = [1, x1, x2] (the default), against the dense GLS estimator."""
    fgk = fgk_mod
    p = workloads.small(601, 1200, 2, nu=1.5, ell=[0.2, 0.25], nrhs=1)
    H = np.column_stack([np.ones(p.N), p.X])
    y = p.V[:, 0] + H @ np.array([2.0, -1.0, 0.5])
    sigma2 = 0.02
    A = dense_A(orc, p, 1, sigma2)
    a_ref, b_ref = osolve.gls(lambda B: np.linalg.solve(A, B), y, H)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        alpha, beta, info, rc = fgk.fgk_cg_solve(h, to_dev(y), sigma2, L=-1, tol=1e-11, mode=mode)
    assert rc == 0
    b = beta.cpu().numpy()[:, 0]
    a = alpha.cpu().numpy()
    cond = np.linalg.cond(A)
    assert np.allclose(b, b_ref, rtol=1e-7, atol=1e-9), (b, b_ref)
    assert np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref) <= cond * 1e-11
    assert len(info["true_resid"]) == 1 + 3


def test_gls_explicit_covariates_and_exact_mean(fgk_mod, orc):
    """y = H beta* exactly: the GLS step returns beta* and alpha = 0."""
    fgk = fgk_mod
    p = workloads.small(602, 900, 3, nu=2.5, ell=[0.3, 0.3, 0.3])
    H = np.column_stack([np.ones(p.N), p.X, p.X[:, 0] * p.X[:, 1]])
    beta_star = np.array([1.0, 0.5, -0.3, 0.2, 0.7])
    y = np.stack([H @ beta_star, 2 * H @ beta_star], axis=1)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        alpha, beta, info, rc = fgk.fgk_cg_solve(h, to_dev(y), 0.01, H=to_dev(H), tol=1e-11, mode="f64")
    assert rc == 0
    b = beta.cpu().numpy()
    assert np.allclose(b[:, 0], beta_star, rtol=1e-6, atol=1e-8)
    assert np.allclose(b[:, 1], 2 * beta_star, rtol=1e-6, atol=1e-8)
    assert np.abs(alpha.cpu().numpy()).max() < 1e-6 * np.abs(y).max()


def test_l1_indefinite_breakdown(fgk_mod, orc):
    """nu = 3/2, d = 2, L1 kernel at the d=2 configuration's lengthscales is
    indefinite (Prop. 4's condition fails); CG meets p^T A p <= 0."""
    fgk = fgk_mod
    p = workloads.c2(N=3000)
    A = dense_A(orc, p, 0, p.sigma2)
    assert np.linalg.eigvalsh(A)[0] < 0
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="l1") as h:
        with pytest.raises(fgk.FgkError) as e:
            fgk.fgk_cg_solve(h, to_dev(p.V), p.sigma2, tol=1e-8, mode="f64")
    assert e.value.code == -5


def test_not_converged_and_zero_rhs(fgk_mod):
    fgk = fgk_mod
    p = workloads.small(603, 2000, 2, nu=1.5, ell=[0.1, 0.3], nrhs=2)
    y = p.V.copy()
    y[:, 1] = 0.0
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        alpha, _, info, rc = fgk.fgk_cg_solve(h, to_dev(y), 0.01, tol=1e-12, maxit=5, mode="f64")
        assert rc == 1
        a = alpha.cpu().numpy()
        assert np.isfinite(a).all() and (a[:, 1] == 0).all()
        assert info["iterations"] <= 5 + 8
        with pytest.raises(fgk.FgkError) as e:
            bad = y.copy()
            bad[5, 0] = np.nan
            fgk.fgk_cg_solve(h, to_dev(bad), 0.01)
        assert e.value.code == -2


@pytest.mark.parametrize("mode", ["mixed", "f64"])
def test_c2_full_size_solve(fgk_mod, orc, mode):
    """The d=2 configuration: N=200000, nu=3/2, ell=(0.1,0.3), sigma^2=0.01,
    product kernel, tolerance 1e-8 on the FP64 true residual.  The residual
    the library reports rests on its FP64 product, which is checked here
    against the brute-force oracle on sampled rows of K alpha."""
    fgk = fgk_mod
    p = workloads.c2()
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        alpha, _, info, rc = fgk.fgk_cg_solve(h, to_dev(p.V), p.sigma2, tol=1e-8, maxit=60000, mode=mode)
        assert rc == 0, info
        assert info["max_true_resid"] <= 1e-8
        Ka = fgk.fgk_matvec(h, alpha.reshape(-1, 1).contiguous(), "f64").cpu().numpy()[:, 0]
    a = alpha.cpu().numpy().reshape(-1)
    rows = np.sort(np.random.default_rng(9).choice(p.N, 300, replace=False))
    ref = orc.mvm_brute(p.X, a, p.nu, p.ell, kind=1, rows=rows)
    assert np.linalg.norm(Ka[rows] - ref) <= 1e-12 * np.linalg.norm(ref)
    r = p.V[:, 0] - Ka - p.sigma2 * a
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(p.V[:, 0])
