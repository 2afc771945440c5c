"""MINRES on the GPU (fgk_minres_solve) for the symmetric systems that the L1
kernel makes indefinite at nu >= 3/2, d >= 2 (App. B, Prop. 4), where CG
breaks down: the solution against dense LAPACK solves at small N, the true
residual recomputed by the brute-force oracle on the d=2 workload's L1
system, and the same answer as the dense solve on a positive definite
system.  Any alpha with true residual <= tol is a correct answer; alpha is
compared with the dense solve within cond(A) tol."""

import numpy as np
import pytest

import workloads
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


# The nugget of the indefinite d = 2 cases is large enough to keep K + sigma2 I
# away from singular (with sigma2 = 0.01 some of its eigenvalues lie within
# 1e-5 of zero on both sides and MINRES, the oracle's as well, stalls); they
# stay indefinite (smallest eigenvalues -0.35 and -0.63, asserted below).
@pytest.mark.parametrize("d,nu,kind,N,sigma2", [(2, 1.5, "l1", 1500, 0.3), (3, 2.5, "l1", 1000, 0.01),
                                                (2, 2.5, "l1", 1200, 0.5), (2, 1.5, "product", 1500, 0.01),
                                                (1, 0.5, "l1", 2000, 0.01)])
def test_minres_matches_dense_solve(fgk_mod, orc, d, nu, kind, N, sigma2):
    fgk = fgk_mod
    p = workloads.small(610 + d, N, d, nu=nu, ell=[0.1, 0.3, 0.2][:d], nrhs=3)
    V = p.V.copy()
    V[:, 2] = 0.0  # a zero column stays zero
    tol = 1e-10
    A = orc.kmat(p.X, p.nu, p.ell, kind=0 if kind == "l1" else 1) + sigma2 * np.eye(p.N)
    if kind == "l1" and d > 1:
        assert np.linalg.eigvalsh(A).min() < 0  # the indefinite case MINRES is for
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind=kind) as h:
        alpha, info, rc = fgk.fgk_minres_solve(h, to_dev(V), sigma2, tol=tol, maxit=50000)
    a = alpha.cpu().numpy()
    assert rc == 0, info
    res = np.linalg.norm(V[:, :2] - A @ a[:, :2], axis=0) / np.linalg.norm(V[:, :2], axis=0)
    assert (res <= tol).all(), res
    assert info["max_true_resid"] <= tol
    assert np.all(a[:, 2] == 0.0)
    ref = np.linalg.solve(A, V[:, :2])
    cond = np.linalg.cond(A)
    assert np.linalg.norm(a[:, :2] - ref) / np.linalg.norm(ref) <= cond * tol


def test_minres_solves_the_d2_workload_l1_system_where_cg_breaks_down(fgk_mod, orc):
    """The d=2 workload's points (N = 5000, nu = 3/2, ell = (0.1, 0.3)) with
    the L1 kernel and sigma2 = 0.3: CG stops with FGK_ERR_BREAKDOWN, MINRES
    reaches a true residual of 1e-8, recomputed here with the brute-force
    oracle.  (At sigma2 = 0.01 this system is nearly singular, eigenvalues
    within 2e-5 of zero on both sides, and unpreconditioned MINRES stalls
    near 1e-2, in the oracle too.)"""
    fgk = fgk_mod
    p = workloads.c2(N=5000)
    y = p.V[:, :1]
    sigma2 = 0.3
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="l1") as h:
        with pytest.raises(fgk.FgkError) as e:
            fgk.fgk_cg_solve(h, to_dev(y), sigma2, tol=1e-8, mode="f64", maxit=20000)
        assert e.value.code == -5  # FGK_ERR_BREAKDOWN
        alpha, info, rc = fgk.fgk_minres_solve(h, to_dev(y), sigma2, tol=1e-8, maxit=200000)
    assert rc == 0, info
    a = alpha.cpu().numpy()
    Ka = orc.mvm_brute(p.X, a, p.nu, p.ell, kind=orc.L1)
    res = np.linalg.norm(y - Ka - sigma2 * a) / np.linalg.norm(y)
    assert res <= 1e-8, (res, info)
