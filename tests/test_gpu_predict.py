"""GPU parity of the posterior mean at new points (eq. gp_mean), through the
C ABI: against the oracle's dense cross-covariance times alpha, the identity
K alpha = y - sigma^2 alpha at the data, and the GLS mean h(z)^T beta."""

import numpy as np
import pytest
import torch

import workloads
from gpu_util import colwise_relerr, to_dev
from oracle import solve as osolve

pytestmark = pytest.mark.gpu

CASES = [  # d, nu, kind, N, M, pattern
    (1, 0.5, "l1", 2500, 700, "uniform"),
    (1, 2.5, "l1", 1100, 3000, "uniform"),
    (2, 1.5, "product", 3000, 900, "uniform"),
    (2, 2.5, "product", 1500, 1, "uniform"),
    (2, 1.5, "l1", 2200, 400, "lattice"),
    (3, 2.5, "product", 1200, 300, "uniform"),
    (3, 0.5, "l1", 900, 500, "dups"),
]


@pytest.mark.parametrize("d,nu,kind,N,M,pattern", CASES)
@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_predict_matches_dense_cross_product(fgk_mod, orc, d, nu, kind, N, M, pattern, precision, tol):
    fgk = fgk_mod
    p = workloads.small(900 + d * 7 + M % 13, N, d, nu=nu, ell=[0.15, 0.3, 0.45][:d], nrhs=2, pattern=pattern,
                        s2=1.4)
    rng = np.random.default_rng(M)
    # new points: inside and outside the data's range, and some exactly on data points
    Z = rng.uniform(-0.25, 1.25, size=(M, d))
    k = min(M // 4, N)
    if k:
        Z[:k] = p.X[rng.choice(N, k, replace=False)]
    alpha = rng.standard_normal((N, 2))
    kk = 0 if kind == "l1" else 1
    ref = osolve.posterior_mean(orc.kcross(p.X, Z, p.nu, p.ell, s2=p.s2, kind=kk), alpha)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, outscale2=p.s2, kind=kind) as h:
        got = fgk.fgk_predict(h, to_dev(alpha), to_dev(Z), precision=precision).cpu().numpy()
    assert (colwise_relerr(got, ref) <= tol).all()


def test_predict_at_the_data_after_a_solve(fgk_mod, orc):
    """(K + sigma^2 I) alpha = y: the mean at the data is y - sigma^2 alpha."""
    fgk = fgk_mod
    p = workloads.small(77, 4000, 2, nu=1.5, ell=[0.15, 0.3], nrhs=1)
    s2n = 0.05
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        alpha, _, info, rc = fgk.fgk_cg_solve(h, to_dev(p.V), s2n, tol=1e-11, mode="f64")
        m = fgk.fgk_predict(h, alpha, to_dev(p.X)).cpu().numpy()
    a = alpha.cpu().numpy()
    assert rc == 0
    assert np.linalg.norm(m - (p.V - s2n * a)) <= 1e-9 * np.linalg.norm(p.V)


def test_predict_with_fixed_effects(fgk_mod, orc):
    fgk = fgk_mod
    p = workloads.small(78, 1200, 2, nu=2.5, ell=[0.2, 0.3], nrhs=1)
    H = np.column_stack([np.ones(p.N), p.X])
    y = p.V[:, 0] + H @ np.array([1.0, -0.5, 2.0])
    s2n = 0.02
    A = orc.kmat(p.X, p.nu, p.ell, kind=1) + s2n * np.eye(p.N)
    a_ref, b_ref = osolve.gls(lambda B: np.linalg.solve(A, B), y, H)
    Z = np.random.default_rng(2).uniform(0, 1, size=(300, 2))
    ref = osolve.posterior_mean(orc.kcross(p.X, Z, p.nu, p.ell, kind=1), a_ref,
                                np.column_stack([np.ones(len(Z)), Z]), b_ref)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        alpha, beta, info, rc = fgk.fgk_cg_solve(h, to_dev(y), s2n, L=-1, tol=1e-12, mode="f64")
        got = fgk.fgk_predict(h, alpha, to_dev(Z), beta=beta, L=-1).cpu().numpy()
        # the same covariates given explicitly
        got2 = fgk.fgk_predict(h, alpha, to_dev(Z), beta=beta,
                               HZ=to_dev(np.column_stack([np.ones(len(Z)), Z]))).cpu().numpy()
    cond = np.linalg.cond(A)
    assert np.linalg.norm(got - ref) <= cond * 1e-12 * np.linalg.norm(ref)
    assert np.allclose(got, got2, rtol=0, atol=1e-14 * np.abs(got).max())


def test_predict_rejects_bad_input(fgk_mod):
    fgk = fgk_mod
    p = workloads.small(79, 300, 2)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        a = torch.zeros((p.N, 1), dtype=torch.float64, device="cuda")
        Z = to_dev(np.array([[0.5, np.nan]]))
        with pytest.raises(fgk.FgkError) as e:
            fgk.fgk_predict(h, a, Z)
        assert e.value.code == -2
        with pytest.raises(ValueError):  # fixed effects without beta (the binding refuses)
            fgk.fgk_predict(h, a, to_dev(np.array([[0.5, 0.5]])), L=-1)
        with pytest.raises(fgk.FgkError) as e:  # L without covariates must be 0 or -1 (the library refuses)
            fgk.fgk_predict(h, a, to_dev(np.array([[0.5, 0.5]])), L=3, beta=to_dev(np.zeros((3, 1))))
        assert e.value.code == -1
