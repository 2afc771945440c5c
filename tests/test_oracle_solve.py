"""Pins for the oracle's CG and GLS (O4): against LAPACK dense solves and the
exact special cases of the GLS estimator."""

import numpy as np
import pytest

import workloads
from oracle import solve


@pytest.mark.parametrize("nu,kind", [(0.5, 0), (1.5, 1), (2.5, 1)])
def test_cg_matches_dense_solve(orc, nu, kind):
    p = workloads.small(31, 400, 2, nu=nu, ell=[0.1, 0.3], nrhs=3)
    sigma2 = 0.01
    K = orc.kmat(p.X, nu, p.ell, kind=kind)

    def A(B):
        return orc.mvm_brute(p.X, B, nu, p.ell, kind=kind) + sigma2 * B

    x, iters = solve.cg(A, p.V, 1e-10, 5000)
    ref = solve.dense_solve(K, sigma2, p.V)
    assert (iters > 0).all()
    res = solve.true_residual(A, x, p.V)
    assert (res <= 2e-10).all()
    cond = np.linalg.cond(K + sigma2 * np.eye(K.shape[0]))
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < cond * 1e-10


def test_gls_exact_mean_is_recovered(orc):
    """y = H beta* exactly: the GLS estimator returns beta* and alpha = 0."""
    p = workloads.small(32, 300, 2, nu=1.5, ell=[0.2, 0.2])
    H = np.column_stack([np.ones(p.N), p.X])
    beta_star = np.array([1.5, -0.7, 2.25])
    y = H @ beta_star
    A = orc.kmat(p.X, 1.5, p.ell, kind=1) + 0.01 * np.eye(p.N)
    alpha, beta = solve.gls(lambda B: np.linalg.solve(A, B), y, H)
    assert np.allclose(beta, beta_star, rtol=1e-9)
    assert np.abs(alpha).max() < 1e-8 * np.abs(y).max()


def test_gls_normal_equations(orc):
    """The GLS beta satisfies H^T A^{-1} (y - H beta) = 0, and alpha solves
    A alpha = y - H beta."""
    p = workloads.small(33, 250, 3, nu=2.5, ell=[0.3, 0.3, 0.3])
    H = np.column_stack([np.ones(p.N), p.X])
    y = p.V[:, 0] + H @ np.array([1.0, 0.5, -0.3, 0.2])
    A = orc.kmat(p.X, 2.5, p.ell, kind=1) + 0.01 * np.eye(p.N)
    alpha, beta = solve.gls(lambda B: np.linalg.solve(A, B), y, H)
    assert np.linalg.norm(H.T @ alpha) < 1e-8 * np.linalg.norm(H.T @ np.linalg.solve(A, y))
    assert np.linalg.norm(A @ alpha - (y - H @ beta)) < 1e-10 * np.linalg.norm(y)


@pytest.mark.parametrize("d,nu,kind", [(1, 0.5, 0), (2, 1.5, 1), (3, 2.5, 1), (2, 2.5, 0)])
def test_posterior_mean_at_the_data_is_y_minus_sigma2_alpha(orc, d, nu, kind):
    """(K + sigma^2 I) alpha = y, so the posterior mean at the training
    points, K alpha (eq. gp_mean_2 with z = x_i), equals y - sigma^2 alpha."""
    p = workloads.small(41 + d, 300, d, nu=nu, ell=[0.2, 0.3, 0.4][:d], nrhs=2)
    s2 = 0.05
    K = orc.kmat(p.X, nu, p.ell, kind=kind)
    alpha = solve.dense_solve(K, s2, p.V)
    m = solve.posterior_mean(orc.kcross(p.X, p.X, nu, p.ell, kind=kind), alpha)
    assert np.allclose(m, p.V - s2 * alpha, rtol=1e-9, atol=1e-10)


def test_posterior_mean_cross_covariance_is_symmetric_and_matches_the_kernel(orc):
    p = workloads.small(47, 50, 2, nu=1.5, ell=[0.2, 0.3])
    Z = np.random.default_rng(3).uniform(-0.2, 1.2, size=(7, 2))
    C = orc.kcross(p.X, Z, 1.5, p.ell, s2=1.7, kind=1)
    # K(z, x) = K(x, z): the data as evaluation points of the new points
    assert np.allclose(C, orc.kcross(Z, p.X, 1.5, p.ell, s2=1.7, kind=1).T, rtol=0, atol=0)
    # the product kernel of the closed-form 1-D kernels
    u = np.abs(Z[:, None, :] - p.X[None, :, :]) * np.sqrt(3.0) / p.ell
    ref = 1.7 * np.prod((1 + u) * np.exp(-u), axis=2)
    assert np.allclose(C, ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_kernel_sums_at_new_points_by_the_decomposition(orc, kind, nu, d):
    """eq. gp_mean's k_z^T V by the ECDF decomposition with sources at the
    data and queries at new points (some of them on data coordinates, so
    ties between the two sets occur) against the dense cross-covariance."""
    p = workloads.small(500 + d, 150, d, nu=nu, ell=[0.3, 0.5, 0.7][:d], nrhs=2, pattern="lattice")
    rng = np.random.default_rng(d)
    Z = np.concatenate([rng.uniform(0, 1, size=(40, d)), p.X[:10]])
    got = orc.mvm_dc_cross(p.X, Z, p.V, nu, p.ell, s2=1.2, kind=kind)
    ref = orc.kcross(p.X, Z, nu, p.ell, s2=1.2, kind=kind) @ p.V
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert (err < 1e-11).all(), err
