"""Pins for the oracle's log marginal likelihood (eq. gp_log_likelihood) and
its gradient (eq. gp_log_likelihood_derivative): scipy's multivariate normal
density, central differences of the likelihood in every log-parameter, and
the mean of the Hutchinson estimate over many probes."""

import numpy as np
import pytest
from scipy import stats

import workloads
from oracle import solve


def problem(orc, seed=3, N=80, kind=1):
    # the L1 kernel is positive definite only for nu = 1/2 (Prop. 4)
    p = workloads.small(seed, N, 2, nu=1.5 if kind == 1 else 0.5, ell=[0.25, 0.4], s2=1.4)
    y = np.sin(4 * p.X[:, 0]) + np.cos(3 * p.X[:, 1]) + 0.1 * np.random.default_rng(seed).standard_normal(N)
    return p, y


def test_loglik_is_the_gaussian_log_density(orc):
    p, y = problem(orc)
    K = orc.kmat(p.X, p.nu, p.ell, s2=p.s2, kind=1)
    A = K + 0.05 * np.eye(p.N)
    ref = stats.multivariate_normal(mean=np.zeros(p.N), cov=A).logpdf(y)
    assert solve.loglik_exact(K, 0.05, y) == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("kind", [0, 1])
def test_gradient_matches_central_differences(orc, kind):
    p, y = problem(orc, kind=kind)
    s2n = 0.05
    K = orc.kmat(p.X, p.nu, p.ell, s2=p.s2, kind=kind)
    eye = np.eye(p.N)
    if kind == 1:
        dKs = [orc.mvm_dlogell_brute(p.X, eye, p.nu, p.ell, dim=m, s2=p.s2, kind=1) for m in range(2)]
    else:
        dKs = [orc.mvm_dlogell_brute(p.X, eye, p.nu, p.ell, dim=-1, s2=p.s2, kind=0)]
    dKs += [K, s2n * eye]  # d/d log s2 (outputscale), d/d log sigma2
    g = solve.loglik_grad_exact(K, dKs, s2n, y)
    h = 1e-5

    def ll(ell, s2, sn):
        return solve.loglik_exact(orc.kmat(p.X, p.nu, ell, s2=s2, kind=kind), sn, y)

    fds = []
    if kind == 1:
        for m in range(2):
            e = np.zeros(2)
            e[m] = h
            fds.append((ll(p.ell * np.exp(e), p.s2, s2n) - ll(p.ell * np.exp(-e), p.s2, s2n)) / (2 * h))
    else:
        fds.append((ll(p.ell * np.exp(h), p.s2, s2n) - ll(p.ell * np.exp(-h), p.s2, s2n)) / (2 * h))
    fds.append((ll(p.ell, p.s2 * np.exp(h), s2n) - ll(p.ell, p.s2 * np.exp(-h), s2n)) / (2 * h))
    fds.append((ll(p.ell, p.s2, s2n * np.exp(h)) - ll(p.ell, p.s2, s2n * np.exp(-h))) / (2 * h))
    np.testing.assert_allclose(g, fds, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("precond", [False, True])
def test_hutchinson_gradient_is_unbiased(orc, precond):
    p, y = problem(orc, seed=8, N=60)
    s2n = 0.05
    K = orc.kmat(p.X, p.nu, p.ell, s2=p.s2, kind=1)
    A = K + s2n * np.eye(p.N)
    eye = np.eye(p.N)
    dKs = [orc.mvm_dlogell_brute(p.X, eye, p.nu, p.ell, dim=m, s2=p.s2, kind=1) for m in range(2)] + [K]
    exact = solve.loglik_grad_exact(K, dKs, s2n, y)
    rng = np.random.default_rng(4)
    nprobe = 4000
    if precond:
        L, _, _ = solve.pivoted_cholesky(lambda i: K[:, i], np.diag(K), 5)
        B = L @ rng.standard_normal((L.shape[1], nprobe)) + np.sqrt(s2n) * rng.standard_normal((p.N, nprobe))
        Pinv = lambda R: solve.woodbury_apply(L, s2n, R)  # noqa: E731
    else:
        B = rng.standard_normal((p.N, nprobe))
        Pinv = None
    Ainv = np.linalg.inv(A)
    est = solve.loglik_grad_estimate(lambda V: Ainv @ V, [lambda V, D=D: D @ V for D in dKs], y, B, Pinv)
    # standard errors of the trace halves
    Z = B if Pinv is None else Pinv(B)
    X = Ainv @ B
    for j, D in enumerate(dKs):
        samples = np.einsum("ij,ij->j", X, D @ Z)
        se = 0.5 * samples.std() / np.sqrt(nprobe)
        assert abs(est[j] - exact[j]) < 4 * se, (j, est[j], exact[j], se)


def test_adam_steps_reach_the_optimum_of_a_concave_quadratic():
    c = np.array([0.3, -0.7, 0.1])
    W = np.diag([2.0, 0.5, 1.0])
    th, _, g = solve.adam_sigma_steps(lambda t, s, j: -W @ (t - c), lambda t, s: 1.0, 1, np.zeros(3), 1.0, 4000,
                                      lr0=0.01, lr1=0.001, n_sched=4000)
    np.testing.assert_allclose(th[-1], c, atol=2e-3)
    # the first Adam step has size lr0 in every coordinate (bias-corrected m/sqrt(v) = sign(g))
    np.testing.assert_allclose(np.abs(th[0]), 0.01, rtol=1e-6)


def test_sigma_update_is_the_profile_maximum_in_sigma2(orc):
    """With varsigma / sigma held, y ~ N(0, sigma^2 (K~ + I)): the update
    sigma^2 = y^T (K~ + I)^{-1} y / N is where the exact log-likelihood is
    stationary in sigma^2."""
    p, y = problem(orc, seed=5, N=70)
    Kt = orc.kmat(p.X, p.nu, p.ell, s2=0.8, kind=1)  # K~ = K(varsigma / sigma, ell)
    Ai = np.linalg.solve(Kt + np.eye(p.N), y)
    s2hat = float(y @ Ai) / p.N
    f = lambda s2: solve.loglik_exact(s2 * Kt, s2, y)  # noqa: E731  K + s2 I = s2 (K~ + I)
    h = 1e-6
    assert abs((f(s2hat * (1 + h)) - f(s2hat * (1 - h))) / (2 * h)) < 1e-5
    # and the form used by the loop: sigma_{j-1}^2 y^T (K + sigma_{j-1}^2 I)^{-1} y / N
    s_prev = 0.3
    K = s_prev * Kt  # K(varsigma_j, ell_j) with varsigma_j^2 = 0.8 sigma_{j-1}^2
    _, sig, _ = solve.adam_sigma_steps(lambda t, s, j: np.zeros(1),
                                       lambda t, s: float(y @ np.linalg.solve(K + s * np.eye(p.N), y)),
                                       p.N, np.zeros(1), s_prev, 1)
    assert sig[0] == pytest.approx(s2hat, rel=1e-12)
