"""The host logic of the fitting loop (paper_2508_01864_gb300.fit.adam_sigma_loop:
Algorithm 1's Adam steps and closed-form nugget update) against the oracle's
own implementation of the same recurrence, both driven by the oracle's exact
dense gradient; and its two stopping rules.  No GPU."""

import math

import numpy as np
import pytest

import workloads
from oracle import solve


def test_loop_follows_the_oracle_recurrence(orc):
    from paper_2508_01864_gb300 import fit

    N, d = 70, 2
    p = workloads.small(17, N, d, nu=1.5, ell=[0.3, 0.3])
    y = np.sin(5 * p.X[:, 0]) + np.cos(3 * p.X[:, 1]) + 0.1 * np.random.default_rng(2).standard_normal(N)
    eye = np.eye(N)

    def grad(theta, s2n):
        ell, s2 = np.exp(theta[:d]), math.exp(theta[d])
        K = orc.kmat(p.X, p.nu, ell, s2=s2, kind=1)
        dKs = [orc.mvm_dlogell_brute(p.X, eye, p.nu, ell, dim=m, s2=s2, kind=1) for m in range(d)] + [K]
        return solve.loglik_grad_exact(K, dKs, s2n, y)

    def quad(theta, s2n):
        K = orc.kmat(p.X, p.nu, np.exp(theta[:d]), s2=math.exp(theta[d]), kind=1)
        return float(y @ np.linalg.solve(K + s2n * eye, y))

    theta0 = np.log([0.3, 0.3, 1.0])
    st = fit.adam_sigma_loop(lambda t, s, j: (grad(t, s), {}), quad, N, theta0, 0.1, 25, lr0=0.05, lr1=0.01,
                             n_sched=25, grad_tol=0.0, param_tol=0.0)
    th, sig, g = solve.adam_sigma_steps(lambda t, s, j: grad(t, s), quad, N, theta0, 0.1, 25, lr0=0.05, lr1=0.01,
                                        n_sched=25)
    np.testing.assert_allclose([h["theta"] for h in st.history], th, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose([h["sigma2"] for h in st.history], sig, rtol=1e-12)
    # and the exact log-likelihood rose
    def ll(theta, s2n):
        K = orc.kmat(p.X, p.nu, np.exp(theta[:d]), s2=math.exp(theta[d]), kind=1)
        return solve.loglik_exact(K, s2n, y)

    assert ll(st.theta, st.sigma2) > ll(theta0, 0.1)


def test_stopping_rules():
    from paper_2508_01864_gb300 import fit

    c = np.array([0.2, -0.1])
    # the gradient of a concave quadratic: stops on the gradient norm
    st = fit.adam_sigma_loop(lambda t, s, j: (-(t - c), {}), lambda t, s: 1.0, 1, np.zeros(2), 1.0, 100000,
                             lr0=0.01, lr1=0.001, n_sched=2000, grad_tol=1e-3, param_tol=0.0)
    assert st.step < 100000 and st.history[-1]["grad_norm"] < 1e-3
    # a vanishing rate: theta stalls, the 100-step change test stops the loop
    st = fit.adam_sigma_loop(lambda t, s, j: (np.ones(2), {}), lambda t, s: 1.0, 1, np.zeros(2), 1.0, 5000,
                             lr0=1e-9, lr1=1e-9, grad_tol=0.0, param_tol=1e-4)
    assert st.step == 101
    # the nugget update: y^T (K + s I)^{-1} y = N is its fixed point, = 2N doubles sigma^2 per step
    st = fit.adam_sigma_loop(lambda t, s, j: (np.zeros(1), {}), lambda t, s: 7.0, 7, np.zeros(1), 0.3, 3,
                             grad_tol=-1.0, param_tol=0.0)
    assert st.sigma2 == pytest.approx(0.3, rel=1e-15)
    st = fit.adam_sigma_loop(lambda t, s, j: (np.zeros(1), {}), lambda t, s: 14.0, 7, np.zeros(1), 0.3, 3,
                             grad_tol=-1.0, param_tol=0.0)
    assert st.sigma2 == pytest.approx(0.3 * 8, rel=1e-15)
