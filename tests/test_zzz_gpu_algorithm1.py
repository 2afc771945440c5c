"""GPU check of Algorithm 1's outer loop (paper_2508_01864_gb300.fit.fit_gls):
GLS estimates from fgk_cg_solve with the covariates H and descents from
fit_adam_sigma (fgk_loglik_grad with Hutchinson probes), against the oracle's
outer loop driven by its dense forms with the same probes."""

import math

import numpy as np
import pytest

import workloads
from oracle import solve

pytestmark = pytest.mark.gpu

N, D, NU = 500, 2, 1.5


def _data():
    p = workloads.small(85, N, D, nu=NU, ell=[0.2, 0.35])
    H = np.column_stack([np.ones(N), p.X])
    rng = np.random.default_rng(85)
    y = H @ np.array([0.5, 1.0, -1.0]) + np.sin(5 * p.X[:, 0]) + np.cos(3 * p.X[:, 1]) \
        + 0.1 * rng.standard_normal(N)
    return p.X, H, y


def _probes(j):
    return np.random.default_rng(2000 + j).standard_normal((N, 8))


def oracle_fit(orc, X, H, y, theta0, sigma2_0, steps, reps):
    eye = np.eye(N)

    def K_of(theta):
        return orc.kmat(X, NU, np.exp(theta[:D]), s2=math.exp(theta[D]), kind=1)

    def descend(yc, theta, s2):
        def grad(th, s, j):
            ell, sc = np.exp(th[:D]), math.exp(th[D])
            K = K_of(th)
            A = K + s * eye
            dKs = [orc.mvm_dlogell_brute(X, eye, NU, ell, dim=m, s2=sc, kind=1) for m in range(D)] + [K, s * eye]
            est = solve.loglik_grad_estimate(lambda V: np.linalg.solve(A, V), [lambda V, M=M: M @ V for M in dKs],
                                             yc, _probes(j))
            return est[:-1]

        def quad(th, s):
            return float(yc @ np.linalg.solve(K_of(th) + s * eye, yc))

        th, sg, _ = solve.adam_sigma_steps(grad, quad, N, theta, s2, steps)
        return th[-1], sg[-1]

    def gls_fn(theta, s2):
        return solve.gls(lambda B: np.linalg.solve(K_of(theta) + s2 * eye, B), y, H)[1]

    return solve.algorithm1_outer(descend, gls_fn, H, y, theta0, sigma2_0, 0.0, reps)


def test_fit_gls_matches_the_oracle(fgk_mod, orc):
    from paper_2508_01864_gb300 import fit

    X, H, y = _data()
    ell0, s20, sig0 = np.array([0.3, 0.3]), 1.0, 0.1
    got = fit.fit_gls(X, y, H, NU, ell0, s20, sig0, _probes, 3, eps_beta=0.0, max_rep=2, tol=1e-11, mode="f64",
                      grad_tol=0.0, param_tol=0.0)
    beta, theta, s2, reps = oracle_fit(orc, X, H, y, np.concatenate([np.log(ell0), [math.log(s20)]]), sig0, 3, 2)
    assert got.reps == len(reps) == 2
    for hist, (b, bavg, _, th, sg) in zip(got.history[1:], reps):
        # beta from solves to 1e-11 at cond(K + sigma^2 I) ~ 2e4: agreement to ~1e-7, tested at 1e-5
        np.testing.assert_allclose(hist["beta_gls"], b, rtol=1e-5, atol=1e-7 * np.abs(b).max())
        np.testing.assert_allclose(hist["beta_avg"], bavg, rtol=1e-5, atol=1e-7 * np.abs(b).max())
        np.testing.assert_allclose(hist["theta"], th, rtol=1e-6, atol=1e-8)
        assert hist["sigma2"] == pytest.approx(sg, rel=1e-6)
    np.testing.assert_allclose(got.beta, beta, rtol=1e-5, atol=1e-7 * np.abs(beta).max())
    np.testing.assert_allclose(got.theta, theta, rtol=1e-6, atol=1e-8)
    assert got.sigma2 == pytest.approx(s2, rel=1e-6)
