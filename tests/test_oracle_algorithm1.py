"""Pins for the oracle's Algorithm 1 outer loop (oracle.solve.algorithm1_outer):
the OLS start against numpy's least squares, the running average and the
stopping rule against a prescribed sequence of GLS estimates, the GLS
estimate at fixed parameters against least squares on data whitened by the
Cholesky factor of K + sigma^2 I, and the recovery of known fixed effects on
data simulated from the model.  No GPU."""

import math

import numpy as np
import pytest
from scipy import linalg

import workloads
from oracle import solve


def _design(seed=3, N=120):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (N, 2))
    H = np.column_stack([np.ones(N), X])
    y = H @ np.array([1.0, -0.5, 2.0]) + 0.3 * rng.standard_normal(N)
    return X, H, y


def test_the_first_descent_gets_the_ols_residual():
    X, H, y = _design()
    seen = []

    def descend(yc, theta, s2):
        seen.append(yc.copy())
        return theta, s2

    solve.algorithm1_outer(descend, lambda t, s: np.zeros(3), H, y, np.zeros(2), 0.1, 1e-9, 1)
    b_ls = np.linalg.lstsq(H, y, rcond=None)[0]
    np.testing.assert_allclose(seen[0], y - H @ b_ls, rtol=0, atol=1e-12)


def test_running_average_and_stopping_rule():
    """A prescribed sequence b_1, b_2, ... of GLS estimates: the descent of
    repetition i sees y - H mean(b_1..b_i), and the loop stops at the first
    i with ||b_i - b_{i-1}|| <= eps (b_0 = beta_OLS)."""
    X, H, y = _design()
    rng = np.random.default_rng(8)
    seq = [np.array([1.0, -0.5, 2.0]) + rng.standard_normal(3) * 0.5 ** k for k in range(8)]
    seq[5] = seq[4] + 1e-4  # the change falls below eps at i = 6
    calls = iter(seq)
    seen = []

    def descend(yc, theta, s2):
        seen.append(yc.copy())
        return theta + 1.0, s2 * 2.0  # marks each descent

    beta, theta, s2, reps = solve.algorithm1_outer(descend, lambda t, s: next(calls), H, y, np.zeros(2), 0.1,
                                                   1e-3, 50)
    assert len(reps) == 6
    np.testing.assert_array_equal(beta, seq[5])
    for i in range(1, 7):
        avg = np.mean(seq[:i], axis=0)
        np.testing.assert_allclose(seen[i], y - H @ avg, rtol=0, atol=1e-12)
        np.testing.assert_allclose(reps[i - 1][1], avg, rtol=1e-14)
    b_ols = np.linalg.lstsq(H, y, rcond=None)[0]
    changes = [np.linalg.norm(seq[0] - b_ols)] + [np.linalg.norm(seq[k] - seq[k - 1]) for k in range(1, 6)]
    np.testing.assert_allclose([r[2] for r in reps], changes, rtol=1e-13)
    # every descent starts where the previous one ended
    assert theta[0] == 7.0 and s2 == pytest.approx(0.1 * 2 ** 7)
    # max_rep bounds the loop when the changes stay large
    calls2 = iter(seq[:3])
    _, _, _, reps2 = solve.algorithm1_outer(descend, lambda t, s: next(calls2), H, y, np.zeros(2), 0.1, 1e-30, 3)
    assert len(reps2) == 3


@pytest.mark.parametrize("kind", [0, 1])
def test_gls_at_fixed_parameters_is_whitened_least_squares(orc, kind):
    """With descents that keep the parameters, every GLS estimate is the same:
    the loop stops at the second repetition with beta_GLS = the least-squares
    fit of C^{-1} y on C^{-1} H, C C^T = K + sigma^2 I."""
    X, H, y = _design(5, 150)
    nu, ell, s2n = 1.5, [0.2, 0.3], 0.05
    K = orc.kmat(X, nu, ell, kind=kind) if kind == 1 else orc.kmat(X, 0.5, ell, kind=kind)
    A = K + s2n * np.eye(len(y))

    def gls_fn(theta, s2):
        return solve.gls(lambda B: np.linalg.solve(A, B), y, H)[1]

    beta, _, _, reps = solve.algorithm1_outer(lambda yc, t, s: (t, s), gls_fn, H, y, np.zeros(3), s2n, 1e-12, 10)
    C = linalg.cholesky(A, lower=True)
    b_white = np.linalg.lstsq(linalg.solve_triangular(C, H, lower=True),
                              linalg.solve_triangular(C, y, lower=True), rcond=None)[0]
    assert len(reps) == 2 and reps[1][2] == 0.0
    np.testing.assert_allclose(beta, b_white, rtol=1e-10)
    np.testing.assert_allclose(reps[1][1], b_white, rtol=1e-10)


def test_recovers_known_fixed_effects(orc):
    """y = H beta* + f + noise with f drawn from the GP: after the loop (dense
    gradients, a few Adam steps per descent) beta_GLS is within 4 standard
    errors sqrt(diag((H^T A^{-1} H)^{-1})) of beta* (about 0.2 here)."""
    p = workloads.small(31, 250, 2, nu=1.5, ell=[0.2, 0.2])
    X, N = p.X, 250
    H = np.column_stack([np.ones(N), X])
    beta_star = np.array([1.0, -0.5, 2.0])
    rng = np.random.default_rng(12)
    ell_t, s2_t, sn_t = np.array([0.2, 0.2]), 0.05, 0.05
    Kt = orc.kmat(X, 1.5, ell_t, s2=s2_t, kind=1)
    f = linalg.cholesky(Kt + 1e-10 * np.eye(N), lower=True) @ rng.standard_normal(N)
    y = H @ beta_star + f + math.sqrt(sn_t) * rng.standard_normal(N)
    eye = np.eye(N)

    def descend(yc, theta, s2):
        def grad(th, s, j):
            ell, sc = np.exp(th[:2]), math.exp(th[2])
            K = orc.kmat(X, 1.5, ell, s2=sc, kind=1)
            dKs = [orc.mvm_dlogell_brute(X, eye, 1.5, ell, dim=m, s2=sc, kind=1) for m in range(2)] + [K]
            return solve.loglik_grad_exact(K, dKs, s, yc)

        def quad(th, s):
            K = orc.kmat(X, 1.5, np.exp(th[:2]), s2=math.exp(th[2]), kind=1)
            return float(yc @ np.linalg.solve(K + s * eye, yc))

        th, sg, _ = solve.adam_sigma_steps(grad, quad, N, theta, s2, 8, lr0=0.05, lr1=0.05, n_sched=8)
        return th[-1], sg[-1]

    def gls_fn(theta, s2):
        K = orc.kmat(X, 1.5, np.exp(theta[:2]), s2=math.exp(theta[2]), kind=1)
        return solve.gls(lambda B: np.linalg.solve(K + s2 * eye, B), y, H)[1]

    beta, theta, s2, reps = solve.algorithm1_outer(descend, gls_fn, H, y, np.log([0.3, 0.3, 0.1]), 0.2, 1e-3, 6)
    A = orc.kmat(X, 1.5, ell_t, s2=s2_t, kind=1) + sn_t * eye
    cov = np.linalg.inv(H.T @ np.linalg.solve(A, H))
    se = np.sqrt(np.diag(cov))
    assert se.max() < 0.25
    assert (np.abs(beta - beta_star) < 4 * se).all(), (beta, beta_star, se)
    assert 2 <= len(reps) <= 6
