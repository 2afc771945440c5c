"""Pins for the oracle's preconditioner (App. A.3): the rank-k pivoted
Cholesky factor, the Woodbury apply, the Sylvester log-determinant and
Algorithm 2 with s_P = P^{-1}, against LAPACK and the definitions."""

import numpy as np
import pytest

import workloads
from oracle import solve


def _kfuns(orc, p, kind):
    K = orc.kmat(p.X, p.nu, p.ell, kind=kind)
    return K, (lambda i: orc.kcols(p.X, [i], p.nu, p.ell, kind=kind)[:, 0])


@pytest.mark.parametrize("d,nu,kind", [(1, 0.5, 0), (2, 1.5, 1), (3, 2.5, 1), (2, 2.5, 1)])
def test_full_rank_is_the_pivoted_cholesky_factor(orc, d, nu, kind):
    """k = N: L L^T = K and the rows of L in pivot order form the lower
    triangular Cholesky factor of K permuted by the pivots."""
    p = workloads.small(61 + d, 60, d, nu=nu, ell=[0.4, 0.6, 0.5][:d])
    K, col = _kfuns(orc, p, kind)
    L, piv, dres = solve.pivoted_cholesky(col, np.diag(K), p.N)
    assert L.shape[1] == p.N and sorted(piv.tolist()) == list(range(p.N))
    assert np.abs(L @ L.T - K).max() <= 1e-10 * np.abs(K).max()
    Lp = L[piv]
    assert np.abs(np.triu(Lp, 1)).max() <= 1e-12
    ref = np.linalg.cholesky(K[np.ix_(piv, piv)])
    assert np.abs(Lp - ref).max() <= 1e-9
    assert np.abs(dres).max() <= 1e-10


def test_greedy_pivots_and_residual_diagonal(orc):
    """Each pivot is the largest diagonal entry of K - L_m L_m^T (computed
    densely), the residual diagonal equals that diagonal, and its trace
    (the approximation error) falls with the rank."""
    p = workloads.small(65, 300, 2, nu=1.5, ell=[0.15, 0.3])
    K, col = _kfuns(orc, p, 1)
    L, piv, dres = solve.pivoted_cholesky(col, np.diag(K), 40)
    traces = []
    for m in range(L.shape[1]):
        rdiag = np.diag(K) - (L[:, :m] ** 2).sum(axis=1)
        assert rdiag[piv[m]] >= rdiag.max() * (1 - 1e-12)
        traces.append(rdiag.sum())
    assert np.allclose(dres, np.diag(K - L @ L.T), atol=1e-12)
    assert all(b < a for a, b in zip(traces, traces[1:]))


def test_first_pivots_on_a_line(orc):
    """A stationary kernel has a constant diagonal: the first pivot is index
    0 (ties go to the first index); the second is the point where k(x_0, .)
    is smallest, i.e. the farthest one on a line."""
    rng = np.random.default_rng(7)
    X = rng.uniform(0, 1, size=(200, 1))
    p = workloads.Problem("line", X, 1.5, np.array([0.2]), sigma2=0.01, V=None)
    K, col = _kfuns(orc, p, 0)
    L, piv, _ = solve.pivoted_cholesky(col, np.diag(K), 2)
    assert piv[0] == 0
    assert piv[1] == int(np.argmax(np.abs(X[:, 0] - X[0, 0])))


def test_woodbury_and_sylvester(orc):
    rng = np.random.default_rng(3)
    L = rng.standard_normal((120, 7))
    R = rng.standard_normal((120, 3))
    for s2 in (0.01, 1.0, 30.0):
        P = L @ L.T + s2 * np.eye(120)
        assert np.allclose(solve.woodbury_apply(L, s2, R), np.linalg.solve(P, R), rtol=1e-10, atol=1e-12)
        sign, ld = np.linalg.slogdet(P)
        assert sign > 0 and abs(solve.precond_logdet(L, s2) - ld) <= 1e-10 * abs(ld)


def test_pcg_with_the_exact_preconditioner_takes_one_iteration(orc):
    p = workloads.small(66, 80, 2, nu=1.5, ell=[0.3, 0.3], nrhs=2)
    K, col = _kfuns(orc, p, 1)
    L, _, _ = solve.pivoted_cholesky(col, np.diag(K), p.N)
    s2 = 0.05

    def A(B):
        return K @ B + s2 * B

    x, iters = solve.cg(A, p.V, 1e-10, 50, apply_Pinv=lambda R: solve.woodbury_apply(L, s2, R))
    assert (iters == 1).all()
    assert (solve.true_residual(A, x, p.V) <= 1e-9).all()


@pytest.mark.parametrize("nu,kind", [(1.5, 1), (2.5, 1), (0.5, 0)])
def test_pcg_matches_dense_solve_with_fewer_iterations(orc, nu, kind):
    p = workloads.small(67, 500, 2, nu=nu, ell=[0.1, 0.3], nrhs=2)
    K, col = _kfuns(orc, p, kind)
    s2 = 0.01
    L, _, _ = solve.pivoted_cholesky(col, np.diag(K), 60)

    def A(B):
        return K @ B + s2 * B

    x, it_pc = solve.cg(A, p.V, 1e-10, 5000, apply_Pinv=lambda R: solve.woodbury_apply(L, s2, R))
    _, it_plain = solve.cg(A, p.V, 1e-10, 5000)
    assert (solve.true_residual(A, x, p.V) <= 2e-10).all()
    ref = solve.dense_solve(K, s2, p.V)
    cond = np.linalg.cond(K + s2 * np.eye(p.N))
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < cond * 1e-10
    assert (it_pc < it_plain).all(), (it_pc, it_plain)


def test_forced_pivots_are_checked(orc):
    p = workloads.small(68, 100, 2, nu=1.5, ell=[0.2, 0.2])
    K, col = _kfuns(orc, p, 1)
    L, piv, _ = solve.pivoted_cholesky(col, np.diag(K), 10)
    L2, piv2, _ = solve.pivoted_cholesky(col, np.diag(K), 10, forced=piv)
    assert (piv2 == piv).all() and np.array_equal(L, L2)
    bad = piv.copy()
    bad[3] = piv[0]  # an exhausted pivot is never a largest residual
    with pytest.raises(ValueError):
        solve.pivoted_cholesky(col, np.diag(K), 10, forced=bad)


def test_factor_stored_in_fp32(orc):
    """store = f32_store: every stored entry is an FP32 value; the
    recurrence runs on the stored columns, so the residual diagonal is
    exactly diag(K - L L^T) of the stored factor (each pivot the largest of
    it), and the next columns take up each rounding: the residual trace at
    the same rank equals the unrounded factor's to 1e-6."""
    p = workloads.small(66, 500, 2, nu=1.5, ell=[0.15, 0.3], s2=1.7)
    K = orc.kmat(p.X, p.nu, p.ell, s2=1.7, kind=1)
    col = lambda i: K[:, i]  # noqa: E731
    L, piv, dres = solve.pivoted_cholesky(col, np.diag(K), 80, store=solve.f32_store)
    Lx, _, dx = solve.pivoted_cholesky(col, np.diag(K), 80)
    assert np.array_equal(L.astype(np.float32).astype(np.float64), L)
    assert np.allclose(dres, np.diag(K - L @ L.T), rtol=0, atol=1e-13)
    for m in range(L.shape[1]):
        rdiag = np.diag(K) - (L[:, :m] ** 2).sum(axis=1)
        assert rdiag[piv[m]] >= rdiag.max() * (1 - 1e-12)
    assert abs(dres.sum() - dx.sum()) <= 1e-6 * dx.sum()
    # a matrix of exact rank 12 (12 points, each twice): the rounding of the
    # stored columns leaves a residual that a few more columns take up
    base = workloads.small(31, 12, 2, nu=1.5, ell=[0.3, 0.3])
    X2 = np.concatenate([base.X, base.X])
    K2 = orc.kmat(X2, 1.5, np.array([0.3, 0.3]), kind=1)
    L2, _, d2 = solve.pivoted_cholesky(lambda i: K2[:, i], np.diag(K2), 40, store=solve.f32_store)
    assert 12 <= L2.shape[1] < 24 and d2.max() <= 1e-12
