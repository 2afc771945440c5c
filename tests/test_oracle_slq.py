"""Pins for the log-determinant oracle (App. A.2: Lanczos matrices from the CG
coefficients of Algorithm 2, eq. approximationLogDet, the preconditioned form
of App. A.3), each against something other than itself: an explicit Lanczos
recurrence with full reorthogonalisation, the polynomial exactness of Gauss
quadrature, dense matrix logarithms, and the mean over many probes against
numpy's slogdet."""

import numpy as np
import pytest

import workloads
from oracle import solve


def spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    return (Q * lam) @ Q.T


def fn_of(A, f):
    w, V = np.linalg.eigh(A)
    return (V * f(w)) @ V.T


def explicit_lanczos(A, b, m):
    """Textbook Lanczos tridiagonalisation started at b / ||b||, with full
    reorthogonalisation (T from the three-term recurrence)."""
    n = b.size
    Vs = np.zeros((n, m))
    a, bt = np.zeros(m), np.zeros(m)
    v = b / np.linalg.norm(b)
    prev, bprev = np.zeros(n), 0.0
    for j in range(m):
        Vs[:, j] = v
        w = A @ v - bprev * prev
        a[j] = v @ w
        w -= a[j] * v
        w -= Vs[:, : j + 1] @ (Vs[:, : j + 1].T @ w)
        bt[j] = np.linalg.norm(w)
        prev, bprev, v = v, bt[j], w / bt[j]
    return np.diag(a) + np.diag(bt[: m - 1], 1) + np.diag(bt[: m - 1], -1)


def test_cg_coefficients_give_the_lanczos_matrix():
    A = spd(60, 1)
    b = np.random.default_rng(2).standard_normal(60)
    _, al, be, ga = solve.cg_lanczos(lambda V: A @ V, b, 1e-30, 15)
    T = solve.lanczos_T(al[0], be[0])
    np.testing.assert_allclose(T, explicit_lanczos(A, b, 15), rtol=1e-9, atol=1e-9 * np.abs(T).max())
    assert ga[0] == pytest.approx(b @ b, rel=1e-15)


@pytest.mark.parametrize("m", [1, 2, 6])
def test_gauss_quadrature_is_exact_for_polynomials(m):
    A = spd(50, 3, cond=50.0)
    b = np.random.default_rng(4).standard_normal(50)
    _, al, be, ga = solve.cg_lanczos(lambda V: A @ V, b, 1e-30, m)
    T = solve.lanczos_T(al[0], be[0])
    for p in range(2 * m):
        quad = ga[0] * np.linalg.matrix_power(T, p)[0, 0]
        exact = b @ np.linalg.matrix_power(A, p) @ b
        assert quad == pytest.approx(exact, rel=1e-9), p
    # and not beyond: degree 2m differs
    quad = ga[0] * np.linalg.matrix_power(T, 2 * m)[0, 0]
    assert abs(quad - b @ np.linalg.matrix_power(A, 2 * m) @ b) > 1e-8 * abs(quad)


def test_converged_quadrature_is_the_quadratic_form_of_the_logarithm():
    A = spd(40, 5, cond=1e4)
    B = np.random.default_rng(6).standard_normal((40, 3))
    est, quad, steps, X = solve.slq_logdet(lambda V: A @ V, B, 200, 1e-13)
    logA = fn_of(A, np.log)
    np.testing.assert_allclose(quad, np.einsum("ij,ij->j", B, logA @ B), rtol=1e-9)
    np.testing.assert_allclose(X, np.linalg.solve(A, B), rtol=1e-8)
    assert (steps < 200).all()  # converged (finite precision may take more than N steps)


def test_preconditioned_quadrature_is_that_of_the_split_operator(orc):
    p = workloads.small(8, 60, 2, nu=1.5, ell=[0.3, 0.4])
    K = orc.kmat(p.X, p.nu, p.ell, kind=1)
    s2 = 0.05
    A = K + s2 * np.eye(60)
    L, _, _ = solve.pivoted_cholesky(lambda i: K[:, i], np.diag(K), 6)
    P = L @ L.T + s2 * np.eye(60)
    B = np.random.default_rng(9).standard_normal((60, 2))
    _, quad, _, _ = solve.slq_logdet(lambda V: A @ V, B, 200, 1e-13, lambda R: solve.woodbury_apply(L, s2, R),
                                     solve.precond_logdet(L, s2))
    Pmh = fn_of(P, lambda w: w ** -0.5)
    At = Pmh @ A @ Pmh
    Bt = Pmh @ B
    np.testing.assert_allclose(quad, np.einsum("ij,ij->j", Bt, fn_of(At, np.log) @ Bt), rtol=1e-8)


@pytest.mark.parametrize("precond", [False, True])
def test_slq_estimate_is_unbiased(orc, precond):
    p = workloads.small(12, 40, 2, nu=2.5, ell=[0.3, 0.3])
    K = orc.kmat(p.X, p.nu, p.ell, kind=1)
    s2 = 0.1
    A = K + s2 * np.eye(40)
    exact = np.linalg.slogdet(A)[1]
    rng = np.random.default_rng(13)
    nprobe = 3000
    if precond:
        L, _, _ = solve.pivoted_cholesky(lambda i: K[:, i], np.diag(K), 4)
        B = L @ rng.standard_normal((L.shape[1], nprobe)) + np.sqrt(s2) * rng.standard_normal((40, nprobe))
        Pinv = lambda R: solve.woodbury_apply(L, s2, R)  # noqa: E731
        ldp = solve.precond_logdet(L, s2)
    else:
        B = rng.standard_normal((40, nprobe))
        Pinv, ldp = None, 0.0
    est, quad, _, _ = solve.slq_logdet(lambda V: A @ V, B, 100, 1e-12, Pinv, ldp)
    se = quad.std() / np.sqrt(nprobe)
    assert abs(est - exact) < 4 * se + 1e-9 * abs(exact), (est, exact, se)
