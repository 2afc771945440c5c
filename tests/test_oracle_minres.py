"""Pins of the oracle's MINRES (Paige and Saunders; the solver for the
symmetric systems K + sigma^2 I that the L1 kernel makes indefinite at
nu >= 3/2, d >= 2, App. B, Prop. 4) against what the mathematics fixes: the
dense solution, the minimal residual over an explicit Krylov basis (least
squares), the monotone residual, the recursive residual equal to the true
one, and the indefinite L1 kernel matrix of the oracle itself."""

import numpy as np
import pytest

import workloads
from oracle import solve


def sym_matrix(n, seed, neg=0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(0.5, 3.0, size=n)
    lam[:neg] *= -1.0
    return (Q * lam) @ Q.T, lam


@pytest.mark.parametrize("neg", [0, 5, 20])
def test_minres_solves_symmetric_systems(neg):
    A, _ = sym_matrix(60, 3 + neg, neg)
    b = np.random.default_rng(1).standard_normal(60)
    x, k, hist = solve.minres(lambda v: A @ v, b, 1e-12, 500)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
    assert np.allclose(x, ref, rtol=1e-9, atol=1e-10)
    assert k <= 60 + 5


def test_minres_minimises_the_residual_over_the_krylov_space():
    A, _ = sym_matrix(40, 7, neg=8)
    b = np.random.default_rng(2).standard_normal(40)
    for m in (1, 3, 6, 10):
        x, k, hist = solve.minres(lambda v: A @ v, b, 0.0, m)
        # explicit Krylov basis, orthonormalised, and the least-squares minimiser
        K = np.empty((40, m))
        v = b.copy()
        for j in range(m):
            K[:, j] = v
            v = A @ v
        Qk, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(A @ Qk, b, rcond=None)
        best = np.linalg.norm(b - A @ (Qk @ y))
        got = np.linalg.norm(b - A @ x)
        assert abs(got - best) <= 1e-10 * np.linalg.norm(b), (m, got, best)
        assert abs(hist[-1] - got) <= 1e-10 * np.linalg.norm(b)  # recursive = true residual


def test_minres_residual_never_grows():
    A, _ = sym_matrix(80, 11, neg=30)
    b = np.random.default_rng(3).standard_normal(80)
    _, _, hist = solve.minres(lambda v: A @ v, b, 1e-10, 200)
    assert np.all(np.diff(hist) <= 1e-12 * np.linalg.norm(b))


def test_minres_on_the_indefinite_l1_kernel(orc):
    """The L1 kernel at nu = 3/2, d = 2 (indefinite, Prop. 4 fails), where CG
    meets p^T A p <= 0: MINRES reaches the dense solution."""
    p = workloads.small(41, 400, 2, nu=1.5, ell=[0.1, 0.3])
    K = orc.kmat(p.X, p.nu, p.ell, kind=orc.L1)
    A = K + 0.01 * np.eye(p.N)
    assert np.linalg.eigvalsh(A).min() < 0  # indefinite
    x, k, _ = solve.minres(lambda v: A @ v, p.V[:, 0], 1e-10, 20000)
    assert np.linalg.norm(p.V[:, 0] - A @ x) <= 1.5e-10 * np.linalg.norm(p.V[:, 0])
    ref = np.linalg.solve(A, p.V[:, 0])
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.cond(A) * np.linalg.norm(ref)


def test_a_planted_sign_error_fails_the_pins():
    """The recurrence is sensitive to the rotation's sign convention: flipping
    the sign of gamma^(1) (a plausible slip) breaks the minimal-residual pin."""
    A, _ = sym_matrix(30, 5, neg=6)
    b = np.random.default_rng(4).standard_normal(30)
    src = solve.minres.__code__
    import types
    bad_src = __import__("inspect").getsource(solve.minres).replace(
        "gamma1 = s_prev * delta1 - c_prev * alpha", "gamma1 = c_prev * alpha - s_prev * delta1")
    ns = {"np": np}
    exec(bad_src, ns)
    x, _, _ = ns["minres"](lambda v: A @ v, b, 1e-12, 200)
    assert np.linalg.norm(b - A @ x) > 1e-6 * np.linalg.norm(b)
    assert src is solve.minres.__code__
