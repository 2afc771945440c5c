"""GPU parity of the pivoted-Cholesky preconditioner (App. A.3) and of the
preconditioned solve, through the C ABI: the pivots and the factor against
the oracle's pivoted Cholesky (same pivots; each GPU pivot checked to be a
largest residual diagonal entry of the oracle's own computation), the
Woodbury apply and the Sylvester log-determinant against the oracle's, and
the preconditioned CG against dense solves and the brute-force product."""

import numpy as np
import pytest
import torch

import workloads
from gpu_util import colwise_relerr, to_dev
from oracle import solve as osolve

pytestmark = pytest.mark.gpu

CASES = [  # d, nu, kind, N, pattern
    (1, 0.5, "l1", 1537, "uniform"),
    (1, 2.5, "l1", 3001, "uniform"),
    (2, 1.5, "product", 2500, "uniform"),
    (2, 2.5, "product", 1800, "uniform"),
    (2, 1.5, "l1", 2200, "uniform"),
    (3, 2.5, "product", 1200, "uniform"),
    (3, 1.5, "l1", 1000, "uniform"),
    (2, 1.5, "product", 1600, "lattice"),
    (2, 0.5, "product", 900, "dups"),
    (2, 3.5, "product", 1500, "uniform"),
    (1, 4.5, "l1", 1200, "uniform"),
    (3, 3.5, "product", 800, "uniform"),
]


def oracle_factor(orc, p, kind, rank, forced):
    kk = 0 if kind == "l1" else 1
    col = lambda i: orc.kcols(p.X, [i], p.nu, p.ell, s2=p.s2, kind=kk)[:, 0]  # noqa: E731
    # the library stores its factor in FP32 and runs the recurrence on the
    # stored columns: the oracle follows the same rounding
    return osolve.pivoted_cholesky(col, np.full(p.N, p.s2), rank, forced=forced, tie_rtol=1e-9,
                                   tie_atol=1e-12 * p.s2, store=osolve.f32_store)


@pytest.mark.parametrize("d,nu,kind,N,pattern", CASES)
def test_factor_pivots_trace_logdet(fgk_mod, orc, d, nu, kind, N, pattern):
    p = workloads.small(700 + d * 10 + N % 7, N, d, nu=nu, ell=[0.2, 0.35, 0.5][:d], pattern=pattern, s2=1.3)
    check_factor(fgk_mod, orc, p, kind, pattern, free_pivots=pattern == "uniform" and nu <= 2.5)


@pytest.mark.parametrize("kind", ["product", "l1"])
def test_factor_with_coordinates_beyond_the_exponential_tables(fgk_mod, orc, kind):
    """Points on [-50, 50]^2 with lengthscales (0.1, 0.12): scaled
    coordinates reach 866 and 722, beyond the 700 up to which the pivot steps
    take e^{-|x_i - x_p|} from tables of e^{+-x}, so rows (and pivots) outside
    them fall back to the exponential within the same factorisation."""
    p = workloads.small(9001, 1200, 2, nu=1.5, ell=[0.1, 0.12], pattern="wide", s2=1.3)
    a = np.sqrt(3.0) / np.array([0.1, 0.12])
    out = np.abs(p.X * a).max(axis=1) > 700.0
    assert 0.05 < out.mean() < 0.5  # both kinds of rows are present
    check_factor(fgk_mod, orc, p, kind, "wide", free_pivots=False)


def check_factor(fgk, orc, p, kind, pattern, free_pivots):
    rank, s2n = 60, 0.02
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, outscale2=p.s2, kind=kind) as h:
        with fgk.fgk_precond_build(h, rank, s2n) as pc:
            info = fgk.fgk_precond_info(pc)
            L = fgk.fgk_precond_factor(pc).cpu().numpy()
            R = np.random.default_rng(5).standard_normal((p.N, 3))
            Z = fgk.fgk_precond_apply(pc, to_dev(R)).cpu().numpy()
    piv = np.array(info["pivots"])
    Lo, pivo, dres = oracle_factor(orc, p, kind, rank, forced=piv)
    assert info["rank"] == Lo.shape[1] == len(piv)
    # both sides round each new column to FP32 from values that agree to
    # ~1e-14 (float pairs vs FP64); an entry that sits on a rounding boundary
    # differs by one FP32 step (6e-8 relative), and a differing pivot row
    # carries that into the later columns, divided by sqrt(d_m) of their
    # pivots: the bound grows as sqrt(s2 / d_min) once pivot residuals are small
    d_min = min(Lo[piv[m], m] ** 2 for m in range(len(piv)))
    tol_L = 1e-5 * np.sqrt(p.s2) * max(1.0, np.sqrt(1e-4 * p.s2 / d_min))
    assert np.abs(L - Lo).max() <= tol_L, (np.abs(L - Lo).max(), tol_L)
    if free_pivots:  # generic positions: the same pivots without forcing
        # (the smoother kernels leave near-ties between residual diagonals, which
        # two roundings may order differently; the forced comparison above covers them)
        _, free, _ = oracle_factor(orc, p, kind, rank, forced=None)
        assert np.array_equal(free, piv)
    assert abs(info["trace_resid"] - dres.sum()) <= 1e-9 * p.N * p.s2
    # the apply inverts the SPD matrix of its own stored factor,
    # (L L^T + sigma^2 I) Z = R (a validity check, no oracle value), to a
    # residual of its float-pair arithmetic (~2^-48) times cond(P)
    PZ = L @ (L.T @ Z) + s2n * Z
    kappa = (np.linalg.norm(L, 2) ** 2 + s2n) / s2n
    assert (colwise_relerr(PZ, R) <= 1e-13 * kappa).all()
    # and agrees with the oracle's Woodbury apply and Sylvester log det of the factor
    assert abs(info["logdet"] - osolve.precond_logdet(L, s2n)) <= 1e-10 * abs(info["logdet"]) + 1e-8
    Zo = osolve.woodbury_apply(Lo, s2n, R)
    assert (colwise_relerr(Z, Zo) <= 1e-5).all()


def test_rank_exhaustion_and_rank_zero(fgk_mod, orc):
    fgk = fgk_mod
    # 12 distinct points, each twice: K has rank 12.  The factor stops once
    # the largest residual diagonal is at most 1e-12 s2: at rank 12 in exact
    # arithmetic; the FP32 rounding of the stored columns leaves a residual
    # that a few more columns take up, so it stops before the 22 asked for
    base = workloads.small(31, 12, 2, nu=1.5, ell=[0.3, 0.3])
    X = np.concatenate([base.X, base.X])
    p = workloads.Problem("dup2", X, 1.5, np.array([0.3, 0.3]))
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        with fgk.fgk_precond_build(h, 22, 0.1) as pc:
            info = fgk.fgk_precond_info(pc)
        assert info["rank_requested"] == 22 and 12 <= info["rank"] < 22, info["rank"]
        Lo, pivo, dres = oracle_factor(orc, p, "product", 22, forced=np.array(info["pivots"]))
        assert Lo.shape[1] == info["rank"] and dres.max() <= 1e-10 * p.s2
        with fgk.fgk_precond_build(h, 0, 0.1) as pc0:  # P = sigma^2 I
            R = np.random.default_rng(1).standard_normal((p.N, 2))
            Z = fgk.fgk_precond_apply(pc0, to_dev(R)).cpu().numpy()
            assert np.allclose(Z, R / 0.1, rtol=1e-15, atol=0)
            assert fgk.fgk_precond_info(pc0)["rank"] == 0


@pytest.mark.parametrize("d,nu", [(1, 2.5), (2, 1.5), (2, 2.5), (3, 1.5), (2, 3.5), (2, 4.5)])
@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_pcg_matches_dense_solve(fgk_mod, orc, d, nu, mode):
    fgk = fgk_mod
    p = workloads.small(800 + d, 1500, d, nu=nu, ell=[0.15, 0.3, 0.45][:d], nrhs=3)
    sigma2, tol = 0.01, 1e-10
    A = orc.kmat(p.X, p.nu, p.ell, kind=1) + sigma2 * np.eye(p.N)
    ref = np.linalg.solve(A, p.V)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        with fgk.fgk_precond_build(h, 80, sigma2) as pc:
            alpha, _, info, rc = fgk.fgk_cg_solve(h, to_dev(p.V), sigma2, tol=tol, mode=mode, precond=pc)
        _, _, plain, _ = fgk.fgk_cg_solve(h, to_dev(p.V), sigma2, tol=tol, mode=mode)
    a = alpha.cpu().numpy()
    assert rc == 0
    res = np.linalg.norm(p.V - A @ a, axis=0) / np.linalg.norm(p.V, axis=0)
    assert (res <= tol).all(), res
    cond = np.linalg.cond(A)
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) <= cond * tol
    assert info["iterations"] < plain["iterations"], (info, plain)


def test_pcg_gls_matches_dense_gls(fgk_mod, orc):
    fgk = fgk_mod
    p = workloads.small(611, 1300, 2, nu=2.5, ell=[0.2, 0.3], nrhs=1)
    H = np.column_stack([np.ones(p.N), p.X])
    y = p.V[:, 0] + H @ np.array([1.0, 0.5, -2.0])
    sigma2 = 0.01
    A = orc.kmat(p.X, p.nu, p.ell, kind=1) + sigma2 * np.eye(p.N)
    a_ref, b_ref = osolve.gls(lambda B: np.linalg.solve(A, B), y, H)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        with fgk.fgk_precond_build(h, 100, sigma2) as pc:
            alpha, beta, info, rc = fgk.fgk_cg_solve(h, to_dev(y), sigma2, L=-1, tol=1e-11, mode="mixed",
                                                     precond=pc)
    assert rc == 0
    cond = np.linalg.cond(A)
    b = beta.cpu().numpy()[:, 0]
    assert np.linalg.norm(b - b_ref) <= cond * 1e-11 * np.linalg.norm(b_ref)
    a = alpha.cpu().numpy()
    assert np.linalg.norm(a - a_ref) <= cond * 1e-11 * np.linalg.norm(a_ref)


def test_precond_must_match_plan_and_sigma2(fgk_mod):
    fgk = fgk_mod
    p = workloads.small(5, 500, 2, nu=1.5)
    q = workloads.small(6, 500, 2, nu=1.5)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h, \
            fgk.fgk_build(to_dev(q.X), q.nu, q.ell, kind="product") as h2:
        with fgk.fgk_precond_build(h, 10, 0.01) as pc:
            y = to_dev(p.V)
            with pytest.raises(fgk.FgkError) as e:
                fgk.fgk_cg_solve(h, y, 0.02, precond=pc)
            assert e.value.code == -1
            with pytest.raises(fgk.FgkError):
                fgk.fgk_cg_solve(h2, y, 0.01, precond=pc)


@pytest.mark.parametrize("mode", ["mixed", "f64"])
def test_c2_full_size_pcg(fgk_mod, orc, mode):
    """The d=2 configuration with the paper's rank-100 preconditioner: the
    tolerance 1e-8 on the FP64 true residual, recomputed here from the
    library's FP64 product (checked against the brute-force oracle on
    sampled rows), in far fewer iterations than without it."""
    fgk = fgk_mod
    p = workloads.c2()
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        with fgk.fgk_precond_build(h, 100, p.sigma2) as pc:
            alpha, _, info, rc = fgk.fgk_cg_solve(h, to_dev(p.V), p.sigma2, tol=1e-8, maxit=20000, mode=mode,
                                                  precond=pc)
        assert rc == 0, info
        assert info["max_true_resid"] <= 1e-8
        assert info["iterations"] < 3000, info
        Ka = fgk.fgk_matvec(h, alpha.reshape(-1, 1).contiguous(), "f64").cpu().numpy()[:, 0]
    a = alpha.cpu().numpy().reshape(-1)
    rows = np.sort(np.random.default_rng(10).choice(p.N, 200, replace=False))
    ref = orc.mvm_brute(p.X, a, p.nu, p.ell, kind=1, rows=rows)
    assert np.linalg.norm(Ka[rows] - ref) <= 1e-12 * np.linalg.norm(ref)
    r = p.V[:, 0] - Ka - p.sigma2 * a
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(p.V[:, 0])
