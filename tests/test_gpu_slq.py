"""GPU checks of the log-determinant by stochastic Lanczos quadrature
(fgk_slq_logdet: Algorithm 2's Lanczos matrices from the library's FP64 CG,
eq. approximationLogDet, the preconditioned form of App. A.3) and of the
Hutchinson trace term of eq. gp_log_likelihood_derivative built from its
solves and fgk_matvec_dlogell, through the C ABI, against the oracle."""

import numpy as np
import pytest
import torch

import workloads
from gpu_util import to_dev
from oracle import solve

pytestmark = pytest.mark.gpu


def _apply_A(orc, p, kind, s2):
    return lambda V: orc.mvm_brute(p.X, V, p.nu, p.ell, kind=kind).reshape(V.shape) + s2 * V


@pytest.mark.parametrize("d,nu,N", [(1, 0.5, 2500), (2, 1.5, 3000), (3, 2.5, 1500)])
def test_quadratures_match_the_oracle_over_fixed_steps(fgk_mod, orc, d, nu, N):
    """Ten steps: before the Ritz values converge, where finite-precision
    Lanczos is still insensitive to rounding (the oracle's own quadratures
    move by ~1e-14 under 1e-15 perturbations of the products at ten steps,
    by ~1e-4 at 25 once orthogonality is lost; the accuracy of converged
    estimates is checked against the exact log-determinant below)."""
    fgk = fgk_mod
    s2, m, nprobe = 0.1, 10, 6
    p = workloads.small(300 + d, N, d, nu=nu, ell=[0.2, 0.3, 0.25][:d])
    B = np.random.default_rng(d).standard_normal((N, nprobe))
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        got = fgk.fgk_slq_logdet(h, to_dev(B), s2, m, tol=1e-30, want_solves=True)
    est, quad, steps, X = solve.slq_logdet(_apply_A(orc, p, 1, s2), B, m, 1e-30)
    assert got["steps"] == [m] * nprobe and (steps == m).all()
    np.testing.assert_allclose(got["quad"], quad, rtol=1e-10)
    assert got["logdet"] == pytest.approx(est, rel=1e-10)
    # the partial solves after ten steps amplify the products' rounding more
    # (~1e-10 per 1e-15 of product error at d = 1 on the CPU; the FP64 scans
    # differ from the brute force by up to ~1e-13)
    np.testing.assert_allclose(got["X"].cpu().numpy(), X, rtol=0, atol=1e-8 * np.abs(X).max())


def test_preconditioned_probes_and_quadratures_match_the_oracle(fgk_mod, orc):
    fgk = fgk_mod
    s2, rank, m, nprobe, N = 0.05, 20, 20, 4, 2000
    p = workloads.small(41, N, 2, nu=1.5, ell=[0.15, 0.3])
    rng = np.random.default_rng(42)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h, fgk.fgk_precond_build(h, rank, s2) as pc:
        info = fgk.fgk_precond_info(pc)
        k = info["rank"]
        Er = rng.standard_normal((k, nprobe))
        En = rng.standard_normal((N, nprobe))
        Bg = fgk.fgk_precond_sample(pc, to_dev(Er), to_dev(En))
        got = fgk.fgk_slq_logdet(h, Bg, s2, m, tol=1e-30, pc=pc)
    # the oracle's own factor, following the library's pivots after checking
    # each is a largest residual diagonal entry
    K = orc.kmat(p.X, p.nu, p.ell, kind=1)
    # (the library stores its factor in FP32, the recurrence run on the stored columns)
    L, _, _ = solve.pivoted_cholesky(lambda i: K[:, i], np.diag(K), k, forced=info["pivots"], tie_rtol=1e-9,
                                     tie_atol=1e-12 * K[0, 0], store=solve.f32_store)
    B = L @ Er + np.sqrt(s2) * En
    np.testing.assert_allclose(Bg.cpu().numpy(), B, rtol=0, atol=1e-6 * np.abs(B).max())
    est, quad, steps, _ = solve.slq_logdet(_apply_A(orc, p, 1, s2), B, m, 1e-30,
                                           lambda R: solve.woodbury_apply(L, s2, R), solve.precond_logdet(L, s2))
    assert got["logdet_precond"] == pytest.approx(solve.precond_logdet(L, s2), rel=1e-7)
    # P of the library is its FP32-stored factor's, which the oracle's factor
    # reproduces (up to an entry on a rounding boundary)
    np.testing.assert_allclose(got["quad"], quad, rtol=1e-6)


@pytest.mark.parametrize("rank", [0, 30])
def test_estimate_is_within_its_standard_error_of_the_exact_log_determinant(fgk_mod, orc, rank):
    fgk = fgk_mod
    s2, N, nprobe = 0.05, 1500, 64
    p = workloads.small(77, N, 2, nu=2.5, ell=[0.2, 0.2])
    K = orc.kmat(p.X, p.nu, p.ell, kind=1)
    exact = np.linalg.slogdet(K + s2 * np.eye(N))[1]
    rng = np.random.default_rng(5)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        if rank:
            with fgk.fgk_precond_build(h, rank, s2) as pc:
                k = fgk.fgk_precond_info(pc)["rank"]
                B = fgk.fgk_precond_sample(pc, to_dev(rng.standard_normal((k, nprobe))),
                                           to_dev(rng.standard_normal((N, nprobe))))
                got = fgk.fgk_slq_logdet(h, B, s2, 2000, tol=1e-10, pc=pc)
        else:
            got = fgk.fgk_slq_logdet(h, to_dev(rng.standard_normal((N, nprobe))), s2, 2000, tol=1e-10)
    q = np.array(got["quad"])
    se = q.std() / np.sqrt(nprobe)
    assert got["solve_status"] == 0 and got["max_true_resid"] <= 1e-10
    assert abs(got["logdet"] - exact) < 4 * se, (got["logdet"], exact, se)


def test_hutchinson_trace_of_the_likelihood_gradient(fgk_mod, orc):
    """tr((K + s2 I)^{-1} dK/d log ell_m) by Hutchinson probes: the solves of
    fgk_slq_logdet times the gradient product, against the dense trace."""
    fgk = fgk_mod
    s2, N, nprobe = 0.05, 1200, 64
    p = workloads.small(91, N, 2, nu=1.5, ell=[0.2, 0.35])
    A = orc.kmat(p.X, p.nu, p.ell, kind=1) + s2 * np.eye(N)
    Ainv = np.linalg.inv(A)
    rng = np.random.default_rng(17)
    B = rng.standard_normal((N, nprobe))
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        got = fgk.fgk_slq_logdet(h, to_dev(B), s2, 3000, tol=1e-10, want_solves=True)
        X = got["X"]
        for dim in (0, 1):
            D = fgk.fgk_matvec_dlogell(h, to_dev(B), dim, "f64")
            samples = (X * D).sum(0).cpu().numpy()  # b^T A^{-1} dK b
            dK = orc.mvm_dlogell_brute(p.X, np.eye(N), p.nu, p.ell, dim=dim, kind=1)
            exact = float(np.sum(Ainv * dK.T))
            se = samples.std() / np.sqrt(nprobe)
            assert abs(samples.mean() - exact) < 4 * se, (dim, samples.mean(), exact, se)
