"""GPU checks of the log-likelihood gradient (fgk_loglik_grad, eq.
gp_log_likelihood_derivative with Hutchinson probes) and of Algorithm 1's
gradient-descent loop built on it (paper_2508_01864_gb300.fit), against the
oracle's dense forms with the same probes."""

import math

import numpy as np
import pytest
import torch

import workloads
from gpu_util import to_dev
from oracle import solve

pytestmark = pytest.mark.gpu


def _problem(seed, N, d, nu):
    p = workloads.small(seed, N, d, nu=nu, ell=[0.2, 0.35, 0.3][:d], s2=1.3)
    y = np.sin(5 * p.X[:, 0]) + 0.1 * np.random.default_rng(seed).standard_normal(N)
    if d > 1:
        y += np.cos(3 * p.X[:, 1])
    return p, y


def _oracle_grad(orc, p, y, kind, s2n, ell, s2, B, apply_Pinv=None):
    kk = 0 if kind == "l1" else 1
    K = orc.kmat(p.X, p.nu, ell, s2=s2, kind=kk)
    A = K + s2n * np.eye(p.N)
    eye = np.eye(p.N)
    d = p.X.shape[1]
    if kind == "product" and d > 1:
        dKs = [orc.mvm_dlogell_brute(p.X, eye, p.nu, ell, dim=m, s2=s2, kind=kk) for m in range(d)]
    else:
        dKs = [orc.mvm_dlogell_brute(p.X, eye, p.nu, ell, dim=-1, s2=s2, kind=kk)]
    dKs += [K, s2n * eye]
    est = solve.loglik_grad_estimate(lambda V: np.linalg.solve(A, V), [lambda V, D=D: D @ V for D in dKs], y, B,
                                     apply_Pinv)
    return est, K


@pytest.mark.parametrize("d,nu,kind,N", [(2, 1.5, "product", 900), (2, 0.5, "l1", 700), (1, 2.5, "l1", 800),
                                         (3, 1.5, "product", 500)])
def test_gradient_matches_the_oracle_with_the_same_probes(fgk_mod, orc, d, nu, kind, N):
    fgk = fgk_mod
    s2n = 0.05
    p, y = _problem(60 + d, N, d, nu)
    B = np.random.default_rng(7).standard_normal((N, 8))
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, outscale2=p.s2, kind=kind) as h:
        got = fgk.fgk_loglik_grad(h, to_dev(y), to_dev(B), s2n, tol=1e-11, mode="f64")
    ref, _ = _oracle_grad(orc, p, y, kind, s2n, p.ell, p.s2, B)
    assert len(got["grad"]) == len(ref)
    np.testing.assert_allclose(got["grad"], ref, rtol=1e-7, atol=1e-8 * np.abs(ref).max())
    A = orc.kmat(p.X, p.nu, p.ell, s2=p.s2, kind=0 if kind == "l1" else 1) + s2n * np.eye(N)
    assert got["yAy"] == pytest.approx(float(y @ np.linalg.solve(A, y)), rel=1e-9)


def test_preconditioned_gradient_matches_the_oracle(fgk_mod, orc):
    fgk = fgk_mod
    s2n, N, rank, n = 0.05, 1200, 20, 8
    p, y = _problem(71, N, 2, 1.5)
    rng = np.random.default_rng(3)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, outscale2=p.s2, kind="product") as h, \
            fgk.fgk_precond_build(h, rank, s2n) as pc:
        info = fgk.fgk_precond_info(pc)
        k = info["rank"]
        Er, En = rng.standard_normal((k, n)), rng.standard_normal((N, n))
        Bg = fgk.fgk_precond_sample(pc, to_dev(Er), to_dev(En))
        got = fgk.fgk_loglik_grad(h, to_dev(y), Bg, s2n, tol=1e-11, mode="f64", pc=pc)
    K = orc.kmat(p.X, p.nu, p.ell, s2=p.s2, kind=1)
    # (the library stores its factor in FP32, the recurrence run on the stored columns)
    L, _, _ = solve.pivoted_cholesky(lambda i: K[:, i], np.diag(K), k, forced=info["pivots"], tie_rtol=1e-9,
                                     tie_atol=1e-12 * K[0, 0], store=solve.f32_store)
    B = L @ Er + math.sqrt(s2n) * En
    ref, _ = _oracle_grad(orc, p, y, "product", s2n, p.ell, p.s2, B, lambda R: solve.woodbury_apply(L, s2n, R))
    # the library's probes and P use its FP32-stored factor, which the oracle's reproduces
    np.testing.assert_allclose(got["grad"], ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def test_fit_steps_match_the_oracle(fgk_mod, orc):
    """Six steps of Algorithm 1's loop (Adam on log ell, log varsigma^2; the
    closed-form nugget) with the same probes on both sides."""
    from paper_2508_01864_gb300 import fit

    N, d, nu = 600, 2, 1.5
    p, y = _problem(81, N, d, nu)
    ell0, s20, sig0 = np.array([0.3, 0.3]), 1.0, 0.1

    def probes(j):
        return np.random.default_rng(1000 + j).standard_normal((N, 8))

    st = fit.fit_adam_sigma(p.X, y, nu, ell0, s20, sig0, probes, max_steps=6, tol=1e-11, mode="f64",
                            grad_tol=0.0, param_tol=0.0)

    def grad_fn(theta, s2n, j):
        ell, s2 = np.exp(theta[:d]), math.exp(theta[d])
        est, _ = _oracle_grad(orc, p, y, "product", s2n, ell, s2, probes(j))
        return est[:-1]

    def quad_fn(theta, s2n):
        K = orc.kmat(p.X, nu, np.exp(theta[:d]), s2=math.exp(theta[d]), kind=1)
        return float(y @ np.linalg.solve(K + s2n * np.eye(N), y))

    th, sig, _ = solve.adam_sigma_steps(grad_fn, quad_fn, N, np.concatenate([np.log(ell0), [math.log(s20)]]), sig0, 6)
    got_th = np.array([hh["theta"] for hh in st.history])
    got_sig = np.array([hh["sigma2"] for hh in st.history])
    np.testing.assert_allclose(got_th, th, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(got_sig, sig, rtol=1e-7)


def test_fit_raises_the_exact_likelihood(fgk_mod, orc):
    from paper_2508_01864_gb300 import fit

    N, d, nu = 500, 2, 1.5
    p, y = _problem(91, N, d, nu)
    rng = np.random.default_rng(5)
    st = fit.fit_adam_sigma(p.X, y, nu, [0.6, 0.6], 0.5, 0.3, lambda j: rng.standard_normal((N, 16)),
                            max_steps=40, lr0=0.05, lr1=0.05, grad_tol=0.0, param_tol=0.0)

    def ll(theta, s2n):
        K = orc.kmat(p.X, nu, np.exp(theta[:d]), s2=math.exp(theta[d]), kind=1)
        return solve.loglik_exact(K, s2n, y)

    start = ll(np.log([0.6, 0.6, 0.5]), 0.3)
    assert ll(st.theta, st.sigma2) > start + 1.0


def test_fit_with_a_preconditioner_raises_the_exact_likelihood(fgk_mod, orc):
    """The loop with rank-20 preconditioners (N(0, P) probes from the caller's
    standard normal numbers) on 15 distinct points each repeated 20 times, so
    the factor stops at rank 15 and only the first 15 rows of each E_r are
    used: the exact log-likelihood rises (by about 350 with exact gradients)."""
    from paper_2508_01864_gb300 import fit

    base = workloads.small(93, 15, 2, nu=1.5, ell=[0.2, 0.35])
    X = np.repeat(base.X, 20, axis=0)
    N, d, nu, rank = X.shape[0], 2, 1.5, 20
    rng = np.random.default_rng(4)
    y = np.repeat(np.sin(5 * base.X[:, 0]) + np.cos(3 * base.X[:, 1]), 20) + 0.1 * rng.standard_normal(N)
    st = fit.fit_adam_sigma(X, y, nu, [0.6, 0.6], 0.5, 0.3,
                            lambda j: (rng.standard_normal((rank, 16)), rng.standard_normal((N, 16))),
                            max_steps=30, precond_rank=rank, lr0=0.05, lr1=0.05, grad_tol=0.0, param_tol=0.0)

    def ll(theta, s2n):
        K = orc.kmat(X, nu, np.exp(theta[:d]), s2=math.exp(theta[d]), kind=1)
        return solve.loglik_exact(K, s2n, y)

    assert st.step == 30
    assert ll(st.theta, st.sigma2) > ll(np.log([0.6, 0.6, 0.5]), 0.3) + 50.0
