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


def _dense_descent(orc, X, nu, n_steps):
    """One Algorithm 1 descent from dense matrices: the oracle's Adam/sigma
    recurrence on the exact gradient of the centred data."""
    N, d = X.shape
    eye = np.eye(N)

    def run(yc, theta, s2):
        def grad(th, s, j):
            ell, sc = np.exp(th[:d]), math.exp(th[d])
            K = orc.kmat(X, nu, ell, s2=sc, kind=1)
            dKs = [orc.mvm_dlogell_brute(X, eye, nu, ell, dim=m, s2=sc, kind=1) for m in range(d)] + [K]
            return solve.loglik_grad_exact(K, dKs, s, yc)

        def quad(th, s):
            K = orc.kmat(X, nu, np.exp(th[:d]), s2=math.exp(th[d]), kind=1)
            return float(yc @ np.linalg.solve(K + s * eye, yc))

        th, sg, _ = solve.adam_sigma_steps(grad, quad, N, theta, s2, n_steps, lr0=0.05, lr1=0.02, n_sched=n_steps)
        return th[-1], sg[-1]

    return run


def test_outer_loop_follows_the_oracle(orc):
    """fit.gls_outer_loop against the oracle's Algorithm 1 outer loop, both
    driven by the same dense descents and dense GLS estimates."""
    from paper_2508_01864_gb300 import fit

    N, d, nu = 80, 2, 1.5
    p = workloads.small(19, N, d, nu=nu, ell=[0.3, 0.3])
    H = np.column_stack([np.ones(N), p.X])
    y = H @ np.array([0.5, 1.0, -1.0]) + np.sin(5 * p.X[:, 0]) + 0.1 * np.random.default_rng(4).standard_normal(N)
    run = _dense_descent(orc, p.X, nu, 4)

    def gls_fn(theta, s2):
        K = orc.kmat(p.X, nu, np.exp(theta[:d]), s2=math.exp(theta[d]), kind=1)
        return solve.gls(lambda B: np.linalg.solve(K + s2 * np.eye(N), B), y, H)[1]

    theta0 = np.log([0.3, 0.3, 1.0])
    got = fit.gls_outer_loop(lambda yc, t, s: (*run(yc, t, s), {}), gls_fn, H, y, theta0, 0.1, eps_beta=1e-4,
                             max_rep=5)
    beta, theta, s2, reps = solve.algorithm1_outer(run, gls_fn, H, y, theta0, 0.1, 1e-4, 5)
    assert got.reps == len(reps) >= 2
    np.testing.assert_allclose(got.beta, beta, rtol=1e-12)
    np.testing.assert_allclose(got.theta, theta, rtol=1e-12)
    assert got.sigma2 == pytest.approx(s2, rel=1e-12)
    for hist, (b, bavg, ch, th, sg) in zip(got.history[1:], reps):
        np.testing.assert_allclose(hist["beta_gls"], b, rtol=1e-12)
        np.testing.assert_allclose(hist["beta_avg"], bavg, rtol=1e-12)
        assert hist["change"] == pytest.approx(ch, rel=1e-10)


def test_fit_gls_maps_parameters_and_frees_its_plans(monkeypatch):
    """The GPU wrapper's glue with fakes for the descents and the library:
    theta maps to (ell, varsigma^2) for both layouts, each descent restarts
    from the previous parameters, each GLS estimate builds one plan (and
    preconditioner) at those parameters and frees it."""
    import torch

    from paper_2508_01864_gb300 import fit

    calls, live = [], set()

    class Obj:
        def __init__(self, tag):
            self.ptr = (tag, len(calls))
            live.add(self.ptr)

    def fake_adam(X, y, nu, ell, s2, sigma2, probes, steps, **kw):
        calls.append(("descend", np.array(ell), s2, sigma2, kw["kind"], kw["precond_rank"]))
        st = fit.FitState(theta=np.concatenate([np.log(np.array(ell)) + 0.1, [math.log(s2) + 0.1]])
                          if kw["kind"] == "product" and X.shape[1] > 1
                          else np.array([math.log(ell[0]) + 0.1, math.log(s2) + 0.1]), sigma2=sigma2 * 0.9, step=steps)
        return st

    def fake_build(X, nu, ell, outscale2=1.0, kind="product", stream=None):
        calls.append(("build", np.array(ell), outscale2))
        return Obj("plan")

    def fake_pc(h, rank, s2, stream=None):
        calls.append(("pc", rank, s2))
        return Obj("pc")

    def fake_solve(h, y, s2, H=None, tol=None, mode=None, precond=None, **kw):
        calls.append(("solve", s2, precond is not None, tuple(H.shape)))
        return None, torch.tensor([[1.0], [2.0], [3.0]], dtype=torch.float64), {}, 0

    def free(o):
        live.discard(o.ptr)

    monkeypatch.setattr(fit, "fit_adam_sigma", fake_adam)
    monkeypatch.setattr(fit.fgk, "fgk_build", fake_build)
    monkeypatch.setattr(fit.fgk, "fgk_precond_build", fake_pc)
    monkeypatch.setattr(fit.fgk, "fgk_cg_solve", fake_solve)
    monkeypatch.setattr(fit.fgk, "fgk_destroy", free)
    monkeypatch.setattr(fit.fgk, "fgk_precond_destroy", free)
    monkeypatch.setattr(torch, "as_tensor", lambda a, **kw: torch.from_numpy(np.asarray(a)))

    rng = np.random.default_rng(0)
    X = rng.uniform(size=(30, 2))
    H = np.column_stack([np.ones(30), X])
    y = rng.standard_normal(30)
    out = fit.fit_gls(X, y, H, 1.5, [0.2, 0.4], 2.0, 0.1, None, 3, eps_beta=0.0, max_rep=2, precond_rank=5)
    assert out.reps == 2 and not live
    np.testing.assert_array_equal(out.beta, [1.0, 2.0, 3.0])
    kinds = [c[0] for c in calls]
    assert kinds == ["descend", "build", "pc", "solve", "descend", "build", "pc", "solve", "descend"]
    # descent 1 from the initial values; each later step from the previous one's result
    np.testing.assert_allclose(calls[0][1], [0.2, 0.4])
    assert calls[0][2] == pytest.approx(2.0) and calls[0][3] == 0.1
    np.testing.assert_allclose(calls[1][1], np.array([0.2, 0.4]) * math.exp(0.1))
    assert calls[1][2] == pytest.approx(2.0 * math.exp(0.1))
    assert calls[2] == ("pc", 5, pytest.approx(0.09)) and calls[3][0:3] == ("solve", pytest.approx(0.09), True)
    np.testing.assert_allclose(calls[4][1], np.array([0.2, 0.4]) * math.exp(0.1))
    # the L1 kernel: one lengthscale entry, the ratio of the initial lengthscales kept
    calls.clear()
    fit.fit_gls(X, y, H, 1.5, [0.2, 0.4], 2.0, 0.1, None, 3, eps_beta=0.0, max_rep=1, kind="l1")
    np.testing.assert_allclose(calls[1][1], np.array([0.2, 0.4]) * math.exp(0.1))
    assert [c[0] for c in calls] == ["descend", "build", "solve", "descend"] and not live
