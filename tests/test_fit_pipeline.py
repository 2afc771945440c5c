"""Algorithm 1 end to end on the host, without a GPU: fit.fit_gls and
fit.fit_adam_sigma run unchanged while the library calls they make
(fgk_build, fgk_loglik_grad, fgk_cg_solve with H, fgk_destroy) are served by
a dense stand-in built from the oracle.  The trajectory must equal the
oracle's own Algorithm 1 with the same probes, so every step of the host
glue (parameter maps, probe handling, the gradient entries kept, the GLS
call) is checked; only the GPU arithmetic is left to the GPU test."""

import math

import numpy as np
import pytest
import torch

import workloads
from oracle import solve

N, D, NU = 150, 2, 1.5


def _data():
    p = workloads.small(86, N, D, nu=NU, ell=[0.2, 0.35])
    H = np.column_stack([np.ones(N), p.X])
    rng = np.random.default_rng(86)
    y = H @ np.array([0.5, 1.0, -1.0]) + np.sin(5 * p.X[:, 0]) + np.cos(3 * p.X[:, 1]) \
        + 0.1 * rng.standard_normal(N)
    return p.X, H, y


def _probes(j):
    return np.random.default_rng(3000 + j).standard_normal((N, 8))


class DenseLibrary:
    """The library calls of the fitting code, computed densely by the oracle."""

    def __init__(self, orc):
        self.orc = orc
        self.live = 0

    class Plan:
        def __init__(self, X, nu, ell, s2, kind):
            self.X, self.nu, self.ell, self.s2, self.kind = X, nu, np.asarray(ell, dtype=np.float64), s2, kind
            self.ptr = 1

    def fgk_build(self, X, nu, ell, outscale2=1.0, kind="l1", stream=None):
        self.live += 1
        return self.Plan(np.asarray(X), nu, ell, outscale2, kind)

    def fgk_destroy(self, h):
        self.live -= 1

    def _K(self, h):
        return self.orc.kmat(h.X, h.nu, h.ell, s2=h.s2, kind=0 if h.kind == "l1" else 1)

    def fgk_loglik_grad(self, h, y, B, sigma2, tol=1e-8, maxit=20000, mode="mixed", pc=None, stream=None):
        assert pc is None
        y = np.asarray(y, dtype=np.float64).reshape(-1)
        K = self._K(h)
        A = K + sigma2 * np.eye(len(y))
        a = np.linalg.solve(A, y)
        if B is None:
            return {"grad": [0.5 * a @ K @ a], "yAy": float(y @ a), "iterations": 0}
        eye = np.eye(len(y))
        dKs = [self.orc.mvm_dlogell_brute(h.X, eye, h.nu, h.ell, dim=m, s2=h.s2, kind=1)
               for m in range(h.X.shape[1])] + [K, sigma2 * eye]
        g = solve.loglik_grad_estimate(lambda V: np.linalg.solve(A, V), [lambda V, M=M: M @ V for M in dKs], y,
                                       np.asarray(B))
        return {"grad": list(g), "yAy": float(y @ a), "iterations": 0}

    def fgk_cg_solve(self, h, y, sigma2, H=None, tol=1e-8, mode="mixed", precond=None, **kw):
        y = np.asarray(y, dtype=np.float64).reshape(-1)
        A = self._K(h) + sigma2 * np.eye(len(y))
        alpha, beta = solve.gls(lambda V: np.linalg.solve(A, V), y, np.asarray(H))
        return torch.from_numpy(alpha.reshape(-1, 1)), torch.from_numpy(beta.reshape(-1, 1)), {}, 0


def test_fit_gls_host_pipeline_equals_the_oracle(orc, monkeypatch):
    from paper_2508_01864_gb300 import fit

    lib = DenseLibrary(orc)
    for name in ("fgk_build", "fgk_destroy", "fgk_loglik_grad", "fgk_cg_solve"):
        monkeypatch.setattr(fit.fgk, name, getattr(lib, name))
    monkeypatch.setattr(torch, "as_tensor", lambda a, **kw: torch.from_numpy(np.array(a, dtype=np.float64)))

    X, H, y = _data()
    ell0, s20, sig0 = np.array([0.3, 0.3]), 1.0, 0.1
    got = fit.fit_gls(X, y, H, NU, ell0, s20, sig0, _probes, 3, eps_beta=0.0, max_rep=2, tol=1e-11, mode="f64",
                      grad_tol=0.0, param_tol=0.0)
    assert lib.live == 0

    eye = np.eye(N)

    def K_of(theta):
        return orc.kmat(X, NU, np.exp(theta[:D]), s2=math.exp(theta[D]), kind=1)

    def descend(yc, theta, s2):
        def grad(th, s, j):
            ell, sc = np.exp(th[:D]), math.exp(th[D])
            K = K_of(th)
            A = K + s * eye
            dKs = [orc.mvm_dlogell_brute(X, eye, NU, ell, dim=m, s2=sc, kind=1) for m in range(D)] + [K, s * eye]
            return solve.loglik_grad_estimate(lambda V: np.linalg.solve(A, V), [lambda V, M=M: M @ V for M in dKs],
                                              yc, _probes(j))[:-1]

        def quad(th, s):
            return float(yc @ np.linalg.solve(K_of(th) + s * eye, yc))

        th, sg, _ = solve.adam_sigma_steps(grad, quad, N, theta, s2, 3)
        return th[-1], sg[-1]

    def gls_fn(theta, s2):
        return solve.gls(lambda B: np.linalg.solve(K_of(theta) + s2 * eye, B), y, H)[1]

    beta, theta, s2, reps = solve.algorithm1_outer(descend, gls_fn, H, y,
                                                   np.concatenate([np.log(ell0), [math.log(s20)]]), sig0, 0.0, 2)
    assert got.reps == len(reps) == 2
    for hist, (b, bavg, _, th, sg) in zip(got.history[1:], reps):
        np.testing.assert_allclose(hist["beta_gls"], b, rtol=1e-11)
        np.testing.assert_allclose(hist["beta_avg"], bavg, rtol=1e-11)
        np.testing.assert_allclose(hist["theta"], th, rtol=1e-11, atol=1e-13)
        assert hist["sigma2"] == pytest.approx(sg, rel=1e-11)
    np.testing.assert_allclose(got.theta, theta, rtol=1e-11, atol=1e-13)
