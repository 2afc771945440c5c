"""Hyperparameter fitting: the gradient-descent loop of Algorithm 1.

Each step takes the log-likelihood gradient (eq. gp_log_likelihood_derivative)
in theta = (log ell_1 .. log ell_d, log varsigma^2) at the current sigma^2
from ``fgk_loglik_grad`` (one CG solve of [y, probes] on the GPU, the trace
terms by Hutchinson probes), moves theta by an Adam ascent step whose rate
falls linearly from 0.005 to 0.0005 over 20000 steps (Sec. 3.1), and then
updates the nugget in closed form, (sigma_j)^2 = y^T (K~ + I)^{-1} y / N with
K~ = K(varsigma_j / sigma_{j-1}, ell_j), i.e. sigma_{j-1}^2 y^T
(K(theta_j) + sigma_{j-1}^2 I)^{-1} y / N (one more solve).  The loop stops
after ``max_steps``, once the gradient norm is below ``grad_tol``, or once
theta has moved by less than ``param_tol`` over the last 100 steps (the
paper's two criteria).  The plan and the preconditioner are built for every
parameter value; all vector work runs in libfgk, this module holds only the
scalar Adam and sigma recurrences.

The probes are standard normal numbers the caller supplies per step
(``probes(j)`` returning an N x n array, or (E_r, E_n) pairs with a
preconditioner, from which ``fgk_precond_sample`` forms N(0, P) probes).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import fgk


@dataclass
class FitState:
    theta: np.ndarray          # log ell_1 .. log ell_d, log varsigma^2
    sigma2: float
    step: int = 0
    m: np.ndarray | None = None
    v: np.ndarray | None = None
    history: list = field(default_factory=list)


def _lr(j: int, lr0: float, lr1: float, n_sched: int) -> float:
    return lr0 + (lr1 - lr0) * min(j / n_sched, 1.0)


def fit_adam_sigma(X: np.ndarray, y: np.ndarray, nu: float, ell0, outscale2_0: float, sigma2_0: float,
                   probes, max_steps: int, kind: str = "product", precond_rank: int = 0, lr0: float = 0.005,
                   lr1: float = 0.0005, n_sched: int = 20000, grad_tol: float = 1e-3, param_tol: float = 1e-4,
                   tol: float = 1e-8, mode: str = "mixed", b1: float = 0.9, b2: float = 0.999,
                   eps: float = 1e-8) -> FitState:
    X_dev = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float64), device="cuda")
    y_dev = torch.as_tensor(np.ascontiguousarray(y, dtype=np.float64), device="cuda")
    N, d = X_dev.shape[0], X_dev.shape[1] if X_dev.dim() == 2 else 1
    ell0 = np.broadcast_to(np.asarray(ell0, dtype=np.float64), (d,)).copy()
    st = FitState(theta=np.concatenate([np.log(ell0), [math.log(outscale2_0)]]), sigma2=float(sigma2_0))
    per_dim = kind == "product" and d > 1
    if not per_dim:  # one lengthscale entry in the gradient: all scaled together
        st.theta = np.concatenate([[math.log(ell0[0])], [math.log(outscale2_0)]])
        ratio = ell0 / ell0[0]  # the lengthscales keep their ratios
    st.m = np.zeros_like(st.theta)
    st.v = np.zeros_like(st.theta)

    def ells(theta):
        return np.exp(theta[:d]) if per_dim else math.exp(theta[0]) * ratio

    def plan(theta, sigma2):
        h = fgk.fgk_build(X_dev, nu, ells(theta), outscale2=math.exp(theta[-1]), kind=kind)
        pc = fgk.fgk_precond_build(h, precond_rank, sigma2) if precond_rank > 0 else None
        return h, pc

    window = []
    for j in range(max_steps):
        h, pc = plan(st.theta, st.sigma2)
        try:
            pr = probes(j)
            if pc is not None:
                B = fgk.fgk_precond_sample(pc, torch.as_tensor(pr[0], device="cuda"),
                                           torch.as_tensor(pr[1], device="cuda"))
            else:
                B = torch.as_tensor(np.ascontiguousarray(pr, dtype=np.float64), device="cuda")
            r = fgk.fgk_loglik_grad(h, y_dev, B, st.sigma2, tol=tol, mode=mode, pc=pc)
        finally:
            if pc is not None:
                fgk.fgk_precond_destroy(pc)
            fgk.fgk_destroy(h)
        g = np.array(r["grad"][:-1])  # theta's entries (the nugget follows the closed form)
        st.m = b1 * st.m + (1 - b1) * g
        st.v = b2 * st.v + (1 - b2) * g * g
        mh = st.m / (1 - b1 ** (j + 1))
        vh = st.v / (1 - b2 ** (j + 1))
        old = st.theta.copy()
        st.theta = st.theta + _lr(j, lr0, lr1, n_sched) * mh / (np.sqrt(vh) + eps)
        # sigma_j^2 = sigma_{j-1}^2 y^T (K(theta_j) + sigma_{j-1}^2 I)^{-1} y / N
        h, pc = plan(st.theta, st.sigma2)
        try:
            q = fgk.fgk_loglik_grad(h, y_dev, None, st.sigma2, tol=tol, mode=mode, pc=pc)["yAy"]
        finally:
            if pc is not None:
                fgk.fgk_precond_destroy(pc)
            fgk.fgk_destroy(h)
        st.sigma2 = st.sigma2 * q / N
        st.step = j + 1
        gnorm = float(np.linalg.norm(g))
        st.history.append({"theta": st.theta.copy(), "sigma2": st.sigma2, "grad": g, "grad_norm": gnorm,
                           "iterations": r["iterations"]})
        window.append(old)
        if gnorm < grad_tol:
            break
        if len(window) > 100:
            window.pop(0)
            if np.linalg.norm(st.theta - window[0]) < param_tol:
                break
    return st
