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
scalar Adam and sigma recurrences (``adam_sigma_loop``, which takes the two
evaluations as callables).

The probes are standard normal numbers the caller supplies per step
(``probes(j)`` returning an N x n array, or with a preconditioner an (E_r, E_n)
pair of precond_rank x n and N x n arrays, from which ``fgk_precond_sample``
forms N(0, P) probes with the first k rows of E_r, k the factor's rank).
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


def adam_sigma_loop(eval_grad, eval_quad, n_points: int, theta0, sigma2_0: float, max_steps: int,
                    lr0: float = 0.005, lr1: float = 0.0005, n_sched: int = 20000, grad_tol: float = 1e-3,
                    param_tol: float = 1e-4, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> FitState:
    """Algorithm 1's inner loop on host scalars.  eval_grad(theta, sigma2, j)
    returns (g, info): the log-likelihood gradient in theta at (theta, sigma2)
    and a dict kept in the history; eval_quad(theta, sigma2) returns
    y^T (K(theta) + sigma2 I)^{-1} y."""
    st = FitState(theta=np.array(theta0, dtype=np.float64), sigma2=float(sigma2_0))
    st.m = np.zeros_like(st.theta)
    st.v = np.zeros_like(st.theta)
    window = []
    for j in range(max_steps):
        g, info = eval_grad(st.theta, st.sigma2, j)
        g = np.asarray(g, dtype=np.float64)
        st.m = b1 * st.m + (1 - b1) * g
        st.v = b2 * st.v + (1 - b2) * g * g
        mh = st.m / (1 - b1 ** (j + 1))
        vh = st.v / (1 - b2 ** (j + 1))
        old = st.theta.copy()
        st.theta = st.theta + _lr(j, lr0, lr1, n_sched) * mh / (np.sqrt(vh) + eps)
        # sigma_j^2 = sigma_{j-1}^2 y^T (K(theta_j) + sigma_{j-1}^2 I)^{-1} y / N
        st.sigma2 = st.sigma2 * eval_quad(st.theta, st.sigma2) / n_points
        st.step = j + 1
        gnorm = float(np.linalg.norm(g))
        st.history.append({"theta": st.theta.copy(), "sigma2": st.sigma2, "grad": g, "grad_norm": gnorm, **info})
        window.append(old)
        if gnorm < grad_tol:
            break
        if len(window) > 100:
            window.pop(0)
            if np.linalg.norm(st.theta - window[0]) < param_tol:
                break
    return st


def fit_adam_sigma(X: np.ndarray, y: np.ndarray, nu: float, ell0, outscale2_0: float, sigma2_0: float,
                   probes, max_steps: int, kind: str = "product", precond_rank: int = 0, lr0: float = 0.005,
                   lr1: float = 0.0005, n_sched: int = 20000, grad_tol: float = 1e-3, param_tol: float = 1e-4,
                   tol: float = 1e-8, mode: str = "mixed", b1: float = 0.9, b2: float = 0.999,
                   eps: float = 1e-8) -> FitState:
    """``adam_sigma_loop`` with every evaluation on the GPU: a plan (and a
    preconditioner of ``precond_rank``) for each parameter value,
    ``fgk_loglik_grad`` with the step's probes for the gradient, and
    ``fgk_loglik_grad`` without probes for y^T A^{-1} y."""
    X_dev = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float64), device="cuda")
    y_dev = torch.as_tensor(np.ascontiguousarray(y, dtype=np.float64), device="cuda")
    N, d = X_dev.shape[0], X_dev.shape[1] if X_dev.dim() == 2 else 1
    ell0 = np.broadcast_to(np.asarray(ell0, dtype=np.float64), (d,)).copy()
    per_dim = kind == "product" and d > 1
    if per_dim:
        theta0 = np.concatenate([np.log(ell0), [math.log(outscale2_0)]])
    else:  # one lengthscale entry in the gradient: all scaled together, keeping their ratios
        theta0 = np.concatenate([[math.log(ell0[0])], [math.log(outscale2_0)]])
    ratio = ell0 / ell0[0]

    def ells(theta):
        return np.exp(theta[:d]) if per_dim else math.exp(theta[0]) * ratio

    def with_plan(theta, sigma2, fn):
        h = fgk.fgk_build(X_dev, nu, ells(theta), outscale2=math.exp(theta[-1]), kind=kind)
        pc = None
        try:
            if precond_rank > 0:
                pc = fgk.fgk_precond_build(h, precond_rank, sigma2)
            return fn(h, pc)
        finally:
            if pc is not None:
                fgk.fgk_precond_destroy(pc)
            fgk.fgk_destroy(h)

    def eval_grad(theta, sigma2, j):
        def run(h, pc):
            pr = probes(j)
            if pc is not None:  # the factor may have stopped below precond_rank: its first k rows
                k = pc.rank
                Er = np.ascontiguousarray(np.asarray(pr[0], dtype=np.float64)[:k])
                B = fgk.fgk_precond_sample(pc, torch.as_tensor(Er, device="cuda"),
                                           torch.as_tensor(np.ascontiguousarray(pr[1], dtype=np.float64),
                                                           device="cuda"))
            else:
                B = torch.as_tensor(np.ascontiguousarray(pr, dtype=np.float64), device="cuda")
            return fgk.fgk_loglik_grad(h, y_dev, B, sigma2, tol=tol, mode=mode, pc=pc)

        r = with_plan(theta, sigma2, run)
        # theta's entries (the nugget follows the closed form)
        return np.array(r["grad"][:-1]), {"iterations": r["iterations"]}

    def eval_quad(theta, sigma2):
        return with_plan(theta, sigma2,
                         lambda h, pc: fgk.fgk_loglik_grad(h, y_dev, None, sigma2, tol=tol, mode=mode, pc=pc)["yAy"])

    return adam_sigma_loop(eval_grad, eval_quad, N, theta0, sigma2_0, max_steps, lr0=lr0, lr1=lr1, n_sched=n_sched,
                           grad_tol=grad_tol, param_tol=param_tol, b1=b1, b2=b2, eps=eps)


# ------------------------------------------------------------ Algorithm 1, outer loop
@dataclass
class GlsFit:
    beta: np.ndarray        # the last GLS estimate of the fixed effects
    beta_avg: np.ndarray    # the running average subtracted from y before the last descent
    theta: np.ndarray
    sigma2: float
    reps: int               # GLS repetitions
    history: list = field(default_factory=list)


def gls_outer_loop(descend, beta_gls, H, y, theta0, sigma2_0: float, eps_beta: float = 1e-3,
                   max_rep: int = 20) -> GlsFit:
    """Algorithm 1 (Sec. 3.1) on host values: a damped fixed-point iteration
    between the fixed effects and the kernel parameters.

    The two depend on each other.  descend(y_c, theta, sigma2) fits the
    parameters to data centred by a mean H b and returns (theta, sigma2,
    info); beta_gls(theta, sigma2) is the GLS estimate
    (H^T A^{-1} H)^{-1} H^T A^{-1} y, A = K(theta) + sigma2 I, at those
    parameters.  Writing P(b) for the parameters fitted to y - H b, a
    consistent pair is a fixed point b = beta_gls(P(b)).  The iteration
    starts from the least-squares mean b_0 = beta_OLS (the normal equations
    of H) and feeds each new estimate b_r = beta_gls(P(m_{r-1})) back through
    the mean m_r of all estimates so far, which damps it; it stops once two
    successive estimates agree to eps_beta (b_1 is compared with beta_OLS)
    or after max_rep estimates.  The parameters returned are P(m_r) of the
    last repetition."""
    H = np.asarray(H, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    b_ols = np.linalg.solve(H.T @ H, H.T @ y)

    def agree(b_new, b_old):
        return float(np.linalg.norm(b_new - b_old)) <= eps_beta

    theta, sigma2, info = descend(y - H @ b_ols, np.array(theta0, dtype=np.float64), float(sigma2_0))
    fit = GlsFit(beta=b_ols.copy(), beta_avg=np.zeros(H.shape[1]), theta=np.asarray(theta, dtype=np.float64),
                 sigma2=float(sigma2), reps=0)
    fit.history.append({"beta_ols": b_ols.copy(), "theta": fit.theta.copy(), "sigma2": fit.sigma2, **info})
    estimates = [b_ols]  # b_0, b_1, ..., b_r; the mean is over b_1 .. b_r
    while len(estimates) <= max_rep:
        b = np.asarray(beta_gls(fit.theta, fit.sigma2), dtype=np.float64).reshape(-1)
        estimates.append(b)
        m = np.sum(estimates[1:], axis=0) / (len(estimates) - 1)
        theta, sigma2, info = descend(y - H @ m, fit.theta, fit.sigma2)
        fit.beta, fit.beta_avg, fit.reps = b.copy(), m, len(estimates) - 1
        fit.theta, fit.sigma2 = np.asarray(theta, dtype=np.float64), float(sigma2)
        fit.history.append({"beta_gls": b.copy(), "beta_avg": m.copy(),
                            "change": float(np.linalg.norm(b - estimates[-2])), "theta": fit.theta.copy(),
                            "sigma2": fit.sigma2, **info})
        if agree(b, estimates[-2]):
            break
    return fit


def fit_gls(X: np.ndarray, y: np.ndarray, H: np.ndarray, nu: float, ell0, outscale2_0: float, sigma2_0: float,
            probes, steps_per_descent: int, eps_beta: float = 1e-3, max_rep: int = 20, kind: str = "product",
            precond_rank: int = 0, tol: float = 1e-8, mode: str = "mixed", **adam) -> GlsFit:
    """Algorithm 1 on the GPU: ``gls_outer_loop`` whose descents are
    ``fit_adam_sigma`` runs (each restarting Adam and its rate schedule, at
    most ``steps_per_descent`` steps; ``adam`` passes lr0, lr1, n_sched,
    grad_tol, param_tol, b1, b2, eps) and whose GLS estimates come from
    ``fgk_cg_solve`` with the covariates H (N x L, e.g. [1, x_1 .. x_d]) at
    the current parameters.  theta is (log ell_1 .. log ell_d, log
    varsigma^2) for the product kernel with d > 1, else (log ell, log
    varsigma^2) with the lengthscales scaled together."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    d = X.shape[1]
    ell0 = np.broadcast_to(np.asarray(ell0, dtype=np.float64), (d,)).copy()
    per_dim = kind == "product" and d > 1
    ratio = ell0 / ell0[0]
    theta0 = np.concatenate([np.log(ell0) if per_dim else [math.log(ell0[0])], [math.log(outscale2_0)]])

    def params(theta):
        ell = np.exp(theta[:d]) if per_dim else math.exp(theta[0]) * ratio
        return ell, math.exp(theta[-1])

    def descend(yc, theta, sigma2):
        ell, s2 = params(theta)
        st = fit_adam_sigma(X, yc, nu, ell, s2, sigma2, probes, steps_per_descent, kind=kind,
                            precond_rank=precond_rank, tol=tol, mode=mode, **adam)
        return st.theta, st.sigma2, {"steps": st.step}

    X_dev = torch.as_tensor(X, device="cuda")
    y_dev = torch.as_tensor(np.ascontiguousarray(y, dtype=np.float64).reshape(-1), device="cuda")
    H_dev = torch.as_tensor(np.ascontiguousarray(H, dtype=np.float64), device="cuda")

    def beta_gls(theta, sigma2):
        ell, s2 = params(theta)
        h = fgk.fgk_build(X_dev, nu, ell, outscale2=s2, kind=kind)
        pc = None
        try:
            if precond_rank > 0:
                pc = fgk.fgk_precond_build(h, precond_rank, sigma2)
            _, beta, _, _ = fgk.fgk_cg_solve(h, y_dev, sigma2, H=H_dev, tol=tol, mode=mode, precond=pc)
            return beta.cpu().numpy().reshape(-1)
        finally:
            if pc is not None:
                fgk.fgk_precond_destroy(pc)
            fgk.fgk_destroy(h)

    return gls_outer_loop(descend, beta_gls, H, y, theta0, sigma2_0, eps_beta, max_rep)
