"""O4: the linear-algebra layer of the GP solve, plainly (numpy, FP64).

TEST INFRASTRUCTURE ONLY.

* ``cg``          Algorithm 2 (App. A.1) with a zero initial guess and the
                  preconditioner apply s_P (default: the identity), several
                  right-hand sides, each column stopped once its own relative
                  residual ||r_j|| / ||b_j|| is at most ``tol`` (the
                  algorithm's block test on ||R||^2 read per column and
                  unsquared).
* ``pivoted_cholesky``  the rank-k pivoted Cholesky factor L of K
                  (App. A.3, after Harbrecht et al.): at each step the pivot
                  is the largest remaining diagonal entry (first index among
                  equal ones) and L gains the column of K at the pivot minus
                  what the earlier columns explain, divided by the square
                  root of that diagonal entry.
* ``woodbury_apply``  P^{-1} R for P = L L^T + sigma^2 I by the Woodbury
                  formula of App. A.3.
* ``precond_logdet``  log det P by Sylvester's determinant theorem (App. A.3).
* ``dense_solve`` (K + sigma^2 I)^{-1} B via numpy, eq. gp_mean_system.
* ``gls``         the generalised least-squares fixed effects
                  beta = (H^T A^{-1} H)^{-1} H^T A^{-1} y (Sec. 3.2, the GLS
                  estimator and Algorithm 1), then alpha = A^{-1}(y - H beta),
                  the weights of eq. gp_mean with m(x) = H beta.
* ``true_residual``  ||b - A x|| / ||b|| per column, A applied by a callable.
* ``cg_lanczos``  Algorithm 2 again, recording per column the CG
                  coefficients alpha_k of every step and beta_k of every step
                  that continued, from which ``lanczos_T`` assembles the
                  tridiagonal Lanczos matrix: T[k][k] = 1/alpha_k +
                  beta_{k-1}/alpha_{k-1}, T[k+1][k] = sqrt(beta_k)/alpha_k.
* ``slq_quadrature``  gamma e_1^T log(T) e_1 (eigen-decomposition of T: the
                  Gauss quadrature of eq. approximationLogDet, gamma the
                  squared norm of the Lanczos start vector); ``slq_logdet``
                  the Hutchinson average over probes plus log det P.
* ``loglik_exact`` / ``loglik_grad_exact``  the log marginal likelihood
                  (eq. gp_log_likelihood) and its gradient
                  (eq. gp_log_likelihood_derivative) from dense matrices:
                  1/2 a^T dK a - 1/2 tr(A^{-1} dK), a = A^{-1} y.
* ``loglik_grad_estimate``  the same gradient with the trace term by
                  Hutchinson probes (App. A.2): mean_i (A^{-1} b_i)^T dK
                  (P^{-1} b_i), the probes N(0, P) (N(0, I) without P).
* ``adam_sigma_steps``  the gradient-descent loop of Algorithm 1: Adam
                  ascent steps on theta = (log ell_k, log varsigma^2) with the
                  learning rate falling linearly from 0.005 to 0.0005 over
                  20000 iterations (Sec. 3.1), each followed by the closed-form
                  update (sigma_j)^2 = y^T (K~ + I)^{-1} y / N with
                  K~ = K(varsigma_j / sigma_{j-1}, ell_j).
* ``algorithm1_outer``  Algorithm 1 around its gradient descents: the OLS
                  start, then GLS estimates of beta at the current
                  parameters, their running average subtracted from y before
                  the next descent, until successive GLS estimates differ by
                  at most eps_beta.
* ``minres``      the minimum-residual method of Paige and Saunders for a
                  symmetric system that need not be positive definite, such as
                  K + sigma^2 I with the L1 kernel at nu >= 3/2, d >= 2
                  (App. B, Prop. 4: not positive definite there, so CG can
                  break down).  Lanczos vectors started at b, the tridiagonal
                  T_k reduced to upper-triangular form by Givens rotations as it
                  grows, x_k = the minimiser of ||b - A x|| over the Krylov
                  space K_k(A, b), updated through the direction vectors of the
                  triangular factor; stop once the recursive residual norm
                  |phi_k| <= tol ||b||.  One column at a time.
* ``posterior_mean``  E[f(z) | x, y] = k_z^T alpha + h(z)^T beta (eq. gp_mean,
                  with alpha = (K + sigma^2 I)^{-1}(y - H beta) as eq. gp_mean_2),
                  given the cross-covariance rows k_z^T.
"""

from __future__ import annotations

import numpy as np


def cg(apply_A, B, tol: float, maxit: int, apply_Pinv=None):
    """Algorithm 2: returns (X, iterations per column)."""
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    B = B.reshape(B.shape[0], -1)
    n, m = B.shape
    s_P = (lambda R: R.copy()) if apply_Pinv is None else (lambda R: np.asarray(apply_Pinv(R)).reshape(n, m))
    X = np.zeros_like(B)
    R = B - apply_A(X)
    Pb = s_P(R)
    k = np.einsum("ij,ij->j", Pb, R)
    bnorm = np.linalg.norm(B, axis=0)
    done = np.linalg.norm(R, axis=0) <= tol * bnorm
    iters = np.zeros(m, dtype=np.int64)
    for it in range(maxit):
        if done.all():
            break
        T = apply_A(Pb)
        pt = np.einsum("ij,ij->j", Pb, T)
        alpha = np.where(done, 0.0, k / np.where(pt == 0, 1.0, pt))
        X += alpha * Pb
        R -= alpha * T
        iters[~done] += 1
        now = np.linalg.norm(R, axis=0) <= tol * bnorm
        done = done | now
        Z = s_P(R)
        k_prev = k
        k = np.einsum("ij,ij->j", Z, R)
        beta = np.where(done, 0.0, k / np.where(k_prev == 0, 1.0, k_prev))
        Pb = Z + beta * Pb
    return (X[:, 0] if vec else X), iters


def f32_store(l):
    """A factor column as stored in FP32 (round to nearest)."""
    return np.asarray(l, dtype=np.float64).astype(np.float32).astype(np.float64)


def pivoted_cholesky(column, diag, k: int, forced=None, tie_rtol: float = 0.0, eps: float = 1e-12,
                     tie_atol: float = 0.0, store=None):
    """Rank-k pivoted Cholesky of the SPD matrix with diagonal ``diag`` and
    columns ``column(i)``.  Returns (L (N x r), pivots (r,), residual
    diagonal) with r <= k: the factorisation stops early once the largest
    residual diagonal entry is at most ``eps`` times the largest diagonal
    entry of the matrix (numerically exhausted: the paper leaves this case
    open; dividing by the square root of a rounding-level residual would only
    add noise columns).

    ``forced``: follow these pivots instead of choosing them, after checking
    that each is a largest remaining diagonal entry within a relative
    ``tie_rtol`` or an absolute ``tie_atol`` (for comparing with a computation
    whose rounding may break near-ties the other way: a residual diagonal
    s2 - sum_m l_m^2 carries an absolute rounding error on the scale of the
    diagonal s2, so once the residuals are small the absolute term decides).

    ``store``: the rounding applied to each new column before it is kept
    (a factor stored in fewer bits, e.g. ``f32_store``); the later columns and
    the residual diagonal then use the stored values, so the factor is the
    exact pivoted Cholesky recurrence of its own stored columns."""
    d = np.array(diag, dtype=np.float64, copy=True)
    N = d.size
    floor = eps * float(d.max()) if N else 0.0
    L = np.zeros((N, k))
    piv = []
    for m in range(k):
        top = d.max()
        if forced is not None:
            if m >= len(forced):
                break
            i = int(forced[m])
            if not d[i] >= top * (1.0 - tie_rtol) - tie_atol:
                raise ValueError(f"step {m}: pivot {i} has residual {d[i]!r}, the largest is {top!r}")
        else:
            i = int(np.argmax(d))
        if not d[i] > floor:
            break
        c = np.asarray(column(i), dtype=np.float64).reshape(N)
        l = (c - L[:, :m] @ L[i, :m]) / np.sqrt(d[i])
        if store is not None:
            l = store(l)
        L[:, m] = l
        d = d - l * l
        piv.append(i)
    r = len(piv)
    return L[:, :r], np.array(piv, dtype=np.int64), d


def woodbury_apply(L, sigma2: float, R):
    """(L L^T + sigma2 I)^{-1} R = R / sigma2 - L (I_k + L^T L / sigma2)^{-1} L^T R / sigma2^2."""
    L = np.asarray(L, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    k = L.shape[1]
    C = np.eye(k) + (L.T @ L) / sigma2
    return R / sigma2 - (L @ np.linalg.solve(C, L.T @ R)) / (sigma2 * sigma2)


def precond_logdet(L, sigma2: float) -> float:
    """log det(L L^T + sigma2 I_N) = N log sigma2 + log det(I_k + L^T L / sigma2)."""
    L = np.asarray(L, dtype=np.float64)
    N, k = L.shape
    sign, ld = np.linalg.slogdet(np.eye(k) + (L.T @ L) / sigma2)
    assert sign > 0
    return N * np.log(sigma2) + ld


def dense_solve(K, sigma2: float, B):
    A = K + sigma2 * np.eye(K.shape[0])
    return np.linalg.solve(A, B)


def gls(solve, y, H):
    """``solve(B)`` returns A^{-1} B.  Returns (alpha, beta)."""
    y = np.asarray(y, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    Ai_y = solve(y)
    Ai_H = solve(H)
    beta = np.linalg.solve(H.T @ Ai_H, H.T @ Ai_y)
    alpha = Ai_y - Ai_H @ beta
    return alpha, beta


def true_residual(apply_A, X, B):
    B = np.asarray(B, dtype=np.float64).reshape(np.shape(B)[0], -1)
    X = np.asarray(X, dtype=np.float64).reshape(B.shape)
    R = B - apply_A(X)
    return np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)


def posterior_mean(Kzx, alpha, Hz=None, beta=None):
    """Kzx: M x N cross-covariance; alpha: N (x nrhs); Hz: M x L, beta: L (x nrhs)."""
    out = np.asarray(Kzx, dtype=np.float64) @ np.asarray(alpha, dtype=np.float64)
    if Hz is not None:
        out = out + np.asarray(Hz, dtype=np.float64) @ np.asarray(beta, dtype=np.float64)
    return out


def cg_lanczos(apply_A, B, tol: float, maxit: int, apply_Pinv=None):
    """Algorithm 2 with the Lanczos coefficients: returns (X, alphas, betas,
    gammas) with alphas[j] the alpha of every step of column j, betas[j] the
    beta of every step after which column j continued, and gammas[j] =
    b_j^T s_P(b_j), the squared norm of the Lanczos start vector."""
    B = np.asarray(B, dtype=np.float64)
    B = B.reshape(B.shape[0], -1)
    n, m = B.shape
    s_P = (lambda R: R.copy()) if apply_Pinv is None else (lambda R: np.asarray(apply_Pinv(R)).reshape(n, m))
    X = np.zeros_like(B)
    R = B - apply_A(X)
    Pb = s_P(R)
    k = np.einsum("ij,ij->j", Pb, R)
    gammas = k.copy()
    bnorm = np.linalg.norm(B, axis=0)
    done = np.linalg.norm(R, axis=0) <= tol * bnorm
    alphas = [[] for _ in range(m)]
    betas = [[] for _ in range(m)]
    for _ in range(maxit):
        if done.all():
            break
        T = apply_A(Pb)
        pt = np.einsum("ij,ij->j", Pb, T)
        alpha = np.where(done, 0.0, k / np.where(pt == 0, 1.0, pt))
        X += alpha * Pb
        R -= alpha * T
        for j in range(m):
            if not done[j]:
                alphas[j].append(float(alpha[j]))
        now = np.linalg.norm(R, axis=0) <= tol * bnorm
        newly = now & ~done
        Z = s_P(R)
        k_prev = k
        k = np.einsum("ij,ij->j", Z, R)
        beta = k / np.where(k_prev == 0, 1.0, k_prev)
        for j in range(m):
            if not done[j] and not newly[j]:
                betas[j].append(float(beta[j]))
        done = done | now
        beta = np.where(done, 0.0, beta)
        Pb = Z + beta * Pb
    return X, alphas, betas, gammas


def lanczos_T(alphas, betas):
    """The tridiagonal Lanczos matrix of len(alphas) CG steps (Algorithm 2's
    entries; the steps' betas between them)."""
    a = np.asarray(alphas, dtype=np.float64)
    b = np.asarray(betas, dtype=np.float64)[: max(len(a) - 1, 0)]
    mm = a.size
    T = np.zeros((mm, mm))
    for i in range(mm):
        T[i, i] = 1.0 / a[i] + (b[i - 1] / a[i - 1] if i > 0 else 0.0)
        if i + 1 < mm:
            T[i + 1, i] = T[i, i + 1] = np.sqrt(b[i]) / a[i]
    return T


def slq_quadrature(alphas, betas, gamma: float) -> float:
    """gamma e_1^T log(T) e_1 = gamma sum_i v_i[0]^2 log(lambda_i) over the
    eigenpairs of T."""
    lam, V = np.linalg.eigh(lanczos_T(alphas, betas))
    return float(gamma * np.sum(V[0, :] ** 2 * np.log(lam)))


def slq_logdet(apply_A, B, m: int, tol: float, apply_Pinv=None, logdet_P: float = 0.0):
    """log det A ~ log det P + mean over the probe columns of B of their
    quadratures (eq. approximationLogDet with the exact start-vector norms;
    with a preconditioner the probes are N(0, P) draws).  Returns
    (estimate, per-probe quadratures, Lanczos steps per probe, solves)."""
    X, al, be, ga = cg_lanczos(apply_A, B, tol, m, apply_Pinv)
    quad = np.array([slq_quadrature(al[j], be[j], ga[j]) if al[j] else 0.0 for j in range(len(al))])
    return logdet_P + float(quad.mean()), quad, np.array([len(a) for a in al]), X


def loglik_exact(K, sigma2: float, y) -> float:
    """eq. gp_log_likelihood: -1/2 y^T A^{-1} y - 1/2 log det A - N/2 log(2 pi), A = K + sigma2 I."""
    K = np.asarray(K, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    A = K + sigma2 * np.eye(K.shape[0])
    return float(-0.5 * y @ np.linalg.solve(A, y) - 0.5 * np.linalg.slogdet(A)[1]
                 - 0.5 * y.size * np.log(2 * np.pi))


def loglik_grad_exact(K, dKs, sigma2: float, y) -> np.ndarray:
    """eq. gp_log_likelihood_derivative for each dK in dKs:
    1/2 a^T dK a - 1/2 tr(A^{-1} dK), a = A^{-1} y."""
    K = np.asarray(K, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    A = K + sigma2 * np.eye(K.shape[0])
    a = np.linalg.solve(A, y)
    Ainv = np.linalg.inv(A)
    return np.array([0.5 * a @ dK @ a - 0.5 * float(np.sum(Ainv * dK.T)) for dK in dKs])


def loglik_grad_estimate(apply_Ainv, apply_dKs, y, B, apply_Pinv=None) -> np.ndarray:
    """The gradient with the trace by Hutchinson probes: for each dK,
    1/2 a^T dK a - 1/2 mean_i (A^{-1} b_i)^T dK (P^{-1} b_i)."""
    y = np.asarray(y, dtype=np.float64).reshape(-1, 1)
    B = np.asarray(B, dtype=np.float64)
    a = apply_Ainv(y)
    X = apply_Ainv(B)
    Z = B if apply_Pinv is None else apply_Pinv(B)
    out = []
    for f in apply_dKs:
        quad = float(a[:, 0] @ f(a)[:, 0])
        tr = float(np.mean(np.einsum("ij,ij->j", X, f(Z))))
        out.append(0.5 * quad - 0.5 * tr)
    return np.array(out)


def adam_sigma_steps(grad_fn, quad_fn, n_points: int, theta0, sigma2_0: float, n_steps: int, lr0: float = 0.005,
                     lr1: float = 0.0005, n_sched: int = 20000, b1: float = 0.9, b2: float = 0.999,
                     eps: float = 1e-8):
    """n_steps of Algorithm 1's inner loop.  grad_fn(theta, sigma2, j) is the
    log-likelihood gradient in theta at (theta, sigma2); quad_fn(theta,
    sigma2) = y^T (K(theta) + sigma2 I)^{-1} y.  Adam (Kingma and Ba) ascends
    the log-likelihood; the step size of iteration j (from 0) is
    lr0 + (lr1 - lr0) min(j / n_sched, 1).  Returns the thetas, sigma2s and
    gradients of every step."""
    theta = np.array(theta0, dtype=np.float64)
    sigma2 = float(sigma2_0)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    thetas, sigmas, grads = [], [], []
    for j in range(n_steps):
        g = np.asarray(grad_fn(theta, sigma2, j), dtype=np.float64)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        mh = m / (1 - b1 ** (j + 1))
        vh = v / (1 - b2 ** (j + 1))
        lr = lr0 + (lr1 - lr0) * min(j / n_sched, 1.0)
        theta = theta + lr * mh / (np.sqrt(vh) + eps)
        # (K~ + I) = (K(theta) + sigma_{j-1}^2 I) / sigma_{j-1}^2
        sigma2 = sigma2 * quad_fn(theta, sigma2) / n_points
        thetas.append(theta.copy())
        sigmas.append(sigma2)
        grads.append(g)
    return np.array(thetas), np.array(sigmas), np.array(grads)


def algorithm1_outer(descend, beta_gls, H, y, theta0, sigma2_0: float, eps_beta: float, max_rep: int):
    """Algorithm 1 with its gradient descents supplied: descend(y_c, theta,
    sigma2) runs one descent (Adam steps on theta with the sigma update) on
    the centred data y_c from (theta, sigma2) and returns the final
    (theta, sigma2); beta_gls(theta, sigma2) returns
    (H^T (K + sigma^2 I)^{-1} H)^{-1} H^T (K + sigma^2 I)^{-1} y for the
    parameters theta (K = K(varsigma, ell)).  In the algorithm's order:
    beta_OLS = (H^T H)^{-1} H^T y and a descent on y - H beta_OLS; then, for
    i = 1, 2, ..., beta_GLS at the current parameters, beta_AVG = (i-1)/i
    beta_AVG + beta_GLS / i, a descent on y - H beta_AVG, and the change
    ||beta_GLS - beta_old|| (beta_old starting at beta_OLS), until the change
    is at most eps_beta or max_rep repetitions.  Returns the final beta_GLS,
    theta, sigma2 and per repetition (beta_GLS, beta_AVG, change, theta,
    sigma2)."""
    H = np.asarray(H, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    beta_ols = np.linalg.solve(H.T @ H, H.T @ y)
    theta, sigma2 = descend(y - H @ beta_ols, np.array(theta0, dtype=np.float64), float(sigma2_0))
    beta_avg = np.zeros(H.shape[1])
    beta_old = beta_ols
    reps = []
    beta = beta_ols
    for i in range(1, max_rep + 1):
        beta = np.asarray(beta_gls(theta, sigma2), dtype=np.float64)
        beta_avg = (i - 1) / i * beta_avg + beta / i
        theta, sigma2 = descend(y - H @ beta_avg, theta, sigma2)
        change = float(np.linalg.norm(beta - beta_old))
        beta_old = beta
        reps.append((beta.copy(), beta_avg.copy(), change, np.array(theta, dtype=np.float64), float(sigma2)))
        if change <= eps_beta:
            break
    return beta, theta, sigma2, reps


def minres(apply_A, b, tol: float, maxit: int):
    """x with ||b - A x|| <= tol ||b|| (recursive estimate), A symmetric.
    Returns (x, iterations, residual norms |phi_k| per iteration)."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    n = b.size
    x = np.zeros(n)
    beta1 = float(np.linalg.norm(b))
    if beta1 == 0.0:
        return x, 0, []
    v_prev = np.zeros(n)
    v = b / beta1
    beta = beta1                      # beta_k: the Lanczos coefficient below v_k
    c_prev, s_prev = -1.0, 0.0        # the previous rotation (c_0 = -1, s_0 = 0)
    delta1, eps = 0.0, 0.0            # delta_k^(1), eps_k: T's entries above the diagonal, rotated
    phi = beta1                       # |phi_k| = ||r_k||
    d_prev = np.zeros(n)
    d_pp = np.zeros(n)
    history = []
    k = 0
    while k < maxit:
        k += 1
        # Lanczos: beta_{k+1} v_{k+1} = A v_k - alpha_k v_k - beta_k v_{k-1}
        p = apply_A(v)
        alpha = float(v @ p)
        p = p - alpha * v - beta * v_prev
        beta_next = float(np.linalg.norm(p))
        # the previous rotation applied to column k of T: (delta_k, alpha_k, beta_{k+1})
        delta2 = c_prev * delta1 + s_prev * alpha
        gamma1 = s_prev * delta1 - c_prev * alpha
        eps_next = s_prev * beta_next
        delta1_next = -c_prev * beta_next
        # a new rotation annihilates beta_{k+1}
        gamma2 = float(np.hypot(gamma1, beta_next))
        if gamma2 == 0.0:
            break
        c, s = gamma1 / gamma2, beta_next / gamma2
        tau = c * phi
        phi = s * phi
        d = (v - delta2 * d_prev - eps * d_pp) / gamma2
        x = x + tau * d
        history.append(phi)
        if phi <= tol * beta1 or beta_next == 0.0:
            break
        d_pp, d_prev = d_prev, d
        v_prev, v = v, p / beta_next
        beta, delta1, eps = beta_next, delta1_next, eps_next
        c_prev, s_prev = c, s
    return x, k, history
