"""O4: the linear-algebra layer of the GP solve, plainly (numpy, FP64).

TEST INFRASTRUCTURE ONLY.

* ``cg``          Algorithm 2 (App. A.1) with the identity preconditioner
                  s_P = I and a zero initial guess, several right-hand sides,
                  each column stopped once its own relative residual
                  ||r_j|| / ||b_j|| is at most ``tol`` (the algorithm's block
                  test on ||R||^2 read per column and unsquared).
* ``dense_solve`` (K + sigma^2 I)^{-1} B via numpy, eq. gp_mean_system.
* ``gls``         the generalised least-squares fixed effects
                  beta = (H^T A^{-1} H)^{-1} H^T A^{-1} y (Sec. 3.2, the GLS
                  estimator and Algorithm 1), then alpha = A^{-1}(y - H beta),
                  the weights of eq. gp_mean with m(x) = H beta.
* ``true_residual``  ||b - A x|| / ||b|| per column, A applied by a callable.
"""

from __future__ import annotations

import numpy as np


def cg(apply_A, B, tol: float, maxit: int):
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    B = B.reshape(B.shape[0], -1)
    n, m = B.shape
    X = np.zeros_like(B)
    R = B - apply_A(X)
    Pb = R.copy()
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
        k_prev = k
        k = np.einsum("ij,ij->j", R, R)
        beta = np.where(done, 0.0, k / np.where(k_prev == 0, 1.0, k_prev))
        Pb = R + beta * Pb
    return (X[:, 0] if vec else X), iters


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
