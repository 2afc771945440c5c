"""The d=3 workload solved at full size: N = 500 000 points of an eight-component
Gaussian mixture in [0,1]^3, nu = 5/2, ell = 0.1054, product kernel, sigma^2 =
0.01, GLS with H = [1, x] (Sec. 3.2), FP32 scans with FP64 residual
replacement and a rank-400 pivoted-Cholesky preconditioner (App. A.3).

Checked against what holds at any size:
- the solver's own FP64 true residuals (one per column of [y, H]) are at
  most 1e-8 of their right-hand sides;
- on sampled rows, the residual of (K + sigma^2 I) alpha = y - H beta with
  K alpha from the brute-force oracle is within the bound the column
  residuals imply (each row of a vector is at most its 2-norm);
- the GLS optimality condition H^T alpha = 0 (beta solves the normal
  equations H^T A^-1 (y - H beta) = 0).
"""

import time

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-8
RANK = 400


def test_c3_full_size_gls_solve(fgk_mod, orc):
    fgk = fgk_mod
    p = workloads.c3()
    y = p.V[:, 0]
    H = p.H
    t0 = time.perf_counter()
    with fgk.fgk_build(torch.as_tensor(p.X, device="cuda"), p.nu, p.ell, kind="product") as h:
        with fgk.fgk_precond_build(h, RANK, p.sigma2) as pc:
            alpha, beta, info, rc = fgk.fgk_cg_solve(h, torch.as_tensor(y, device="cuda"), p.sigma2,
                                                     H=torch.as_tensor(H, device="cuda"), tol=TOL, mode="mixed",
                                                     precond=pc)
            torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert rc == 0, info
    a = alpha.cpu().numpy()
    b = beta.cpu().numpy()[:, 0]
    print(f"\nC3 solve: {elapsed:.1f} s, {info['iterations']} iterations, {info['mvm_f64']} FP64 products, "
          f"true residuals {info['true_resid']}")
    # the solver's FP64 check of every column of [y, H]
    assert max(info["true_resid"]) <= TOL, info["true_resid"]
    # sampled rows of (K + sigma^2 I) alpha - (y - H beta) against the oracle
    rows = np.sort(np.random.default_rng(34).choice(p.N, size=40, replace=False))
    Ka = orc.mvm_brute(p.X, a[:, None], p.nu, p.ell, kind=1, rows=rows)[:, 0]
    r = Ka + p.sigma2 * a[rows] - (y[rows] - H[rows] @ b)
    bound = TOL * (np.linalg.norm(y) + np.sum(np.abs(b) * np.linalg.norm(H, axis=0)))
    assert np.all(np.abs(r) <= bound), (np.abs(r).max(), bound)
    # GLS: H^T alpha = 0 up to the columns' residuals
    hta = H.T @ a
    assert np.all(np.abs(hta) <= 1e-6 * np.linalg.norm(H, axis=0) * np.linalg.norm(a)), hta
