"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and lays them out; it contains none of
the method's arithmetic, and it is the one module that both the oracle-side
tests and the CUDA path's tests/benchmark take their inputs from.

The paper's simulated experiments draw x uniformly on [0,1]^d with a
lengthscale near 0.1 (Sec. 3.1) and its real-data experiment uses 2-D spatial
coordinates with an affine mean (Sec. 3.2).  These generators stand in for
those workloads (the temperature dataset of Sec. 3.2 is not used):

* ``c1``  d=1, N=4096, nu=1/2, ell=0.2, x ~ U[0,1], v ~ N(0,1); one K v.
* ``c2``  d=2, N=200000, nu=3/2, ell=(0.1,0.3), x ~ U[0,1]^2,
          y = sin(2 pi x1) + cos(2 pi x2) + N(0, 0.1^2), sigma^2 = 0.01.
* ``c3``  d=3, N=500000, nu=5/2, ell=0.1054 per dimension, sigma^2 = 0.01,
          x from an 8-component Gaussian mixture (weights Dirichlet(1), means
          U[0.15,0.85]^3, isotropic std U[0.03,0.12]),
          y = 1 + 0.5 x1 - 0.3 x2 + 0.2 x3 + sin(2 pi x1) cos(2 pi x2)
              + N(0, 0.1^2); fixed effects H = [1, x1, x2, x3].
* ``c4``  64 problems, N log-uniform on [1e3, 1e5], d in {1,2}, nu in
          {1/2,3/2,5/2}, ell log-uniform on [0.05, 0.5] (isotropic),
          16 N(0,1) right-hand sides each, sigma^2 = 0.01.
* ``c5``  2000 requests, N log-uniform on [2e3, 3e5], d in {1,2,3}, mixed
          nu, x ~ U[0,1]^d, ell log-uniform on [0.05, 0.5], sigma^2 = 0.01,
          y as in c2 (plus x3 when d = 3); exponential inter-arrival gaps of
          mean 1 (scaled by the caller to the wanted rate).
* ``small`` generic seeded problems for tests (uniform, lattice with ties,
          duplicated points).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    name: str
    X: np.ndarray  # N x d, float64, row-major
    nu: float
    ell: np.ndarray  # d lengthscales
    s2: float = 1.0  # outputscale squared (varsigma^2)
    sigma2: float = 0.0  # noise variance
    V: np.ndarray | None = None  # N x nrhs right-hand sides / MVM operands
    H: np.ndarray | None = None  # N x L fixed-effect covariates
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]


def c1(seed: int = 1) -> Problem:
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(4096, 1))
    v = rng.standard_normal((4096, 1))
    return Problem("c1_d1_N4096_nu0.5", X, 0.5, np.array([0.2]), V=v)


def c2(seed: int = 2, N: int = 200_000) -> Problem:
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(N, 2))
    noise = rng.normal(0.0, 0.1, size=N)
    y = np.sin(2 * np.pi * X[:, 0]) + np.cos(2 * np.pi * X[:, 1]) + noise
    return Problem(f"c2_d2_N{N}_nu1.5", X, 1.5, np.array([0.1, 0.3]), sigma2=0.01, V=y[:, None])


def c3(seed: int = 3, N: int = 500_000) -> Problem:
    rng = np.random.default_rng(seed)
    w = rng.dirichlet(np.ones(8))
    means = rng.uniform(0.15, 0.85, size=(8, 3))
    stds = rng.uniform(0.03, 0.12, size=8)
    comp = rng.choice(8, size=N, p=w)
    X = means[comp] + stds[comp, None] * rng.standard_normal((N, 3))
    noise = rng.normal(0.0, 0.1, size=N)
    y = (1.0 + 0.5 * X[:, 0] - 0.3 * X[:, 1] + 0.2 * X[:, 2]
         + np.sin(2 * np.pi * X[:, 0]) * np.cos(2 * np.pi * X[:, 1]) + noise)
    H = np.column_stack([np.ones(N), X])
    return Problem(f"c3_d3_N{N}_nu2.5", X, 2.5, np.full(3, 0.1054), sigma2=0.01, V=y[:, None], H=H)


def c4(seed: int = 4, n_problems: int = 64, nrhs: int = 16) -> list[Problem]:
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n_problems):
        N = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e5)))))
        d = int(rng.integers(1, 3))
        nu = float(rng.choice([0.5, 1.5, 2.5]))
        ell = float(np.exp(rng.uniform(np.log(0.05), np.log(0.5))))
        X = rng.uniform(0.0, 1.0, size=(N, d))
        V = rng.standard_normal((N, nrhs))
        out.append(Problem(f"c4_p{p}_d{d}_N{N}_nu{nu}", X, nu, np.full(d, ell), sigma2=0.01, V=V))
    return out


def c5(seed: int = 5, n_requests: int = 2000, n_min: int = 2000, n_max: int = 300_000):
    """Returns (requests, gaps): gaps are unit-mean exponential draws."""
    rng = np.random.default_rng(seed)
    reqs = []
    gaps = rng.exponential(1.0, size=n_requests)
    for r in range(n_requests):
        N = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        d = int(rng.integers(1, 4))
        nu = float(rng.choice([0.5, 1.5, 2.5]))
        ell = float(np.exp(rng.uniform(np.log(0.05), np.log(0.5))))
        X = rng.uniform(0.0, 1.0, size=(N, d))
        noise = rng.normal(0.0, 0.1, size=N)
        y = np.sin(2 * np.pi * X[:, 0]) + noise
        if d >= 2:
            y = y + np.cos(2 * np.pi * X[:, 1])
        if d >= 3:
            y = y + X[:, 2]
        reqs.append(Problem(f"c5_r{r}_d{d}_N{N}_nu{nu}", X, nu, np.full(d, ell), sigma2=0.01, V=y[:, None]))
    return reqs, gaps


def small(seed: int, N: int, d: int, nu: float = 1.5, ell=0.2, nrhs: int = 1, pattern: str = "uniform",
          s2: float = 1.0) -> Problem:
    """Generic seeded test problem.

    pattern: "uniform" (U[0,1]^d), "lattice" (coordinates on a coarse integer
    grid scaled to [0,1], so many ties per coordinate), "dups" (uniform, with
    about a quarter of the points repeated exactly), "negzero" (lattice with
    -0.0 and +0.0 both present), "wide" (U[-50, 50]^d).
    """
    rng = np.random.default_rng(seed)
    if pattern == "uniform":
        X = rng.uniform(0.0, 1.0, size=(N, d))
    elif pattern == "lattice":
        X = rng.integers(0, 7, size=(N, d)).astype(np.float64) / 6.0
    elif pattern == "dups":
        X = rng.uniform(0.0, 1.0, size=(N, d))
        if N > 1:
            k = max(1, N // 4)
            src = rng.integers(0, N, size=k)
            dst = rng.integers(0, N, size=k)
            X[dst] = X[src]
    elif pattern == "negzero":
        X = rng.integers(-2, 3, size=(N, d)).astype(np.float64) / 2.0
        X[X == 0.0] = np.where(rng.uniform(size=int((X == 0.0).sum())) < 0.5, -0.0, 0.0)
    elif pattern == "wide":
        X = rng.uniform(-50.0, 50.0, size=(N, d))
    else:
        raise ValueError(pattern)
    V = rng.standard_normal((N, nrhs))
    ell = np.broadcast_to(np.asarray(ell, dtype=np.float64), (d,)).copy()
    return Problem(f"small_{pattern}_s{seed}_N{N}_d{d}", X, nu, ell, s2=s2, V=V)
