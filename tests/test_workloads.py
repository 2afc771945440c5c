"""The seeded synthetic inputs follow their stated recipes (shapes, kernel
parameters, value ranges, the noise of y) and are reproducible."""

import numpy as np

import workloads


def test_d1_workload():
    p = workloads.c1()
    assert p.X.shape == (4096, 1) and p.nu == 0.5 and np.allclose(p.ell, [0.2])
    assert 0.0 <= p.X.min() and p.X.max() <= 1.0
    assert abs(p.V.mean()) < 0.05 and abs(p.V.std() - 1.0) < 0.05
    assert np.array_equal(p.X, workloads.c1().X)


def test_d2_workload():
    p = workloads.c2()
    assert p.X.shape == (200_000, 2) and p.nu == 1.5 and np.allclose(p.ell, [0.1, 0.3]) and p.sigma2 == 0.01
    resid = p.V[:, 0] - (np.sin(2 * np.pi * p.X[:, 0]) + np.cos(2 * np.pi * p.X[:, 1]))
    assert abs(resid.std() - 0.1) < 2e-3 and abs(resid.mean()) < 2e-3
    assert np.array_equal(p.V, workloads.c2().V)


def test_d3_workload():
    p = workloads.c3(N=60_000)
    assert p.X.shape == (60_000, 3) and p.nu == 2.5 and np.allclose(p.ell, 0.1054) and p.sigma2 == 0.01
    assert np.allclose(p.H, np.column_stack([np.ones(p.N), p.X]))
    x1, x2, x3 = p.X.T
    mean = 1.0 + 0.5 * x1 - 0.3 * x2 + 0.2 * x3 + np.sin(2 * np.pi * x1) * np.cos(2 * np.pi * x2)
    assert abs((p.V[:, 0] - mean).std() - 0.1) < 3e-3
    # an 8-component mixture: the points sit in clusters, far tighter than U[0,1]^3
    assert p.X.std(axis=0).max() < 0.3


def test_batched_workload():
    probs = workloads.c4()
    assert len(probs) == 64
    for p in probs:
        assert 1_000 <= p.N <= 100_000 and p.X.shape[1] in (1, 2) and p.nu in (0.5, 1.5, 2.5)
        assert 0.05 <= p.ell[0] <= 0.5 and np.all(p.ell == p.ell[0]) and p.sigma2 == 0.01
        assert p.V.shape == (p.N, 16)
    assert {p.X.shape[1] for p in probs} == {1, 2} and {p.nu for p in probs} == {0.5, 1.5, 2.5}


def test_serving_workload():
    reqs, gaps = workloads.c5(n_requests=60)
    assert len(reqs) == 60 and gaps.shape == (60,) and np.all(gaps > 0)
    for p in reqs:
        assert 2_000 <= p.N <= 300_000 and p.X.shape[1] in (1, 2, 3) and 0.05 <= p.ell[0] <= 0.5
    big, g2 = workloads.c5(n_requests=2000, n_min=2, n_max=3)  # cheap: the gap law only
    assert abs(g2.mean() - 1.0) < 0.08
