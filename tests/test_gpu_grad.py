"""GPU parity of the lengthscale-gradient product (dK/d log ell) V
(fgk_matvec_dlogell; the gradient formulas of App. C.1, the product that the
trace term of eq. gp_log_likelihood_derivative needs) against the oracle's
definition, through the C ABI: FP64 within 1e-12 and FP32 within 1e-5
normwise relative error per column, the same bars as the product K V."""

import numpy as np
import pytest
import torch

import workloads
from gpu_util import colwise_relerr, to_dev

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5

CASES = [
    # N, d, pattern, nrhs: several tiles (2048 entries), long segments, ragged tails
    (1, 1, "uniform", 1), (2, 2, "uniform", 1), (3, 3, "uniform", 2), (64, 2, "lattice", 1),
    (1000, 1, "dups", 2), (2500, 2, "uniform", 1), (3001, 3, "uniform", 1), (5000, 2, "dups", 2),
    (4097, 1, "uniform", 1), (2049, 3, "lattice", 1), (600, 2, "wide", 1),
]


def _dims(d, kind):
    if kind == "product" and d > 1:
        return [-1] + list(range(d))
    return [-1] if d > 1 else [-1, 0]


# at d = 1 the product kernel is the L1 kernel: above N = 100 only the L1 case runs
PARITY = [(N, d, pattern, nrhs, nu, kind) for kind in ("l1", "product") for nu in (0.5, 1.5, 2.5)
          for (N, d, pattern, nrhs) in CASES if not (kind == "product" and d == 1 and N > 100)]
# nu = 7/2 (eq. dmatern72_dl): the scans with five moments
PARITY += [(N, d, pattern, nrhs, 3.5, kind) for kind in ("l1", "product")
           for (N, d, pattern, nrhs) in [(1000, 1, "dups", 2), (2500, 2, "uniform", 1), (600, 2, "wide", 1)]
           if not (kind == "product" and d == 1)]


@pytest.mark.parametrize("N,d,pattern,nrhs,nu,kind", PARITY)
def test_gradient_product_parity(fgk_mod, orc, N, d, pattern, nrhs, nu, kind):
    fgk = fgk_mod
    ell = [0.2, 0.35, 0.5][:d] if pattern != "wide" else [10.0, 20.0, 30.0][:d]
    p = workloads.small(11 * N + d, N, d, nu=nu, ell=ell, nrhs=nrhs, pattern=pattern, s2=1.3)
    kcode = 0 if kind == "l1" else 1
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, outscale2=p.s2, kind=kind) as h:
        for dim in _dims(d, kind):
            ref = orc.mvm_dlogell_brute(p.X, p.V, nu, p.ell, dim=dim, s2=p.s2, kind=kcode).reshape(N, -1)
            y64 = fgk.fgk_matvec_dlogell(h, to_dev(p.V), dim, "f64").cpu().numpy().reshape(N, -1)
            y32 = fgk.fgk_matvec_dlogell(h, to_dev(p.V, torch.float32), dim, "f32").cpu().numpy().reshape(N, -1)
            if N == 1:
                assert (y64 == 0).all() and (y32 == 0).all()
                continue
            e64, e32 = colwise_relerr(y64, ref), colwise_relerr(y32, ref)
            assert (e64 <= TOL64).all(), (dim, e64)
            assert (e32 <= TOL32).all(), (dim, e32)


def test_gradient_sums_over_lengthscales(fgk_mod):
    fgk = fgk_mod
    p = workloads.small(77, 3000, 3, nu=2.5, ell=[0.2, 0.3, 0.25], nrhs=2)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        V = to_dev(p.V)
        parts = sum(fgk.fgk_matvec_dlogell(h, V, m, "f64") for m in range(3)).cpu().numpy()
        allm = fgk.fgk_matvec_dlogell(h, V, -1, "f64").cpu().numpy()
        assert (colwise_relerr(allm, parts) <= 1e-13).all()


def test_l1_per_lengthscale_derivative_is_rejected(fgk_mod):
    fgk = fgk_mod
    p = workloads.small(5, 100, 2, nu=1.5, ell=[0.2, 0.3])
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="l1") as h:
        with pytest.raises(RuntimeError, match="L1"):
            fgk.fgk_matvec_dlogell(h, to_dev(p.V), 0, "f64")
        with pytest.raises(RuntimeError):
            fgk.fgk_matvec_dlogell(h, to_dev(p.V), 2, "f64")


@pytest.mark.parametrize("prec,tol", [("f64", TOL64), ("f32", TOL32)])
def test_gradient_product_d2_workload_sampled(fgk_mod, orc, prec, tol):
    """The d=2 workload at full size (N = 200000, nu = 3/2, ell = (0.1, 0.3),
    product kernel), every lengthscale, on 300 output rows computed by the
    oracle."""
    fgk = fgk_mod
    p = workloads.c2()
    rng = np.random.default_rng(9)
    V = rng.standard_normal(p.N)
    rows = np.sort(rng.choice(p.N, size=300, replace=False))
    dt = torch.float64 if prec == "f64" else torch.float32
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        for dim in (-1, 0, 1):
            y = fgk.fgk_matvec_dlogell(h, to_dev(V, dt), dim, prec).cpu().numpy().astype(np.float64)
            ref = orc.mvm_dlogell_brute(p.X, V, p.nu, p.ell, dim=dim, kind=1, rows=rows)
            err = np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref)
            assert err <= tol, (dim, err)


@pytest.mark.parametrize("d,nu", [(2, 4.5), (3, 3.5)])
def test_gradient_beyond_the_built_orders_is_rejected(fgk_mod, d, nu):
    """The nu = 9/2 derivative needs six moments and the nu = 7/2 one at d = 3
    five moments with two split dimensions: neither is built, both refused."""
    fgk = fgk_mod
    p = workloads.small(78, 500, d, nu=nu, ell=[0.2, 0.3, 0.25][:d])
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        with pytest.raises(fgk.FgkError) as e:
            fgk.fgk_matvec_dlogell(h, to_dev(p.V), 0, "f64")
        assert e.value.code == -1
