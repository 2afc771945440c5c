"""Pins for the oracle's lengthscale-gradient product (dK/d log ell) V, the
matrix-vector product of the trace term of eq. gp_log_likelihood_derivative
(App. C.1 prints the gradients of the Matérn kernels).  Each check ties the
closed forms to something other than themselves: central finite differences
of scipy's Bessel form and of the oracle's own (already pinned) product, the
symmetry of dK, the sum over lengthscales and the zero self-term."""

import numpy as np
import pytest
from scipy import special

import workloads

NUS = (0.5, 1.5, 2.5)
NUS_ALL = NUS + (3.5, 4.5)  # eqs. dmatern72_dl, dmatern92_dl


def bessel_k(nu, u):
    """eq. matern_general (scipy's modified Bessel function of the 2nd kind)."""
    u = np.abs(np.asarray(u, dtype=np.float64))
    z = np.sqrt(2 * nu) * u
    out = np.ones_like(z)
    nz = z > 0
    out[nz] = z[nz] ** nu / (2 ** (nu - 1) * special.gamma(nu)) * special.kv(nu, z[nz])
    return out


@pytest.mark.parametrize("nu", NUS_ALL)
def test_kernel_dlog_is_the_log_lengthscale_derivative_of_the_bessel_form(orc, nu):
    u = np.linspace(0.0, 6.0, 61)
    h = 1e-5
    # k(|x| / l) with l -> l e^{+-h}: u -> u e^{-+h}
    fd = (bessel_k(nu, u * np.exp(-h)) - bessel_k(nu, u * np.exp(h))) / (2 * h)
    np.testing.assert_allclose(orc.kernel_dlog(nu, u, which=0), fd, rtol=1e-7, atol=1e-10)
    uu = u[1:]
    fd1 = (bessel_k(nu, uu - h) - bessel_k(nu, uu + h)) / (2 * h)  # -k'(u)
    np.testing.assert_allclose(orc.kernel_dlog(nu, uu, which=1), fd1, rtol=1e-7, atol=1e-10)


def _fd_product(orc, X, V, nu, ell, dim, kind, h=1e-5):
    ell = np.asarray(ell, dtype=np.float64)
    step = np.zeros_like(ell)
    if dim < 0:
        step[:] = h
    else:
        step[dim] = h
    yp = orc.mvm_brute(X, V, nu, ell * np.exp(step), kind=kind)
    ym = orc.mvm_brute(X, V, nu, ell * np.exp(-step), kind=kind)
    return (yp - ym) / (2 * h)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("nu", NUS_ALL)
@pytest.mark.parametrize("d", [1, 2, 3])
def test_gradient_product_matches_finite_differences(orc, kind, nu, d):
    p = workloads.small(700 + d, 150, d, nu=nu, ell=[0.2, 0.35, 0.15][:d], nrhs=2)
    dims = [-1] + list(range(d))
    for dim in dims:
        got = orc.mvm_dlogell_brute(p.X, p.V, nu, p.ell, dim=dim, kind=kind)
        fd = _fd_product(orc, p.X, p.V, nu, p.ell, dim, kind)
        err = np.linalg.norm(got - fd, axis=0) / np.linalg.norm(fd, axis=0)
        assert (err < 1e-7).all(), (dim, err)


@pytest.mark.parametrize("kind", [0, 1])
def test_gradient_product_on_ties_and_duplicates(orc, kind):
    for name in ("lattice", "dups"):
        p = workloads.small(11, 120, 2, pattern=name)
        for dim in (-1, 0, 1):
            got = orc.mvm_dlogell_brute(p.X, p.V, 1.5, [0.3, 0.2], dim=dim, kind=kind)
            fd = _fd_product(orc, p.X, p.V, 1.5, [0.3, 0.2], dim, kind)
            assert np.linalg.norm(got - fd) <= 1e-7 * np.linalg.norm(fd), (name, dim)


@pytest.mark.parametrize("kind", [0, 1])
def test_gradient_matrix_is_symmetric_with_zero_diagonal_and_sums_over_dims(orc, kind):
    p = workloads.small(31, 60, 3, nu=2.5, ell=[0.2, 0.3, 0.25])
    eye = np.eye(p.N)
    G = [orc.mvm_dlogell_brute(p.X, eye, 2.5, p.ell, dim=m, kind=kind) for m in range(3)]
    Gall = orc.mvm_dlogell_brute(p.X, eye, 2.5, p.ell, dim=-1, kind=kind)
    for g in G + [Gall]:
        np.testing.assert_allclose(g, g.T, rtol=0, atol=1e-14)
        np.testing.assert_array_equal(np.diag(g), 0.0)
    np.testing.assert_allclose(G[0] + G[1] + G[2], Gall, rtol=0, atol=1e-13)


def test_gradient_of_one_point_is_zero_and_outputscale_is_linear(orc):
    X = np.array([[0.3, 0.7]])
    assert orc.mvm_dlogell_brute(X, np.array([2.0]), 1.5, [0.1, 0.2], kind=1)[0] == 0.0
    p = workloads.small(5, 80, 2, nu=0.5, ell=[0.1, 0.2])
    a = orc.mvm_dlogell_brute(p.X, p.V, 0.5, p.ell, dim=1, s2=2.5, kind=1)
    b = orc.mvm_dlogell_brute(p.X, p.V, 0.5, p.ell, dim=1, s2=1.0, kind=1)
    np.testing.assert_allclose(a, 2.5 * b, rtol=1e-15)


def test_gradient_rejects_a_dimension_out_of_range(orc):
    p = workloads.small(6, 10, 2, nu=1.5, ell=[0.1, 0.2])
    with pytest.raises(ValueError):
        orc.mvm_dlogell_brute(p.X, p.V, 1.5, p.ell, dim=2)


@pytest.mark.parametrize("nu", NUS)
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("pattern", ["uniform", "lattice", "dups"])
def test_printed_l1_gradient_decomposition_equals_the_definition(orc, nu, d, pattern):
    """App. C.1's gradient decompositions of the L1 kernels (the ECDF form,
    evaluated on the literal divide and conquer) against the brute-force
    derivative."""
    # lengthscales of the O2 pins: the literal form's raw e^{a delta.x} weights cancel
    p = workloads.small(900 + d, 120, d, nu=nu, ell=[0.3, 0.5, 0.7][:d], nrhs=2, pattern=pattern, s2=1.3)
    got = orc.mvm_dc_dlogell_l1(p.X, p.V, nu, p.ell, s2=p.s2)
    ref = orc.mvm_dlogell_brute(p.X, p.V, nu, p.ell, dim=-1, s2=p.s2, kind=0)
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert (err < 1e-11).all(), err


@pytest.mark.parametrize("nu", NUS)
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("pattern", ["uniform", "lattice", "dups"])
def test_product_gradient_through_proposition_2_equals_the_definition(orc, nu, d, pattern):
    p = workloads.small(950 + d, 100, d, nu=nu, ell=[0.3, 0.5, 0.7][:d], nrhs=2, pattern=pattern, s2=1.3)
    for dim in [-1] + list(range(d)):
        got = orc.mvm_dc_dlogell_product(p.X, p.V, nu, p.ell, dim=dim, s2=p.s2)
        ref = orc.mvm_dlogell_brute(p.X, p.V, nu, p.ell, dim=dim, s2=p.s2, kind=1)
        err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert (err < 1e-11).all(), (dim, err)
