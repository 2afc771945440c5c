"""Pins for the oracle: each check ties it to something other than itself
(scipy's Bessel function, a state-space model, a textbook closed-form
inverse, a Kronecker identity, limits, brute force on tiny inputs, the
paper's own second algorithm)."""

import math

import numpy as np
import pytest
from scipy import linalg, special
from scipy.spatial.distance import cdist

import workloads
from oracle import structure

NUS = (0.5, 1.5, 2.5)
# the closed forms of eqs. matern_7_2 and matern_9_2: the definition-based
# entries take them (the decompositions O2 and phi stop at 5/2)
NUS_ALL = NUS + (3.5, 4.5)


def matern_bessel(nu, u):
    """eq. matern_general: (sqrt(2nu)|u|)^nu / (2^(nu-1) Gamma(nu)) K_nu(sqrt(2nu)|u|)."""
    u = np.abs(np.asarray(u, dtype=np.float64))
    z = np.sqrt(2 * nu) * u
    out = np.ones_like(z)
    nz = z > 0
    out[nz] = z[nz] ** nu / (2 ** (nu - 1) * special.gamma(nu)) * special.kv(nu, z[nz])
    return out


def matern_general(p, u):
    """eq. matern_explicit for nu = p + 1/2."""
    u = np.abs(np.asarray(u, dtype=np.float64))
    s = np.zeros_like(u)
    c = math.sqrt(2 * p + 1)
    for i in range(p + 1):
        s += (math.comb(p, i) * math.factorial(2 * p - i) / math.factorial(2 * p)) * (2 * c * u) ** i
    return s * np.exp(-c * u)


def matern_state_space(nu, tau):
    """Stationary covariance of the Matérn SDE in companion form
    ((d/dt + lam)^P f = white noise, lam = sqrt(2 nu)), normalised to 1 at 0."""
    P = int(nu + 0.5)
    lam = math.sqrt(2 * nu)
    coeffs = [math.comb(P, j) * lam ** (P - j) for j in range(P)]  # of (s + lam)^P
    F = np.zeros((P, P))
    F[:-1, 1:] = np.eye(P - 1)
    F[-1, :] = -np.array(coeffs)
    Lq = np.zeros((P, P))
    Lq[-1, -1] = 1.0
    Pinf = linalg.solve_continuous_lyapunov(F, -Lq)
    return np.array([(linalg.expm(F * t) @ Pinf)[0, 0] / Pinf[0, 0] for t in np.atleast_1d(tau)])


def dense_ref(X, ell, nu, kind):
    """K from scipy pieces only: cityblock distances and the Bessel form."""
    U = np.asarray(X, dtype=np.float64) / np.asarray(ell)[None, :]
    if kind == 0:
        return matern_bessel(nu, cdist(U, U, metric="cityblock"))
    K = np.ones((U.shape[0], U.shape[0]))
    for k in range(U.shape[1]):
        K *= matern_bessel(nu, cdist(U[:, k:k + 1], U[:, k:k + 1], metric="cityblock"))
    return K


def relerr(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# --------------------------------------------------------------------------
# kernel values
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nu", NUS_ALL)
def test_kernel_closed_form_vs_bessel(orc, nu):
    u = np.concatenate([[0.0], np.geomspace(1e-4, 25.0, 200)])
    got = orc.kernel(nu, u)
    ref = matern_bessel(nu, u)
    assert np.allclose(got, ref, rtol=2e-13, atol=1e-300)
    assert orc.kernel(nu, 0.0) == 1.0


@pytest.mark.parametrize("nu", NUS_ALL)
def test_kernel_closed_form_vs_general_formula(orc, nu):
    u = np.linspace(0, 12, 97)
    assert np.allclose(orc.kernel(nu, u), matern_general(int(nu - 0.5), u), rtol=1e-14, atol=1e-300)


@pytest.mark.parametrize("nu", NUS_ALL)
def test_kernel_closed_form_vs_state_space(orc, nu):
    tau = np.linspace(0, 4, 17)
    assert np.allclose(orc.kernel(nu, tau), matern_state_space(nu, tau), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("nu", NUS)
def test_phi_factorisation(orc, nu):
    """Assumption 1: sum_p phi1_p(u) phi2_p(v) = k(u - v) for u >= v, with k
    taken from the Bessel form (eqs. k12/k32/k52_decomposition)."""
    rng = np.random.default_rng(11)
    v = rng.uniform(-3, 3, 300)
    u = v + rng.uniform(0, 4, 300)
    P = int(nu + 0.5)
    s = sum(orc.phi(nu, 1, p, u) * orc.phi(nu, 2, p, v) for p in range(P))
    assert np.allclose(s, matern_bessel(nu, u - v), rtol=1e-11, atol=1e-13)


# --------------------------------------------------------------------------
# O1: brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("nu", NUS_ALL)
@pytest.mark.parametrize("kind", [0, 1])
def test_brute_vs_scipy_dense(orc, d, nu, kind):
    p = workloads.small(100 + d, 150, d, nu=nu, ell=[0.2, 0.35, 0.5][:d], nrhs=3, s2=1.7)
    K = dense_ref(p.X, p.ell, nu, kind)
    got = orc.mvm_brute(p.X, p.V, nu, p.ell, s2=p.s2, kind=kind)
    assert relerr(got, p.s2 * K @ p.V) < 1e-13
    assert np.allclose(orc.kmat(p.X, nu, p.ell, p.s2, kind), p.s2 * K, rtol=1e-13, atol=1e-300)


def test_brute_rows_subset(orc):
    p = workloads.small(5, 300, 2, nu=2.5, nrhs=2)
    full = orc.mvm_brute(p.X, p.V, 2.5, p.ell, kind=1)
    rows = np.array([0, 7, 299, 150, 7])
    part = orc.mvm_brute(p.X, p.V, 2.5, p.ell, kind=1, rows=rows)
    assert np.array_equal(part, full[rows])


def test_ou_closed_form_inverse(orc):
    """nu=1/2, d=1: the Ornstein-Uhlenbeck covariance on sorted points has the
    tridiagonal inverse Q with rho_i = exp(-(t_{i+1}-t_i)/ell):
    Q_ii = 1/(1-rho_{i-1}^2) + 1/(1-rho_i^2) - 1, Q_{i,i+1} = -rho_i/(1-rho_i^2)
    (end rows drop the missing term).  K (Q v) = v."""
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0, 1, 400))
    ell = 0.2
    rho = np.exp(-np.diff(t) / ell)
    a = 1.0 / (1.0 - rho ** 2)
    diag = np.ones(t.size)
    diag[:-1] += a - 1.0
    diag[1:] += a - 1.0
    off = -rho * a
    v = rng.standard_normal(t.size)
    Qv = diag * v
    Qv[:-1] += off * v[1:]
    Qv[1:] += off * v[:-1]
    perm = rng.permutation(t.size)  # the oracle must not care about order
    got = orc.mvm_brute(t[perm, None], Qv[perm], 0.5, [ell])
    assert relerr(got, v[perm]) < 1e-11


@pytest.mark.parametrize("nu", NUS_ALL)
def test_kronecker_tensor_grid(orc, nu):
    """Product kernel on a tensor grid: K = K1 (x) K2 (eq. product_kernel);
    at nu = 1/2 the L1 kernel is the same matrix (eq. matern_l1_12)."""
    rng = np.random.default_rng(4)
    g1 = np.sort(rng.uniform(0, 1, 13))
    g2 = np.sort(rng.uniform(0, 1, 9))
    ell = np.array([0.15, 0.4])
    X = np.array([[a, b] for a in g1 for b in g2])
    V = rng.standard_normal((13, 9))
    K1 = np.stack([orc.mvm_brute(g1[:, None], e, nu, ell[:1]) for e in np.eye(13)], axis=1)
    K2 = np.stack([orc.mvm_brute(g2[:, None], e, nu, ell[1:]) for e in np.eye(9)], axis=1)
    ref = (K1 @ V @ K2.T).ravel()
    got = orc.mvm_brute(X, V.ravel(), nu, ell, kind=1)
    assert relerr(got, ref) < 1e-13
    if nu == 0.5:
        assert relerr(orc.mvm_brute(X, V.ravel(), nu, ell, kind=0), ref) < 1e-13


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("nu", NUS_ALL)
def test_lengthscale_limits(orc, kind, nu):
    rng = np.random.default_rng(6)
    X = rng.uniform(0, 1, (60, 2))
    v = rng.standard_normal(60)
    big = orc.mvm_brute(X, v, nu, [1e12, 1e12], s2=2.0, kind=kind)
    assert np.allclose(big, 2.0 * v.sum(), rtol=1e-9)
    Xg = np.array([[i * 1e-2, j * 1e-2] for i in range(6) for j in range(10)])
    tiny = orc.mvm_brute(Xg, v, nu, [1e-5, 1e-5], s2=2.0, kind=kind)
    assert np.allclose(tiny, 2.0 * v, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("kind", [0, 1])
def test_symmetry_and_linearity(orc, kind):
    p = workloads.small(8, 250, 3, nu=2.5, nrhs=2)
    u, v = p.V[:, 0], p.V[:, 1]
    Ku = orc.mvm_brute(p.X, u, 2.5, p.ell, kind=kind)
    Kv = orc.mvm_brute(p.X, v, 2.5, p.ell, kind=kind)
    assert abs(u @ Kv - v @ Ku) < 1e-11 * abs(u @ Kv)
    Kuv = orc.mvm_brute(p.X, 2 * u - 3 * v, 2.5, p.ell, kind=kind)
    assert relerr(Kuv, 2 * Ku - 3 * Kv) < 1e-13


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("nu", NUS)
def test_positive_definiteness(orc, d, nu):
    """Prop. 3: the product kernel is PD; Prop. 4: the L1 kernel is PD for
    nu = 1/2 (completely monotone k).  For nu >= 3/2 the sufficient
    condition of Prop. 4 fails and the L1 matrix is indefinite."""
    rng = np.random.default_rng(20 + d)
    X = rng.uniform(0, 1, (300, d))
    ell = np.full(d, 0.3)
    lam_prod = np.linalg.eigvalsh(orc.kmat(X, nu, ell, kind=1))[0]
    assert lam_prod > 0
    lam_l1 = np.linalg.eigvalsh(orc.kmat(X, nu, ell, kind=0))[0]
    if nu == 0.5:
        assert lam_l1 > 0
    else:
        assert lam_l1 < 0


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("nu", (3.5, 4.5))
def test_positive_definiteness_of_the_smoother_kernels(orc, d, nu):
    """Props. 3-4 at nu = 7/2, 9/2 (lengthscale 0.15, where the smallest
    eigenvalue of the product kernel stays far above eigvalsh's rounding):
    the product kernel is PD, the L1 kernel indefinite."""
    rng = np.random.default_rng(20 + d)
    X = rng.uniform(0, 1, (300, d))
    ell = np.full(d, 0.15)
    w = np.linalg.eigvalsh(orc.kmat(X, nu, ell, kind=1))
    assert w[0] > 1e3 * X.shape[0] * np.finfo(float).eps * w[-1]
    assert np.linalg.eigvalsh(orc.kmat(X, nu, ell, kind=0))[0] < -1e-2


def test_decompositions_stop_at_five_halves(orc):
    """The paper prints the decompositions (O2, the phi pairs) for nu <= 5/2
    only: those entries refuse nu = 7/2, while the definition accepts it."""
    p = workloads.small(5, 20, 2, nu=1.5)
    assert np.isfinite(orc.mvm_brute(p.X, p.V, 3.5, p.ell, kind=1)).all()
    for call in (lambda: orc.mvm_dc(p.X, p.V, 3.5, p.ell, kind=1),
                 lambda: orc.mvm_dc(p.X, p.V, 4.5, p.ell, kind=0),
                 lambda: orc.mvm_dc_dlogell_l1(p.X, p.V, 3.5, p.ell),
                 lambda: orc.mvm_dc_dlogell_product(p.X, p.V, 3.5, p.ell),
                 lambda: orc.mvm_dc_cross(p.X, p.X[:3], p.V, 3.5, p.ell),
                 lambda: orc.phi(3.5, 1, 0, 0.5)):
        with pytest.raises(ValueError):
            call()
    with pytest.raises(ValueError):
        orc.kernel(3.0, 0.5)  # not a half-integer


# --------------------------------------------------------------------------
# O2: the paper's decomposition, against O1
# --------------------------------------------------------------------------

CASES = [(1, "uniform"), (2, "uniform"), (3, "uniform"), (7, "lattice"), (33, "dups"),
         (64, "lattice"), (64, "negzero"), (100, "uniform"), (37, "wide")]


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("nu", NUS)
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("N,pattern", CASES)
def test_dc_vs_brute(orc, d, nu, kind, N, pattern):
    ell = [0.3, 0.5, 0.7][:d] if pattern != "wide" else [20.0, 30.0, 40.0][:d]
    p = workloads.small(N + 7 * d, N, d, nu=nu, ell=ell, nrhs=2, pattern=pattern, s2=1.3)
    ref = orc.mvm_brute(p.X, p.V, nu, p.ell, s2=p.s2, kind=kind)
    got = orc.mvm_dc(p.X, p.V, nu, p.ell, s2=p.s2, kind=kind)
    # the printed recombinations subtract terms of size ~ (a delta.z)^p F_0
    assert relerr(got, ref) < 1e-11


@pytest.mark.parametrize("d", [1, 2, 3])
def test_dc_product32_printed_reading(orc, d):
    p = workloads.small(40 + d, 80, d, nu=1.5, ell=[0.25, 0.4, 0.6][:d], pattern="dups")
    ref = orc.mvm_dc(p.X, p.V[:, 0], 1.5, p.ell, kind=1)
    got = orc.mvm_dc_product32_printed(p.X, p.V[:, 0], p.ell)
    assert relerr(got, ref) < 1e-12


# --------------------------------------------------------------------------
# O3: structure
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N,d,pattern", [(1, 2, "uniform"), (2, 2, "uniform"), (5, 2, "lattice"),
                                         (37, 2, "dups"), (64, 2, "lattice"), (100, 3, "uniform"),
                                         (33, 3, "lattice"), (70, 3, "negzero"), (50, 1, "dups")])
def test_structure_covers_each_pair_once(N, d, pattern):
    p = workloads.small(N * 3 + d, N, d, nu=1.5, ell=[0.2, 0.3, 0.4][:d], pattern=pattern)
    Xs = structure.scaled(p.X, p.nu, p.ell)
    perms, ranks = structure.permutations(p.X, p.nu, p.ell)
    # permutations: ascending, ties by index
    for k in range(d):
        key = list(zip(Xs[perms[k], k], perms[k]))
        assert key == sorted(key)
    levs = structure.levels(p.X, p.nu, p.ell)
    assert len(levs) == structure.n_levels(N, d)
    q2pt = perms[0]
    cover = np.zeros((N, N), dtype=np.int64)
    for lev in levs:
        q = lev["q"].astype(np.int64)
        assert np.array_equal(np.sort(q), np.arange(N))
        S = lev["S"]
        pts = q2pt[q]
        xs = Xs[pts, d - 1]
        for s0 in range(0, N, S):
            seg = slice(s0, min(s0 + S, N))
            sp = pts[seg]
            # sorted by the sweep coordinate, ties by original index
            key = list(zip(xs[seg], sp))
            assert key == sorted(key)
            assert lev["dl64"][s0] == 0.0
            assert np.all(lev["dl64"][seg] >= 0)
            if d == 1:
                continue
            cnt = sp.size
            roles = lev["r1"][seg].astype(np.int64)
            if d == 3:
                roles = roles * 2 + lev["r2"][seg]
            nch = 2 if d == 2 else 4
            for a in range(cnt):
                for b in range(cnt):
                    if roles[a] + roles[b] == nch - 1:  # complementary roles
                        cover[sp[a], sp[b]] += 1
                        # offsets add up to the split-dimension distances
                        for k in range(d - 1):
                            dist = abs(Xs[sp[a], k] - Xs[sp[b], k])
                            s = lev["off64"][s0 + a, k] + lev["off64"][s0 + b, k]
                            assert abs(s - dist) <= 4e-16 * max(abs(Xs[:, k]).max(), 1.0)
                        # the summed gaps give the sweep distance
                        lo, hi = sorted((a, b))
                        D = lev["dl64"][s0 + lo + 1:s0 + hi + 1].sum()
                        assert abs(D - abs(xs[s0 + a] - xs[s0 + b])) <= 1e-14 * max(abs(xs).max(), 1.0)
    if d >= 2:
        assert np.array_equal(cover, 1 - np.eye(N, dtype=np.int64))


def test_structure_scaling_canonical():
    X = np.array([[-0.0, 1.0], [0.0, -0.0], [0.5, 0.25]])
    Xs = structure.scaled(X, 1.5, [0.2, 0.4])
    assert not np.signbit(Xs).any()
    assert Xs[2, 0] == 0.5 * (np.sqrt(3.0) / 0.2)
