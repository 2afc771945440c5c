"""GPU parity of the build (sort permutations, dominance levels: bit-exact)
and of the product K V (FP64 within 1e-12, FP32 within 1e-5 normwise
relative error per column) against the oracle, through the C ABI."""

import numpy as np
import pytest
import torch

import workloads
from oracle import structure
from gpu_util import colwise_relerr, to_dev

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def build(fgk, p, kind):
    return fgk.fgk_build(to_dev(p.X), p.nu, p.ell, outscale2=p.s2, kind=kind)


STRUCT_CASES = [
    (1, 1, "uniform"), (2, 2, "uniform"), (5, 2, "lattice"), (37, 2, "dups"), (1000, 2, "uniform"),
    (1025, 2, "lattice"), (3000, 2, "dups"), (5000, 2, "uniform"), (2, 3, "uniform"), (33, 3, "lattice"),
    (700, 3, "negzero"), (2500, 3, "uniform"), (4097, 3, "dups"), (3000, 1, "dups"), (9, 1, "negzero"),
]


@pytest.mark.parametrize("N,d,pattern", STRUCT_CASES)
def test_structure_bit_exact(fgk_mod, N, d, pattern):
    fgk = fgk_mod
    p = workloads.small(N + 13 * d, N, d, nu=2.5, ell=[0.13, 0.29, 0.41][:d], pattern=pattern)
    perms, _ = structure.permutations(p.X, p.nu, p.ell)
    levs = structure.levels(p.X, p.nu, p.ell)
    with build(fgk, p, "product") as h:
        info = fgk.fgk_get_info(h)
        assert info["n_levels"] == len(levs) == structure.n_levels(N, d)
        for k in range(d):
            assert np.array_equal(fgk.fgk_get_permutation(h, k), perms[k].astype(np.int32)), f"perm {k}"
        for li, ref in enumerate(levs):
            got = fgk.fgk_get_level(h, li)
            assert got["S"] == ref["S"]
            assert np.array_equal(got["q"], ref["q"]), f"level {li} q"
            roles = np.zeros(N, dtype=np.uint8)
            if d >= 2:
                roles |= ref["r1"]
            if d == 3:
                roles |= ref["r2"] << 1
            assert np.array_equal(got["roles"], roles), f"level {li} roles"
            assert np.array_equal(got["dl64"].view(np.uint64), ref["dl64"].view(np.uint64)), f"level {li} dl64"
            assert np.array_equal(got["dl32"].view(np.uint32), ref["dl32"].view(np.uint32)), f"level {li} dl32"
            if d >= 2:
                assert np.array_equal(got["off64"].view(np.uint64), ref["off64"].view(np.uint64)), f"level {li} off"
                assert np.array_equal(got["off32"].view(np.uint32), ref["off32"].view(np.uint32))


MVM_CASES = [
    # N, d, pattern, nrhs
    (1, 1, "uniform", 1), (2, 2, "uniform", 2), (3, 3, "uniform", 1), (7, 1, "lattice", 2),
    (64, 2, "lattice", 1), (100, 3, "dups", 3), (1000, 1, "uniform", 2), (1500, 2, "negzero", 1),
    (2500, 2, "dups", 2), (3001, 3, "uniform", 2), (5000, 1, "dups", 1), (5000, 2, "uniform", 3),
    (2049, 3, "lattice", 1), (600, 2, "wide", 2),
]


# at nu = 1/2 or d = 1 the product kernel is the L1 kernel: above N = 100 only
# the L1 case runs
PARITY = [(N, d, pattern, nrhs, nu, kind) for kind in ("l1", "product") for nu in (0.5, 1.5, 2.5)
          for (N, d, pattern, nrhs) in MVM_CASES if not (kind == "product" and (nu == 0.5 or d == 1) and N > 100)]


@pytest.mark.parametrize("N,d,pattern,nrhs,nu,kind", PARITY)
def test_mvm_parity(fgk_mod, orc, N, d, pattern, nrhs, nu, kind):
    fgk = fgk_mod
    ell = [0.2, 0.35, 0.5][:d] if pattern != "wide" else [10.0, 20.0, 30.0][:d]
    p = workloads.small(7 * N + d, N, d, nu=nu, ell=ell, nrhs=nrhs, pattern=pattern, s2=1.7)
    kcode = 0 if kind == "l1" else 1
    ref = orc.mvm_brute(p.X, p.V, nu, p.ell, s2=p.s2, kind=kcode)
    with build(fgk, p, kind) as h:
        y64 = fgk.fgk_matvec(h, to_dev(p.V), "f64").cpu().numpy()
        y32 = fgk.fgk_matvec(h, to_dev(p.V, torch.float32), "f32").cpu().numpy()
    e64 = colwise_relerr(y64, ref)
    e32 = colwise_relerr(y32, ref)
    assert (e64 <= TOL64).all(), e64
    assert (e32 <= TOL32).all(), e32


def test_mvm_c1_full(fgk_mod, orc):
    """The d=1 configuration at full size (N=4096, nu=1/2, ell=0.2)."""
    fgk = fgk_mod
    p = workloads.c1()
    ref = orc.mvm_brute(p.X, p.V, p.nu, p.ell)
    with build(fgk, p, "l1") as h:
        for prec, tol, dt in (("f64", TOL64, torch.float64), ("f32", TOL32, torch.float32)):
            y = fgk.fgk_matvec(h, to_dev(p.V, dt), prec).cpu().numpy()
            assert (colwise_relerr(y, ref) <= tol).all()


def sampled_rows(N, k, seed):
    rng = np.random.default_rng(seed)
    rows = rng.choice(N, size=min(k, N), replace=False)
    return np.sort(np.concatenate([rows, [0, N - 1]]))


@pytest.mark.parametrize("kind", ["product", "l1"])
def test_mvm_c2_full_size_sampled(fgk_mod, orc, kind):
    """d=2, N=200000, nu=3/2, ell=(0.1,0.3): every output row is computed on
    the GPU, 400 sampled rows are checked against the brute-force oracle."""
    fgk = fgk_mod
    p = workloads.c2()
    rng = np.random.default_rng(22)
    V = rng.standard_normal((p.N, 2))
    rows = sampled_rows(p.N, 400, 5)
    ref = orc.mvm_brute(p.X, V, p.nu, p.ell, kind=0 if kind == "l1" else 1, rows=rows)
    with build(fgk, p, kind) as h:
        y64 = fgk.fgk_matvec(h, to_dev(V), "f64").cpu().numpy()[rows]
        y32 = fgk.fgk_matvec(h, to_dev(V, torch.float32), "f32").cpu().numpy()[rows]
    assert (colwise_relerr(y64, ref) <= TOL64).all()
    assert (colwise_relerr(y32, ref) <= TOL32).all()


def test_mvm_c3_full_size_sampled(fgk_mod, orc):
    """d=3, N=500000, nu=5/2, product kernel on the Gaussian-mixture points."""
    fgk = fgk_mod
    p = workloads.c3()
    rng = np.random.default_rng(33)
    V = rng.standard_normal((p.N, 1))
    rows = sampled_rows(p.N, 150, 6)
    ref = orc.mvm_brute(p.X, V, p.nu, p.ell, kind=1, rows=rows)
    with build(fgk, p, "product") as h:
        y64 = fgk.fgk_matvec(h, to_dev(V), "f64").cpu().numpy()[rows]
        y32 = fgk.fgk_matvec(h, to_dev(V, torch.float32), "f32").cpu().numpy()[rows]
    assert (colwise_relerr(y64, ref) <= TOL64).all()
    assert (colwise_relerr(y32, ref) <= TOL32).all()


def test_nonfinite_input_rejected(fgk_mod):
    fgk = fgk_mod
    X = np.random.default_rng(1).uniform(size=(50, 2))
    X[17, 1] = np.nan
    with pytest.raises(fgk.FgkError) as e:
        fgk.fgk_build(to_dev(X), 1.5, [0.2, 0.2])
    assert e.value.code == -2
    X[17, 1] = np.inf
    with pytest.raises(fgk.FgkError):
        fgk.fgk_build(to_dev(X), 1.5, [0.2, 0.2])


def test_invalid_arguments(fgk_mod):
    fgk = fgk_mod
    X = to_dev(np.random.default_rng(2).uniform(size=(20, 2)))
    with pytest.raises(ValueError):
        fgk.fgk_build(X, 1.0, [0.2, 0.2])
    with pytest.raises(fgk.FgkError):
        fgk.fgk_build(X, 1.5, [0.2, 0.0])
    with fgk.fgk_build(X, 1.5, [0.2, 0.2]) as h:
        with pytest.raises(TypeError):
            fgk.fgk_matvec(h, torch.zeros(20, dtype=torch.float32, device="cuda"), "f64")


def test_permutation_equivariance_and_linearity(fgk_mod):
    fgk = fgk_mod
    p = workloads.small(77, 3000, 2, nu=1.5, ell=[0.1, 0.3], nrhs=2)
    perm = np.random.default_rng(3).permutation(p.N)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h1, \
            fgk.fgk_build(to_dev(p.X[perm]), p.nu, p.ell, kind="product") as h2:
        y1 = fgk.fgk_matvec(h1, to_dev(p.V)).cpu().numpy()
        y2 = fgk.fgk_matvec(h2, to_dev(p.V[perm])).cpu().numpy()
        assert np.allclose(y2, y1[perm], rtol=1e-12, atol=1e-12 * np.abs(y1).max())
        comb = fgk.fgk_matvec(h1, to_dev(2 * p.V[:, :1] - 3 * p.V[:, 1:])).cpu().numpy()
        assert np.allclose(comb, 2 * y1[:, :1] - 3 * y1[:, 1:], atol=1e-12 * np.abs(y1).max())


@pytest.mark.parametrize("d,nu,N,nrhs", [(2, 1.5, 200000, 1), (2, 2.5, 60000, 3), (3, 2.5, 20000, 2),
                                         (1, 0.5, 50000, 2)])
def test_product_bit_reproducible(fgk_mod, d, nu, N, nrhs):
    """S5: the levels are summed in a fixed order, so the same product is
    bit-identical call after call, in both precisions, also with another
    plan's product launched in between on another stream."""
    fgk = fgk_mod
    p = workloads.small(300 + d, N, d, nu=nu, ell=[0.1, 0.3, 0.2][:d], nrhs=nrhs)
    other = workloads.small(301 + d, 7000, 2, nu=1.5, ell=[0.2, 0.2], nrhs=4)
    with build(fgk, p, "product") as h, build(fgk, other, "product") as h2:
        for dt, prec in ((torch.float32, "f32"), (torch.float64, "f64")):
            V = to_dev(p.V, dt)
            first = fgk.fgk_matvec(h, V, prec).cpu().numpy()
            side = torch.cuda.Stream()
            with torch.cuda.stream(side):
                fgk.fgk_matvec(h2, to_dev(other.V, dt), prec, stream=side)
            again = fgk.fgk_matvec(h, V, prec).cpu().numpy()
            torch.cuda.synchronize()
            bits = np.uint32 if dt == torch.float32 else np.uint64
            assert np.array_equal(first.view(bits), again.view(bits)), prec


# nu = 7/2 and 9/2 (eqs. matern_7_2, matern_9_2): the scans with four and five
# moments and the coefficients of eq. matern_explicit passed at run time
HIGH_NU_CASES = [(N, d, pattern, nrhs, nu, kind)
                 for nu in (3.5, 4.5)
                 for (N, d, pattern, nrhs, kind) in [
                     (1, 1, "uniform", 1, "l1"), (700, 1, "dups", 2, "l1"), (5000, 1, "uniform", 1, "l1"),
                     (64, 2, "lattice", 1, "product"), (2500, 2, "dups", 2, "product"),
                     (5000, 2, "uniform", 1, "product"), (3000, 2, "uniform", 2, "l1"),
                     (100, 3, "dups", 1, "product"), (3001, 3, "uniform", 1, "product"),
                     (2049, 3, "lattice", 1, "l1"), (600, 2, "wide", 2, "product")]
                 if not (nu == 4.5 and d == 3)]


def test_nine_halves_at_d3_is_refused(fgk_mod):
    """nu = 9/2 is built for d <= 2: the library refuses d = 3."""
    fgk = fgk_mod
    p = workloads.small(5, 100, 3, nu=4.5, ell=[0.2, 0.3, 0.4])
    with pytest.raises(fgk.FgkError) as e:
        fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product")
    assert e.value.code == -1


@pytest.mark.parametrize("N,d,pattern,nrhs,nu,kind", HIGH_NU_CASES)
def test_mvm_parity_higher_nu(fgk_mod, orc, N, d, pattern, nrhs, nu, kind):
    fgk = fgk_mod
    ell = [0.2, 0.35, 0.5][:d] if pattern != "wide" else [10.0, 20.0, 30.0][:d]
    p = workloads.small(11 * N + d, N, d, nu=nu, ell=ell, nrhs=nrhs, pattern=pattern, s2=1.3)
    ref = orc.mvm_brute(p.X, p.V, nu, p.ell, s2=p.s2, kind=0 if kind == "l1" else 1)
    with build(fgk, p, kind) as h:
        y64 = fgk.fgk_matvec(h, to_dev(p.V), "f64").cpu().numpy()
        y32 = fgk.fgk_matvec(h, to_dev(p.V, torch.float32), "f32").cpu().numpy()
    assert (colwise_relerr(y64, ref) <= TOL64).all(), colwise_relerr(y64, ref)
    assert (colwise_relerr(y32, ref) <= TOL32).all(), colwise_relerr(y32, ref)


def test_mvm_higher_nu_c2_shape_sampled(fgk_mod, orc):
    """nu = 9/2 on the d=2 workload's points (N = 200000), 200 sampled rows."""
    fgk = fgk_mod
    p = workloads.c2()
    V = np.random.default_rng(45).standard_normal((p.N, 1))
    rows = sampled_rows(p.N, 200, 9)
    ref = orc.mvm_brute(p.X, V, 4.5, p.ell, kind=1, rows=rows)
    with fgk.fgk_build(to_dev(p.X), 4.5, p.ell, kind="product") as h:
        y64 = fgk.fgk_matvec(h, to_dev(V), "f64").cpu().numpy()[rows]
        y32 = fgk.fgk_matvec(h, to_dev(V, torch.float32), "f32").cpu().numpy()[rows]
    assert (colwise_relerr(y64, ref) <= TOL64).all()
    assert (colwise_relerr(y32, ref) <= TOL32).all()


@pytest.mark.parametrize("d,nu,kind", [(1, 1.5, "l1"), (2, 1.5, "product"), (2, 2.5, "l1"), (2, 0.5, "l1")])
def test_mvm_parity_mixed_gap_scales(fgk_mod, orc, d, nu, kind):
    """Dense clusters next to points spaced three scaled units apart along
    every coordinate: some threads' eight entries span more than the FP32
    scans' anchored-walk limit (20 scaled units) and take the plain walk,
    others take the anchored one, within the same product."""
    fgk = fgk_mod
    rng = np.random.default_rng(4242 + 10 * d)
    ell = np.full(d, 0.25)
    a = np.sqrt(2 * nu) / ell[0]
    n_sparse, n_dense = 1500, 2500
    sparse = (3.0 / a) * np.arange(n_sparse)[:, None] + rng.uniform(0, 0.1 / a, size=(n_sparse, d))
    dense = rng.uniform(0, 0.05, size=(n_dense, d)) + sparse[n_sparse // 2]
    X = np.concatenate([sparse, dense])[rng.permutation(n_sparse + n_dense)]
    V = rng.standard_normal((X.shape[0], 2)) * np.exp(rng.uniform(-3, 3, size=(X.shape[0], 1)))
    ref = orc.mvm_brute(X, V, nu, ell, kind=0 if kind == "l1" else 1)
    with fgk.fgk_build(to_dev(X), nu, ell, kind=kind) as h:
        y32 = fgk.fgk_matvec(h, to_dev(V, torch.float32), "f32").cpu().numpy()
        y64 = fgk.fgk_matvec(h, to_dev(V), "f64").cpu().numpy()
    assert (colwise_relerr(y64, ref) <= TOL64).all()
    assert (colwise_relerr(y32, ref) <= TOL32).all(), colwise_relerr(y32, ref)
