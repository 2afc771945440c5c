"""The C ABI without a GPU: the library builds, loads, exports every function
that include/fgk.h declares, and rejects invalid arguments before touching
the device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_01864_gb300 import build, fgk

    build.build()
    return fgk.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fgk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(fgk_[a-z_0-9]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["fgk_build", "fgk_matvec", "fgk_cg_solve", "fgk_bytes_estimate", "fgk_destroy", "fgk_last_error",
              "fgk_set_allocator"]:
        assert n in names


def test_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n
    from paper_2508_01864_gb300 import fgk

    assert sorted(fgk.EXPORTS) == declared_functions()


def test_bytes_estimate(lib):
    from paper_2508_01864_gb300 import fgk

    assert fgk.fgk_bytes_estimate(0, 2, 1.5) == 0
    assert fgk.fgk_bytes_estimate(1000, 4, 1.5) == 0
    small = fgk.fgk_bytes_estimate(10_000, 2, 1.5, "product", 1)
    big = fgk.fgk_bytes_estimate(200_000, 2, 1.5, "product", 1)
    d3 = fgk.fgk_bytes_estimate(200_000, 3, 2.5, "product", 5)
    assert 0 < small < big < d3
    # the structure of d=3 holds about L(L+1)/2 entries per point
    assert d3 > 200_000 * 18 * 19 // 2 * 16


def test_invalid_arguments_rejected_without_gpu(lib):
    out = ctypes.c_void_p()
    ell = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    # N = 0, d = 4, two_nu = 2, ell <= 0, kind = 7: all rejected before any CUDA call
    assert lib.fgk_build(1, 0, 2, 3, ell, 1.0, 0, None, ctypes.byref(out)) == -1
    assert b"N" in lib.fgk_last_error()
    assert lib.fgk_build(1, 10, 4, 3, ell, 1.0, 0, None, ctypes.byref(out)) == -1
    assert lib.fgk_build(1, 10, 2, 2, ell, 1.0, 0, None, ctypes.byref(out)) == -1
    bad_ell = (ctypes.c_double * 3)(0.1, -1.0, 0.1)
    assert lib.fgk_build(1, 10, 2, 3, bad_ell, 1.0, 0, None, ctypes.byref(out)) == -1
    assert lib.fgk_build(1, 10, 2, 3, ell, 1.0, 7, None, ctypes.byref(out)) == -1
    assert lib.fgk_build(1, 10, 2, 3, ell, 0.0, 0, None, ctypes.byref(out)) == -1
    assert out.value is None
    assert lib.fgk_matvec(None, 1, 1, 1, 0, None) == -1
    assert lib.fgk_destroy(None) == 0
    assert lib.fgk_set_allocator(1, None, None) == -1
    assert lib.fgk_set_allocator(None, None, None) == 0
    # preconditioner: NULL plan, bad rank or sigma2
    pc = ctypes.c_void_p()
    assert lib.fgk_precond_build(None, 10, 0.01, None, ctypes.byref(pc)) == -1
    assert lib.fgk_precond_build(1, -1, 0.01, None, ctypes.byref(pc)) == -1
    assert lib.fgk_precond_build(1, 10, 0.0, None, ctypes.byref(pc)) == -1
    assert lib.fgk_precond_build(1, 5000, 0.01, None, ctypes.byref(pc)) == -1
    assert pc.value is None
    assert lib.fgk_precond_info(None, None, None) == -1
    assert lib.fgk_precond_apply(None, 1, 1, 1, None) == -1
    assert lib.fgk_precond_destroy(None) == 0
    # MINRES: NULL handle or outputs, nrhs outside [1, 64], sigma2 < 0, tol <= 0, maxit < 1
    for args in [(None, 1, 1, 0.01, 1e-8, 10, 1), (1, None, 1, 0.01, 1e-8, 10, 1), (1, 1, 1, 0.01, 1e-8, 10, None),
                 (1, 1, 0, 0.01, 1e-8, 10, 1), (1, 1, 65, 0.01, 1e-8, 10, 1), (1, 1, 1, -1.0, 1e-8, 10, 1),
                 (1, 1, 1, 0.01, 0.0, 10, 1), (1, 1, 1, 0.01, 1e-8, 0, 1)]:
        assert lib.fgk_minres_solve(*args, None, None) == -1, args
    # nu = 9/2 is built for d <= 2 only
    assert lib.fgk_build(1, 10, 3, 9, ell, 1.0, 1, None, ctypes.byref(out)) == -1
    assert b"9/2" in lib.fgk_last_error()
    assert lib.fgk_bytes_estimate(1000, 3, 9, 1, 1) == 0 and lib.fgk_bytes_estimate(1000, 3, 7, 1, 1) > 0


def test_likelihood_entries_reject_invalid_arguments_without_gpu(lib):
    """The gradient product, the probes, the log-determinant and the
    likelihood gradient validate their arguments before any CUDA call."""
    from paper_2508_01864_gb300 import fgk

    # NULL handle / arrays, nrhs < 1, a bad precision
    assert lib.fgk_matvec_dlogell(None, 1, 1, 1, 0, 0, None) == -1
    assert b"dlogell" in lib.fgk_last_error()
    assert lib.fgk_matvec_dlogell(1, 1, 0, 1, 0, 0, None) == -1
    assert lib.fgk_matvec_dlogell(1, 1, 1, 1, 0, 7, None) == -1
    assert lib.fgk_precond_sample(None, 1, 1, 1, 1, None) == -1
    assert b"precond_sample" in lib.fgk_last_error()
    rep = fgk.fgk_slq_report()
    for args in [(None, None, 0.1, 1, 4, 10, 1e-8), (1, None, 0.1, None, 4, 10, 1e-8), (1, None, 0.1, 1, 0, 10, 1e-8),
                 (1, None, 0.1, 1, 65, 10, 1e-8), (1, None, 0.1, 1, 4, 0, 1e-8), (1, None, -1.0, 1, 4, 10, 1e-8),
                 (1, None, 0.1, 1, 4, 10, 0.0)]:
        assert lib.fgk_slq_logdet(*args, None, None, None, ctypes.byref(rep), None) == -1, args
    assert b"slq_logdet" in lib.fgk_last_error()
    g = (ctypes.c_double * 8)()
    grep = fgk.fgk_grad_report()
    for args in [(None, None, 0.1, 1, 1, 4, 1e-8, 10, 2), (1, None, 0.1, None, 1, 4, 1e-8, 10, 2),
                 (1, None, 0.1, 1, None, 4, 1e-8, 10, 2), (1, None, 0.0, 1, 1, 4, 1e-8, 10, 2),
                 (1, None, 0.1, 1, 1, 64, 1e-8, 10, 2), (1, None, 0.1, 1, 1, 4, 1e-8, 0, 2),
                 (1, None, 0.1, 1, 1, 4, 1e-8, 10, 1)]:
        assert lib.fgk_loglik_grad(*args, g, ctypes.byref(grep), None) == -1, args
    assert b"loglik_grad" in lib.fgk_last_error()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2508_01864_gb300 import fgk

    with pytest.raises(FileNotFoundError):
        fgk.load.__wrapped__ if hasattr(fgk.load, "__wrapped__") else None
        saved = fgk._lib
        fgk._lib = None
        try:
            fgk.load(str(tmp_path / "missing.so"))
        finally:
            fgk._lib = saved
