"""ctypes wrapper around ``fgk_oracle.c`` (O1 brute force, O2 literal divide
and conquer).  Test infrastructure only; see the package docstring."""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

L1 = 0
PRODUCT = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fgk_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libfgk_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE semantics, OpenMP) if it is missing
    or older than its source.  Returns the path of the shared library."""
    os.makedirs(_LIBDIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        Lp = ctypes.POINTER(ctypes.c_long)
        lib.orc_kernel.restype = ctypes.c_double
        lib.orc_kernel.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_mvm_brute.restype = ctypes.c_int
        lib.orc_mvm_brute.argtypes = [D, ctypes.c_long, ctypes.c_int, ctypes.c_int, D, ctypes.c_double,
                                      ctypes.c_int, D, ctypes.c_int, Lp, ctypes.c_long, D, ctypes.c_int]
        lib.orc_kmat.restype = ctypes.c_int
        lib.orc_kmat.argtypes = [D, ctypes.c_long, ctypes.c_int, ctypes.c_int, D, ctypes.c_double,
                                 ctypes.c_int, D]
        lib.orc_kcols.restype = ctypes.c_int
        lib.orc_kcols.argtypes = [D, ctypes.c_long, ctypes.c_int, ctypes.c_int, D, ctypes.c_double,
                                  ctypes.c_int, Lp, ctypes.c_long, D]
        lib.orc_kcross.restype = ctypes.c_int
        lib.orc_kcross.argtypes = [D, ctypes.c_long, D, ctypes.c_long, ctypes.c_int, ctypes.c_int, D,
                                   ctypes.c_double, ctypes.c_int, D]
        lib.orc_kernel_dlog.restype = ctypes.c_double
        lib.orc_kernel_dlog.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        lib.orc_mvm_dlogell_brute.restype = ctypes.c_int
        lib.orc_mvm_dlogell_brute.argtypes = [D, ctypes.c_long, ctypes.c_int, ctypes.c_int, D, ctypes.c_double,
                                              ctypes.c_int, ctypes.c_int, D, ctypes.c_int, Lp, ctypes.c_long, D,
                                              ctypes.c_int]
        lib.orc_mvm_dc_dlogell_l1.restype = ctypes.c_int
        lib.orc_mvm_dc_dlogell_l1.argtypes = [D, ctypes.c_long, ctypes.c_int, ctypes.c_int, D, ctypes.c_double, D,
                                              ctypes.c_int, D]
        lib.orc_mvm_dc_dlogell_product.restype = ctypes.c_int
        lib.orc_mvm_dc_dlogell_product.argtypes = [D, ctypes.c_long, ctypes.c_int, ctypes.c_int, D, ctypes.c_double,
                                                   ctypes.c_int, D, ctypes.c_int, D]
        lib.orc_mvm_dc_cross.restype = ctypes.c_int
        lib.orc_mvm_dc_cross.argtypes = [D, ctypes.c_long, D, ctypes.c_long, ctypes.c_int, ctypes.c_int, D,
                                         ctypes.c_double, ctypes.c_int, D, ctypes.c_int, D]
        lib.orc_mvm_dc.restype = ctypes.c_int
        lib.orc_mvm_dc.argtypes = [D, ctypes.c_long, ctypes.c_int, ctypes.c_int, D, ctypes.c_double,
                                   ctypes.c_int, D, ctypes.c_int, D]
        lib.orc_mvm_dc_product32_printed.restype = ctypes.c_int
        lib.orc_mvm_dc_product32_printed.argtypes = [D, ctypes.c_long, ctypes.c_int, D, ctypes.c_double, D, D]
        lib.orc_phi.restype = ctypes.c_int
        lib.orc_phi.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, D]
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_max_threads.argtypes = []
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _prep(X, ell):
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    d = X.shape[1]
    ell = np.ascontiguousarray(np.broadcast_to(np.asarray(ell, dtype=np.float64), (d,)))
    return X, d, ell


def _two_nu(nu) -> int:
    """2 nu for nu = 1/2 .. 9/2 (the closed forms of App. C.1); the
    decomposition entries (O2) reject nu > 5/2 themselves."""
    t = int(round(2 * float(nu)))
    if t not in (1, 3, 5, 7, 9) or abs(2 * float(nu) - t) > 1e-12:
        raise ValueError(f"nu must be 1/2, 3/2, 5/2, 7/2 or 9/2, got {nu}")
    return t


def kernel(nu, u) -> np.ndarray:
    """Closed-form unit-lengthscale Matérn kernel k_nu(|u|) (App. C.1)."""
    lib = _load()
    t = _two_nu(nu)
    u = np.asarray(u, dtype=np.float64)
    return np.vectorize(lambda x: lib.orc_kernel(t, float(x)), otypes=[np.float64])(u)


def phi(nu, which: int, p: int, x) -> np.ndarray:
    """One-dimensional factor phi_{which, p+1} of Assumption 1 (0-based p)."""
    lib = _load()
    t = _two_nu(nu)
    out = ctypes.c_double()

    def one(v):
        if lib.orc_phi(t, which, p, float(v), ctypes.byref(out)) != 0:
            raise ValueError("bad phi index")
        return out.value

    return np.vectorize(one, otypes=[np.float64])(np.asarray(x, dtype=np.float64))


def mvm_brute(X, V, nu, ell, s2: float = 1.0, kind: int = L1, rows=None, nthreads: int = 0) -> np.ndarray:
    """O1: Y = s2 * K V from the definition.  ``rows`` selects output rows."""
    lib = _load()
    X, d, ell = _prep(X, ell)
    N = X.shape[0]
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V = np.ascontiguousarray(V.reshape(N, -1))
    nrhs = V.shape[1]
    if rows is None:
        Y = np.empty((N, nrhs))
        rc = lib.orc_mvm_brute(_dp(X), N, d, _two_nu(nu), _dp(ell), float(s2), int(kind), _dp(V), nrhs,
                               None, 0, _dp(Y), int(nthreads))
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        Y = np.empty((rows.size, nrhs))
        rc = lib.orc_mvm_brute(_dp(X), N, d, _two_nu(nu), _dp(ell), float(s2), int(kind), _dp(V), nrhs,
                               rows.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), rows.size, _dp(Y),
                               int(nthreads))
    if rc != 0:
        raise ValueError("orc_mvm_brute rejected its arguments")
    return Y[:, 0] if vec else Y


def kernel_dlog(nu, u, which: int = 0) -> np.ndarray:
    """which=0: -u k'(u) (= l d/dl of k(|x|/l)); which=1: -k'(u) (App. C.1)."""
    lib = _load()
    t = _two_nu(nu)
    u = np.asarray(u, dtype=np.float64)
    return np.vectorize(lambda x: lib.orc_kernel_dlog(t, int(which), float(x)), otypes=[np.float64])(u)


def mvm_dlogell_brute(X, V, nu, ell, dim: int = -1, s2: float = 1.0, kind: int = L1, rows=None,
                      nthreads: int = 0) -> np.ndarray:
    """Y = s2 * (dK/d log ell_dim) V from the definition (dim = -1: all
    lengthscales scaled together).  ``rows`` selects output rows."""
    lib = _load()
    X, d, ell = _prep(X, ell)
    N = X.shape[0]
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V = np.ascontiguousarray(V.reshape(N, -1))
    nrhs = V.shape[1]
    rp, nr = None, 0
    if rows is not None:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        rp, nr = rows.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), rows.size
    Y = np.empty((N if rows is None else nr, nrhs))
    rc = lib.orc_mvm_dlogell_brute(_dp(X), N, d, _two_nu(nu), _dp(ell), float(s2), int(kind), int(dim), _dp(V),
                                   nrhs, rp, nr, _dp(Y), int(nthreads))
    if rc != 0:
        raise ValueError("orc_mvm_dlogell_brute rejected its arguments")
    return Y[:, 0] if vec else Y


def kmat(X, nu, ell, s2: float = 1.0, kind: int = L1) -> np.ndarray:
    """Dense K (small N)."""
    lib = _load()
    X, d, ell = _prep(X, ell)
    N = X.shape[0]
    K = np.empty((N, N))
    if lib.orc_kmat(_dp(X), N, d, _two_nu(nu), _dp(ell), float(s2), int(kind), _dp(K)) != 0:
        raise ValueError("orc_kmat rejected its arguments")
    return K


def kcols(X, idx, nu, ell, s2: float = 1.0, kind: int = L1) -> np.ndarray:
    """Columns K[:, idx] (N x len(idx)) from the definition."""
    lib = _load()
    X, d, ell = _prep(X, ell)
    N = X.shape[0]
    idx = np.ascontiguousarray(np.atleast_1d(idx), dtype=np.int64)
    C = np.empty((N, idx.size))
    if lib.orc_kcols(_dp(X), N, d, _two_nu(nu), _dp(ell), float(s2), int(kind),
                     idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), idx.size, _dp(C)) != 0:
        raise ValueError("orc_kcols rejected its arguments")
    return C


def kcross(X, Z, nu, ell, s2: float = 1.0, kind: int = L1) -> np.ndarray:
    """Dense cross-covariance [K(z_j, x_i)] (M x N), the rows k_z^T of eq. gp_mean."""
    lib = _load()
    X, d, ell = _prep(X, ell)
    Z = np.ascontiguousarray(np.asarray(Z, dtype=np.float64).reshape(-1, d))
    N, M = X.shape[0], Z.shape[0]
    C = np.empty((M, N))
    if lib.orc_kcross(_dp(X), N, _dp(Z), M, d, _two_nu(nu), _dp(ell), float(s2), int(kind), _dp(C)) != 0:
        raise ValueError("orc_kcross rejected its arguments")
    return C


def mvm_dc(X, V, nu, ell, s2: float = 1.0, kind: int = L1) -> np.ndarray:
    """O2: Y = s2 * K V by the paper's ECDF decomposition (literal, slow)."""
    lib = _load()
    X, d, ell = _prep(X, ell)
    N = X.shape[0]
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V = np.ascontiguousarray(V.reshape(N, -1))
    Y = np.empty_like(V)
    if lib.orc_mvm_dc(_dp(X), N, d, _two_nu(nu), _dp(ell), float(s2), int(kind), _dp(V), V.shape[1], _dp(Y)) != 0:
        raise ValueError("orc_mvm_dc rejected its arguments")
    return Y[:, 0] if vec else Y


def mvm_dc_cross(X, Z, V, nu, ell, s2: float = 1.0, kind: int = L1) -> np.ndarray:
    """Kernel sums at the new points Z over the data X (the k_z^T V of
    eq. gp_mean) by the paper's ECDF decomposition (literal, slow)."""
    lib = _load()
    X, d, ell = _prep(X, ell)
    N = X.shape[0]
    Z = np.ascontiguousarray(np.asarray(Z, dtype=np.float64).reshape(-1, d))
    M = Z.shape[0]
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V = np.ascontiguousarray(V.reshape(N, -1))
    Y = np.empty((M, V.shape[1]))
    if lib.orc_mvm_dc_cross(_dp(X), N, _dp(Z), M, d, _two_nu(nu), _dp(ell), float(s2), int(kind), _dp(V),
                            V.shape[1], _dp(Y)) != 0:
        raise ValueError("orc_mvm_dc_cross rejected its arguments")
    return Y[:, 0] if vec else Y


def mvm_dc_dlogell_l1(X, V, nu, ell, s2: float = 1.0) -> np.ndarray:
    """The L1 kernel's log-lengthscale gradient product by the paper's printed
    ECDF decompositions (every lengthscale scaled together)."""
    lib = _load()
    X, d, ell = _prep(X, ell)
    N = X.shape[0]
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V = np.ascontiguousarray(V.reshape(N, -1))
    Y = np.empty_like(V)
    if lib.orc_mvm_dc_dlogell_l1(_dp(X), N, d, _two_nu(nu), _dp(ell), float(s2), _dp(V), V.shape[1], _dp(Y)) != 0:
        raise ValueError("orc_mvm_dc_dlogell_l1 rejected its arguments")
    return Y[:, 0] if vec else Y


def mvm_dc_dlogell_product(X, V, nu, ell, dim: int = -1, s2: float = 1.0) -> np.ndarray:
    """The product kernel's log-lengthscale gradient product through
    Proposition 2's weighted ECDFs with one factor differentiated."""
    lib = _load()
    X, d, ell = _prep(X, ell)
    N = X.shape[0]
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V = np.ascontiguousarray(V.reshape(N, -1))
    Y = np.empty_like(V)
    if lib.orc_mvm_dc_dlogell_product(_dp(X), N, d, _two_nu(nu), _dp(ell), float(s2), int(dim), _dp(V),
                                      V.shape[1], _dp(Y)) != 0:
        raise ValueError("orc_mvm_dc_dlogell_product rejected its arguments")
    return Y[:, 0] if vec else Y


def mvm_dc_product32_printed(X, v, ell, s2: float = 1.0) -> np.ndarray:
    """The printed product Matérn-3/2 example, under the binomial reading."""
    lib = _load()
    X, d, ell = _prep(X, ell)
    N = X.shape[0]
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(N)
    Y = np.empty(N)
    if lib.orc_mvm_dc_product32_printed(_dp(X), N, d, _dp(ell), float(s2), _dp(v), _dp(Y)) != 0:
        raise ValueError("bad arguments")
    return Y


def max_threads() -> int:
    return int(_load().orc_max_threads())
