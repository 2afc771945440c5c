"""The library's host-side Lanczos quadrature (fgk_lanczos_logquad: the
implicit symmetric QR eigen-decomposition of the tridiagonal matrix built
from CG coefficients, no GPU work) against the oracle's (numpy eigh)."""

import numpy as np
import pytest

from oracle import solve


def spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    return (Q * lam) @ Q.T


def test_library_host_quadrature_matches_the_oracle():
    from paper_2508_01864_gb300 import build, fgk

    build.build()
    rng = np.random.default_rng(21)
    for n, cond, m in [(80, 1e2, 1), (80, 1e2, 2), (120, 1e4, 40), (300, 1e6, 250), (60, 10.0, 60)]:
        A = spd(n, int(cond) % 97 + m, cond=cond)
        b = rng.standard_normal(n)
        _, al, be, ga = solve.cg_lanczos(lambda V: A @ V, b, 1e-30, m)
        al, be = al[0], be[0][: len(al[0]) - 1]
        got = fgk.fgk_lanczos_logquad(al, be)
        ref = solve.slq_quadrature(al, be, 1.0)
        assert got == pytest.approx(ref, rel=1e-11, abs=1e-12), (n, cond, m)
    with pytest.raises(RuntimeError):
        fgk.fgk_lanczos_logquad([1.0, -2.0], [0.5])
    with pytest.raises(RuntimeError):
        fgk.fgk_lanczos_logquad([], [])
