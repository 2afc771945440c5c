"""fgk_matvec_q_noalloc, the product for callers that may not allocate device
memory during the call (their memory is planned before they start).  It must
give the same product as fgk_matvec_q, call after call, while its scratch
lives in the library's fixed device array.  Collected last on purpose."""

import ctypes

import numpy as np
import pytest
import torch

import workloads
from gpu_util import colwise_relerr, to_dev

pytestmark = pytest.mark.gpu


def raw_noalloc(fgk, h, Vq, Yq, precision):
    """Straight through the C ABI."""
    lib = fgk.load()
    prec = fgk.FGK_F64 if precision == "f64" else fgk.FGK_F32
    return lib.fgk_matvec_q_noalloc(ctypes.c_void_p(h.ptr), Vq.data_ptr(), Vq.shape[1], Yq.data_ptr(), prec,
                                    torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("d,nu,N,nrhs", [(2, 1.5, 60000, 2), (1, 0.5, 5000, 3), (3, 2.5, 20000, 1)])
def test_noalloc_matches_matvec_q_twice(fgk_mod, d, nu, N, nrhs):
    fgk = fgk_mod
    p = workloads.small(4242 + d, N, d, nu=nu, ell=[0.1, 0.3, 0.2][:d], nrhs=nrhs)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        for prec, dt, tol in (("f32", torch.float32, 1e-5), ("f64", torch.float64, 1e-12)):
            Vq = to_dev(p.V, dt)
            ref = fgk.fgk_matvec_q(h, Vq, prec).cpu().numpy().astype(np.float64)
            for _ in range(2):  # two calls in a row share the scratch array
                Yq = torch.full_like(Vq, float("nan"))
                assert raw_noalloc(fgk, h, Vq, Yq, prec) == 0, fgk.fgk_last_error()
                got = Yq.cpu().numpy().astype(np.float64)
                assert np.isfinite(got).all()
                assert (colwise_relerr(got, ref) <= tol).all()


def test_noalloc_rejects_products_beyond_its_scratch(fgk_mod):
    fgk = fgk_mod
    p = workloads.c2(N=200000)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        # 512 FP64 columns: the tile aggregates and carries of the 7+ long
        # levels alone are far beyond 16 MiB
        nrhs = 512
        Vq = torch.zeros(p.N, nrhs, dtype=torch.float64, device="cuda")
        Yq = torch.empty_like(Vq)
        assert raw_noalloc(fgk, h, Vq, Yq, "f64") == -1
        assert "scratch" in fgk.fgk_last_error()
