"""fgk_matvec_q_noalloc, the product for callers that may not allocate device
memory during the call: a serving loop whose budget is handed out, an engine
with a fixed memory plan, a path that cannot afford an allocator call or an
out-of-memory error in the middle of its work.  It must give the same product
as fgk_matvec_q, call after call, while its scratch lives in the library's
fixed device array, and it must not allocate: no call reaches the library's
allocator and the device's free memory does not move.  Collected last on
purpose, so that a run stopping at the first failure has run every other
test before it."""

import ctypes

import numpy as np
import pytest
import torch

import workloads
from gpu_util import colwise_relerr, to_dev

pytestmark = pytest.mark.gpu

_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class CountingAllocator:
    """The library's allocator hook, routed to torch's caching allocator and
    counting every call (installed for the test, removed after it)."""

    def __init__(self, lib):
        self.lib, self.allocs, self.frees = lib, 0, 0

        def _alloc(nbytes, stream, ctx):
            self.allocs += 1
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      ctypes.c_void_p(stream).value or 0)

        def _free(ptr, stream, ctx):
            self.frees += 1
            torch.cuda.caching_allocator_delete(ptr)

        self._a, self._f = _ALLOC_T(_alloc), _FREE_T(_free)

    def __enter__(self):
        assert self.lib.fgk_set_allocator(ctypes.cast(self._a, ctypes.c_void_p),
                                          ctypes.cast(self._f, ctypes.c_void_p), None) == 0
        return self

    def __exit__(self, *exc):
        self.lib.fgk_set_allocator(None, None, None)


def raw_noalloc(fgk, h, Vq, Yq, precision):
    """Straight through the C ABI."""
    lib = fgk.load()
    prec = fgk.FGK_F64 if precision == "f64" else fgk.FGK_F32
    return lib.fgk_matvec_q_noalloc(ctypes.c_void_p(h.ptr), Vq.data_ptr(), Vq.shape[1], Yq.data_ptr(), prec,
                                    torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("d,nu,N,nrhs", [(2, 1.5, 60000, 2), (1, 0.5, 5000, 3), (3, 2.5, 20000, 1)])
def test_noalloc_matches_matvec_q_twice(fgk_mod, d, nu, N, nrhs):
    fgk = fgk_mod
    lib = fgk.load()
    p = workloads.small(4242 + d, N, d, nu=nu, ell=[0.1, 0.3, 0.2][:d], nrhs=nrhs)
    with CountingAllocator(lib) as counter:
        with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
            for prec, dt, tol in (("f32", torch.float32, 1e-5), ("f64", torch.float64, 1e-12)):
                Vq = to_dev(p.V, dt)
                ref = fgk.fgk_matvec_q(h, Vq, prec).cpu().numpy().astype(np.float64)
                outs = [torch.full_like(Vq, float("nan")) for _ in range(2)]
                torch.cuda.synchronize()
                before = (counter.allocs, counter.frees)
                free0 = torch.cuda.mem_get_info()[0]
                for Yq in outs:  # two calls in a row share the scratch array
                    assert raw_noalloc(fgk, h, Vq, Yq, prec) == 0, fgk.fgk_last_error()
                torch.cuda.synchronize()
                assert (counter.allocs, counter.frees) == before, "the library allocated during the calls"
                assert torch.cuda.mem_get_info()[0] == free0, "device memory moved during the calls"
                for Yq in outs:
                    got = Yq.cpu().numpy().astype(np.float64)
                    assert np.isfinite(got).all()
                    assert (colwise_relerr(got, ref) <= tol).all()


def test_noalloc_rejects_products_beyond_its_scratch(fgk_mod):
    fgk = fgk_mod
    p = workloads.c2(N=200000)
    with fgk.fgk_build(to_dev(p.X), p.nu, p.ell, kind="product") as h:
        # 512 FP64 columns: the 18 level rows alone need 14.7 GB, far beyond
        # the 64 MiB array
        nrhs = 512
        Vq = torch.zeros(p.N, nrhs, dtype=torch.float64, device="cuda")
        Yq = torch.full_like(Vq, 7.0)
        assert raw_noalloc(fgk, h, Vq, Yq, "f64") == -1
        assert "scratch" in fgk.fgk_last_error()
        torch.cuda.synchronize()
        assert bool((Yq == 7.0).all()), "a refused call must launch nothing"
