"""The library's device scratch routed through torch's caching allocator
(fgk.use_torch_allocator, which installs callbacks with fgk_set_allocator):
the same product and the same preconditioned solve as with the library's own
allocator, bit for bit, and the allocations visible in torch's counters."""

import numpy as np
import pytest
import torch

import workloads
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def test_product_and_solve_through_torch_allocator(fgk_mod):
    fgk = fgk_mod
    p = workloads.small(515, 4000, 2, nu=1.5, ell=[0.2, 0.3], nrhs=2)
    X, V = to_dev(p.X), to_dev(p.V)

    def run():
        with fgk.fgk_build(X, p.nu, p.ell, kind="product") as h:
            y = fgk.fgk_matvec(h, V, "f64").cpu().numpy()
            with fgk.fgk_precond_build(h, 40, 0.05) as pc:
                a, _, info, rc = fgk.fgk_cg_solve(h, V[:, :1].contiguous(), 0.05, tol=1e-10, mode="mixed",
                                                  precond=pc)
        torch.cuda.synchronize()
        return y, a.cpu().numpy(), rc

    y0, a0, rc0 = run()
    before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    fgk.use_torch_allocator(True)
    try:
        y1, a1, rc1 = run()
        after = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    finally:
        fgk.use_torch_allocator(False)
    assert after > before  # the scratch came from torch's allocator
    assert rc0 == rc1 == 0
    assert np.array_equal(y0, y1)
    assert np.array_equal(a0, a1)
