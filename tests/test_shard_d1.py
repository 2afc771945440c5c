"""The sharded d = 1 product on the CPU: two gloo ranks, each holding a
contiguous range of the sorted points, exchange their moments by one
all-gather and compose the cross-shard terms; the product each rank returns
for its rows equals the brute-force oracle (O1) on those rows.  The device
calls of a shard (its plan's product, its moments, the fix-up) are played
by a stand-in written here from their stated definitions, so that the
exchange and the composition are what is tested.  No GPU."""

import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def matern_c(P):
    """c_p of k(r) = sum_p c_p r^p e^{-r} for nu = P - 1/2 (eqs. matern_1_2 ... matern_9_2)."""
    from math import factorial as f

    return [f(P - 1) * f(2 * P - 2 - q) * 2 ** q / (f(2 * P - 2) * f(q) * f(P - 1 - q)) for q in range(P)]


class CpuShard:
    """Stand-in for the device side: the shard's own product by the oracle,
    the moments and the fix-up straight from their definitions."""

    def __init__(self, x, nu, ell, s2=1.0):
        import oracle

        self.x, self.nu, self.ell, self.s2 = x, nu, ell, s2
        self.P = int(round(nu + 0.5))
        self.a = np.sqrt(2 * nu) / ell
        self.orc = oracle

    def local_product(self, V):
        return self.orc.mvm_brute(self.x[:, None], V, self.nu, [self.ell], s2=self.s2)

    def moments(self, V):
        xs = self.a * self.x
        xf, xl = xs.min(), xs.max()
        M = np.zeros((V.shape[1], 2, self.P))
        for dirn, dl in ((0, xl - xs), (1, xs - xf)):
            for q in range(self.P):
                M[:, dirn, q] = (V * (dl ** q * np.exp(-dl))[:, None]).sum(axis=0)
        return xf, xl, M

    def fixup(self, carry, Y):
        from math import comb

        xs = self.a * self.x
        c = matern_c(self.P)
        for dirn, D in ((0, xs - xs.min()), (1, xs.max() - xs)):
            for p in range(self.P):
                for q in range(p + 1):
                    Y += self.s2 * c[p] * comb(p, q) * (np.exp(-D) * D ** (p - q))[:, None] * carry[:, dirn, q][None, :]
        return Y


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, nu, out_q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import workloads
    from paper_2508_01864_gb300 import shard

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        p = workloads.small(909, 3001, 1, nu=nu, ell=0.05, nrhs=2, pattern="dups")
        order = np.argsort(p.X[:, 0], kind="stable")
        mine = np.array_split(order, ws)[rank]  # a contiguous range of the sorted order
        sh = CpuShard(p.X[mine, 0], nu, 0.05)
        Y = shard.sharded_matvec(sh, p.V[mine].copy(), rank, ws)
        out_q.put((rank, mine, Y))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("nu", [0.5, 2.5, 4.5])
def test_two_gloo_ranks_compose_the_full_product(orc, nu):
    import torch.multiprocessing as mp

    import workloads

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, nu, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=180) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = workloads.small(909, 3001, 1, nu=nu, ell=0.05, nrhs=2, pattern="dups")
    ref = orc.mvm_brute(p.X, p.V, nu, [0.05])
    for rank, mine, Y in res:
        err = np.linalg.norm(Y - ref[mine], axis=0) / np.linalg.norm(ref[mine], axis=0)
        assert (err <= 1e-12).all(), (rank, err)
    # the cross-shard terms matter: the local products alone are far off
    for rank, mine, _ in res:
        loc = orc.mvm_brute(p.X[mine], p.V[mine], nu, [0.05])
        assert np.linalg.norm(loc - ref[mine]) > 1e-6 * np.linalg.norm(ref[mine])


def test_three_shards_in_one_process_and_the_step_rule(orc):
    """world_size 1 per call, three shards composed by hand: the same
    composition as the exchange gives O1; and the binomial step equals the
    moments recomputed from their definition at the moved anchor."""
    sys.path.insert(0, ROOT)
    import workloads
    from paper_2508_01864_gb300 import shard

    p = workloads.small(5, 2000, 1, nu=1.5, ell=0.1, nrhs=1)
    order = np.argsort(p.X[:, 0], kind="stable")
    parts = np.array_split(order, 3)
    shs = [CpuShard(p.X[m, 0], 1.5, 0.1) for m in parts]
    mom = [s.moments(p.V[m]) for s, m in zip(shs, parts)]
    ref = orc.mvm_brute(p.X, p.V, 1.5, [0.1])
    for r, (s, m) in enumerate(zip(shs, parts)):
        Y = s.local_product(p.V[m])
        s.fixup(shard.compose_carries(mom, r), Y)
        assert np.linalg.norm(Y - ref[m]) <= 1e-12 * np.linalg.norm(ref[m])
    # step rule: moments of shard 0 seen from shard 1's first point
    xs0 = np.sqrt(3.0) / 0.1 * p.X[parts[0], 0]
    x1 = np.sqrt(3.0) / 0.1 * p.X[parts[1], 0].min()
    direct = np.array([(p.V[parts[0], 0] * (x1 - xs0) ** q * np.exp(-(x1 - xs0))).sum() for q in range(2)])
    stepped = shard.step_moments(mom[0][2][:, 0], x1 - mom[0][1])[0]
    assert np.allclose(stepped, direct, rtol=1e-12, atol=1e-300)
    with pytest.raises(ValueError):
        shard.step_moments(mom[0][2][:, 0], -1.0)
