"""One d = 1 problem over several devices: the points split into shards,
contiguous ranges of the sorted order, one per rank.

Each rank's plan covers the pairs inside its shard.  The pairs between
shards act through P moments per shard and direction (Sec. 2.1, fast sum
updating: the running sums of a sweep, taken relative to an anchor point so
that every factor lies in [0, 1]): fgk_shard_moments gives, per column, the
moments of the shard's sources seen from its last point (forward) and from
its first point (backward).  One all-gather exchanges them (2 + 2 nrhs P
numbers per rank); every rank then composes, in shard order, the moments of
all earlier shards at its own first point and of all later shards at its own
last point by the binomial step over each gap,
    M'_q = e^{-g} sum_{t<=q} C(q,t) g^{q-t} M_t,
and fgk_shard_fixup adds their contributions to its rows of Y.  The product
therefore needs one exchange of a few hundred bytes per call, whatever N.
"""

from __future__ import annotations

from math import comb

import numpy as np


def step_moments(M, g: float):
    """Moments M[..., q] relative to an anchor moved a distance g >= 0 further
    from the sources: M'_q = e^{-g} sum_{t<=q} C(q,t) g^{q-t} M_t."""
    if not g >= 0.0:
        raise ValueError(f"shards must be in sorted order (gap {g})")
    M = np.asarray(M, dtype=np.float64)
    P = M.shape[-1]
    out = np.zeros_like(M)
    e = np.exp(-g)
    for q in range(P):
        acc = np.zeros(M.shape[:-1])
        for t in range(q + 1):
            acc = acc + comb(q, t) * g ** (q - t) * M[..., t]
        out[..., q] = e * acc
    return out


def compose_carries(shards, rank: int):
    """shards: per rank, in shard order, (x_first, x_last, M[nrhs, 2, P]) as
    fgk_shard_moments returns them.  Returns carry[nrhs, 2, P] for ``rank``:
    dir 0 the points of every earlier shard anchored at this shard's first
    point, dir 1 those of every later shard anchored at its last point (the
    shards added in order, so every rank composes the same way)."""
    xf_r, xl_r, M_r = shards[rank]
    carry = np.zeros_like(np.asarray(M_r, dtype=np.float64))
    for s, (xf, xl, M) in enumerate(shards):
        M = np.asarray(M, dtype=np.float64)
        if s < rank:
            carry[:, 0] += step_moments(M[:, 0], xf_r - xl)
        elif s > rank:
            carry[:, 1] += step_moments(M[:, 1], xf - xl_r)
    return carry


class GpuShard:
    """The device side of one shard: its plan's product and the two calls
    around the exchange."""

    def __init__(self, h):
        self.h = h

    def local_product(self, V):
        from . import fgk

        return fgk.fgk_matvec(self.h, V, "f64")

    def moments(self, V):
        from . import fgk

        return fgk.fgk_shard_moments(self.h, V)

    def fixup(self, carry, Y):
        from . import fgk

        return fgk.fgk_shard_fixup(self.h, carry, Y)


def exchange(local, world_size: int, device="cpu"):
    """All-gather of (x_first, x_last, M) over the default process group
    (gloo on the CPU, NCCL between GPUs); a single rank returns [local]."""
    xf, xl, M = local
    M = np.asarray(M, dtype=np.float64)
    if world_size == 1:
        return [(xf, xl, M)]
    import torch
    import torch.distributed as dist

    flat = torch.as_tensor(np.concatenate([[xf, xl], M.reshape(-1)]), dtype=torch.float64, device=device)
    parts = [torch.empty_like(flat) for _ in range(world_size)]
    dist.all_gather(parts, flat)
    out = []
    for t in parts:
        a = t.cpu().numpy()
        out.append((float(a[0]), float(a[1]), a[2:].reshape(M.shape)))
    return out


def sharded_matvec(shard, V, rank: int, world_size: int, device="cpu"):
    """Y = K V on this rank's rows (its shard, original order within it):
    local product, one all-gather of the moments, composed carries, fix-up."""
    Y = shard.local_product(V)
    shards = exchange(shard.moments(V), world_size, device)
    for s in range(1, len(shards)):
        if shards[s][0] < shards[s - 1][1]:
            raise ValueError(f"shard {s} starts before shard {s - 1} ends: shards must be contiguous in sorted order")
    shard.fixup(compose_carries(shards, rank), Y)
    return Y
