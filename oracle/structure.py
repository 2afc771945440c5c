"""O3: canonical sort permutations and dominance-level arrays (numpy).

TEST INFRASTRUCTURE ONLY.  This builds, independently of the CUDA path, the
exact arrays the device build must produce, so that the two can be compared
bit for bit.

The structure stores the sorted subsets of the divide and conquer once, before
any product is taken (Sec. 2.2.3: the sorted subsets for each coordinate are
kept in a data structure and every later sort is replaced by a look-up).  Its
canonical form, fixed here because the paper gives none:

* scaled coordinates  x'_k = x_k * (sqrt(2 nu) / ell_k)  in FP64, -0 -> +0
  (eq. scaled_kernel with one lengthscale per dimension);
* perm_k = stable ascending argsort of x'_k (ties by original index),
  rank_k = its inverse; q = rank_1 is the point's index in x'_1 order;
* L = ceil(log2 N); a "level" lists all N points once, grouped into aligned
  segments of a power-of-two size S (segment j holds positions
  [j S, min((j+1) S, N))), each segment ordered by the last coordinate
  (the sweep dimension).
* d = 1: one level, S = 2^L, q = 0..N-1.
* d = 2: level l = 0..L-1, S = 2^(L-l), segment id q >> (L-l), role
  r1 = bit (L-1-l) of q (0: low half of the segment in x'_1).
* d = 3: outer level l1 = 0..L-1 (S1 = 2^(L-l1), outer segment o = q >> (L-l1),
  role r1 = bit (L-1-l1) of q); inside each outer segment the points are
  ranked by x'_2 (local rank lr2), and inner level l2 = 0..L-l1-1 has
  S = S1 >> l2, inner segment h = lr2 >> (L-l1-l2), role r2 = bit
  (L-l1-1-l2) of lr2.  Level index = sum_{l'<l1} (L-l') + l2.
* per entry: dl = x'_d(this) - x'_d(previous entry of the same segment)
  (0 at a segment start), and for each split dimension an offset
  |x' - split|, split being x' of the last point of the segment's low half
  (clamped to the segment's last point).  FP32 copies are the FP64 values
  rounded to nearest.

A pair of distinct points is handled at exactly one level: the one where they
share a segment but not a role, in every split dimension.
"""

from __future__ import annotations

import numpy as np


def n_levels(N: int, d: int) -> int:
    L = ceil_log2(N)
    if d == 1:
        return 1
    if d == 2:
        return L
    return L * (L + 1) // 2


def ceil_log2(N: int) -> int:
    return 0 if N <= 1 else int(N - 1).bit_length()


def scaled(X, nu, ell) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    d = X.shape[1]
    two_nu = int(round(2 * float(nu)))
    ell = np.broadcast_to(np.asarray(ell, dtype=np.float64), (d,))
    a = np.sqrt(float(two_nu)) / ell
    Xs = X * a[None, :]
    return Xs + 0.0  # -0 -> +0


def permutations(X, nu, ell):
    Xs = scaled(X, nu, ell)
    perms, ranks = [], []
    for k in range(Xs.shape[1]):
        p = np.argsort(Xs[:, k], kind="stable").astype(np.int64)
        r = np.empty_like(p)
        r[p] = np.arange(p.size)
        perms.append(p)
        ranks.append(r)
    return perms, ranks


def _finish(q, S, x_sweep_q, roles, offs64):
    N = q.size
    pos = np.arange(N)
    xs = x_sweep_q[q]
    dl = np.zeros(N)
    inner = (pos % S) != 0
    dl[inner] = xs[inner] - xs[np.nonzero(inner)[0] - 1]
    lev = {
        "S": int(S),
        "q": q.astype(np.uint32),
        "dl64": dl,
        "dl32": dl.astype(np.float32),
    }
    for name, r in roles.items():
        lev[name] = r.astype(np.uint8)
    if offs64:
        off = np.stack(offs64, axis=1)
        lev["off64"] = off
        lev["off32"] = off.astype(np.float32)
    return lev


def levels(X, nu, ell):
    """All levels of the canonical structure, as a list of dicts."""
    Xs = scaled(X, nu, ell)
    N, d = Xs.shape
    perms, ranks = permutations(X, nu, ell)
    L = ceil_log2(N)
    p1 = perms[0]
    x1q = Xs[p1, 0]  # x'_1 by q
    out = []
    if d == 1:
        q = np.arange(N)
        out.append(_finish(q, 1 << L, x1q, {}, []))
        return out
    qall = np.arange(N)
    r2q = ranks[1][p1]
    x2q = Xs[p1, 1]
    if d == 2:
        for lev in range(L):
            S = 1 << (L - lev)
            g = qall >> (L - lev)
            q = qall[np.lexsort((r2q, g))]
            r1 = (q >> (L - 1 - lev)) & 1
            gq = q >> (L - lev)
            split = np.minimum(gq * S + S // 2 - 1, N - 1)
            off1 = np.abs(x1q[q] - x1q[split])
            out.append(_finish(q, S, x2q, {"r1": r1}, [off1]))
        return out
    r3q = ranks[2][p1]
    x3q = Xs[p1, 2]
    for l1 in range(L):
        S1 = 1 << (L - l1)
        o_all = qall >> (L - l1)
        pi = qall[np.lexsort((r2q, o_all))]  # outer order: (o, rank2)
        lr2 = np.empty(N, dtype=np.int64)
        lr2[pi] = np.arange(N) - ((pi >> (L - l1)) << (L - l1))
        for l2 in range(L - l1):
            S = S1 >> l2
            h_all = lr2 >> (L - l1 - l2)
            q = qall[np.lexsort((r3q, h_all, o_all))]
            o = q >> (L - l1)
            h = lr2[q] >> (L - l1 - l2)
            r1 = (q >> (L - 1 - l1)) & 1
            r2 = (lr2[q] >> (L - l1 - 1 - l2)) & 1
            split1 = np.minimum(o * S1 + S1 // 2 - 1, N - 1)
            cnt1 = np.minimum(S1, N - o * S1)
            split2_pos = o * S1 + np.minimum(h * S + S // 2 - 1, cnt1 - 1)
            off1 = np.abs(x1q[q] - x1q[split1])
            off2 = np.abs(x2q[q] - x2q[pi[split2_pos]])
            out.append(_finish(q, S, x3q, {"r1": r1, "r2": r2}, [off1, off2]))
    return out
