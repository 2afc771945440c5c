"""Writes tests/golden/oracle_values.txt: reference values computed by the
oracle alone (the paper prints no numerical example of the product, so no
value here is the paper's).  They freeze the oracle's output on small seeded
inputs so that a change to its arithmetic shows up as a failing test.

    python tests/golden/make_golden.py
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

CASES = [  # seed, N, d, nu, ell, kind
    (11, 300, 1, 0.5, [0.2], oracle.L1),
    (12, 400, 2, 1.5, [0.1, 0.3], oracle.PRODUCT),
    (13, 250, 3, 2.5, [0.3, 0.2, 0.4], oracle.PRODUCT),
    (14, 350, 2, 2.5, [0.25, 0.15], oracle.L1),
    (15, 300, 2, 3.5, [0.2, 0.3], oracle.PRODUCT),
]
ROWS = [0, 7, 42, 123, 249]
DISTANCES = [0.0, 0.1, 0.5, 1.0, 2.5]


def lines():
    out = ["# kernel <2nu> <u> <k(u)>: closed forms of App. C.1 at u = |x| / ell",
           "# mvm <seed> <N> <d> <nu> <ell...> <kind> <row> <Y[row]>: O1, s2 = 1, V = the seeded N(0,1) column"]
    for nu in (0.5, 1.5, 2.5, 3.5, 4.5):
        for u in DISTANCES:
            out.append(f"kernel {int(2 * nu)} {u!r} {float(oracle.kernel(nu, u))!r}")
    for seed, N, d, nu, ell, kind in CASES:
        p = workloads.small(seed, N, d, nu=nu, ell=ell)
        y = oracle.mvm_brute(p.X, p.V[:, 0], nu, ell, kind=kind, rows=np.array(ROWS), nthreads=1)
        for r, v in zip(ROWS, y):
            out.append(f"mvm {seed} {N} {d} {nu!r} {' '.join(repr(e) for e in ell)} {kind} {r} {float(v)!r}")
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_values.txt"), "w") as f:
        f.write("\n".join(lines()) + "\n")
