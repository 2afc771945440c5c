"""Oracle for the exact fast Matérn kernel MVM and the GP solve built on it.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product package never imports it, and it never imports the product package.
Everything here is plain FP64 on the CPU:

* ``mvm_brute``  O1, the definition of K V (C, OpenMP, compensated sums);
* ``kmat``       the dense matrix K for small N; ``kcols`` selected columns;
  ``kcross``      the cross-covariance between evaluation points and the data
  (the vector k_z of the posterior mean, eq. gp_mean);
* ``mvm_dlogell_brute``  the lengthscale-gradient product (dK/d log ell) V
  from the definition, with ``kernel_dlog`` the closed-form derivatives
  (App. C.1 gradient formulas);
* ``mvm_dc``     O2, the paper's ECDF decomposition evaluated literally by a
  re-sorting divide and conquer (C);
* ``structure``  O3, canonical sort permutations and the dominance-level
  arrays (numpy);
* ``solve``      O4, conjugate gradients (Algorithm 2, with the identity or
  the pivoted-Cholesky preconditioner of App. A.3: the rank-k pivoted
  Cholesky factor, the Woodbury apply and the Sylvester log-determinant),
  dense solves and the GLS fixed-effects step (numpy).
"""

from .core import (  # noqa: F401
    L1,
    PRODUCT,
    build,
    kcols,
    kcross,
    kernel,
    kernel_dlog,
    kmat,
    max_threads,
    mvm_brute,
    mvm_dc,
    mvm_dc_cross,
    mvm_dc_dlogell_l1,
    mvm_dc_dlogell_product,
    mvm_dc_product32_printed,
    mvm_dlogell_brute,
    phi,
)
