"""GB300-native exact fast Matérn-kernel MVM and GP solve (arXiv 2508.01864).

The compute path is libfgk (hand-written CUDA for sm_103a behind a C ABI,
``include/fgk.h``); ``fgk`` is its thin Python binding.
"""

from .fgk import (  # noqa: F401
    Batch,
    fgk_batch_cg_solve,
    fgk_batch_create,
    fgk_batch_destroy,
    fgk_batch_matvec_q,
    FGK_F32,
    FGK_F64,
    FGK_L1,
    FGK_MIXED,
    FGK_PRODUCT,
    FgkError,
    Handle,
    fgk_build,
    fgk_bytes_estimate,
    fgk_cg_solve,
    fgk_destroy,
    fgk_get_info,
    fgk_get_level,
    fgk_get_permutation,
    fgk_last_error,
    fgk_kernel_launches,
    fgk_matvec,
    fgk_matvec_q,
    fgk_matvec_q_noalloc,
    fgk_scan_timing,
    load,
    use_torch_allocator,
)
