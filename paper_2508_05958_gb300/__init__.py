"""GB300-native (sm_103a) HTLR library: Construct and HMultVec of hierarchical Tucker
low-rank matrices (Li & Liu, arXiv 2508.05958) behind a C ABI (include/htlr.h)."""
from .htlr import (  # noqa: F401
    HTLRError, Operator, htlr_construct, htlr_free, htlr_info, htlr_last_error,
    htlr_last_launch_count, htlr_matvec, htlr_matvec_host, htlr_matvec_timed, htlr_set_stream, htlr_sync, load,
    K_LOG, K_INV_R, K_EXP_R, K_GAUSS, K_POLY, K_CONST, STORE_AUTO, STORE_STORED, STORE_SHARED,
)
