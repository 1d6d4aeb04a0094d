"""GB300 (sm_103a) connected components: the adaptive Hook-Compress method of Sutton, Ben-Nun,
Barak, Pai and Pingali (arXiv:1612.01178) as a CUDA library with a C ABI (include/cc.h) and this
thin Python binding."""
from .cc import (CC_FLAG_SYMMETRIC, CC_FLAG_SYNC, CC_FLAG_VALIDATE, CC_MODE_AUTO, CC_MODE_CLUSTER, CC_MODE_FILTERED,
                 CC_MODE_MULTI_LAUNCH, CC_MODE_PERSISTENT, CCError, ConnectedComponents, cc_create, cc_destroy,
                 cc_labels_batched, cc_labels_coo, cc_labels_csr, cc_labels_csr64, cc_labels_csr_host,
                 cc_labels_csr_noalloc, cc_last_run_info, cc_set_launch_status, cc_set_options, cc_set_stream,
                 cc_sync, default_options, load)

__all__ = [
    "CC_FLAG_SYMMETRIC", "CC_FLAG_SYNC", "CC_FLAG_VALIDATE", "CC_MODE_AUTO", "CC_MODE_CLUSTER", "CC_MODE_FILTERED",
    "CC_MODE_MULTI_LAUNCH", "CC_MODE_PERSISTENT", "CCError", "ConnectedComponents", "cc_create", "cc_destroy",
    "cc_labels_batched", "cc_labels_coo", "cc_labels_csr", "cc_labels_csr64", "cc_labels_csr_host",
    "cc_labels_csr_noalloc", "cc_last_run_info", "cc_set_launch_status", "cc_set_options", "cc_set_stream",
    "cc_sync", "default_options", "load",
]
