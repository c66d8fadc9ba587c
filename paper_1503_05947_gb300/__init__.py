"""GB300-native Reduced Basis Decomposition (Y. Chen, arXiv 1503.05947).

The greedy compression X ~ Y T of Algorithm 1 runs in hand-written CUDA kernels for sm_103a
behind the C ABI of include/rbd.h (librbd.so); ``rbd`` is its thin Python binding.
"""
from .rbd import (  # noqa: F401
    BatchPlan,
    Compressed,
    RbdError,
    as_colmajor,
    colmajor_empty,
    compress,
    compress_host,
    compress_noalloc,
    compress_resume,
    compress_rows,
    grad,
    grad_batched,
    get_profile,
    load,
    project,
    reconstruct,
    set_profiling,
    set_wait_limit,
    status_string,
    version,
    workspace_bytes,
)
from .buildlib import build  # noqa: F401
from .autograd import RBDLoss, RBDLossBatched, rbd_loss, rbd_loss_batched  # noqa: F401
