"""GB300 (sm_103a) DMRG operator rotation.

Python face of the C ABI in ``include/dmrg_rotate.h``: functions carry the C
names and only marshal torch tensors (device memory, streams) into the
library's calls.  The computation, O'_k = U^T (O_k (x) I_d) U for a batch of
block operators (Rincon, Garcia, Hallberg, Sec. 2 step 5 and Sec. 3.2), runs in
the library's CUDA kernels; importing the rotation functions without the built
library raises.
"""
from .api import (  # noqa: F401
    Handle,
    default_handle,
    dmrg_rotate_ops,
    dmrg_rotate_ops_workspace,
    dmrg_rotate_ops_noalloc,
    dmrg_rotate_ops_host,
    dmrg_autotune_rotate_ops,
    dmrg_rotate_ops_backward,
    dmrg_rotate_site_ops,
    dmrg_orthonormality_error,
    dmrg_correlations,
    dmrg_expectation,
    dmrg_cross_correlations,
    dmrg_structure_factor,
    dmrg_truncation,
    dmrg_set_option,
    dmrg_kernel_timing,
    dmrg_sync_status,
    BlockedPlan,
    dmrg_blocked_plan_create,
    dmrg_rotate_ops_blocked,
    PRECISIONS,
)
from .partition import umd_partition  # noqa: F401
from .autograd import DmrgRotate, rotate  # noqa: F401
