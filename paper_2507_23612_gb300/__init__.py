"""Real-space DFT+U Chebyshev-filtered subspace iteration on GB300 (sm_103a).

A thin Python binding over the C ABI of ``libhub.so`` (declared in ``include/hub.h``).  It
only marshals arguments: every step on grid data runs in the library's CUDA kernels.
Tensors are torch CUDA tensors; a block of ``ncol`` orbitals is a tensor of shape
``(ncol, ld)`` (row ``j`` = orbital ``j``), which is the column-major ``ld x ncol`` layout the
library expects.  There is no CPU fallback: if the library cannot be loaded, importing the
binding's entry points raises.
"""
from .binding import (  # noqa: F401
    HubError, Hub, load_library, library_path, HUB_F64, HUB_F32, HUB_MIXED_BF16, HUB_MIXED_F16,
    KERNEL_KINDS, scf_params, STATUS_NAMES, batch_filter, MLP, descriptors,
)
