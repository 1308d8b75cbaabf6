"""GB300-native Nested Neumann (NN) iterative matrix inversion.

The compute path is ``lib/libnn.so`` (CUDA kernels for sm_103a behind the C ABI in
``include/nn.h``); ``abi`` is its thin Python binding. Build with
``python -m paper_2212_02406_gb300.build``.
"""
from . import abi  # noqa: F401
from .abi import (  # noqa: F401
    nn_init_precond,
    nn_invert,
    nn_invert_host,
    nn_residual,
    nn_csr_workspace_bytes,
    nn_solve_csr,
    nn_batched_plan,
    nn_batched_plan_classes,
    nn_invert_batched_c64,
    nn_workspace_bytes,
    nn_workspace_bytes_host,
)
