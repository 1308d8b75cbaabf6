"""Batched oracle: the dense NN loop over many small complex Hermitian matrices.

Test infrastructure only. Each matrix runs its own right-multiplied NN (see
``oracle.dense``) in complex128 from the Jacobi start X_0 = c diag(A)^-1 (a diagonal
Theta, Appendix 1), for a fixed number of nests (tol <= 0), exactly as a massive-MIMO
receiver would (Corollary 4 discusses Chebyshev steps for mMIMO detection).
"""
from __future__ import annotations

import numpy as np

from .dense import nn_invert, precond_jacobi


def nn_batched(matrices, depth: int, nests: int, damping=1.0):
    """Returns a list of ``NNRun`` (x, nests, residual history, status) per matrix.

    ``damping`` is a scalar, or a callable of the matrix size U giving the scalar.
    """
    out = []
    for a in matrices:
        a = np.asarray(a, dtype=np.complex128)
        c = damping(a.shape[0]) if callable(damping) else damping
        x0 = precond_jacobi(a, c)
        out.append(nn_invert(a, x0, depth, tol=0.0, max_nests=nests))
    return out
