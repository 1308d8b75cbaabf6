"""CPU oracle for the Nested Neumann (NN) matrix inversion method.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow FP64 / complex128 (and, for
tiny inputs, exact rational) restatement of what the method computes, written from
the paper "Generalization of higher order methods for fast iterative matrix
inversion via GPU acceleration" (Engsig, Yang, Mehouachi). It exists to check the
CUDA path. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the library in ``paper_2212_02406_gb300`` never
does, and this package imports nothing from that library.

Modules
-------
``dense``    Neumann series, Newton and Chebyshev iterations, NN (Algorithm 1 and
             the right-multiplied form), the explicit product form, preconditioners,
             the residual, the stop/divergence rule, and general solves through the
             normal equations (Corollary 3).
``exact``    the same recursions over ``fractions.Fraction`` for N <= 4.
``sparse``   the explicit NN product form applied to right-hand sides through a
             CSR matrix (Corollary 1, Corollary 6, Algorithm 2).
``batched``  a loop of the dense oracle over small complex Hermitian matrices.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against a
fact the paper or the mathematics fixes (exact rational identities, closed forms on
diagonal and known-spectrum matrices, Newton/Chebyshev special cases, library
inverses, Jacobi sweeps, the convergence order).
"""
from .dense import (  # noqa: F401
    STATUS_OK,
    STATUS_DIVERGED,
    STATUS_NOT_CONVERGED,
    NNRun,
    chebyshev_iteration,
    neumann_series,
    neumann_series_right,
    newton_iteration,
    nn_alg1,
    nn_explicit,
    nn_invert,
    nn_normal_solve,
    nn_step_right,
    precond_jacobi,
    precond_pan_schreiber,
    precond_scalar,
    precond_theta2,
    precond_trace,
    residual,
    theta2,
    rms_frob,
)
