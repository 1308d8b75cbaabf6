"""Sparse oracle: the explicit NN product form applied to right-hand sides.

Test infrastructure only. Follows Corollary 1 (Eq. (NNexplicit)) with phi^(0) a
diagonal matrix D^-1 (Jacobi), read per Corollary 6 and Algorithm 2 as a chain of
sparse matrix-vector products that never forms a dense matrix:

    x = D^-1 prod_{j=0}^{k-1} ( sum_{n=0}^{L} P^{n (L+1)^j} ) b,   P = I - A D^-1.

Readings: Algorithm 2 prints "Z = B; P_id = 1 - Z W_tilde" with mismatched shapes; it
is read as P = I - A D^-1 applied to vectors (the right-multiplied form of
I - D^-1 A, since (I - D^-1 A)^n D^-1 = D^-1 (I - A D^-1)^n). The printed loop
covers L + 1 = 2; here the factor for general L is applied as L successive blocks of
(L+1)^j products with P, summed. The product of the k factors is the Neumann series
of order (L+1)^k - 1 (Corollary 2), i.e. (L+1)^k - 1 sparse products in all.
"""
from __future__ import annotations

import numpy as np


def apply_p(a, dinv: np.ndarray, v: np.ndarray) -> np.ndarray:
    """P v = v - A (D^-1 v) with A a SciPy CSR matrix (library SpMV as the primitive)."""
    return v - a @ (dinv[:, None] * v if v.ndim == 2 else dinv * v)


def nn_sparse_solve(a, b: np.ndarray, depth: int, nests: int, dinv: np.ndarray | None = None) -> np.ndarray:
    """x = D^-1 prod_j sum_n P^{n (L+1)^j} b for ``nests`` factors (FP64 or as given)."""
    return nn_sparse_solve_sched(a, b, [depth] * nests, dinv)


def nn_sparse_solve_sched(a, b: np.ndarray, depths, dinv: np.ndarray | None = None) -> np.ndarray:
    """The factor product with a depth per factor:

        x = D^-1 prod_j ( sum_{n=0}^{L_j} P^{n m_j} ) b,   m_j = prod_{q<j} (L_q + 1),

    the Chebyshev-then-Neumann (CNS) construction of Corollary 4 and Corollary 6 when the
    first factors have L = 2 (Chebyshev nests) and the rest L = 1 (the factorised series
    prod_t (I + P^{2^t}) on the preconditioner those nests built). The product is the
    Neumann series of order prod_j (L_j + 1) - 1, in that many sparse products.
    """
    if dinv is None:
        dinv = 1.0 / a.diagonal()
    z = np.array(b, copy=True)
    t = 1
    for depth in depths:
        acc = z.copy()
        u = z
        for _n in range(depth):
            for _ in range(t):
                u = apply_p(a, dinv, u)
            acc = acc + u
        z = acc
        t *= depth + 1
    return (dinv[:, None] * z) if z.ndim == 2 else dinv * z


def relative_residual(a, x: np.ndarray, b: np.ndarray) -> float:
    """||b - A x||_2 / ||b||_2 (Frobenius over all right-hand sides)."""
    return float(np.linalg.norm(b - a @ x) / np.linalg.norm(b))
