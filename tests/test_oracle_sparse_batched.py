"""Pins of the sparse-chain and batched oracles.

Sparse (Corollary 1, Corollary 6, Algorithm 2): k factors of depth L are the Neumann
series of order (L+1)^k - 1 applied to b, which is exactly (L+1)^k Jacobi sweeps from
x = 0 (a textbook iteration), and, for the 5-point Laplacian whose diagonal is a
constant, the error obeys ||x* - x|| <= rho(P)^m ||x*|| with rho(P) known in closed form.

Batched: each matrix's iterate equals the Neumann series of the same order
(Corollary 2) from the Jacobi start; converging cases approach the library inverse.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import batched, dense, sparse


def _jacobi_sweeps(a, b, sweeps):
    d = a.diagonal()
    x = np.zeros_like(b)
    for _ in range(sweeps):
        x = x + (b - a @ x) / (d[:, None] if b.ndim == 2 else d)
    return x


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("kind", ["laplacian", "random"])
def test_sparse_chain_equals_jacobi_sweeps(depth, kind):
    if kind == "laplacian":
        m = synth.laplacian_5pt(9, 7, shift=0.5)
    else:
        m = synth.random_sparse_spd(70, per_row=5, seed=3)
    a = m.to_scipy()
    b = synth.gaussian_rhs(m.n, 2, seed=1)
    for nests in range(0, 4):
        x = sparse.nn_sparse_solve(a, b, depth, nests)
        want = _jacobi_sweeps(a, b, (depth + 1) ** nests)
        assert np.linalg.norm(x - want) <= 1e-12 * np.linalg.norm(want)


@pytest.mark.parametrize("depths", [[2, 1, 1], [2, 2, 1, 1, 1], [1, 2], [3, 1, 2]])
def test_sparse_schedule_equals_jacobi_sweeps(depths):
    # a depth per factor (CNS: Chebyshev factors, then the factorised Neumann series) is the
    # Neumann series of order prod (L_j + 1) - 1: exactly prod (L_j + 1) Jacobi sweeps
    m = synth.random_sparse_spd(60, per_row=5, seed=9)
    a = m.to_scipy()
    b = synth.gaussian_rhs(m.n, 2, seed=4)
    x = sparse.nn_sparse_solve_sched(a, b, depths)
    want = _jacobi_sweeps(a, b, int(np.prod([d + 1 for d in depths])))
    assert np.linalg.norm(x - want) <= 1e-12 * np.linalg.norm(want)


@pytest.mark.parametrize("depth", [1, 2])
def test_sparse_chain_equals_dense_explicit_form(depth):
    m = synth.random_sparse_spd(40, per_row=4, seed=8)
    a = m.to_scipy()
    ad = a.toarray()
    b = synth.gaussian_rhs(m.n, 1, seed=2)[:, 0]
    dinv = 1.0 / np.diag(ad)
    for nests in (1, 2, 3):
        xd = dense.nn_explicit(ad, dinv, depth, nests) @ b
        xs = sparse.nn_sparse_solve(a, b, depth, nests)
        assert np.linalg.norm(xs - xd) <= 1e-12 * np.linalg.norm(xd)


def test_sparse_laplacian_error_bound_closed_form():
    nx, shift, depth = 16, 0.5, 2
    m = synth.laplacian_5pt(nx, shift=shift)
    a = m.to_scipy().tocsc()
    b = synth.gaussian_rhs(m.n, 1, seed=4)[:, 0]
    xs = spla.spsolve(a, b)
    rho = 4.0 * math.cos(math.pi / (nx + 1)) / (4.0 + shift)
    for nests in range(1, 5):
        terms = (depth + 1) ** nests
        x = sparse.nn_sparse_solve(a.tocsr(), b, depth, nests)
        err = np.linalg.norm(xs - x) / np.linalg.norm(xs)
        assert err <= rho ** terms * (1 + 1e-9) + 1e-14
    assert err < 1e-5


def test_batched_matches_neumann_and_library():
    bt = synth.mimo_gram_batch(12, seed=5, dtype=np.complex128)
    runs = batched.nn_batched([bt.matrix(b) for b in range(bt.count)], depth=2, nests=3)
    for b, run in enumerate(runs):
        a = bt.matrix(b)
        x0 = dense.precond_jacobi(a)
        rho = np.max(np.abs(np.linalg.eigvals(np.eye(a.shape[0]) - a @ x0)))
        if rho < 1:
            ns = dense.neumann_series_right(a, x0, 3 ** 3 - 1)
            assert np.linalg.norm(run.x - ns) <= 1e-11 * np.linalg.norm(ns)
            assert run.status == dense.STATUS_OK
            # residual after 3 nests is the 27th power of R_0 (Appendix 2)
            r27 = np.linalg.matrix_power(np.eye(a.shape[0]) - a @ x0, 27)
            s = np.linalg.norm(r27) / a.shape[0]
            assert abs(run.history[-1] - s) <= 1e-9 * s + 1e-14
        if rho > 1.3:
            assert run.status == dense.STATUS_DIVERGED


def test_batched_damped_jacobi_converges():
    # Damped start X_0 = diag(A)^-1 / (1 + U/128) keeps rho(I - A X_0) < 1 for every U.
    bt = synth.mimo_gram_batch(12, seed=6, dtype=np.complex128)
    mats = [bt.matrix(b) for b in range(bt.count)]
    runs = batched.nn_batched(mats, depth=2, nests=5, damping=lambda u: 1.0 / (1.0 + u / 128.0))
    for a, run in zip(mats, runs):
        assert run.status == dense.STATUS_OK
        inv = np.linalg.inv(a)
        assert np.linalg.norm(run.x - inv) <= 1e-5 * np.linalg.norm(inv)
