"""Pins of the exact (rational) oracle and of the FP64 oracle against it.

Every identity here is one the paper proves, checked with exact arithmetic:
* Corollary 2 / Appendix 4: k nests of depth L equal the Neumann series of order
  (L+1)^k - 1 from the same X_0.
* Appendix 2: I - W X_{k+1} = (I - W X_k)^(L+1).
* Section II-D: the left (Algorithm 1) and right-multiplied forms give the same iterate.
* Corollary 4: L = 1 is Newton iteration (Eq. (newtoniteration)), L = 2 is Chebyshev
  iteration (Eq. (cheby)).
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import dense, exact


def _theta(w):
    return Fraction(1) / exact.trace(w)


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (4, 2)])
@pytest.mark.parametrize("depth", [1, 2, 3])
def test_nn_equals_neumann_of_order(n, seed, depth):
    w = exact.mat(synth.rational_spd(n, seed))
    x0 = exact.scale(exact.eye(n), _theta(w))
    nests = 2 if depth < 3 or n < 4 else 1
    its = exact.nn_right(w, x0, depth, nests)
    for k, xk in enumerate(its):
        assert xk == exact.neumann_right(w, x0, (depth + 1) ** k - 1)


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_residual_power_law(depth):
    w = exact.mat(synth.rational_spd(3, 5))
    x0 = exact.scale(exact.eye(3), _theta(w))
    its = exact.nn_right(w, x0, depth, 2)
    for k in range(2):
        rk = exact.residual(w, its[k])
        assert exact.residual(w, its[k + 1]) == exact.power(rk, depth + 1)


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_left_form_equals_right_form(depth):
    w = exact.mat(synth.rational_spd(3, 7))
    th = _theta(w)
    x0 = exact.scale(exact.eye(3), th)
    right = exact.nn_right(w, x0, depth, 2)[2]
    left = exact.nn_alg1(w, th, depth, 2)
    assert left == right


def test_left_neumann_equals_right_neumann_with_matrix_theta():
    # Appendix 1 allows a matrix Theta; the identity (I - X W)^n X = X (I - W X)^n
    # makes the printed left form and the right form the same series.
    w = exact.mat(synth.rational_spd(3, 9))
    dinv = [[(Fraction(1) / w[i][i] if i == j else Fraction(0)) for j in range(3)] for i in range(3)]
    for order in range(5):
        assert exact.neumann_left(w, dinv, order) == exact.neumann_right(w, dinv, order)


def test_depth1_is_newton_depth2_is_chebyshev():
    w = exact.mat(synth.rational_spd(3, 11))
    th = _theta(w)
    w_t = exact.scale(w, th)
    i3 = exact.eye(3)
    for k in range(3):
        nn1 = exact.nn_alg1(w, th, 1, k)
        nn2 = exact.nn_alg1(w, th, 2, k)
        assert nn1 == exact.scale(exact.newton(w_t, i3, k), th)
        assert nn2 == exact.scale(exact.chebyshev(w_t, i3, k), th)


def test_depth_zero_is_identity_map():
    # Appendix 2, case L = 0: phi^(i+1) = phi^(i); the library rejects depth 0 instead.
    w = exact.mat(synth.rational_spd(2, 3))
    x0 = exact.scale(exact.eye(2), _theta(w))
    assert exact.nn_right(w, x0, 0, 3)[-1] == x0


def _to_np(m):
    return np.array([[float(v) for v in row] for row in m])


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_fp64_oracle_matches_exact(depth):
    n = 4
    w = exact.mat(synth.rational_spd(n, 13))
    th = _theta(w)
    x0 = exact.scale(exact.eye(n), th)
    nests = 2
    ex = exact.nn_right(w, x0, depth, nests)
    wf = _to_np(w)
    run = dense.nn_invert(wf, _to_np(x0), depth, tol=0.0, max_nests=nests)
    ref = _to_np(ex[-1])
    assert np.linalg.norm(run.x - ref) <= 1e-13 * np.linalg.norm(ref)
    # Algorithm 1 and the explicit product form in FP64, same input
    alg1 = dense.nn_alg1(wf, float(th), depth, nests)
    expl = dense.nn_explicit(wf, float(th), depth, nests)
    assert np.linalg.norm(alg1 - ref) <= 1e-13 * np.linalg.norm(ref)
    assert np.linalg.norm(expl - ref) <= 1e-13 * np.linalg.norm(ref)
    # residual history against the exact residual norms
    for k in range(nests + 1):
        rk = _to_np(exact.residual(w, ex[k]))
        s_exact = np.linalg.norm(rk) / n
        assert abs(run.history[k] - s_exact) <= 1e-12 * max(s_exact, 1e-300) + 1e-15
