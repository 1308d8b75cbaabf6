"""Exact rational oracle of the Nested Neumann (NN) method for tiny matrices.

Test infrastructure only. Matrices are lists of lists of ``fractions.Fraction``;
every operation is exact, so identities the paper proves hold with equality:
* Corollary 2 / Appendix 4: NN after k nests equals the Neumann series of order
  (L+1)^k - 1 from the same starting matrix.
* Appendix 2: I - W X_{k+1} = (I - W X_k)^(L+1).
* Corollary 4: L = 1 is Newton iteration, L = 2 is Chebyshev iteration.
"""
from __future__ import annotations

from fractions import Fraction

Mat = list  # list[list[Fraction]]


def mat(rows) -> Mat:
    return [[Fraction(v) for v in row] for row in rows]


def eye(n: int) -> Mat:
    return [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]


def add(a: Mat, b: Mat) -> Mat:
    return [[x + y for x, y in zip(ra, rb)] for ra, rb in zip(a, b)]


def sub(a: Mat, b: Mat) -> Mat:
    return [[x - y for x, y in zip(ra, rb)] for ra, rb in zip(a, b)]


def scale(a: Mat, c) -> Mat:
    c = Fraction(c)
    return [[c * x for x in row] for row in a]


def matmul(a: Mat, b: Mat) -> Mat:
    n, m, p = len(a), len(b), len(b[0])
    return [[sum((a[i][k] * b[k][j] for k in range(m)), Fraction(0)) for j in range(p)] for i in range(n)]


def power(a: Mat, e: int) -> Mat:
    out = eye(len(a))
    for _ in range(e):
        out = matmul(out, a)
    return out


def trace(a: Mat) -> Fraction:
    return sum((a[i][i] for i in range(len(a))), Fraction(0))


def residual(w: Mat, x: Mat) -> Mat:
    """R = I - W X."""
    return sub(eye(len(w)), matmul(w, x))


def neumann_right(w: Mat, x0: Mat, order: int) -> Mat:
    """x0 sum_{n=0}^{order} (I - W x0)^n, Eq. (Neumann) multiplied out on the right."""
    r = residual(w, x0)
    acc = [[Fraction(0)] * len(w) for _ in w]
    term = eye(len(w))
    for _ in range(order + 1):
        acc = add(acc, term)
        term = matmul(term, r)
    return matmul(x0, acc)


def neumann_left(w: Mat, phi: Mat, order: int) -> Mat:
    """sum_{n=0}^{order} (I - phi W)^n phi, Eq. (Neumann) as printed."""
    p = sub(eye(len(w)), matmul(phi, w))
    acc = [[Fraction(0)] * len(w) for _ in w]
    term = eye(len(w))
    for _ in range(order + 1):
        acc = add(acc, term)
        term = matmul(term, p)
    return matmul(acc, phi)


def nn_right(w: Mat, x0: Mat, depth: int, nests: int) -> list:
    """Iterates X_0..X_nests of X <- X (I + R (I + R (...))), R = I - W X (L factors)."""
    n = len(w)
    out = [x0]
    x = x0
    for _ in range(nests):
        r = residual(w, x)
        s = eye(n)
        for _l in range(depth):
            s = add(eye(n), matmul(r, s))
        x = matmul(x, s)
        out.append(x)
    return out


def nn_alg1(w: Mat, theta, depth: int, nests: int) -> Mat:
    """Algorithm 1 (left form, power sum, phi^(0) = I) with a scalar Theta; returns Z Theta."""
    n = len(w)
    w_t = scale(w, theta)
    z = eye(n)
    for _ in range(nests):
        p = sub(eye(n), matmul(z, w_t))
        s = eye(n)
        pl = eye(n)
        for _l in range(depth):
            pl = matmul(pl, p)
            s = add(s, pl)
        z = matmul(s, z)
    return scale(z, theta)


def newton(w_t: Mat, z0: Mat, steps: int) -> Mat:
    """Z <- Z (2I - W~ Z), Eq. (newtoniteration)."""
    n = len(w_t)
    z = z0
    for _ in range(steps):
        z = matmul(z, sub(scale(eye(n), 2), matmul(w_t, z)))
    return z


def chebyshev(w_t: Mat, z0: Mat, steps: int) -> Mat:
    """Z <- Z [3I - W~ Z (3I - W~ Z)], Eq. (cheby)."""
    n = len(w_t)
    z = z0
    three = scale(eye(n), 3)
    for _ in range(steps):
        wz = matmul(w_t, z)
        z = matmul(z, sub(three, matmul(wz, sub(three, wz))))
    return z
