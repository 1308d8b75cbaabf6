"""Dense FP64 oracle of the Nested Neumann (NN) method. Test infrastructure only.

Notation follows the paper: W is the matrix to invert, Theta the normalisation
(scalar or matrix) with W~ = Theta W, phi^(i) the preconditioning matrix after i
nests, L the inception depth. The library's right-multiplied iterate is
X_k = phi^(k) Theta, with X_0 = Theta (phi^(0) = I), and its residual is
R_k = I - W X_k.

Readings of the paper used here (the paper is terse or has typos at these points):
* Algorithm 1 writes "phi = Trace(W); W_tilde = phi W; return Z phi": read as
  Theta = 1/Tr(W), W~ = Theta W, return Z Theta (consistent with Eq. (trace)).
* Algorithm 1 writes "P = 1 - Z W_tilde": read as P = I - Z W~ (identity matrix).
* Eq. (newtoniteration) writes Z(2I - W Z~): read as Z(2I - W~ Z).
* The paper iterates on the left (Z <- S Z, P = I - Z W~). The right-multiplied form
  X <- X sum_n (I - W X)^n is the same sequence, because X (I - W X)^n = (I - X W)^n X.
  ``nn_invert`` runs the right form, which is what the GPU path computes;
  ``nn_alg1`` runs Algorithm 1 as printed. Tests check the two agree.
* Stop test (the paper names only a "root mean Frobenius norm error"):
  s_k = ||I - W X_k||_F / N. The loop stops at the first k with s_k < tol and
  returns X_k, the iterate whose residual was measured. tol <= 0 runs exactly
  ``max_nests`` nests.
* Divergence (the paper gives no rule): s_k non-finite, or k >= 1 with s_k >= 1 and
  s_k > s_{k-1}. Convergence needs spectral radius rho(I - W X_0) < 1
  (Appendix 2 shows I - W X_{k+1} = (I - W X_k)^(L+1)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

STATUS_OK = 0
STATUS_DIVERGED = 2
STATUS_NOT_CONVERGED = 3


def _eye_like(w: np.ndarray) -> np.ndarray:
    return np.eye(w.shape[0], dtype=w.dtype)


def _as_matrix(theta, n: int, dtype) -> np.ndarray:
    """A scalar Theta becomes Theta*I; a vector becomes diag(Theta); a matrix is kept."""
    t = np.asarray(theta)
    if t.ndim == 0:
        return np.eye(n, dtype=dtype) * t
    if t.ndim == 1:
        return np.diag(t.astype(dtype))
    return t.astype(dtype)


# ---------------------------------------------------------------------------
# Preconditioners (Section II-A, Eq. (normalization) and Eq. (trace)).
# ---------------------------------------------------------------------------

def precond_trace(w: np.ndarray) -> np.ndarray:
    """X_0 = Theta_1 I with Theta_1 = 1 / Tr(W), Eq. (trace)."""
    n = w.shape[0]
    return np.eye(n, dtype=w.dtype) * (1.0 / np.trace(w).real)


def theta2(w: np.ndarray, k: int, v: np.ndarray) -> float:
    """Theta_2(k) of Eq. (trace), read as (k/(k+1)) ||W^k v||^2 / <W^k v, W^(k+1) v>.

    The printed ratio ||W^k v||^2 / ||W^(k+1) v||^2 has the dimension of 1/lambda^2 and
    cannot normalise W; the inverse Rayleigh quotient of the k-th power iterate has dimension
    1/lambda, tends to 1/lambda_max from above (for PD W and a start v with a component on
    the top eigenvector), and with the paper's safety factor k/(k+1) gives
    Theta_2 lambda_max <= 1 up to the iteration's error, so rho(I - Theta_2 W) < 1.
    The k products W^j v are taken one after another from the given start vector.
    """
    u = np.array(v, dtype=w.dtype, copy=True)
    for _ in range(k):
        u = w @ u
    wu = w @ u
    return float((k / (k + 1.0)) * np.vdot(u, u).real / np.vdot(u, wu).real)


def precond_theta2(w: np.ndarray, k: int, v: np.ndarray) -> np.ndarray:
    """X_0 = Theta_2(k) I, Eq. (trace)."""
    return np.eye(w.shape[0], dtype=w.dtype) * theta2(w, k, v)


def precond_scalar(n: int, alpha: float, dtype=np.float64) -> np.ndarray:
    """X_0 = alpha I: a scalar Theta (Appendix 1 allows any Theta with ||I - Theta W||_2 < 1)."""
    return np.eye(n, dtype=dtype) * alpha


def precond_jacobi(w: np.ndarray, damping: float = 1.0) -> np.ndarray:
    """X_0 = damping * diag(W)^-1: a diagonal matrix Theta (Appendix 1: Theta may be a matrix)."""
    return np.diag(damping / np.diag(w))


def precond_pan_schreiber(w: np.ndarray) -> np.ndarray:
    """X_0 = W^H / (||W||_1 ||W||_inf): the Pan-Schreiber starting matrix for Newton
    iteration (the reference the paper follows in Section II-C), which gives
    ||I - W X_0||_2 < 1 for any nonsingular W."""
    n1 = np.max(np.sum(np.abs(w), axis=0))
    ninf = np.max(np.sum(np.abs(w), axis=1))
    return w.conj().T / (n1 * ninf)


# ---------------------------------------------------------------------------
# Residual and norm.
# ---------------------------------------------------------------------------

def residual(w: np.ndarray, x: np.ndarray) -> np.ndarray:
    """R = I - W X."""
    return _eye_like(w) - w @ x


def rms_frob(r: np.ndarray) -> float:
    """Root-mean Frobenius norm ||R||_F / N (the paper's error measure, Section II)."""
    return float(np.linalg.norm(r, "fro") / r.shape[0])


# ---------------------------------------------------------------------------
# Neumann series, Eq. (Neumann).
# ---------------------------------------------------------------------------

def neumann_series(w: np.ndarray, phi: np.ndarray, order: int) -> np.ndarray:
    """sum_{n=0}^{order} (I - phi W)^n phi, Eq. (Neumann) as printed (left form)."""
    i = _eye_like(w)
    p = i - phi @ w
    acc = np.zeros_like(w)
    term = i.copy()
    for _ in range(order + 1):
        acc = acc + term
        term = term @ p
    return acc @ phi


def neumann_series_right(w: np.ndarray, x0: np.ndarray, order: int) -> np.ndarray:
    """x0 sum_{n=0}^{order} (I - W x0)^n: Eq. (Neumann) multiplied out on the right."""
    i = _eye_like(w)
    r = i - w @ x0
    acc = np.zeros_like(w)
    term = i.copy()
    for _ in range(order + 1):
        acc = acc + term
        term = term @ r
    return x0 @ acc


# ---------------------------------------------------------------------------
# Newton and Chebyshev iterations (Section II-B, II-C).
# ---------------------------------------------------------------------------

def newton_iteration(w_t: np.ndarray, z0: np.ndarray, steps: int) -> np.ndarray:
    """Z <- Z (2I - W~ Z), Eq. (newtoniteration) (read with W~ Z)."""
    i = _eye_like(w_t)
    z = z0
    for _ in range(steps):
        z = z @ (2.0 * i - w_t @ z)
    return z


def chebyshev_iteration(w_t: np.ndarray, z0: np.ndarray, steps: int) -> np.ndarray:
    """Z <- Z [3I - W~ Z (3I - W~ Z)], Eq. (cheby)."""
    i = _eye_like(w_t)
    z = z0
    for _ in range(steps):
        wz = w_t @ z
        z = z @ (3.0 * i - wz @ (3.0 * i - wz))
    return z


# ---------------------------------------------------------------------------
# Nested Neumann.
# ---------------------------------------------------------------------------

def nn_alg1(w: np.ndarray, theta, depth: int, nests: int) -> np.ndarray:
    """Algorithm 1 as printed (left form, power sum), with phi^(0) = I.

    W~ = Theta W; Z = I; each nest: P = I - Z W~, S = I + sum_{l=1}^{L} P^l, Z = S Z.
    Returns Z Theta, the approximation of W^-1.
    """
    n = w.shape[0]
    th = _as_matrix(theta, n, w.dtype)
    w_t = th @ w
    i = _eye_like(w)
    z = i.copy()
    for _ in range(nests):
        p = i - z @ w_t
        s = i.copy()
        pl = i.copy()
        for _l in range(depth):
            pl = pl @ p
            s = s + pl
        z = s @ z
    return z @ th


def nn_explicit(w: np.ndarray, theta, depth: int, nests: int) -> np.ndarray:
    """Eq. (NNexplicit), Corollary 1: phi^(i) = prod_{j=0}^{i-1} sum_{n=0}^{L} P0^{n (L+1)^j} phi^(0),
    with P0 = I - phi^(0) W~ and phi^(0) = I; returns phi^(i) Theta.

    (The printed equation is indexed for phi^(i+1); ``nests`` here is the number of
    factors, i.e. of nests applied.)
    """
    n = w.shape[0]
    th = _as_matrix(theta, n, w.dtype)
    i = _eye_like(w)
    p0 = i - th @ w  # phi^(0) = I
    prod = i.copy()
    for j in range(nests):
        base = np.linalg.matrix_power(p0, (depth + 1) ** j)
        fac = i.copy()
        pw = i.copy()
        for _n in range(depth):
            pw = pw @ base
            fac = fac + pw
        prod = prod @ fac
    return prod @ th


def nn_step_right(w: np.ndarray, x: np.ndarray, depth: int, r: np.ndarray | None = None) -> np.ndarray:
    """One nest of the right-multiplied NN: X <- X (I + R (I + R (... (I + R)))), L factors of R.

    Horner form of X sum_{n=0}^{L} R^n with R = I - W X (Theorem, Eq. (nestedneumann),
    multiplied out on the right).
    """
    i = _eye_like(w)
    if r is None:
        r = i - w @ x
    s = i.copy()
    for _ in range(depth):
        s = i + r @ s
    return x @ s


@dataclass
class NNRun:
    x: np.ndarray
    nests: int
    history: list = field(default_factory=list)
    status: int = STATUS_OK


def nn_invert(w: np.ndarray, x0: np.ndarray, depth: int, tol: float, max_nests: int = 64,
              depth_schedule=None) -> NNRun:
    """NN outer loop with the stop and divergence rules stated in the module docstring.

    ``depth_schedule`` (optional) gives nest k the depth depth_schedule[min(k, len - 1)]
    instead of ``depth``: e.g. [2, 2, 1] runs two Chebyshev nests, then Newton nests, the
    matrix form of the CNS construction (Corollary 4, Corollary 6). After nests of depths
    L_0 .. L_{k-1} the iterate is the Neumann series of order prod (L_j + 1) - 1.
    """
    if depth < 1 or (depth_schedule is not None and min(depth_schedule) < 1):
        raise ValueError("inception depth must be >= 1")
    i = _eye_like(w)
    n = w.shape[0]
    x = x0.astype(w.dtype, copy=True)
    hist: list[float] = []
    for k in range(max_nests + 1):
        r = i - w @ x
        s = float(np.linalg.norm(r, "fro") / n)
        hist.append(s)
        if not np.isfinite(s):
            return NNRun(x, k, hist, STATUS_DIVERGED)
        if k >= 1 and s >= 1.0 and s > hist[-2]:
            return NNRun(x, k, hist, STATUS_DIVERGED)
        if tol > 0 and s < tol:
            return NNRun(x, k, hist, STATUS_OK)
        if k == max_nests:
            break
        d = depth if not depth_schedule else depth_schedule[min(k, len(depth_schedule) - 1)]
        x = nn_step_right(w, x, d, r)
    return NNRun(x, max_nests, hist, STATUS_NOT_CONVERGED if tol > 0 else STATUS_OK)


# ---------------------------------------------------------------------------
# General (non-Hermitian, complex) systems through the normal equations (Corollary 3).
# ---------------------------------------------------------------------------

def nn_normal_solve(a: np.ndarray, b: np.ndarray, depth: int, tol: float, max_nests: int = 64):
    """Solve A x = B for any nonsingular A (real or complex) as Corollary 3 does.

    W = A^H A is Hermitian positive definite; the NN runs on W from X_0 = Theta I with
    Theta = 1 / Tr(W) (the trace normalisation of Eq. (trace)); the solution is
    x = X_k A^H B, the right-form counterpart of prod_j sum_n (I - Theta W)^{n (L+1)^j} Theta A^H B
    (Eq. (nnlinearsystem)). The stop rule is the one of ``nn_invert`` applied to W.
    Returns (x, run).
    """
    ah = a.conj().T
    w = ah @ a
    theta = 1.0 / np.trace(w).real
    x0 = np.eye(w.shape[0], dtype=w.dtype) * theta
    run = nn_invert(w, x0, depth, tol, max_nests)
    return run.x @ (ah @ b), run
