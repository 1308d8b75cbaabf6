"""Pins of the FP64 dense oracle against closed forms, textbook special cases and
library inverses (nothing here re-types the oracle's own formula)."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U64 = np.finfo(np.float64).eps / 2


# --- closed form on diagonal matrices ------------------------------------------------
# With A = diag(lambda) and X_0 = alpha I everything commutes, and Appendix 2's identity
# R_k = R_0^((L+1)^k) gives X_k = diag((1 - (1 - alpha lambda)^((L+1)^k)) / lambda).

@pytest.mark.parametrize("depth", [1, 2, 3])
def test_diagonal_closed_form(depth):
    lam = np.array([0.3, 1.0, 2.5, 7.0, 11.0, 19.5])
    alpha = 2.0 / (lam.min() + lam.max())
    a = np.diag(lam)
    x = dense.precond_scalar(len(lam), alpha)
    for k in range(6):
        m = (depth + 1) ** k
        want = (1.0 - (1.0 - alpha * lam) ** m) / lam
        got = np.diag(x)
        assert np.allclose(got, want, rtol=64 * U64 * m, atol=0)
        assert np.count_nonzero(x - np.diag(got)) == 0
        x = dense.nn_step_right(a, x, depth)


# --- closed-form residual on a known spectrum ----------------------------------------
# A = Q diag(lambda) Q^T, X_0 = alpha I: ||R_k||_F / N = sqrt(sum_j (1-alpha lambda_j)^(2 (L+1)^k)) / N.

@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("kappa", [1e2, 1e4])
def test_known_spectrum_residual_history(depth, kappa):
    n = 96
    a, q, lam = synth.spd_spectrum(n, kappa, seed=3)
    alpha = 2.0 / (lam[0] + lam[-1])
    run = dense.nn_invert(a, dense.precond_scalar(n, alpha), depth, tol=1e-6, max_nests=40)
    assert run.status == dense.STATUS_OK
    pred = []
    for k in range(len(run.history)):
        m = (depth + 1) ** k
        pred.append(math.sqrt(float(np.sum((1.0 - alpha * lam) ** (2 * m)))) / n)
    floor = 50 * kappa * U64
    for s, p in zip(run.history, pred):
        if p > floor:
            assert abs(s - p) <= 1e-6 * p + floor
    # first nest under tol agrees with the prediction
    k_pred = next(k for k, p in enumerate(pred) if p < 1e-6)
    assert run.nests == k_pred


# --- textbook special cases (Corollary 4) -----------------------------------------

def test_depth1_newton_depth2_chebyshev_fp64():
    a = synth.spd_wishart(40, seed=1)
    th = 1.0 / np.trace(a)
    w_t = th * a
    i = np.eye(40)
    for k in range(5):
        x1 = dense.nn_invert(a, th * i, 1, tol=0.0, max_nests=k).x
        x2 = dense.nn_invert(a, th * i, 2, tol=0.0, max_nests=k).x
        n1 = dense.newton_iteration(w_t, i, k) * th
        c2 = dense.chebyshev_iteration(w_t, i, k) * th
        assert np.linalg.norm(x1 - n1) <= 1e-12 * np.linalg.norm(n1)
        assert np.linalg.norm(x2 - c2) <= 1e-12 * np.linalg.norm(c2)


# --- Corollary 2 and the left/right forms in FP64 ---------------------------------

@pytest.mark.parametrize("depth", [1, 2, 3])
def test_nn_vs_neumann_and_alg1_fp64(depth):
    a = synth.spd_wishart(48, seed=2)
    x0 = dense.precond_pan_schreiber(a)
    nests = 3
    x_nn = dense.nn_invert(a, x0, depth, tol=0.0, max_nests=nests).x
    x_ns = dense.neumann_series_right(a, x0, (depth + 1) ** nests - 1)
    x_ns_left = dense.neumann_series(a, x0, (depth + 1) ** nests - 1)
    x_alg1 = dense.nn_alg1(a, x0, depth, nests)
    x_expl = dense.nn_explicit(a, x0, depth, nests)
    ref = np.linalg.norm(x_ns)
    for other in (x_nn, x_ns_left, x_alg1, x_expl):
        assert np.linalg.norm(other - x_ns) <= 1e-11 * ref


# --- library inverse, order of convergence, stop rule (config: N=256 Wishart) ------

@pytest.mark.parametrize("depth,nests_expected", [(1, 15), (2, 10), (3, 8)])
def test_wishart_256_converges_to_library_inverse(depth, nests_expected):
    a = synth.spd_wishart(256, seed=0)
    x0 = dense.precond_pan_schreiber(a)
    run = dense.nn_invert(a, x0, depth, tol=1e-10, max_nests=64)
    assert run.status == dense.STATUS_OK
    assert run.nests == nests_expected
    inv = np.linalg.inv(a)
    kappa = np.linalg.cond(a)
    assert np.linalg.norm(run.x - inv) <= 100 * kappa * U64 * np.linalg.norm(inv)
    assert run.history[-1] < 1e-10 <= run.history[-2]


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_order_of_convergence(depth):
    # Appendix 5: order L+1. On A = diag with one dominant residual eigenvalue rho,
    # log(s_{k+1}/s_k) / log(s_k/s_{k-1}) -> L+1.
    n = 64
    rho = 0.999
    lam = np.linspace(0.2, 1.0 - rho + 1.0, n)  # residual eigenvalues 1 - lam
    lam[0] = 1.0 - rho
    a = np.diag(lam)
    run = dense.nn_invert(a, np.eye(n), depth, tol=0.0, max_nests=12)
    h = run.history
    ratios = []
    for k in range(1, len(h) - 1):
        if h[k + 1] > 1e-12:  # stay well above the FP64 rounding floor
            num = math.log(h[k + 1] / h[k])
            den = math.log(h[k] / h[k - 1])
            if abs(den) > 1e-3:
                ratios.append(num / den)
    assert ratios, "no measurable nests"
    assert abs(ratios[-1] - (depth + 1)) < 1e-3


def test_divergence_is_reported():
    lam = np.array([1.0, 2.0, 4.0])
    a = np.diag(lam)
    x0 = dense.precond_scalar(3, 0.9)   # 1 - 0.9*4 = -2.6: rho(R0) > 1
    run = dense.nn_invert(a, x0, 2, tol=1e-12, max_nests=30)
    assert run.status == dense.STATUS_DIVERGED
    x0 = dense.precond_scalar(3, 0.4)   # rho(R0) = 0.6
    run = dense.nn_invert(a, x0, 2, tol=1e-12, max_nests=30)
    assert run.status == dense.STATUS_OK


def test_not_converged_when_capped():
    a = synth.spd_wishart(32, seed=4)
    run = dense.nn_invert(a, dense.precond_trace(a), 1, tol=1e-300, max_nests=3)
    assert run.status == dense.STATUS_NOT_CONVERGED and run.nests == 3
    assert len(run.history) == 4


def test_preconditioners_satisfy_norm_condition():
    r = synth.rng(5)
    g = r.standard_normal((30, 30))
    assert np.linalg.norm(np.eye(30) - g @ dense.precond_pan_schreiber(g), 2) < 1.0
    a = synth.spd_wishart(30, seed=5)
    assert np.max(np.abs(np.linalg.eigvals(np.eye(30) - a @ dense.precond_trace(a)))) < 1.0
    dd = a + np.diag(np.sum(np.abs(a), axis=1))
    assert np.max(np.abs(np.linalg.eigvals(np.eye(30) - dd @ dense.precond_jacobi(dd)))) < 1.0


def test_pan_schreiber_complex_start():
    # Section II allows W in C^{N x N}: X_0 = W^H / (||W||_1 ||W||_inf) makes W X_0 Hermitian
    # positive definite with eigenvalues sigma_i^2 / (||W||_1 ||W||_inf) in (0, 1] (sigma_max^2 <=
    # ||W||_1 ||W||_inf), so I - W X_0 has its spectrum in [0, 1) and the NN loop converges to
    # W^-1. A dropped conjugate (W^T) breaks the Hermitian property and the convergence.
    r = synth.rng(6)
    n = 24
    w = r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))
    x0 = dense.precond_pan_schreiber(w)
    m = w @ x0
    assert np.allclose(m, m.conj().T, rtol=0, atol=1e-14)
    ev = np.linalg.eigvalsh(m)
    assert ev.min() > 0 and ev.max() <= 1 + 1e-12
    assert np.linalg.norm(np.eye(n) - m, 2) < 1.0
    run = dense.nn_invert(w, x0, 2, tol=1e-12, max_nests=40)
    assert run.status == dense.STATUS_OK
    assert np.linalg.norm(run.x @ w - np.eye(n)) < 1e-9
    # the transpose without conjugation is not a convergent start for this W
    bad = w.T / (np.max(np.sum(np.abs(w), axis=0)) * np.max(np.sum(np.abs(w), axis=1)))
    assert np.max(np.abs(np.linalg.eigvals(np.eye(n) - w @ bad))) >= 1.0


# --- the paper's only printed numeric claim (Corollary 3) ---------------------------

def test_corollary3_normal_equations_claim():
    with open(os.path.join(GOLDEN, "cor3_normal_equations.json")) as f:
        claim = json.load(f)
    n = 12
    cond = claim["cond_A"]
    r = synth.rng(21)
    u, _ = np.linalg.qr(r.standard_normal((n, n)))
    v, _ = np.linalg.qr(r.standard_normal((n, n)))
    sig = np.geomspace(1.0, 1.0 / cond, n)
    a = (u * sig) @ v.T
    w = a.T @ a
    th = 1.0 / np.trace(w)
    # Closed form: residual eigenvalues (1 - th sigma_j^2)^((L+1)^nests), worst at sigma_min.
    worst = (1.0 - th * sig[-1] ** 2) ** ((claim["inception_depth"] + 1) ** claim["nests"])
    assert worst < 1e-300 or worst == 0.0
    x = dense.nn_alg1(w, th, claim["inception_depth"], claim["nests"])
    b = r.standard_normal(n)
    sol = x @ (a.T @ b)
    true = np.linalg.solve(a, b)
    # FP64 floor of the normal equations: relative error of order cond(W) u = cond(A)^2 u
    assert np.linalg.norm(sol - true) <= cond * cond * U64 * np.linalg.norm(true)


def test_optimal_depth_claim():
    # Appendix 6: for a budget of K matrix products, nests = K/(L+1) and the Neumann
    # order reached is (L+1)^(K/(L+1)); the integer optimum is L = 2.
    with open(os.path.join(GOLDEN, "optimal_depth.json")) as f:
        claim = json.load(f)
    k_budget = 36
    orders = {L: (L + 1) ** (k_budget // (L + 1)) for L in (1, 2, 3, 4, 5)}
    assert max(orders, key=orders.get) == claim["optimal_inception_depth"]


# --- Theta_2 power-iteration normalisation (Eq. (trace), read as an inverse Rayleigh quotient) ---

def test_theta2_bounds_and_limit():
    # On a diagonal matrix the k-th power iterate's Rayleigh quotient is computable by hand:
    # with v = ones, u = W^k v has entries lambda_j^k, so <u, W u> / <u, u> =
    # sum lambda^(2k+1) / sum lambda^(2k), which increases to lambda_max.
    lam = np.array([1.0, 2.0, 5.0, 10.0])
    w = np.diag(lam)
    v = np.ones(4)
    for k in (1, 2, 4, 8, 16):
        rq = float(np.sum(lam ** (2 * k + 1)) / np.sum(lam ** (2 * k)))
        assert abs(dense.theta2(w, k, v) - (k / (k + 1)) / rq) <= 1e-14 / rq
        # never above 1 / lambda_max, so I - Theta_2 W keeps its spectrum in [0, 1)
        assert dense.theta2(w, k, v) * lam.max() < 1.0
    # rho(I - Theta_2 W) < 1 on an SPD matrix, and Theta_2 beats the trace normalisation
    a, q, lamq = synth.spd_spectrum(200, 1e3, seed=4)
    v = synth.rng(9).standard_normal(200)
    t2 = dense.theta2(a, 8, v)
    rho2 = np.max(np.abs(1.0 - t2 * lamq))
    rho1 = np.max(np.abs(1.0 - lamq / np.trace(a)))
    assert rho2 < 1.0 and rho2 < rho1


# --- general systems through the normal equations (Corollary 3) -----------------------

@pytest.mark.parametrize("depth", [1, 2, 3])
def test_normal_solve_diagonal_complex_closed_form(depth):
    # A = diag(a_j), complex: W = A^H A = diag(|a_j|^2), Theta = 1 / sum |a_j|^2 and
    # X_k = diag((1 - (1 - Theta |a_j|^2)^((L+1)^k)) / |a_j|^2), so x_j = X_k,jj conj(a_j) b_j.
    # A dropped conjugate, a missing Theta or a wrong power fails this.
    r = synth.rng(3)
    n = 9
    a = (r.uniform(0.5, 2.0, n) * np.exp(1j * r.uniform(0, 2 * np.pi, n)))
    b = r.standard_normal(n) + 1j * r.standard_normal(n)
    for nests in (0, 1, 3, 6):
        x, run = dense.nn_normal_solve(np.diag(a), b, depth, 0.0, nests)
        th = 1.0 / np.sum(np.abs(a) ** 2)
        xk = (1.0 - (1.0 - th * np.abs(a) ** 2) ** ((depth + 1) ** nests)) / np.abs(a) ** 2
        want = xk * a.conj() * b
        assert run.nests == nests
        assert np.max(np.abs(x - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("complex_", [False, True])
def test_normal_solve_spectral_nest_count(complex_):
    # R_k = (I - Theta W)^((L+1)^k) with W = V diag(sigma^2) V^H, so
    # s_k = sqrt(sum_j (1 - Theta sigma_j^2)^(2 (L+1)^k)) / N: the nest count is known in advance.
    n, cond, depth, tol = 48, 20.0, 2, 1e-9
    a, sig = synth.general_svd(n, cond, seed=5, complex_=complex_)
    b = synth.gaussian_rhs(n, 2, seed=6)
    th = 1.0 / np.sum(sig ** 2)
    pred = [math.sqrt(np.sum((1.0 - th * sig ** 2) ** (2 * (depth + 1) ** k))) / n for k in range(40)]
    k_stop = next(k for k, s in enumerate(pred) if s < tol)
    x, run = dense.nn_normal_solve(a, b, depth, tol, 40)
    assert run.status == dense.STATUS_OK and run.nests == k_stop
    for k in range(k_stop + 1):
        assert abs(run.history[k] - pred[k]) <= 1e-9 * pred[k] + 1e3 * U64
    # and the solution solves A x = b: with X_k = W^-1 (I - R_k) and R_k a polynomial in W,
    # x - x* = -R_k x*, so the relative error is at most ||R_k||_2 <= N s_k, plus the FP64 floor
    true = np.linalg.solve(a, b)
    err = np.linalg.norm(x - true) / np.linalg.norm(true)
    assert err <= n * run.history[-1] + 64 * cond ** 2 * U64


def test_normal_solve_nonsymmetric_matches_library():
    # a general complex matrix with cond(A) = 1e3: the converged NN solution equals
    # numpy.linalg.solve within the normal equations' FP64 error bound c cond(A)^2 u
    n, cond = 40, 1e3
    a, _ = synth.general_svd(n, cond, seed=11, complex_=True)
    b = synth.gaussian_rhs(n, 3, seed=12) + 1j * synth.gaussian_rhs(n, 3, seed=13)
    x, run = dense.nn_normal_solve(a, b, 2, 1e-13, 64)
    assert run.status in (dense.STATUS_OK, dense.STATUS_NOT_CONVERGED)
    true = np.linalg.solve(a, b)
    assert np.linalg.norm(x - true) <= 64 * cond ** 2 * U64 * np.linalg.norm(true)


# --- a depth per nest (CNS: Chebyshev nests, then Newton nests; Corollary 4, Corollary 6) ---

@pytest.mark.parametrize("sched", [[2, 2, 1], [2, 1, 1, 1], [1, 3, 2], [3]])
def test_depth_schedule_is_neumann_of_product_order(sched):
    # After nests of depths L_0 .. L_{k-1} the iterate is the Neumann series of order
    # prod (L_j + 1) - 1 (Corollary 2 with R_{k+1} = R_k^(L_k + 1)); on a diagonal matrix with a
    # scalar start this is the closed form (1 - (1 - alpha lambda)^m) / lambda.
    lam = np.array([0.2, 0.7, 1.0, 1.9, 3.0])
    alpha = 2.0 / (lam.min() + lam.max())
    nests = len(sched) + 1   # the last depth repeats
    run = dense.nn_invert(np.diag(lam), dense.precond_scalar(5, alpha), 1, 0.0, nests, depth_schedule=sched)
    m = int(np.prod([sched[min(k, len(sched) - 1)] + 1 for k in range(nests)]))
    want = (1.0 - (1.0 - alpha * lam) ** m) / lam
    assert np.allclose(np.diag(run.x), want, rtol=64 * U64 * m, atol=0)
    # and on a full SPD matrix it equals the right Neumann series of that order
    a = synth.spd_wishart(24, seed=6)
    x0 = dense.precond_trace(a)
    run = dense.nn_invert(a, x0, 1, 0.0, 3, depth_schedule=sched)
    m = int(np.prod([sched[min(k, len(sched) - 1)] + 1 for k in range(3)]))
    ns = dense.neumann_series_right(a, x0, m - 1)
    assert np.linalg.norm(run.x - ns) <= 1e-11 * np.linalg.norm(ns)
