"""GPU tests of the serving runtime (continuous batching of NN inversions and solves).

* Every request's result is the same alone and in the mix: the kernels are deterministic
  (static tile schedules, fixed reduction orders), so a request run by itself and the same
  request run among concurrent ones on other streams give identical bits.
* Results are correct: every served X is the FP64 oracle's NN iterate (Algorithm 1, same A,
  same X_0 = I / Tr(A), same number of nests) up to what the residuals allow,
  ||X - X_ora||_F <= ||A^-1||_2 ||R - R_ora||_F since X - X_ora = A^-1 (R_ora - R); mixed
  requests (BF16 pieces, then emulated FP64 nests where the pieces cannot certify tol) all reach
  tol = 1e-6 in FP64 terms; Y = X B solves A Y = B to within N s (A Y - B = -(I - A X) B).
* The arena budget is never exceeded; a request that can never fit is refused at submission.
"""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nn():
    from paper_2212_02406_gb300 import abi, build

    build.build()
    abi.lib()
    return abi


def _requests(count, seed=0, n_max=600):
    reqs = synth.request_stream(count, rate_per_s=1000.0, seed=seed, n_max=n_max, max_rhs=8)
    out = []
    for r in reqs:
        a, q, lam = synth.spd_spectrum(r.n, r.kappa, seed=r.seed)
        b = synth.rng(r.seed + 1).standard_normal((r.n, r.nrhs))
        out.append((r, np.ascontiguousarray(a), np.ascontiguousarray(b)))
    return out


def _dt(r):
    return "f32" if r.dtype == "f32" else "mixed_emu"


def _run(nn, reqs, max_active, arena_bytes=None, stagger=0.0):
    import torch

    need = max(nn.nn_server_request_bytes(r.n, r.nrhs, _dt(r)) for r, _, _ in reqs)
    arena = torch.empty(int(arena_bytes or 8 * need), dtype=torch.uint8, device="cuda")
    srv = nn.Server(arena, max_active=max_active, depth=2, tol=1e-6, max_nests=40)
    outs = {}
    try:
        for r, a, b in reqs:
            y = np.empty_like(b)
            x = np.empty_like(a)
            dt = _dt(r)
            assert srv.submit(r.rid, a, B=b, Y=y, X=x, dtype=dt, precond="trace") == nn.NN_OK
            outs[r.rid] = (x, y)
            if stagger:
                time.sleep(stagger)
        assert srv.wait_idle(300.0) == nn.NN_OK
        comps = {c["id"]: c for c in srv.poll(1024)}
        stats = srv.stats()
    finally:
        srv.close()
    return outs, comps, stats, arena.numel()


def test_alone_equals_mix(nn):
    reqs = _requests(10, seed=1)
    alone, comps1, _, _ = _run(nn, reqs, max_active=1)
    mixed, comps2, _, _ = _run(nn, reqs, max_active=4, stagger=0.002)
    for r, a, b in reqs:
        assert comps1[r.rid]["status"] == comps2[r.rid]["status"]
        assert comps1[r.rid]["nests"] == comps2[r.rid]["nests"]
        xa, ya = alone[r.rid]
        xm, ym = mixed[r.rid]
        assert np.array_equal(xa, xm) and np.array_equal(ya, ym), r.rid


def test_results_are_correct(nn):
    from oracle import dense

    reqs = _requests(8, seed=2)
    outs, comps, _, _ = _run(nn, reqs, max_active=3)
    tol = 1e-6
    for r, a, b in reqs:
        c = comps[r.rid]
        x, y = outs[r.rid]
        r_gpu = dense.residual(a, x)
        s64 = dense.rms_frob(r_gpu)
        if r.dtype == "f32":
            assert c["status"] in (nn.NN_OK, nn.NN_ERR_NOT_CONVERGED), c
            assert s64 < 1e-4, (r.rid, r.n, r.kappa, s64, c)
        else:
            # mixed requests reach tol: the certified residual, and the FP64 one
            assert c["status"] == nn.NN_OK, (r.rid, r.n, r.kappa, c)
            assert c["residual"] < tol and s64 < tol, (r.rid, r.n, r.kappa, s64, c)
        # the oracle's iterate after the same nests from the same X_0 (lambda_min = 1: ||A^-1||_2 = 1)
        ora = dense.nn_invert(a, dense.precond_trace(a), 2, tol=0.0, max_nests=c["nests"])
        r_ora = dense.residual(a, ora.x)
        assert np.linalg.norm(x - ora.x) <= np.linalg.norm(r_gpu - r_ora) * (1 + 1e-9) + 1e-12, r.rid
        # A Y - B = -(I - A X) B, so the solve's relative residual is at most ||I - A X||_F = N s
        rel = np.linalg.norm(a @ y - b) / np.linalg.norm(b)
        assert rel <= r.n * s64 * 1.01 + 1e-12, (rel, s64)
        assert np.allclose(y, x @ b, rtol=1e-10, atol=1e-12 * np.abs(y).max())
        assert c["t_submit"] <= c["t_start"] <= c["t_done"]


def test_budget_respected_and_oversize_refused(nn):
    import torch

    reqs = _requests(6, seed=3, n_max=300)
    sizes = [nn.nn_server_request_bytes(r.n, r.nrhs, _dt(r)) for r, _, _ in reqs]
    budget = int(max(sizes) * 1.5)
    outs, comps, stats, cap = _run(nn, reqs, max_active=4, arena_bytes=budget)
    assert len(comps) == len(reqs)
    assert stats["arena_peak"] <= cap and stats["arena_used"] == 0
    arena = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    srv = nn.Server(arena, max_active=1)
    try:
        a = np.eye(512)
        assert srv.submit(99, a, dtype="f64") == nn.NN_ERR_OOM_BUDGET
    finally:
        srv.close()
