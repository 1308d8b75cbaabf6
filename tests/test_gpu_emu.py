"""FP64 products emulated on the BF16 tensor cores with exact slices (NN_F64_EMU).

The emulated product must match FP64: the residual of arbitrary (not inverse) pairs to a
few units of 2^-53 relative, and the whole NN chain must follow the FP64 oracle nest for
nest (same stop, history to 1e-8 above the FP64 floor), including at cond = 1e4 where the
mixed BF16 chain stops at its floor.
"""
import math

import numpy as np
import pytest

import synth
from oracle import dense

pytestmark = pytest.mark.gpu
U64 = np.finfo(np.float64).eps / 2


@pytest.fixture(scope="module")
def nn():
    from paper_2212_02406_gb300 import abi, build

    build.build()
    abi.lib()
    return abi


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [1, 7, 256, 300, 1000])
def test_emulated_residual_matches_fp64(nn, n):
    # I - A X for random A, X: the result is O(1), so the emulated product's error shows directly
    r = synth.rng(n)
    a = r.standard_normal((n, n))
    x = r.standard_normal((n, n)) / n
    x[::3] *= 1e-3          # rows of different scales
    want = np.linalg.norm(np.eye(n) - a @ x) / n
    ws = nn.workspace(n, "f64_emu")
    st, s = nn.nn_residual(_dev(a), _dev(x), "f64_emu", ws)
    assert st == nn.NN_OK
    assert abs(s - want) <= 64 * U64 * want * math.sqrt(n) + 1e-300


@pytest.mark.parametrize("n,kappa", [(256, 1e2), (257, 1e2), (600, 1e4)])
def test_emulated_chain_matches_fp64_oracle(nn, n, kappa):
    import torch

    a, q, lam = synth.spd_spectrum(n, kappa, seed=n)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    tol = 1e-11
    A, X0 = _dev(a), _dev(x0)
    X = torch.empty_like(A)
    ws = nn.workspace(n, "f64_emu")
    st, res = nn.nn_invert(A, X0, nn.make_opts(2, tol, 40, "f64_emu"), X, ws)
    torch.cuda.synchronize()
    run = dense.nn_invert(a, x0, 2, tol, 40)
    assert st == nn.NN_OK and run.status == dense.STATUS_OK
    assert res["nests"] == run.nests
    floor = 50 * kappa * U64
    for s_gpu, s_cpu in zip(res["history"], run.history):
        assert abs(s_gpu - s_cpu) <= 1e-8 * s_cpu + floor
    x = X.cpu().numpy()
    assert np.linalg.norm(x - run.x) <= 100 * kappa * U64 * np.linalg.norm(run.x) * math.sqrt(n)


def test_emulated_chain_reaches_1e10_at_kappa_1e4(nn):
    # where the mixed BF16 chain stops at its arithmetic floor, the emulated FP64 chain goes on
    import torch

    n, kappa = 1024, 1e4
    a, q, lam = synth.spd_spectrum(n, kappa, seed=5)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    A, X0 = _dev(a), _dev(x0)
    X = torch.empty_like(A)
    ws = nn.workspace(n, "f64_emu")
    st, res = nn.nn_invert(A, X0, nn.make_opts(2, 1e-10, 40, "f64_emu"), X, ws)
    torch.cuda.synchronize()
    assert st == nn.NN_OK and res["residual"] < 1e-10
    r = np.eye(n) - a @ X.cpu().numpy()
    assert np.linalg.norm(r) / n < 2e-10


def test_emulated_normal_equations(nn):
    # general solve with W = A^T A formed and inverted with emulated FP64 products
    import torch

    n, cond = 300, 1e3
    a, _ = synth.general_svd(n, cond, seed=3)
    b = synth.gaussian_rhs(n, 2, seed=4)
    A, B = _dev(a), _dev(b)
    X = torch.empty_like(B)
    ws = nn.normal_workspace(n, 2, False, "f64_emu")
    st, res = nn.nn_solve_normal(A, B, nn.make_opts(2, 1e-11, 64, "f64_emu"), X, ws)
    torch.cuda.synchronize()
    assert st in (nn.NN_OK, nn.NN_ERR_NOT_CONVERGED)
    true = np.linalg.solve(a, b)
    err = np.linalg.norm(X.cpu().numpy() - true) / np.linalg.norm(true)
    assert err <= 64 * cond ** 2 * U64 + n * res["residual"]


@pytest.mark.parametrize("n,kappa,tol", [(1024, 1e4, 1e-10), (1024, 1e2, 1e-12), (300, 1e3, 1e-11)])
def test_mixed_then_emulated_reaches_fp64_tolerances(nn, n, kappa, tol):
    # NN_MIXED_EMU: BF16-piece nests until the iterate nears their floor, then emulated FP64
    # nests from it; the returned X meets tolerances the mixed chain alone cannot reach
    import torch

    a, q, lam = synth.spd_spectrum(n, kappa, seed=int(kappa) + n)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    A, X0 = _dev(a), _dev(x0)
    X = torch.empty_like(A)
    ws = nn.workspace(n, "mixed_emu")
    st, res = nn.nn_invert(A, X0, nn.make_opts(2, tol, 40, "mixed_emu"), X, ws)
    torch.cuda.synchronize()
    assert st == nn.NN_OK and res["residual"] < tol
    assert res["pieces"][0] >= 1 and res["pieces"][res["nests"]] == 0  # both stages ran
    r = np.eye(n) - a @ X.cpu().numpy()
    assert np.linalg.norm(r) / n < 2 * tol
    # the history decreases through the handoff and matches the nest count bookkeeping
    assert len(res["history"]) == res["nests"] + 1


def test_mixed_emu_equals_mixed_when_tol_is_reachable(nn):
    # a tolerance the BF16 pieces reach: no handoff, bit-for-bit the mixed chain
    import torch

    n = 512
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=77)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    out = {}
    for dt in ("mixed_bf16", "mixed_emu"):
        A, X0 = _dev(a), _dev(x0)
        X = torch.empty_like(A)
        st, res = nn.nn_invert(A, X0, nn.make_opts(2, 1e-4, 40, dt), X, nn.workspace(n, dt))
        torch.cuda.synchronize()
        out[dt] = (st, res, X.cpu().numpy())
    assert out["mixed_bf16"][0] == out["mixed_emu"][0] == nn.NN_OK
    assert out["mixed_bf16"][1]["nests"] == out["mixed_emu"][1]["nests"]
    assert np.array_equal(out["mixed_bf16"][2], out["mixed_emu"][2])


@pytest.mark.parametrize("n,kappa", [(1024, 1e2), (2048, 1e2), (1024, 1e4), (2048, 1e4)])
def test_refined_result_within_1e6_of_oracle(nn, n, kappa):
    # The refined mode (NN_MIXED_EMU with a forward-error target): BF16-piece nests, then
    # emulated FP64 nests, stopping at N s_k < fwd_tol, which bounds ||X - A^-1||_F / ||A^-1||_F
    # (X - A^-1 = -A^-1 R and ||A^-1||_2 <= ||A^-1||_F). The FP64 oracle runs the same NN
    # (Algorithm 1, depth 2, same X_0) to its own floor; the returned X must lie within 1e-6 of
    # it, relatively, in the Frobenius norm (Section II's error measure against the solution).
    import torch

    a, q, lam = synth.spd_spectrum(n, kappa, seed=n + int(kappa))
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    ora = dense.nn_invert(a, x0, 2, tol=1e-13, max_nests=40)
    A, X0 = _dev(a), _dev(x0)
    X = torch.empty_like(A)
    ws = nn.workspace(n, "mixed_emu")
    opts = nn.make_opts(2, 0.0, 40, "mixed_emu", x0_scalar=alpha, fwd_tol=1e-6)
    st, res = nn.nn_invert(A, X0, opts, X, ws)
    torch.cuda.synchronize()
    assert st == nn.NN_OK, res
    assert n * res["residual"] < 1e-6
    assert res["pieces"][0] >= 1 and res["pieces"][res["nests"]] == 0  # both stages ran
    x = X.cpu().numpy()
    err = np.linalg.norm(x - ora.x) / np.linalg.norm(ora.x)
    assert err <= 1e-6, err
    # the residual the call reports is the FP64 residual of the returned X
    s64 = dense.rms_frob(dense.residual(a, x))
    assert abs(res["residual"] - s64) <= 1e-3 * s64 + 64 * U64 * math.sqrt(n), (res["residual"], s64)
