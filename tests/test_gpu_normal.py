"""GPU parity of general (non-Hermitian, real or complex) solves through the normal equations
(Corollary 3) against the oracle's nn_normal_solve.

Both sides form W = A^H A, start from I / Tr(W) and run the same FP64 iteration; they differ by
rounding order only. The normal equations amplify rounding by cond(W) = cond(A)^2, so the
solution tolerance is c cond(A)^2 u, and the W-residual history agrees to 1e-8 relative above
the FP64 floor.
"""
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


def _solve(nn, a, b, depth, tol, max_nests, dtype="f64"):
    import torch

    A = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    B = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    X = torch.empty_like(B)
    ws = nn.normal_workspace(a.shape[0], b.shape[1], np.iscomplexobj(a), dtype)
    st, res = nn.nn_solve_normal(A, B, nn.make_opts(depth, tol, max_nests, dtype), X, ws)
    torch.cuda.synchronize()
    return st, res, X.cpu().numpy()


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n", [1, 48, 100, 257])
@pytest.mark.parametrize("depth", [1, 2])
def test_normal_solve_matches_oracle(nn, complex_, n, depth):
    cond = 30.0
    a, _ = synth.general_svd(n, cond, seed=n + depth, complex_=complex_)
    b = synth.gaussian_rhs(n, 3, seed=2)
    if complex_:
        b = b + 1j * synth.gaussian_rhs(n, 3, seed=3)
    tol = 1e-10
    st, res, x = _solve(nn, a, b, depth, tol, 60)
    want, run = dense.nn_normal_solve(a, b, depth, tol, 60)
    assert st == nn.NN_OK and run.status == dense.STATUS_OK
    assert res["nests"] == run.nests
    floor = 64 * cond ** 2 * U64
    for s_gpu, s_cpu in zip(res["history"], run.history):
        assert abs(s_gpu - s_cpu) <= 1e-8 * s_cpu + floor
    err = np.linalg.norm(x - want) / np.linalg.norm(want)
    assert err <= 16 * floor, err


def test_normal_solve_badly_conditioned_matches_library(nn):
    # cond(A) = 1e3, cond(W) = 1e6 in FP64: the solution agrees with numpy.linalg.solve within
    # the normal equations' error bound c cond(A)^2 u plus n times the final W residual
    n, cond = 160, 1e3
    a, _ = synth.general_svd(n, cond, seed=31)
    b = synth.gaussian_rhs(n, 2, seed=32)
    st, res, x = _solve(nn, a, b, 2, 1e-12, 64)
    # tol 1e-12 lies below W's FP64 residual floor (about u cond(W)): the run may end capped
    assert st in (nn.NN_OK, nn.NN_ERR_NOT_CONVERGED)
    true = np.linalg.solve(a, b)
    err = np.linalg.norm(x - true) / np.linalg.norm(true)
    assert err <= 64 * cond ** 2 * U64 + n * res["residual"]


@pytest.mark.parametrize("dtype", ["mixed_bf16", "mixed_f16"])
def test_normal_solve_mixed_precision_runs_to_its_floor(nn, dtype):
    # the mixed chains on W (cond(W) = 100): converge to tol 1e-5 and solve to about n tol
    n, cond = 256, 10.0
    a, _ = synth.general_svd(n, cond, seed=41)
    b = synth.gaussian_rhs(n, 1, seed=42)
    st, res, x = _solve(nn, a, b, 2, 1e-5, 40, dtype=dtype)
    assert st == nn.NN_OK and res["residual"] < 1e-5
    true = np.linalg.solve(a, b)
    assert np.linalg.norm(x - true) / np.linalg.norm(true) <= n * 2e-5


def test_normal_solve_argument_errors(nn):
    import torch

    a = torch.eye(4, dtype=torch.float64, device="cuda")
    b = torch.ones(4, 1, dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    ws = nn.normal_workspace(4, 1, False, "f64")
    small = ws[: ws.numel() // 2]
    st, _ = nn.nn_solve_normal(a, b, nn.make_opts(2, 1e-10, 10, "f64"), x, small)
    assert st == nn.NN_ERR_OOM_BUDGET
    st, _ = nn.nn_solve_normal(a, b, nn.make_opts(0, 1e-10, 10, "f64"), x, ws)
    assert st == nn.NN_ERR_ARG
    st, res = nn.nn_solve_normal(a, b, nn.make_opts(2, 1e-10, 10, "f64"), x, ws)
    assert st == nn.NN_OK and np.allclose(x.cpu().numpy(), 1.0, rtol=1e-12)
