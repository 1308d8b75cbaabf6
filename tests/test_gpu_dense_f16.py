"""GPU parity of the dense mixed chain with FP16 operand pieces (NN_MIXED_F16) against the FP64
oracle, and the properties its power-of-two scaling must keep.

The chain is the BF16-piece chain of test_gpu_dense.py with FP16 pieces (11 significant bits
instead of 8) at exact power-of-two scales: A per row, X_k from ||X_k||_F, R and T at 2^12.
The tolerances are the same as there (module docstring of test_gpu_dense.py): the reported
s against an FP64 re-evaluation of the returned X within e_acc(N), the forward error within
2 sqrt(N) s + 16 kappa u32, the certified estimate covering the FP64 residual.
"""
import math

import numpy as np
import pytest

import synth
from oracle import dense

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def nn():
    import torch  # noqa: F401

    from paper_2212_02406_gb300 import abi, build

    build.build()
    abi.lib()
    return abi


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def e_acc(n):
    return 4 * U32 * (1 + math.sqrt(n) / 4)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(nn, a_np, x0_np, depth, tol, max_nests, dtype, **kw):
    import torch

    n = a_np.shape[0]
    A = _dev(a_np)
    X0 = _dev(x0_np)
    X = torch.empty_like(A)
    ws = nn.workspace(n, dtype)
    st, res = nn.nn_invert(A, X0, nn.make_opts(depth, tol, max_nests, dtype, **kw), X, ws)
    torch.cuda.synchronize()
    return st, res, X.cpu().numpy()


@pytest.mark.parametrize("n", [128, 300, 512])
@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("hint", [False, True])
def test_f16_converges_and_matches(nn, n, depth, hint):
    kappa = 1e2
    a, q, lam = synth.spd_spectrum(n, kappa, seed=n + depth)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    st, res, x = _run(nn, a, x0, depth, 1e-6, 40, "mixed_f16", x0_scalar=alpha if hint else 0.0)
    assert st == nn.NN_OK, res
    assert res["residual"] < 1e-6
    s64 = dense.rms_frob(dense.residual(a, x))
    assert abs(s64 - res["residual"]) <= e_acc(n)
    assert s64 < 1e-6
    assert res["residual_est"] < 1e-6 and s64 <= 1.5 * res["residual_est"]
    inv = np.linalg.inv(a)
    assert _rel(x, inv) <= 2 * math.sqrt(n) * s64 + 16 * kappa * U32
    ora = dense.nn_invert(a, x0, depth, tol=1e-6, max_nests=40)
    assert abs(res["nests"] - ora.nests) <= 1


@pytest.mark.parametrize("n,kappa", [(1024, 1e3), (2048, 1e2), (2048, 1e3)])
def test_f16_stop_is_certified(nn, n, kappa):
    # as for the BF16 pieces: NN_OK only when the FP64 residual of the returned X meets tol; a
    # tol under the floor ends NN_ERR_NOT_CONVERGED with an honest estimate
    a, q, lam = synth.spd_spectrum(n, kappa, seed=n + int(kappa) + 5)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    for tol in (1e-5, 1e-6, 3e-7, 1e-7):
        st, res, x = _run(nn, a, x0, 2, tol, 40, "mixed_f16", x0_scalar=alpha)
        s64 = dense.rms_frob(dense.residual(a, x))
        assert st in (nn.NN_OK, nn.NN_ERR_NOT_CONVERGED), res
        assert s64 <= 1.5 * res["residual_est"], (tol, s64, res["residual_est"])
        if st == nn.NN_OK:
            assert res["residual_est"] < tol and s64 < tol, (tol, s64, res)
        else:
            assert res["residual_est"] >= 0.5 * tol, (tol, res)


@pytest.mark.parametrize("k", [-20, 20])
@pytest.mark.parametrize("dtype", ["mixed_f16", "mixed_bf16"])
def test_power_of_two_scaling_is_exact(nn, k, dtype):
    # A -> 2^k A, X_0 -> 2^-k X_0: every piece scale moves by the same power of two, so the FP16
    # chain must return exactly 2^-k X with the same residual history (2^20 A would overflow
    # unscaled FP16 pieces, 2^-20 X_0 would underflow them). The BF16 chain keeps the same
    # property through its exponent range.
    n = 300
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=29)
    alpha = 2.0 / (lam[0] + lam[-1])
    c = 2.0 ** k
    for hint in (False, True):
        st1, res1, x1 = _run(nn, a, dense.precond_scalar(n, alpha), 2, 1e-6, 40, dtype,
                             x0_scalar=alpha if hint else 0.0)
        st2, res2, x2 = _run(nn, a * c, dense.precond_scalar(n, alpha / c), 2, 1e-6, 40, dtype,
                             x0_scalar=alpha / c if hint else 0.0)
        assert st1 == st2 == nn.NN_OK
        assert res1["history"] == res2["history"] and res1["pieces"] == res2["pieces"]
        assert np.array_equal(x1, x2 * c)


def test_f16_takes_no_more_passes_than_bf16(nn):
    # FP16 pieces lower each level's floor, so for the same tol the chain never needs more
    # tensor-core passes than the BF16 one (here fewer: it stays at one piece a nest longer)
    n = 2048
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=3)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    st_b, res_b, _ = _run(nn, a, x0, 2, 1e-6, 40, "mixed_bf16", x0_scalar=alpha)
    st_h, res_h, x_h = _run(nn, a, x0, 2, 1e-6, 40, "mixed_f16", x0_scalar=alpha)
    assert st_b == st_h == nn.NN_OK
    assert res_h["nests"] <= res_b["nests"]
    assert res_h["hw_flops"] < res_b["hw_flops"], (res_h["pieces"], res_b["pieces"])
    assert dense.rms_frob(dense.residual(a, x_h)) < 1e-6


@pytest.mark.parametrize("n", [384, 2048, 2100])
def test_f16_host_calls_equal_device(nn, n):
    # host-buffer calls (panel-wise copy and split from N = 2048, each panel's row scales taken
    # as it arrives) must equal the device call bit for bit
    import torch

    a, q, lam = synth.spd_spectrum(n, 1e2, seed=n + 7)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    ws = nn.workspace(n, "mixed_f16", host=True)
    st1, res1, x1 = _run(nn, a, x0, 2, 1e-6, 40, "mixed_f16", x0_scalar=alpha)
    xh = np.full_like(a, np.nan)
    st2, res2 = nn.nn_invert_host_pc(np.ascontiguousarray(a), "scalar", alpha, nn.make_opts(2, 1e-6, 40, "mixed_f16"),
                                     xh, ws)
    torch.cuda.synchronize()
    assert st1 == st2 == nn.NN_OK
    assert res1["history"] == res2["history"]
    assert np.array_equal(x1, xh)
    st3, res3, x3 = _run(nn, a, x0, 2, 1e-6, 40, "mixed_f16")
    xh3 = np.full_like(a, np.nan)
    st4, res4 = nn.nn_invert_host(np.ascontiguousarray(a), np.ascontiguousarray(x0),
                                  nn.make_opts(2, 1e-6, 40, "mixed_f16"), xh3, ws)
    torch.cuda.synchronize()
    assert st3 == st4 == nn.NN_OK
    assert res3["history"] == res4["history"]
    assert np.array_equal(x3, xh3)


@pytest.mark.parametrize("n", [300, 1024])
@pytest.mark.parametrize("sched", [[1], [2], [3], [1, 2]])
@pytest.mark.parametrize("kappa", [1e2, 1e4])
def test_f16_scalar_hint_matches_explicit_x0(nn, n, sched, kappa):
    a, q, lam = synth.spd_spectrum(n, kappa, seed=int(n + kappa) % 997)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    kw = dict(depth_schedule=sched)
    st1, res1, x1 = _run(nn, a, x0, sched[-1], 1e-6, 40, "mixed_f16", **kw)
    st2, res2, x2 = _run(nn, a, x0, sched[-1], 1e-6, 40, "mixed_f16", x0_scalar=alpha, **kw)
    assert st1 == st2, (res1["history"], res2["history"])
    assert abs(res1["nests"] - res2["nests"]) <= 1
    ainv = (q / lam) @ q.T
    for x, res in ((x1, res1), (x2, res2)):
        s64 = dense.rms_frob(dense.residual(a, x))
        assert abs(s64 - res["residual"]) <= e_acc(n) * max(1.0, kappa / 1e2)
        if st2 == nn.NN_OK:
            assert _rel(x, ainv) <= 2 * math.sqrt(n) * s64 + 16 * kappa * U32
    s0 = dense.rms_frob(np.eye(n) - alpha * a)
    assert abs(res2["history"][0] - s0) <= 1e-6 * s0


@pytest.mark.parametrize("bulk", [1, 2, 3, 4])
def test_f16_every_start_level(nn, bulk):
    n = 300
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=17)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    st1, res1, x1 = _run(nn, a, x0, 2, 1e-6, 40, "mixed_f16", bulk_pieces=bulk)
    st2, res2, x2 = _run(nn, a, x0, 2, 1e-6, 40, "mixed_f16", bulk_pieces=bulk, x0_scalar=alpha)
    assert st1 == st2 == nn.NN_OK
    for x in (x1, x2):
        assert dense.rms_frob(dense.residual(a, x)) < 1e-6 + e_acc(n)


def test_f16_divergence_reported(nn):
    n = 128
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=9)
    x0 = dense.precond_scalar(n, 2.5 / lam[-1])  # rho(R_0) = 1.5
    st, res, _ = _run(nn, a, x0, 2, 1e-8, 30, "mixed_f16")
    assert st == nn.NN_ERR_DIVERGED and res["status"] == nn.NN_ERR_DIVERGED


def test_f16_kappa_1e4_does_not_diverge(nn):
    n = 512
    a, q, lam = synth.spd_spectrum(n, 1e4, seed=5)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    st, res, x = _run(nn, a, x0, 2, 1e-6, 20, "mixed_f16")
    assert st in (nn.NN_OK, nn.NN_ERR_NOT_CONVERGED), res
    s64 = dense.rms_frob(dense.residual(a, x))
    assert s64 < 1e-4
    assert abs(s64 - res["residual"]) <= e_acc(n) * 1e2


def test_f16_general_matrix_pan_schreiber(nn):
    # a nonsymmetric, non-normal A from the Pan-Schreiber start (Section II-A): rows of very
    # different scales exercise the per-row piece scales of A
    n = 256
    rng = synth.rng(77)
    a = np.eye(n) * 4.0 + rng.standard_normal((n, n)) / math.sqrt(n)
    a *= np.exp(rng.uniform(-2, 2, size=(n, 1)))  # row scales over about 2^6
    x0 = dense.precond_pan_schreiber(a)
    tol = 1e-5
    st, res, x = _run(nn, a, x0, 2, tol, 60, "mixed_f16")
    ora = dense.nn_invert(a, x0, 2, tol=tol, max_nests=60)
    assert st == nn.NN_OK and ora.status == 0, (res["history"], ora.history)
    s64 = dense.rms_frob(dense.residual(a, x))
    assert s64 < tol and s64 <= 1.5 * res["residual_est"]
    assert abs(res["nests"] - ora.nests) <= 1
