"""GPU parity of the dense NN path (C ABI) against the FP64 CPU oracle.

Tolerances (derived from the arithmetic):
* FP64 chain vs FP64 oracle after the same nests: both follow the same exact sequence;
  they differ only by rounding, which the self-correcting iteration keeps at the level
  of the conditioning floor: ||X_gpu - X_ora||_F / ||X_ora||_F <= max(1e-12, 16 kappa u64 sqrt(N)).
* FP32 chain: the same with u32 (and kappa u32 for the converged iterate).
* Mixed BF16 tensor-core chain: the accepted residual is evaluated from three BF16 pieces
  per operand (products exact to ~2^-24) but summed by the tensor core in FP32, whose
  rounding over N/16 accumulator updates bounds the reported s against an FP64
  re-evaluation of the returned X by e_acc(N) = 4 u32 (1 + sqrt(N)/4) (the diagonal terms
  drift from 0 to 1, so a per-update error of u32 gives at most u32 N/16 per diagonal entry,
  u32 sqrt(N)/16 in rms). The forward error then follows from X - A^-1 = -A^-1 R:
  ||X - A^-1||_F / ||A^-1||_F <= 2 sqrt(N) s + 16 kappa u32 (the last term is the FP32
  storage of X and the piece representation of A).
"""
import math

import numpy as np
import pytest

import synth
from oracle import dense

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
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
    """Bound on |reported s - FP64 re-evaluation| for the mixed chain (module docstring)."""
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


@pytest.mark.parametrize("kind", ["pan_schreiber", "trace", "scalar", "jacobi", "theta2"])
@pytest.mark.parametrize("n", [1, 17, 256, 257])
def test_precond_parity(nn, kind, n):
    import torch

    a = synth.spd_wishart(n, seed=n)
    A = _dev(a)
    X0 = torch.empty_like(A)
    ws = nn.workspace(n, "f64")
    scalar = {"scalar": 0.37, "theta2": 8}.get(kind, 1.0)
    st = nn.nn_init_precond(A, kind, scalar, X0, ws)
    torch.cuda.synchronize()
    assert st == nn.NN_OK
    want = {"pan_schreiber": dense.precond_pan_schreiber(a), "trace": dense.precond_trace(a),
            "scalar": dense.precond_scalar(n, 0.37), "jacobi": dense.precond_jacobi(a),
            "theta2": dense.precond_theta2(a, 8, np.ones(n))}[kind]
    got = X0.cpu().numpy()
    assert np.allclose(got, want, rtol=1e-14 * max(1, n), atol=0)


@pytest.mark.parametrize("depth,nests_expected", [(1, 15), (2, 10), (3, 8)])
def test_f64_wishart256_matches_oracle(nn, depth, nests_expected):
    # N = 256, A = B B^T / N + 0.5 I, Pan-Schreiber X_0, tol 1e-10.
    a = synth.spd_wishart(256, seed=0)
    x0 = dense.precond_pan_schreiber(a)
    ora = dense.nn_invert(a, x0, depth, tol=1e-10, max_nests=64)
    st, res, x = _run(nn, a, x0, depth, 1e-10, 64, "f64")
    assert st == nn.NN_OK and res["status"] == nn.NN_OK
    assert res["nests"] == ora.nests == nests_expected
    kappa = np.linalg.cond(a)
    tol = max(1e-12, 16 * kappa * U64 * math.sqrt(256))
    assert _rel(x, ora.x) <= tol
    for s_gpu, s_ora in zip(res["history"], ora.history):
        assert abs(s_gpu - s_ora) <= 1e-9 * s_ora + 1e-15
    assert res["gemms"] == (depth + 1) * res["nests"] + 1


@pytest.mark.parametrize("n", [1, 2, 17, 63, 65, 255, 257])
@pytest.mark.parametrize("depth", [1, 2, 3])
def test_f64_ragged_sizes_fixed_nests(nn, n, depth):
    a = synth.spd_wishart(n, seed=100 + n)
    x0 = dense.precond_trace(a)
    nests = 4
    ora = dense.nn_invert(a, x0, depth, tol=0.0, max_nests=nests)
    st, res, x = _run(nn, a, x0, depth, 0.0, nests, "f64")
    assert st == nn.NN_OK and res["nests"] == nests
    assert _rel(x, ora.x) <= max(1e-12, 16 * np.linalg.cond(a) * U64 * math.sqrt(n))


def test_theta2_start_speeds_up_convergence(nn):
    # Theta_2 normalises by an estimate of lambda_max instead of the trace: fewer nests, same answer
    import torch

    n = 300
    a, q, lam = synth.spd_spectrum(n, 1e3, seed=12)
    A = _dev(a)
    ws = nn.workspace(n, "f64")
    nests = {}
    for kind, scalar in (("trace", 1.0), ("theta2", 8)):
        X0 = torch.empty_like(A)
        assert nn.nn_init_precond(A, kind, scalar, X0, ws) == nn.NN_OK
        st, res, x = _run(nn, a, X0.cpu().numpy(), 2, 1e-10, 64, "f64")
        assert st == nn.NN_OK
        ora = dense.nn_invert(a, X0.cpu().numpy(), 2, tol=1e-10, max_nests=64)
        assert res["nests"] == ora.nests
        nests[kind] = res["nests"]
    assert nests["theta2"] < nests["trace"]


def test_f64_zero_nests_returns_x0(nn):
    a = synth.spd_wishart(33, seed=3)
    x0 = dense.precond_trace(a)
    st, res, x = _run(nn, a, x0, 2, 0.0, 0, "f64")
    assert st == nn.NN_OK and res["nests"] == 0 and np.array_equal(x, x0)
    assert abs(res["residual"] - dense.rms_frob(dense.residual(a, x0))) <= 1e-13


@pytest.mark.parametrize("dtype", ["f64", "f32", "mixed_bf16"])
def test_divergence_reported(nn, dtype):
    n = 128
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=9)
    x0 = dense.precond_scalar(n, 2.5 / lam[-1])  # 1 - 2.5 = -1.5: rho(R_0) > 1
    st, res, _ = _run(nn, a, x0, 2, 1e-8, 30, dtype)
    assert st == nn.NN_ERR_DIVERGED and res["status"] == nn.NN_ERR_DIVERGED


def test_not_converged_status(nn):
    a = synth.spd_wishart(64, seed=5)
    st, res, _ = _run(nn, a, dense.precond_trace(a), 1, 1e-300, 2, "f64")
    assert st == nn.NN_ERR_NOT_CONVERGED and res["nests"] == 2


@pytest.mark.parametrize("n", [96, 200])
@pytest.mark.parametrize("depth", [1, 2])
def test_f32_chain(nn, n, depth):
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=n)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    ora = dense.nn_invert(a, x0, depth, tol=1e-6, max_nests=40)
    st, res, x = _run(nn, a, x0, depth, 1e-6, 40, "f32")
    assert st == nn.NN_OK
    assert abs(res["nests"] - ora.nests) <= 1
    inv = np.linalg.inv(a)
    # converged FP32 iterate: forward error ~ kappa u32 sqrt(N) plus sqrt(N) * tol
    assert _rel(x, inv) <= 64 * 1e2 * U32 * math.sqrt(n) + 4 * math.sqrt(n) * 1e-6


@pytest.mark.parametrize("n", [128, 300, 512])
@pytest.mark.parametrize("depth", [1, 2, 3])
def test_mixed_bf16_converges_and_matches(nn, n, depth):
    kappa = 1e2
    a, q, lam = synth.spd_spectrum(n, kappa, seed=n + depth)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    st, res, x = _run(nn, a, x0, depth, 1e-6, 40, "mixed_bf16")
    assert st == nn.NN_OK, res
    assert res["residual"] < 1e-6
    assert res["pieces"][-1] == 3  # the accepted residual was measured at FP32-level accuracy
    # the reported residual agrees with an independent FP64 evaluation of the returned X
    s64 = dense.rms_frob(dense.residual(a, x))
    assert abs(s64 - res["residual"]) <= e_acc(n)
    assert s64 < 1e-6
    # the certified residual (measured value with the arithmetic's floor) covers the truth
    assert res["residual_est"] < 1e-6 and s64 <= 1.5 * res["residual_est"]
    # forward error against the library inverse: residual floor + FP32 rounding of A
    inv = np.linalg.inv(a)
    assert _rel(x, inv) <= 2 * math.sqrt(n) * s64 + 16 * kappa * U32
    # the oracle run to the same tol lands on an iterate equally close
    ora = dense.nn_invert(a, x0, depth, tol=1e-6, max_nests=40)
    assert abs(res["nests"] - ora.nests) <= 1


@pytest.mark.parametrize("n", [128, 256])
def test_mixed_matches_oracle_within_1e6(nn, n):
    # Relative error against the FP64 oracle's converged inverse, at sizes where the FP32
    # accumulation floor keeps sqrt(N) s below the 1e-6 target.
    kappa, depth = 1e2, 2
    a, q, lam = synth.spd_spectrum(n, kappa, seed=11)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    st, res, x = _run(nn, a, x0, depth, 1e-7, 12, "mixed_bf16")
    assert st in (nn.NN_OK, nn.NN_ERR_NOT_CONVERGED), res
    ora = dense.nn_invert(a, x0, depth, tol=1e-13, max_nests=40)
    assert _rel(x, ora.x) <= 1e-6


@pytest.mark.parametrize("n,kappa", [(1024, 1e3), (2048, 1e2), (2048, 1e3)])
def test_mixed_stop_is_certified(nn, n, kappa):
    # The chain converges to the X whose measured (BF16-piece, FP32-accumulated) residual
    # vanishes, so a measured s falls below the truth by about the arithmetic's floor. A stop
    # must pass the certified estimate, residual_est = sqrt(s^2 + e^2): whenever the call reports
    # NN_OK the FP64 residual of the returned X meets tol, and a tol under the floor ends
    # NN_ERR_NOT_CONVERGED with an honest estimate.
    a, q, lam = synth.spd_spectrum(n, kappa, seed=n + int(kappa) + 5)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    for tol in (1e-5, 1e-6, 3e-7):
        st, res, x = _run(nn, a, x0, 2, tol, 40, "mixed_bf16", x0_scalar=alpha)
        s64 = dense.rms_frob(dense.residual(a, x))
        assert st in (nn.NN_OK, nn.NN_ERR_NOT_CONVERGED), res
        assert s64 <= 1.5 * res["residual_est"], (tol, s64, res["residual_est"])
        if st == nn.NN_OK:
            assert res["residual_est"] < tol and s64 < tol, (tol, s64, res)
        else:
            assert res["residual_est"] >= 0.5 * tol, (tol, res)


def test_mixed_kappa_1e4_does_not_diverge(nn):
    # kappa = 1e4 needs more than FP32-level arithmetic to reach 1e-6; the level schedule must
    # still converge to its floor without diverging, and report the floor honestly.
    n = 512
    a, q, lam = synth.spd_spectrum(n, 1e4, seed=5)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    st, res, x = _run(nn, a, x0, 2, 1e-6, 20, "mixed_bf16")
    assert st in (nn.NN_OK, nn.NN_ERR_NOT_CONVERGED), res
    s64 = dense.rms_frob(dense.residual(a, x))
    assert s64 < 1e-4
    assert abs(s64 - res["residual"]) <= e_acc(n) * 1e2  # floor scales with |A||X| ~ kappa


def test_host_variant_equals_device_variant(nn):
    import torch

    n = 160
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=2)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    for dtype in ("f64", "mixed_bf16"):
        st1, res1, x1 = _run(nn, a, x0, 2, 1e-7, 30, dtype)
        xh = np.empty_like(a)
        ws = nn.workspace(n, dtype, host=True)
        st2, res2 = nn.nn_invert_host(np.ascontiguousarray(a), np.ascontiguousarray(x0),
                                      nn.make_opts(2, 1e-7, 30, dtype), xh, ws)
        torch.cuda.synchronize()
        assert st1 == st2 == nn.NN_OK
        assert res1["nests"] == res2["nests"]
        assert np.array_equal(x1, xh)


@pytest.mark.parametrize("tol", [1e-4, 1e-6, 1e-7])
@pytest.mark.parametrize("kappa", [1e1, 1e2, 1e3])
def test_host_pc_variant_and_early_copy_equal_device(nn, tol, kappa):
    # nn_invert_host_pc builds X_0 on the device; for the mixed chain the likely-final iterate is
    # copied to the host on a side stream while its residual runs. Either way the host result
    # must equal the device call's bit for bit, whether or not the prediction held.
    import torch

    n = 384
    a, q, lam = synth.spd_spectrum(n, kappa, seed=int(kappa) + 3)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    for dtype in ("mixed_bf16", "f64"):
        # the host call passes the scalar preconditioner to the chain as the X_0 = alpha I hint
        st1, res1, x1 = _run(nn, a, x0, 2, tol, 40, dtype, x0_scalar=alpha)
        xh = np.full_like(a, np.nan)
        ws = nn.workspace(n, dtype, host=True)
        st2, res2 = nn.nn_invert_host_pc(np.ascontiguousarray(a), "scalar", alpha, nn.make_opts(2, tol, 40, dtype),
                                         xh, ws)
        torch.cuda.synchronize()
        assert st1 == st2
        assert res1["nests"] == res2["nests"] and res1["history"] == res2["history"]
        assert np.array_equal(x1, xh)


@pytest.mark.parametrize("n", [2048, 2100])
def test_host_panel_split_equals_device(nn, n):
    # From N = 2048 the host-buffer calls copy A in row panels on a copy stream and split each
    # panel as soon as it has arrived (the last panel includes the padding rows); the results
    # must equal the device calls bit for bit, with the scalar-X_0 hint and with an explicit X_0.
    import torch

    a, q, lam = synth.spd_spectrum(n, 1e2, seed=n)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    ws = nn.workspace(n, "mixed_bf16", host=True)
    st1, res1, x1 = _run(nn, a, x0, 2, 1e-6, 40, "mixed_bf16", x0_scalar=alpha)
    xh = np.full_like(a, np.nan)
    st2, res2 = nn.nn_invert_host_pc(np.ascontiguousarray(a), "scalar", alpha, nn.make_opts(2, 1e-6, 40, "mixed_bf16"),
                                     xh, ws)
    torch.cuda.synchronize()
    assert st1 == st2 == nn.NN_OK
    assert res1["history"] == res2["history"]
    assert np.array_equal(x1, xh)
    st3, res3, x3 = _run(nn, a, x0, 2, 1e-6, 40, "mixed_bf16")
    xh3 = np.full_like(a, np.nan)
    st4, res4 = nn.nn_invert_host(np.ascontiguousarray(a), np.ascontiguousarray(x0),
                                  nn.make_opts(2, 1e-6, 40, "mixed_bf16"), xh3, ws)
    torch.cuda.synchronize()
    assert st3 == st4 == nn.NN_OK
    assert res3["history"] == res4["history"]
    assert np.array_equal(x3, xh3)


@pytest.mark.parametrize("n,pad", [(300, 0), (300, 1), (517, 3), (1024, 0)])
@pytest.mark.parametrize("tol", [1e-5, 3e-7])
def test_device_early_copy_strided_output(nn, n, pad, tol):
    # For the mixed chain the iterate predicted to be returned is widened into the caller's X by
    # the confirming residual's epilogue (16-byte stores for an even leading dimension, element
    # stores otherwise, ragged last chunk). X must equal the host call's result bit for bit,
    # whether or not the prediction held, and the columns past n stay untouched.
    import torch

    a, q, lam = synth.spd_spectrum(n, 1e2, seed=n + pad)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    xf_dev = torch.full((n, n + pad), 7.0, dtype=torch.float64, device="cuda")
    X = xf_dev[:, :n]
    ws = nn.workspace(n, "mixed_bf16")
    st1, res1 = nn.nn_invert(_dev(a), _dev(x0), nn.make_opts(2, tol, 40, "mixed_bf16"), X, ws)
    torch.cuda.synchronize()
    xh = np.full_like(a, np.nan)
    st2, res2 = nn.nn_invert_host(np.ascontiguousarray(a), np.ascontiguousarray(x0),
                                  nn.make_opts(2, tol, 40, "mixed_bf16"), xh, nn.workspace(n, "mixed_bf16", host=True))
    assert st1 == st2 == nn.NN_OK
    assert res1["history"] == res2["history"]
    xf = xf_dev.cpu().numpy()
    assert np.array_equal(xf[:, :n], xh)
    assert np.all(xf[:, n:] == 7.0)


@pytest.mark.parametrize("n", [300, 1024])
@pytest.mark.parametrize("sched", [[1], [2], [3], [1, 2]])
@pytest.mark.parametrize("kappa", [1e2, 1e4])
def test_scalar_x0_hint_matches_explicit_x0(nn, n, sched, kappa):
    # With x0_scalar the mixed chain forms R_0 = I - alpha A element-wise (FP64) and X_1 =
    # alpha (I + T) in the epilogue of the first nest's last Horner product (depth 1: element-wise)
    # instead of by GEMMs. The iteration is the same; only rounding in the first nest differs, so
    # both runs must end in the same status, within one nest, and each must meet the
    # forward-error bound of the module docstring.
    a, q, lam = synth.spd_spectrum(n, kappa, seed=int(n + kappa) % 997)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    tol = 1e-6
    kw = dict(depth_schedule=sched)
    st1, res1, x1 = _run(nn, a, x0, sched[-1], tol, 40, "mixed_bf16", **kw)
    st2, res2, x2 = _run(nn, a, x0, sched[-1], tol, 40, "mixed_bf16", x0_scalar=alpha, **kw)
    assert st1 == st2, (res1["history"], res2["history"])
    assert abs(res1["nests"] - res2["nests"]) <= 1
    assert res2["gemms"] < res1["gemms"]
    ainv = (q / lam) @ q.T
    for x, res in ((x1, res1), (x2, res2)):
        s64 = dense.rms_frob(dense.residual(a, x))
        assert abs(s64 - res["residual"]) <= e_acc(n) * max(1.0, kappa / 1e2)
        if st2 == nn.NN_OK:
            assert _rel(x, ainv) <= 2 * math.sqrt(n) * s64 + 16 * kappa * U32
    # the first residual of the hinted run is the element-wise I - alpha A
    s0 = dense.rms_frob(np.eye(n) - alpha * a)
    assert abs(res2["history"][0] - s0) <= 1e-6 * s0


@pytest.mark.parametrize("bulk", [1, 2, 3, 4])
@pytest.mark.parametrize("depth", [1, 2])
def test_scalar_x0_first_residual_any_start_level(nn, bulk, depth):
    # With X_0 = alpha I the pass that splits A also writes R_0 = I - alpha A at the starting
    # level's piece count (opts.bulk_pieces); every starting level must give the element-wise s_0
    # and agree with the explicit-X_0 run's status.
    n = 300
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=17)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    st1, res1, x1 = _run(nn, a, x0, depth, 1e-6, 40, "mixed_bf16", bulk_pieces=bulk)
    st2, res2, x2 = _run(nn, a, x0, depth, 1e-6, 40, "mixed_bf16", bulk_pieces=bulk, x0_scalar=alpha)
    assert st1 == st2 == nn.NN_OK
    s0 = dense.rms_frob(np.eye(n) - alpha * a)
    assert abs(res2["history"][0] - s0) <= 1e-6 * s0
    s64 = dense.rms_frob(dense.residual(a, x2))
    assert s64 < 1e-6 + e_acc(n)


@pytest.mark.parametrize("refine", [1e-1, 1e-3])
@pytest.mark.parametrize("hint", [False, True])
def test_level_rise_at_measurement_regenerates_pieces(nn, refine, hint):
    # opts.refine_below raises the level to 3 once s sqrt(N) falls below it, a rise that the
    # per-nest prediction does not foresee: the iterate's BF16 pieces (written for the predicted
    # level only) are split again from its FP32 master before the residual reads them. The run
    # must converge, reach level 3, and report a residual that an FP64 re-evaluation confirms.
    n = 384
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=23)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    kw = dict(refine_below=refine, x0_scalar=alpha if hint else 0.0)
    st, res, x = _run(nn, a, x0, 2, 1e-6, 40, "mixed_bf16", **kw)
    assert st == nn.NN_OK, res
    assert 3 in res["pieces"]
    s64 = dense.rms_frob(dense.residual(a, x))
    assert abs(s64 - res["residual"]) <= e_acc(n)
    ainv = (q / lam) @ q.T
    assert _rel(x, ainv) <= 2 * math.sqrt(n) * s64 + 16 * 1e2 * U32


def test_host_pc_rejects_bad_preconditioner(nn):
    n = 8
    a = np.eye(n)
    xh = np.empty_like(a)
    ws = nn.workspace(n, "f64", host=True)
    st, _ = nn.nn_invert_host_pc(a, "scalar", -1.0, nn.make_opts(2, 1e-8, 10, "f64"), xh, ws)
    assert st == nn.NN_ERR_ARG
    st, _ = nn.nn_invert_host_pc(a, "theta2", 0.0, nn.make_opts(2, 1e-8, 10, "f64"), xh, ws)
    assert st == nn.NN_ERR_ARG


@pytest.mark.parametrize("n", [1, 31, 256, 300])
def test_residual_call(nn, n):
    import torch

    a = synth.spd_wishart(n, seed=7)
    x = np.linalg.inv(a) * (1 + 1e-3)
    ws = nn.workspace(n, "f64")
    st, s = nn.nn_residual(_dev(a), _dev(x), "f64", ws)
    torch.cuda.synchronize()
    assert st == nn.NN_OK
    want = dense.rms_frob(dense.residual(a, x))
    assert abs(s - want) <= 1e-10 * want
    ws32 = nn.workspace(n, "f32")
    st, s32 = nn.nn_residual(_dev(a), _dev(x), "f32", ws32)
    assert st == nn.NN_OK and abs(s32 - want) <= 1e-3 * want + 1e-6


@pytest.mark.parametrize("n", [512, 1024, 4096])
def test_gemm_tilings_agree_bitwise(nn, n):
    # n = 4096: 256 tiles of 256 x 256 on the 2-SM kernel leave a last wave at most half full,
    # which runs as 256 x 128 halves
    # Single-CTA tiles and the 2-SM MMA run the same K-ordered BF16 products into FP32 per
    # output element, so the iterates must agree bit for bit; only the per-CTA grouping of the
    # residual's sum of squares differs.
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=n + 7)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    out = {}
    try:
        assert nn.nn_set_gemm_variant(2) == nn.NN_ERR_ARG
        for variant in (1, 3, 4):
            assert nn.nn_set_gemm_variant(variant) == nn.NN_OK
            out[variant] = _run(nn, a, x0, 2, 1e-6, 40, "mixed_bf16")
    finally:
        nn.nn_set_gemm_variant(0)
    st1, r1, x1 = out[1]
    assert st1 == nn.NN_OK
    for variant in (3, 4):
        st2, r2, x2 = out[variant]
        assert st2 == nn.NN_OK
        assert r1["nests"] == r2["nests"] and r1["pieces"] == r2["pieces"]
        assert np.array_equal(x1, x2)
        for h1, h2 in zip(r1["history"], r2["history"]):
            assert abs(h1 - h2) <= 1e-12 * h1


@pytest.mark.parametrize("sched", [[2, 2, 1], [1, 3], [3, 1, 2]])
def test_depth_schedule_matches_oracle_f64(nn, sched):
    # per-nest depths (the matrix form of the CNS construction): same nest count, history and
    # iterate as the oracle's scheduled loop, and flops counted per nest
    n = 200
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=17)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    st, res, x = _run(nn, a, x0, 2, 1e-10, 40, "f64", depth_schedule=sched)
    run = dense.nn_invert(a, x0, 2, 1e-10, 40, depth_schedule=sched)
    assert st == nn.NN_OK and res["nests"] == run.nests
    for s_gpu, s_cpu in zip(res["history"], run.history):
        assert abs(s_gpu - s_cpu) <= 1e-8 * s_cpu + 1e-13
    assert np.linalg.norm(x - run.x) <= 1e-9 * np.linalg.norm(run.x)
    gemms = 1 + sum(sched[min(k, len(sched) - 1)] + 1 for k in range(run.nests))
    assert res["flops"] == pytest.approx(2.0 * n ** 3 * gemms, rel=1e-12)


def test_depth_schedule_mixed_converges(nn):
    # the tensor-core chain under a Chebyshev-then-Newton schedule reaches tol like the fixed depth
    n = 512
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=19)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    st, res, x = _run(nn, a, x0, 2, 1e-6, 40, "mixed_bf16", depth_schedule=[2, 2, 1])
    assert st == nn.NN_OK and res["residual"] < 1e-6
    r = np.eye(n) - a @ x
    assert np.linalg.norm(r) / n < 1e-6 + 4 * 2.0 ** -24 * (1 + math.sqrt(n) / 4)
