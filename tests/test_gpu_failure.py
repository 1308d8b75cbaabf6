"""Failure detection on the GPU, in the forms that fault nothing.

* A device wait that runs out: nn_debug_withhold_signal makes the next tensor-core GEMM's MMA
  issuer withhold one "accumulator ready" signal that nothing else sets. The epilogue's bounded
  wait (about one second) runs out, the kernel returns, and the call reports NN_ERR_TIMEOUT; the
  context stays usable, and the next call returns the same X as a clean run, bit for bit. The
  same for the batched tensor-core class (every matrix of the class reports NN_ERR_TIMEOUT) and
  for the sparse chain's bulk-copy ring (its first block never fills its first stage).
* Non-finite input: NaN or Inf in A (dense chains, every dtype), in one matrix of a batch, or in
  a right-hand side of the sparse chain must be reported as NN_ERR_DIVERGED (the residual is not
  finite, the divergence rule of Algorithm 1's stop test); the other matrices of a batch are
  unaffected, bit for bit.
"""
import time

import numpy as np
import pytest

import synth
from oracle import dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nn():
    from paper_2212_02406_gb300 import abi, build

    build.build()
    abi.lib()
    return abi


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _invert(nn, a, x0, dtype, tol=1e-6, **kw):
    import torch

    A, X0 = _dev(a), _dev(x0)
    X = torch.empty_like(A)
    st, res = nn.nn_invert(A, X0, nn.make_opts(2, tol, 40, dtype, **kw), X, nn.workspace(a.shape[0], dtype))
    torch.cuda.synchronize()
    return st, res, X.cpu().numpy()


@pytest.mark.parametrize("n,hint", [(512, True), (384, False), (1024, True)])
def test_withheld_signal_times_out_and_context_recovers(nn, n, hint):
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=n)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    kw = dict(x0_scalar=alpha) if hint else {}
    st0, res0, x_clean = _invert(nn, a, x0, "mixed_bf16", **kw)
    assert st0 == nn.NN_OK
    assert nn.nn_debug_withhold_signal(True) == nn.NN_OK
    t0 = time.time()
    st, res, _ = _invert(nn, a, x0, "mixed_bf16", **kw)
    assert st == nn.NN_ERR_TIMEOUT and res["status"] == nn.NN_ERR_TIMEOUT, res
    assert time.time() - t0 < 30.0
    # the hook was taken by that launch; the context is usable and the chain deterministic
    st2, res2, x2 = _invert(nn, a, x0, "mixed_bf16", **kw)
    assert st2 == nn.NN_OK and res2["history"] == res0["history"]
    assert np.array_equal(x2, x_clean)


def _batched(nn, bt, cfg_by_u):
    import torch

    plan_h = nn.nn_batched_plan(bt.sizes, cfg_by_u)
    A = torch.from_numpy(bt.data.astype(np.complex64)).cuda()
    X = torch.empty_like(A)
    res = torch.empty(bt.count, dtype=torch.float32, device="cuda")
    st = torch.empty(bt.count, dtype=torch.int32, device="cuda")
    ws = torch.empty(nn.nn_batched_workspace_bytes(bt.count), dtype=torch.uint8, device="cuda")
    assert nn.nn_invert_batched(A, torch.from_numpy(bt.offsets.astype(np.int64)).cuda(),
                                torch.from_numpy(bt.sizes.astype(np.int32)).cuda(), 2, 3, 1.0 / 128.0,
                                torch.from_numpy(plan_h).cuda(), X, res, st, ws,
                                classes=nn.nn_batched_plan_classes(plan_h)) == nn.NN_OK
    torch.cuda.synchronize()
    return X.cpu().numpy(), st.cpu().numpy()


def test_batched_withheld_signal_times_out_and_recovers(nn):
    # the hook goes to the first tensor-core class (U = 64): every CTA's first MMA chain never
    # signals completion, the workers' bounded wait runs out, and every matrix of that class
    # (those in the slots, the one claimed ahead, the ones still queued) reports NN_ERR_TIMEOUT;
    # the U = 48 class runs untouched, and the next call equals a clean run bit for bit
    bt = synth.mimo_gram_batch(400, seed=61, sizes=(64, 48))
    cfg = {48: 2, 64: 2}
    x_clean, st_clean = _batched(nn, bt, cfg)
    assert np.all(st_clean == nn.NN_OK)
    assert nn.nn_debug_withhold_signal(True) == nn.NN_OK
    t0 = time.time()
    x_bad, st_bad = _batched(nn, bt, cfg)
    assert time.time() - t0 < 30.0
    big = bt.sizes == 64
    assert np.all(st_bad[big] == nn.NN_ERR_TIMEOUT), np.unique(st_bad[big])
    assert np.all(st_bad[~big] == nn.NN_OK)
    for k in np.flatnonzero(~big):
        o, u = int(bt.offsets[k]), int(bt.sizes[k])
        assert np.array_equal(x_bad[o:o + u * u], x_clean[o:o + u * u]), k
    x2, st2 = _batched(nn, bt, cfg)
    assert np.array_equal(st2, st_clean) and np.array_equal(x2, x_clean)


def test_sparse_ring_withheld_stage_times_out_and_recovers(nn):
    # the hook goes to the chain's first product on the bulk-copy ring: its first block never
    # fills its first stage, the consumers' bounded wait runs out, and the solve reports
    # NN_ERR_TIMEOUT; the next solve equals a clean one bit for bit
    import torch

    m = synth.laplacian_5pt(64, shift=0.5)
    b = synth.gaussian_rhs(m.n, 1, seed=3)
    rp = torch.from_numpy(m.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(m.col.astype(np.int32)).cuda()
    val = torch.from_numpy(m.val).cuda()
    B = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    ws = nn.csr_workspace(m.n, m.nnz, 1, "f64")

    def solve():
        X = torch.empty_like(B)
        st, res = nn.nn_solve_csr(rp, col, val, B, 2, 3, 0.0, X, ws)
        torch.cuda.synchronize()
        return st, X.cpu().numpy()

    st0, x0 = solve()
    assert st0 == nn.NN_OK
    assert nn.nn_debug_withhold_signal(True) == nn.NN_OK
    t0 = time.time()
    st1, _ = solve()
    assert st1 == nn.NN_ERR_TIMEOUT, st1
    assert time.time() - t0 < 30.0
    st2, x2 = solve()
    assert st2 == nn.NN_OK and np.array_equal(x2, x0)


def test_disarmed_hook_changes_nothing(nn):
    n = 256
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=3)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    st0, _, x0_run = _invert(nn, a, x0, "mixed_bf16")
    nn.nn_debug_withhold_signal(True)
    nn.nn_debug_withhold_signal(False)
    st1, _, x1_run = _invert(nn, a, x0, "mixed_bf16")
    assert st0 == st1 == nn.NN_OK and np.array_equal(x0_run, x1_run)


@pytest.mark.parametrize("bad", [np.nan, np.inf])
@pytest.mark.parametrize("dtype,hint", [("f64", False), ("f32", False), ("mixed_bf16", False), ("mixed_bf16", True),
                                        ("mixed_f16", False), ("mixed_f16", True), ("mixed_emu", True)])
def test_non_finite_matrix_diverges(nn, bad, dtype, hint):
    n = 200
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=9)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    a = a.copy()
    a[17, 101] = bad
    kw = dict(x0_scalar=alpha) if hint else {}
    st, res, _ = _invert(nn, a, x0, dtype, **kw)
    assert st == nn.NN_ERR_DIVERGED and res["status"] == nn.NN_ERR_DIVERGED, res


def test_non_finite_start_diverges(nn):
    n = 128
    a, q, lam = synth.spd_spectrum(n, 1e2, seed=10)
    x0 = dense.precond_scalar(n, 2.0 / (lam[0] + lam[-1]))
    x0[3, 3] = np.nan
    for dtype in ("f64", "mixed_bf16", "mixed_f16"):
        st, res, _ = _invert(nn, a, x0, dtype)
        assert st == nn.NN_ERR_DIVERGED, (dtype, res)


def test_non_finite_batch_member_diverges_alone(nn):
    import torch

    bt = synth.mimo_gram_batch(40, seed=31)
    data_bad = bt.data.copy()
    k_bad = [3, 17, 29]
    for j, k in enumerate(k_bad):
        data_bad[int(bt.offsets[k]) + (j % 2)] = np.nan if j != 1 else np.inf
    plan_h = nn.nn_batched_plan(bt.sizes, None)
    out = {}
    for label, data in (("clean", bt.data), ("bad", data_bad)):
        A = torch.from_numpy(data.astype(np.complex64)).cuda()
        X = torch.empty_like(A)
        res = torch.empty(bt.count, dtype=torch.float32, device="cuda")
        st = torch.empty(bt.count, dtype=torch.int32, device="cuda")
        ws = torch.empty(nn.nn_batched_workspace_bytes(bt.count), dtype=torch.uint8, device="cuda")
        assert nn.nn_invert_batched(A, torch.from_numpy(bt.offsets.astype(np.int64)).cuda(),
                                    torch.from_numpy(bt.sizes.astype(np.int32)).cuda(), 2, 3, 1.0 / 128.0,
                                    torch.from_numpy(plan_h).cuda(), X, res, st, ws,
                                    classes=nn.nn_batched_plan_classes(plan_h)) == nn.NN_OK
        torch.cuda.synchronize()
        out[label] = (X.cpu().numpy(), st.cpu().numpy())
    xc, sc = out["clean"]
    xb, sb = out["bad"]
    for k in range(bt.count):
        u, o = int(bt.sizes[k]), int(bt.offsets[k])
        if k in k_bad:
            assert sb[k] == nn.NN_ERR_DIVERGED, (k, sb[k])
        else:
            assert sb[k] == sc[k]
            assert np.array_equal(xb[o:o + u * u], xc[o:o + u * u]), k


@pytest.mark.parametrize("u,cfg", [(64, 2), (48, 2), (32, 0), (16, 3)])
def test_non_finite_member_of_a_size_class(nn, u, cfg):
    """One size, one path: NaN or Inf on the diagonal of some matrices (each ends as diverged)
    leaves every other matrix bitwise as in a clean run."""
    import torch

    count = 25
    bt = synth.mimo_gram_batch(count, seed=40 + u, sizes=(u,))
    data_bad = bt.data.copy()
    k_bad = [0, 5, 12, 24]
    for j, k in enumerate(k_bad):
        data_bad[int(bt.offsets[k]) + (j % 3) * (u + 1)] = (np.nan, np.inf, -np.inf, np.nan)[j]
    plan_h = nn.nn_batched_plan(bt.sizes, {u: cfg})
    out = {}
    for label, data in (("clean", bt.data), ("bad", data_bad)):
        A = torch.from_numpy(data.astype(np.complex64)).cuda()
        X = torch.empty_like(A)
        res = torch.empty(bt.count, dtype=torch.float32, device="cuda")
        st = torch.empty(bt.count, dtype=torch.int32, device="cuda")
        ws = torch.empty(nn.nn_batched_workspace_bytes(bt.count), dtype=torch.uint8, device="cuda")
        assert nn.nn_invert_batched(A, torch.from_numpy(bt.offsets.astype(np.int64)).cuda(),
                                    torch.from_numpy(bt.sizes.astype(np.int32)).cuda(), 2, 3, 1.0 / 128.0,
                                    torch.from_numpy(plan_h).cuda(), X, res, st, ws,
                                    classes=nn.nn_batched_plan_classes(plan_h)) == nn.NN_OK
        torch.cuda.synchronize()
        out[label] = (X.cpu().numpy(), st.cpu().numpy(), res.cpu().numpy())
    xc, sc, rc = out["clean"]
    xb, sb, rb = out["bad"]
    assert np.all(sc == nn.NN_OK)
    for k in range(bt.count):
        o = int(bt.offsets[k])
        if k in k_bad:
            assert sb[k] == nn.NN_ERR_DIVERGED, (k, sb[k])
        else:
            assert sb[k] == nn.NN_OK and rb[k] == rc[k], k
            assert np.array_equal(xb[o:o + u * u], xc[o:o + u * u]), k


def test_non_finite_rhs_sparse_diverges(nn):
    import torch

    m = synth.laplacian_5pt(20, shift=0.5)
    b = synth.gaussian_rhs(m.n, 2, seed=2)
    b[7, 1] = np.nan
    rp = torch.from_numpy(m.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(m.col.astype(np.int32)).cuda()
    val = torch.from_numpy(m.val).cuda()
    B = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    X = torch.empty_like(B)
    for tol in (0.0, 1e-6):
        st, res = nn.nn_solve_csr(rp, col, val, B, 2, 3, tol, X, nn.csr_workspace(m.n, m.nnz, 2, "f64"))
        torch.cuda.synchronize()
        assert st == nn.NN_ERR_DIVERGED, (tol, res)
