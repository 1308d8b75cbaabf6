"""GPU parity of the sparse NN chain (nn_solve_csr) against the CPU oracle.

The chain computes X = D^-1 prod_j sum_n P^{n (L+1)^j} B with (L+1)^k - 1 sparse products.
Both sides run the same sequence of products; they differ by the summation order inside
each row (at most max_row_nnz terms) and by the FP64/FP32 rounding of each product, so the
relative difference is bounded by m * u * (1 + max_row_nnz) with m = (L+1)^k - 1 products:
tolerance 8 m u (nnz_row + 1) per dtype, with a 1e-13 floor for FP64. The double-float
arithmetic (FP64 data, hi + lo FP32 pairs) has u = 2^-48.
"""
import math

import numpy as np
import pytest

import synth
from oracle import sparse

pytestmark = pytest.mark.gpu

U = {"f64": 2.0 ** -53, "f64_df": 2.0 ** -48, "f32": 2.0 ** -24}
NP = {"f64": np.float64, "f64_df": np.float64, "f32": np.float32}


@pytest.fixture(scope="module")
def nn():
    from paper_2212_02406_gb300 import abi, build

    build.build()
    abi.lib()
    return abi


def _solve(nn, m, b, depth, nests, tol=0.0, dtype="f64"):
    import torch

    npd = NP[dtype]
    rp = torch.from_numpy(m.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(m.col.astype(np.int32)).cuda()
    val = torch.from_numpy(m.val.astype(npd)).cuda()
    B = torch.from_numpy(np.ascontiguousarray(b.T.astype(npd))).cuda()  # (nrhs, n)
    X = torch.empty_like(B)
    ws = nn.csr_workspace(m.n, m.nnz, B.shape[0], dtype)
    st, res = nn.nn_solve_csr(rp, col, val, B, depth, nests, tol, X, ws, double_float=(dtype == "f64_df"))
    torch.cuda.synchronize()
    return st, res, X.cpu().numpy().T


def _tol(m, depth, nests, dtype):
    terms = (depth + 1) ** nests - 1
    nnz_row = int(np.max(np.diff(m.row_ptr)))
    t = 8 * max(terms, 1) * U[dtype] * (nnz_row + 1)
    return max(t, 1e-13) if dtype == "f64" else t


@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32"])
@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("kind", ["laplacian", "random"])
@pytest.mark.parametrize("nrhs", [1, 3, 6])
def test_chain_matches_oracle(nn, dtype, depth, kind, nrhs):
    m = synth.laplacian_5pt(33, 29, shift=0.5) if kind == "laplacian" else synth.random_sparse_spd(1000, 7, seed=4)
    b = synth.gaussian_rhs(m.n, nrhs, seed=3)
    a64 = m.to_scipy()
    for nests in (0, 1, 3):
        if (depth + 1) ** nests > 100:
            continue
        st, res, x = _solve(nn, m, b, depth, nests, dtype=dtype)
        assert st == nn.NN_OK and res["nests"] == nests
        want = sparse.nn_sparse_solve(a64, b.astype(np.float64), depth, nests)
        err = np.linalg.norm(x - want) / np.linalg.norm(want)
        assert err <= _tol(m, depth, nests, dtype), (nests, err)
        # residual reported for the returned X agrees with the oracle's
        r = sparse.relative_residual(a64, want, b)
        assert abs(res["residual"] - r) <= 1e-6 * r + {"f64": 1e-12, "f64_df": 1e-10, "f32": 1e-5}[dtype]


def test_tol_stops_at_first_factor_below(nn):
    m = synth.laplacian_5pt(40, shift=0.5)
    b = synth.gaussian_rhs(m.n, 1, seed=8)
    a64 = m.to_scipy()
    st, res, x = _solve(nn, m, b, 2, 8, tol=1e-6)
    assert st == nn.NN_OK
    rels = [sparse.relative_residual(a64, sparse.nn_sparse_solve(a64, b, 2, j + 1), b) for j in range(8)]
    k = next(j for j, r in enumerate(rels) if r < 1e-6)
    assert res["nests"] == k + 1
    for j in range(k + 1):
        assert abs(res["history"][j] - rels[j]) <= 1e-8 * rels[j] + 1e-14


def test_edge_cases(nn):
    # n = 1, nests = 0 (X = D^-1 B), a missing diagonal is rejected before the chain runs
    m = synth.Csr(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    st, res, x = _solve(nn, m, np.array([[2.0]]), 2, 3)
    assert st == nn.NN_OK and abs(x[0, 0] - 0.5) < 1e-15
    m = synth.laplacian_5pt(5, shift=0.5)
    b = synth.gaussian_rhs(m.n, 1, seed=1)
    st, res, x = _solve(nn, m, b, 2, 0)
    assert st == nn.NN_OK and np.allclose(x[:, 0], b[:, 0] / m.to_scipy().diagonal(), rtol=1e-15)
    bad = synth.Csr(2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([1.0, 1.0]))
    st, res, x = _solve(nn, bad, np.ones((2, 1)), 2, 1)
    assert st == nn.NN_ERR_ARG


@pytest.mark.parametrize("dtype", ["f64", "f64_df"])
def test_full_size_laplacian_2048(nn, dtype):
    # The benchmarked configuration: 2048 x 2048 grid, shift 0.5, depth 2, 5 factors
    # (242 sparse products), FP64 data, checked element-wise against the oracle.
    m = synth.laplacian_5pt(2048, shift=0.5)
    b = synth.gaussian_rhs(m.n, 1, seed=0)
    st, res, x = _solve(nn, m, b, 2, 5, dtype=dtype)
    assert st == nn.NN_OK
    a64 = m.to_scipy()
    want = sparse.nn_sparse_solve(a64, b, 2, 5)
    err = np.linalg.norm(x - want) / np.linalg.norm(want)
    assert err <= _tol(m, 2, 5, dtype)
    # D = 4.5 I, so b - A x_m = (I - A/4.5)^m b and ||r|| / ||b|| <= rho(P)^m, m = 3^5 terms,
    # down to the FP64 rounding floor
    rho = 4.0 * math.cos(math.pi / 2049) / 4.5
    assert res["residual"] <= rho ** 243 + 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32"])
@pytest.mark.parametrize("case", ["lap_odd_nnz", "random_ragged", "random_long_rows", "tiny"])
def test_product_kernels_agree_bitwise(nn, dtype, case):
    # The bulk-copy ring kernel and the staged-load kernel sum each row's terms in the same
    # order, so iterates and residuals must agree bit for bit. The cases cover a nonzero count
    # that is not a multiple of 4 (elements read past the last staged one), ragged rows, rows
    # longer than one ring stage (a tile split into many chunks) and a single partial tile.
    m = {
        "lap_odd_nnz": lambda: synth.laplacian_5pt(33, 29, shift=0.5),
        "random_ragged": lambda: synth.random_sparse_spd(1000, 7, seed=4),
        "random_long_rows": lambda: synth.random_sparse_spd(3000, 300, seed=1),
        "tiny": lambda: synth.laplacian_5pt(5, shift=0.5),
    }[case]()
    b = synth.gaussian_rhs(m.n, 1, seed=11)
    out = {}
    try:
        for variant in (1, 0):
            assert nn.nn_set_spmv_variant(variant) == nn.NN_OK
            out[variant] = _solve(nn, m, b, 2, 3, tol=1e-30, dtype=dtype)
    finally:
        nn.nn_set_spmv_variant(0)
    (s1, r1, x1), (s0, r0, x0) = out[1], out[0]
    assert s1 == s0 and r1["nests"] == r0["nests"] == 3
    assert np.array_equal(x1, x0)
    assert r1["history"][:3] == r0["history"][:3]


@pytest.mark.parametrize("dtype", ["f64", "f64_df", "f32"])
@pytest.mark.parametrize("depths", [[2, 1, 1], [2, 2, 1, 1, 1], [1, 3, 2]])
def test_schedule_matches_oracle(nn, dtype, depths):
    # a depth per factor (CNS: Chebyshev factors, then the factorised Neumann series)
    import torch

    m = synth.random_sparse_spd(1000, 7, seed=5)
    b = synth.gaussian_rhs(m.n, 1, seed=7)
    npd = NP[dtype]
    rp = torch.from_numpy(m.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(m.col.astype(np.int32)).cuda()
    val = torch.from_numpy(m.val.astype(npd)).cuda()
    B = torch.from_numpy(np.ascontiguousarray(b.T.astype(npd))).cuda()
    X = torch.empty_like(B)
    ws = nn.csr_workspace(m.n, m.nnz, 1, dtype)
    st, res = nn.nn_solve_csr_sched(rp, col, val, B, depths, 0.0, X, ws, double_float=(dtype == "f64_df"))
    torch.cuda.synchronize()
    assert st == nn.NN_OK and res["nests"] == len(depths)
    x = X.cpu().numpy().T
    want = sparse.nn_sparse_solve_sched(m.to_scipy(), b.astype(np.float64), depths)
    terms = int(np.prod([d + 1 for d in depths])) - 1
    nnz_row = int(np.max(np.diff(m.row_ptr)))
    tol = max(8 * terms * U[dtype] * (nnz_row + 1), 1e-13 if dtype == "f64" else 0)
    assert np.linalg.norm(x - want) / np.linalg.norm(want) <= tol


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("sched", [None, [2, 2, 1]])
def test_solve_interface_equals_csr_entry_and_oracle(nn, dtype, sched):
    # nn_solve (A, B, depth, tol, opts, X, result, stream) runs the same chain as nn_solve_csr /
    # nn_solve_csr_sched: bitwise the same X, and the oracle's factor product within the chain
    # tolerance (problem statement; Corollary 1, Eq. (NNexplicit); Algorithm 2)
    import torch

    m = synth.laplacian_5pt(37, 31, shift=0.5)
    b = synth.gaussian_rhs(m.n, 2, seed=5)
    npd = NP[dtype]
    rp = torch.from_numpy(m.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(m.col.astype(np.int32)).cuda()
    val = torch.from_numpy(m.val.astype(npd)).cuda()
    B = torch.from_numpy(np.ascontiguousarray(b.T.astype(npd))).cuda()
    X = torch.empty_like(B)
    ws = nn.csr_workspace(m.n, m.nnz, B.shape[0], dtype)
    opts = nn.make_opts(depth=2, max_nests=3, dtype=dtype, depth_schedule=sched)
    st, res = nn.nn_solve(rp, col, val, B, 2, 0.0, opts, X, ws)
    torch.cuda.synchronize()
    assert st == nn.NN_OK
    X2 = torch.empty_like(B)
    if sched is None:
        st2, res2 = nn.nn_solve_csr(rp, col, val, B, 2, 3, 0.0, X2, ws)
        depths = [2, 2, 2]
    else:
        st2, res2 = nn.nn_solve_csr_sched(rp, col, val, B, sched, 0.0, X2, ws)
        depths = sched
    torch.cuda.synchronize()
    assert st2 == nn.NN_OK and res["nests"] == res2["nests"] == len(depths)
    assert torch.equal(X, X2)
    want = sparse.nn_sparse_solve_sched(m.to_scipy(), b, depths)
    err = np.linalg.norm(X.cpu().numpy().T - want) / np.linalg.norm(want)
    terms = int(np.prod([d + 1 for d in depths])) - 1
    nnz_row = int(np.max(np.diff(m.row_ptr)))
    assert err <= max(8 * terms * U[dtype] * (nnz_row + 1), 1e-13), err


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("world", [2, 3])
def test_row_strips_equal_single_chain_bitwise(nn, dtype, world):
    # The row-strip entry points (nn_csr_strip_*) driven by the sharded host loop, with the halos
    # copied in-process between strips on this GPU: each strip row sums its terms in the order of
    # the single-GPU chain's row, and the loop applies the same products and accumulations, so
    # X must equal nn_solve_csr_sched's bit for bit (Corollary 1 applied per strip).
    import torch

    from paper_2212_02406_gb300 import shard

    npd = NP[dtype]
    m = synth.laplacian_5pt(41, 37, shift=0.5)
    b = synth.gaussian_rhs(m.n, 1, seed=12)[:, 0].astype(npd)
    depths = [2, 2, 1]
    plans = shard.build_halo_plans(m.row_ptr, m.col, shard.partition_rows_by_nnz(m.row_ptr, world))
    strips = [shard.CudaStrip(p, m.row_ptr, m.val.astype(npd), "cuda") for p in plans]
    ex = shard.LocalExchange(plans, "cuda")
    shard.setup_strips(strips, ex)
    xs, rel = shard.sharded_sparse_chain(strips, ex, [torch.from_numpy(b[p.r0:p.r1].copy()).cuda() for p in plans],
                                         depths)
    torch.cuda.synchronize()
    x = torch.cat(xs).cpu().numpy()
    rp = torch.from_numpy(m.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(m.col.astype(np.int32)).cuda()
    val = torch.from_numpy(m.val.astype(npd)).cuda()
    B = torch.from_numpy(b[None, :].copy()).cuda()
    X = torch.empty_like(B)
    st, res = nn.nn_solve_csr_sched(rp, col, val, B, depths, 0.0, X, nn.csr_workspace(m.n, m.nnz, 1, dtype))
    torch.cuda.synchronize()
    assert st == nn.NN_OK
    assert np.array_equal(x, X.cpu().numpy()[0])
    assert abs(rel - res["residual"]) <= 1e-8 * res["residual"] + {"f64": 1e-14, "f32": 1e-6}[dtype]


def test_row_strip_entry_points_reject_bad_arguments(nn):
    import torch

    ws = torch.empty(nn.nn_csr_strip_workspace_bytes(8), dtype=torch.uint8, device="cuda")
    rp = torch.zeros(9, dtype=torch.int32, device="cuda")
    col = torch.zeros(0, dtype=torch.int32, device="cuda")
    val = torch.zeros(0, dtype=torch.float64, device="cuda")
    dinv = torch.empty(8, dtype=torch.float64, device="cuda")
    # rows without a diagonal entry
    assert nn.nn_csr_strip_diag_inv(rp, col, val, dinv, ws) == nn.NN_ERR_ARG
    v = torch.zeros(8, dtype=torch.float64, device="cuda")
    # neither y nor an accumulator to write
    assert nn.nn_csr_strip_product(rp, col, val, v, None, ws) == nn.NN_ERR_ARG
