"""GPU parity of the batched small-complex NN kernel against the complex128 oracle loop.

Both sides run the same fixed-nest loop per matrix. The GPU works in complex64: each complex
product of order U (three BF16 pieces per real operand with FP32 accumulation on the tensor
cores, FP32 FMA chains on the CUDA cores) carries about sqrt(U) u32 of relative rounding, and a
nest of depth L amplifies earlier rounding by (L+1) rho^L along its residual's spectral radius
rho, so matrices that converge agree within C_BATCHED G sqrt(U) u32 (batched_bounds.py: c = 2, G
the nests' amplification from rho(I - A X_0); test_batched_tolerance.py shows on the CPU that a
two-piece product breaks it). Diverging matrices (the plain Jacobi start has rho(I - A X_0) > 1
for most U >= 32) must be reported as diverged on both sides.
"""
import math

import numpy as np
import pytest

import synth
from batched_bounds import C_BATCHED, U32, amplification
from oracle import batched

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nn():
    from paper_2212_02406_gb300 import abi, build

    build.build()
    abi.lib()
    return abi


def _run(nn, bt, depth, nests, damping, cfg_by_u=None, graph=False):
    import torch

    A = torch.from_numpy(bt.data.astype(np.complex64)).cuda()
    offs = torch.from_numpy(bt.offsets.astype(np.int64)).cuda()
    sizes = torch.from_numpy(bt.sizes.astype(np.int32)).cuda()
    plan_host = nn.nn_batched_plan(bt.sizes, cfg_by_u)
    classes = nn.nn_batched_plan_classes(plan_host)
    plan = torch.from_numpy(plan_host).cuda()
    X = torch.empty_like(A)
    res = torch.empty(bt.count, dtype=torch.float32, device="cuda")
    st = torch.empty(bt.count, dtype=torch.int32, device="cuda")
    ws = torch.empty(nn.nn_batched_workspace_bytes(bt.count), dtype=torch.uint8, device="cuda")
    if graph:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            assert nn.nn_invert_batched_c64(A, offs, sizes, plan, depth, nests, damping, X, res, st, ws, s,
                                            classes=classes) == 0
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        X.zero_()
        with torch.cuda.graph(g):
            rc = nn.nn_invert_batched_c64(A, offs, sizes, plan, depth, nests, damping, X, res, st, ws, classes=classes)
        assert rc == 0
        g.replay()
        g.replay()
    else:
        assert nn.nn_invert_batched_c64(A, offs, sizes, plan, depth, nests, damping, X, res, st, ws,
                                        classes=classes) == 0
    torch.cuda.synchronize()
    return X.cpu().numpy(), res.cpu().numpy(), st.cpu().numpy()


def _check(bt, x, res, st, depth, nests, damping, check_all=True):
    mats = [bt.matrix(b).astype(np.complex128) for b in range(bt.count)]
    runs = batched.nn_batched(mats, depth, nests, damping=lambda u: 1.0 / (1.0 + damping * u))
    n_conv = 0
    for b, (a, run) in enumerate(zip(mats, runs)):
        assert int(st[b]) == run.status, (b, bt.sizes[b], st[b], run.status, run.history)
        if run.status != 0:
            continue
        n_conv += 1
        u = a.shape[0]
        o = int(bt.offsets[b])
        xg = x[o:o + u * u].reshape(u, u).astype(np.complex128)
        tol = C_BATCHED * amplification(a, depth, nests, damping) * math.sqrt(u) * U32
        err = np.linalg.norm(xg - run.x) / np.linalg.norm(run.x)
        assert err <= tol, (b, u, err, tol)
        # the reported residual of X (an FP32 product of order U, then the Frobenius sum)
        s = run.history[-1]
        assert abs(res[b] - s) <= tol * s + 8 * math.sqrt(u) * U32, (b, res[b], s)
    return n_conv


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("damping", [0.0, 1.0 / 128.0])
def test_mixed_sizes_match_oracle(nn, depth, damping):
    bt = synth.mimo_gram_batch(96, seed=depth)
    x, res, st = _run(nn, bt, depth, 3, damping)
    n_conv = _check(bt, x, res, st, depth, 3, damping)
    assert n_conv > 0


@pytest.mark.parametrize("cfg", [0, 1, 3])
def test_tile_configs_agree(nn, cfg):
    bt = synth.mimo_gram_batch(48, seed=11, sizes=(8, 24, 40, 64, 5, 17, 33, 63, 1))
    x, res, st = _run(nn, bt, 2, 4, 1.0 / 128.0, cfg_by_u={u: cfg for u in range(1, 65)})
    _check(bt, x, res, st, 2, 4, 1.0 / 128.0)


@pytest.mark.parametrize("cfg", [0, 1])
@pytest.mark.parametrize("depth", [2, 3])
def test_exact_tile_classes_with_padded_rows(nn, cfg, depth):
    # U a multiple of the thread group's side runs the exact class, whose shared-memory rows are
    # padded (pitch != U); several matrices of each size per work item for the 8 x 8 groups,
    # and four buffers per matrix at depth 3
    sizes = (8, 16, 24, 32, 48, 64)
    bt = synth.mimo_gram_batch(72, seed=23 + depth, sizes=sizes)
    assert set(int(u) for u in bt.sizes) == set(sizes)
    x, res, st = _run(nn, bt, depth, 3, 1.0 / 128.0, cfg_by_u={u: cfg for u in range(1, 65)})
    assert _check(bt, x, res, st, depth, 3, 1.0 / 128.0) == bt.count


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("damping", [0.0, 1.0 / 128.0])
def test_tensor_core_items_match_oracle(nn, depth, damping):
    # plan configuration 2 (U in {48, 64}): masters in TMEM, complex products as tcgen05 MMA
    # chains on the real embedding with three BF16 pieces per operand, two matrices per CTA in
    # a pipeline (one at depth 3); other sizes fall back to the CUDA-core classes
    bt = synth.mimo_gram_batch(60, seed=20 + depth, sizes=(16, 32, 48, 64, 8, 24, 40))
    x, res, st = _run(nn, bt, depth, 3, damping, cfg_by_u={u: 2 for u in range(1, 65)})
    n_conv = _check(bt, x, res, st, depth, 3, damping)
    assert n_conv > 0


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_warp_items_match_oracle(nn, depth):
    # plan configuration 3 (U in {8, 16, 24, 32}): one warp per matrix, warp synchronisation
    # only; other sizes fall back to the CTA-wide CUDA-core classes
    bt = synth.mimo_gram_batch(80, seed=40 + depth, sizes=(8, 16, 24, 32, 5, 40, 64))
    x, res, st = _run(nn, bt, depth, 3, 1.0 / 128.0, cfg_by_u={u: 3 for u in range(1, 65)})
    n_conv = _check(bt, x, res, st, depth, 3, 1.0 / 128.0)
    assert n_conv > 0


def test_tensor_core_items_unaligned_offsets(nn):
    # odd sizes before the tensor-core sizes leave their matrices 8- but not 16-byte aligned
    bt = synth.mimo_gram_batch(24, seed=31, sizes=(5, 64, 17, 48, 1, 63))
    x, res, st = _run(nn, bt, 2, 3, 1.0 / 128.0, cfg_by_u={48: 2, 64: 2})
    assert any(int(bt.offsets[b]) % 2 == 1 and int(bt.sizes[b]) in (48, 64) for b in range(bt.count))
    n_conv = _check(bt, x, res, st, 2, 3, 1.0 / 128.0)
    assert n_conv > 0


def test_single_and_tiny(nn):
    bt = synth.mimo_gram_batch(1, seed=2, sizes=(1,))
    x, res, st = _run(nn, bt, 2, 2, 0.0)
    a = bt.matrix(0)
    assert st[0] == 0 and abs(x[0] - 1.0 / a[0, 0]) <= 1e-6 * abs(1.0 / a[0, 0])


def test_all_classes_mask_matches_plan_mask(nn):
    # launching every class (empty ones exit at once) gives the same bits as the plan's mask
    import torch

    bt = synth.mimo_gram_batch(40, seed=6)
    x1, r1, s1 = _run(nn, bt, 2, 3, 1.0 / 128.0)
    A = torch.from_numpy(bt.data.astype(np.complex64)).cuda()
    offs = torch.from_numpy(bt.offsets.astype(np.int64)).cuda()
    sizes = torch.from_numpy(bt.sizes.astype(np.int32)).cuda()
    plan = torch.from_numpy(nn.nn_batched_plan(bt.sizes)).cuda()
    X = torch.empty_like(A)
    res = torch.empty(bt.count, dtype=torch.float32, device="cuda")
    st = torch.empty(bt.count, dtype=torch.int32, device="cuda")
    ws = torch.empty(nn.nn_batched_workspace_bytes(bt.count), dtype=torch.uint8, device="cuda")
    assert nn.nn_invert_batched_c64(A, offs, sizes, plan, 2, 3, 1.0 / 128.0, X, res, st, ws) == 0
    assert nn.nn_invert_batched_c64(A, offs, sizes, plan, 2, 3, 1.0 / 128.0, X, res, st, ws, classes=0) == nn.NN_ERR_ARG
    torch.cuda.synchronize()
    assert np.array_equal(X.cpu().numpy(), x1) and np.array_equal(res.cpu().numpy(), r1)
    assert np.array_equal(st.cpu().numpy(), s1)


def test_graph_capture_replay(nn):
    bt = synth.mimo_gram_batch(64, seed=4)
    x1, r1, s1 = _run(nn, bt, 2, 3, 1.0 / 128.0)
    x2, r2, s2 = _run(nn, bt, 2, 3, 1.0 / 128.0, graph=True)
    assert np.array_equal(x1, x2) and np.array_equal(r1, r2) and np.array_equal(s1, s2)


@pytest.mark.parametrize("cfg_tc", [False, True])
def test_full_batch_16384(nn, cfg_tc):
    # The benchmarked configuration: 16,384 Gram matrices, U uniform over {8..64}, depth 2,
    # 3 nests, damped Jacobi start; every matrix checked against the oracle, with the CUDA-core
    # items only and with the tensor-core items for U in {48, 64}.
    bt = synth.mimo_gram_batch(16384, seed=0)
    table = {48: 2, 64: 2} if cfg_tc else None
    x, res, st = _run(nn, bt, 2, 3, 1.0 / 128.0, cfg_by_u=table)
    n_conv = _check(bt, x, res, st, 2, 3, 1.0 / 128.0)
    assert n_conv == bt.count


def test_batched_interface_equals_c64_entry(nn):
    # nn_invert_batched (batch, depth, nests, X, residuals, stream order) runs the same kernels
    # as nn_invert_batched_c64: bitwise the same X, residuals and statuses (Corollary 4's use)
    import torch

    bt = synth.mimo_gram_batch(64, seed=21)
    x, res, st = _run(nn, bt, 2, 3, 1.0 / 128.0)
    A = torch.from_numpy(bt.data.astype(np.complex64)).cuda()
    offs = torch.from_numpy(bt.offsets.astype(np.int64)).cuda()
    sizes = torch.from_numpy(bt.sizes.astype(np.int32)).cuda()
    plan_host = nn.nn_batched_plan(bt.sizes, None)
    plan = torch.from_numpy(plan_host).cuda()
    X = torch.empty_like(A)
    r2 = torch.empty(bt.count, dtype=torch.float32, device="cuda")
    s2 = torch.empty(bt.count, dtype=torch.int32, device="cuda")
    ws = torch.empty(nn.nn_batched_workspace_bytes(bt.count), dtype=torch.uint8, device="cuda")
    assert nn.nn_invert_batched(A, offs, sizes, 2, 3, 1.0 / 128.0, plan, X, r2, s2, ws,
                                classes=nn.nn_batched_plan_classes(plan_host)) == nn.NN_OK
    torch.cuda.synchronize()
    assert np.array_equal(X.cpu().numpy(), x)
    assert np.array_equal(r2.cpu().numpy(), res) and np.array_equal(s2.cpu().numpy(), st)
