"""Multi-rank host logic on CPU: two gloo ranks (one process each), no GPU.

* The row-strip sharded sparse chain (halo exchange per product, all-reduced residual) gives
  the same X as the single-process oracle.
* The batch shard covers every matrix once and balances sum(U^3); per-rank oracle runs
  gathered together equal the full-batch run.
"""
import os
import socket

import numpy as np
import pytest

import synth
from oracle import batched, sparse
from paper_2212_02406_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _sparse_worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = synth.random_sparse_spd(400, 5, seed=2)
        a = m.to_scipy()
        b = synth.gaussian_rhs(m.n, 1, seed=1)[:, 0]
        ranges = shard.partition_rows_by_nnz(m.row_ptr, world)
        plans = shard.build_halo_plans(m.row_ptr, m.col, ranges)
        p = plans[rank]
        dinv_all = 1.0 / a.diagonal()
        # local rows of A' = A D^-1 in the strip's column numbering
        vals = shard.local_values(m.val, m.row_ptr, p)
        gcols = m.col[int(m.row_ptr[p.r0]):int(m.row_ptr[p.r1])]
        vals_scaled = vals * dinv_all[gcols]
        import scipy.sparse as sp

        nloc = p.r1 - p.r0
        a_loc = sp.csr_matrix((vals_scaled, p.col_local, p.row_ptr), shape=(nloc, nloc + len(p.halo)))
        ex = shard.Exchanger(p, rank)
        b_loc = b[p.r0:p.r1]

        def apply_local(v_ext):
            return v_ext[:nloc] - a_loc @ v_ext

        def residual_local(z_ext):
            return b_loc - a_loc @ z_ext

        x_loc, rel = shard.distributed_sparse_chain(apply_local, ex.extend, b_loc, dinv_all[p.r0:p.r1], 2, 3,
                                                    residual_local)
        out[rank] = (p.r0, p.r1, x_loc, rel)
    finally:
        dist.destroy_process_group()


def _batched_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bt = synth.mimo_gram_batch(40, seed=3, dtype=np.complex128)
        parts = shard.shard_batch(bt.sizes, world)
        mine = parts[rank]
        runs = batched.nn_batched([bt.matrix(int(i)) for i in mine], 2, 3, damping=lambda u: 1 / (1 + u / 128))
        res = torch.tensor([r.history[-1] for r in runs], dtype=torch.float64)
        # gather the per-matrix residuals (the only cross-rank traffic of the batched path)
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([len(mine)], dtype=torch.int64))
        maxlen = int(max(s.item() for s in sizes))
        padded = torch.zeros(maxlen, dtype=torch.float64)
        padded[:len(mine)] = res
        gathered = [torch.zeros(maxlen, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, padded)
        out[rank] = ([p.tolist() for p in parts], [g[:int(s.item())].numpy() for g, s in zip(gathered, sizes)])
    finally:
        dist.destroy_process_group()


def _spawn(fn, world=2):
    import torch.multiprocessing as mp

    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(fn, args=(world, _free_port(), out), nprocs=world, join=True)
    return dict(out)


def test_partitions():
    assert shard.partition_rows(10, 3) == [(0, 4), (4, 7), (7, 10)]
    m = synth.laplacian_5pt(12, shift=0.5)
    rg = shard.partition_rows_by_nnz(m.row_ptr, 4)
    assert rg[0][0] == 0 and rg[-1][1] == m.n and all(a[1] == b[0] for a, b in zip(rg, rg[1:]))
    sizes = synth.mimo_gram_batch(100, seed=1).sizes
    parts = shard.shard_batch(sizes, 4)
    allidx = np.sort(np.concatenate(parts))
    assert np.array_equal(allidx, np.arange(100))
    loads = [float(np.sum(sizes[p].astype(float) ** 3)) for p in parts]
    assert max(loads) <= 1.15 * min(loads) + 64 ** 3


def test_halo_plan_laplacian():
    m = synth.laplacian_5pt(8, shift=0.5)
    plans = shard.build_halo_plans(m.row_ptr, m.col, shard.partition_rows(m.n, 2))
    # a 5-point stencil strip needs exactly one grid row (8 values) from its neighbour
    assert len(plans[0].halo) == 8 and len(plans[1].halo) == 8
    assert np.array_equal(plans[0].send[1], np.arange(24, 32))
    assert np.array_equal(plans[1].send[0], np.arange(0, 8))


def test_sharded_sparse_chain_matches_oracle():
    out = _spawn(_sparse_worker)
    m = synth.random_sparse_spd(400, 5, seed=2)
    a = m.to_scipy()
    b = synth.gaussian_rhs(m.n, 1, seed=1)[:, 0]
    want = sparse.nn_sparse_solve(a, b, 2, 3)
    x = np.zeros(m.n)
    for rank, (r0, r1, xl, rel) in out.items():
        x[r0:r1] = xl
    assert np.linalg.norm(x - want) <= 1e-12 * np.linalg.norm(want)
    rel_want = sparse.relative_residual(a, want, b)
    for _, (_, _, _, rel) in out.items():
        # both are relative to ||b||: a cancellation floor of a few u64 on top of 1e-10 rel
        assert abs(rel - rel_want) <= 1e-10 * rel_want + 64 * 2.0 ** -53


def test_sharded_batch_gathers_full_result():
    out = _spawn(_batched_worker)
    bt = synth.mimo_gram_batch(40, seed=3, dtype=np.complex128)
    full = batched.nn_batched([bt.matrix(b) for b in range(bt.count)], 2, 3, damping=lambda u: 1 / (1 + u / 128))
    parts, gathered = out[0]
    for part, vals in zip(parts, gathered):
        for i, v in zip(part, vals):
            assert abs(v - full[i].history[-1]) <= 1e-15 * max(1.0, abs(v))


def _strip_chain_worker(rank, world, port, out):
    # the host loop of the strip-sharded chain (sharded_sparse_chain) with the host stand-in of
    # the library's strip calls, halos exchanged between gloo ranks (DistExchange)
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = synth.laplacian_5pt(23, 17, shift=0.5)
        b = synth.gaussian_rhs(m.n, 1, seed=6)[:, 0]
        ranges = shard.partition_rows_by_nnz(m.row_ptr, world)
        plans = shard.build_halo_plans(m.row_ptr, m.col, ranges)
        p = plans[rank]
        strip = shard.HostStrip(p, m.row_ptr, m.val)
        ex = shard.DistExchange(p, "cpu")
        shard.setup_strips([strip], ex)
        xs, rel = shard.sharded_sparse_chain([strip], ex, [torch.from_numpy(b[p.r0:p.r1].copy())], [2, 2, 1],
                                             allreduce=shard.allreduce_sum)
        out[rank] = (p.r0, p.r1, xs[0].numpy(), rel)
    finally:
        dist.destroy_process_group()


def test_strip_sharded_chain_two_ranks_matches_oracle():
    out = _spawn(_strip_chain_worker, world=2)
    m = synth.laplacian_5pt(23, 17, shift=0.5)
    b = synth.gaussian_rhs(m.n, 1, seed=6)[:, 0]
    x = np.empty(m.n)
    rels = set()
    for r0, r1, xl, rel in out.values():
        x[r0:r1] = xl
        rels.add(round(rel, 12))
    want = sparse.nn_sparse_solve_sched(m.to_scipy(), b[:, None], [2, 2, 1])[:, 0]
    assert np.linalg.norm(x - want) <= 1e-13 * np.linalg.norm(want)
    assert len(rels) == 1  # one all-reduced residual on both ranks
    assert abs(rels.pop() - sparse.relative_residual(m.to_scipy(), want[:, None], b[:, None])) <= 1e-10


@pytest.mark.parametrize("world", [1, 3, 4])
def test_strip_chain_in_one_process_matches_oracle(world):
    # several strips held by one process, halos copied in-process (LocalExchange): the same loop
    import torch

    m = synth.random_sparse_spd(300, 6, seed=9)
    b = synth.gaussian_rhs(m.n, 1, seed=4)[:, 0]
    plans = shard.build_halo_plans(m.row_ptr, m.col, shard.partition_rows_by_nnz(m.row_ptr, world))
    strips = [shard.HostStrip(p, m.row_ptr, m.val) for p in plans]
    ex = shard.LocalExchange(plans, "cpu")
    shard.setup_strips(strips, ex)
    xs, rel = shard.sharded_sparse_chain(strips, ex, [torch.from_numpy(b[p.r0:p.r1].copy()) for p in plans], [2, 2])
    x = np.concatenate([t.numpy() for t in xs])
    want = sparse.nn_sparse_solve(m.to_scipy(), b[:, None], 2, 2)[:, 0]
    assert np.linalg.norm(x - want) <= 1e-13 * np.linalg.norm(want)
    assert abs(rel - sparse.relative_residual(m.to_scipy(), want[:, None], b[:, None])) <= 1e-10
