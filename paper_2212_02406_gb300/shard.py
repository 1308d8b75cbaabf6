"""Host-side sharding for runs with one process per GPU.

* One dense inversion does not shard without an operand all-gather per GEMM, so the dense
  path runs replicas (each rank its own matrix; no data-path collective).
* A batch of small matrices shards by matrices: ``shard_batch`` balances the estimated work
  (sum of U^3) with a longest-processing-time greedy; ranks only gather statistics at the end.
* The sparse chain shards by row strips: every sparse product needs the neighbours' values of
  the input vector on the strip's halo columns (one exchange per product) and each residual
  check needs one all-reduce of two scalars. ``HaloPlan`` holds the index maps and
  ``distributed_sparse_chain`` the host loop of the explicit NN form (Corollary 1, Corollary 6):
  X = D^-1 prod_j sum_n P^{n (L+1)^j} B with P = I - A D^-1, exactly as the single-GPU chain.

The local product is a callable so the same loop drives the CUDA kernel on a GPU rank and a
NumPy product in the CPU tests; the exchange and reductions go through ``torch.distributed``
(NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def partition_rows(n: int, world: int) -> list[tuple[int, int]]:
    """Contiguous row strips of near-equal size."""
    base, extra = divmod(n, world)
    out, r = [], 0
    for k in range(world):
        m = base + (1 if k < extra else 0)
        out.append((r, r + m))
        r += m
    return out


def partition_rows_by_nnz(row_ptr: np.ndarray, world: int) -> list[tuple[int, int]]:
    """Contiguous row strips holding near-equal numbers of nonzeros."""
    n = row_ptr.shape[0] - 1
    nnz = int(row_ptr[-1])
    cuts = [0]
    for k in range(1, world):
        cuts.append(int(np.searchsorted(row_ptr, k * nnz / world, side="left")))
    cuts.append(n)
    cuts = [min(max(c, 0), n) for c in cuts]
    for k in range(1, len(cuts)):
        cuts[k] = max(cuts[k], cuts[k - 1])
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def shard_batch(sizes: np.ndarray, world: int) -> list[np.ndarray]:
    """Matrix indices per rank, balancing sum(U^3) (largest first onto the lightest rank)."""
    sizes = np.asarray(sizes)
    order = np.argsort(-sizes, kind="stable")
    load = np.zeros(world)
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        k = int(np.argmin(load))
        parts[k].append(int(i))
        load[k] += float(sizes[i]) ** 3
    return [np.sort(np.asarray(p, dtype=np.int64)) for p in parts]


@dataclass
class HaloPlan:
    """Index maps of one rank's row strip [r0, r1) of an n x n CSR matrix.

    ``col_local`` renumbers the strip's columns: owned columns c -> c - r0, halo columns -> the
    position after the owned block in ``halo`` order. ``recv[k]`` lists the global columns this
    rank receives from rank k; ``send[k]`` the owned rows it sends to rank k (positions relative
    to r0), in the order rank k expects them.
    """

    r0: int
    r1: int
    row_ptr: np.ndarray
    col_local: np.ndarray
    halo: np.ndarray
    recv: dict
    send: dict


def build_halo_plans(row_ptr: np.ndarray, col: np.ndarray, ranges: list[tuple[int, int]]) -> list[HaloPlan]:
    owner_starts = np.asarray([r[0] for r in ranges])

    def owner(c):
        return np.searchsorted(owner_starts, c, side="right") - 1

    plans = []
    for k, (r0, r1) in enumerate(ranges):
        e0, e1 = int(row_ptr[r0]), int(row_ptr[r1])
        cols = col[e0:e1].astype(np.int64)
        outside = (cols < r0) | (cols >= r1)
        halo = np.unique(cols[outside])
        pos = np.empty_like(cols)
        pos[~outside] = cols[~outside] - r0
        pos[outside] = (r1 - r0) + np.searchsorted(halo, cols[outside])
        recv = {}
        if halo.size:
            owners = owner(halo)
            for q in np.unique(owners):
                recv[int(q)] = halo[owners == q]
        plans.append(HaloPlan(r0, r1, (row_ptr[r0:r1 + 1] - row_ptr[r0]).astype(np.int64), pos, halo, recv, {}))
    for k, p in enumerate(plans):
        for q, cols in p.recv.items():
            plans[q].send[k] = cols - plans[q].r0
    return plans


def local_values(val: np.ndarray, row_ptr: np.ndarray, plan: HaloPlan) -> np.ndarray:
    return val[int(row_ptr[plan.r0]):int(row_ptr[plan.r1])]


class Exchanger:
    """Halo exchange through torch.distributed point-to-point operations."""

    def __init__(self, plan: HaloPlan, rank: int, dtype=np.float64):
        self.plan = plan
        self.rank = rank
        self.dtype = dtype

    def extend(self, v_local: np.ndarray) -> np.ndarray:
        """[owned values | halo values] for the strip's local column numbering."""
        import torch
        import torch.distributed as dist

        p = self.plan
        reqs = []
        bufs = {}
        for q, cols in p.recv.items():
            bufs[q] = torch.empty(len(cols), dtype=torch.float64)
            reqs.append(dist.irecv(bufs[q], src=q))
        sends = []
        for q, rows in p.send.items():
            t = torch.from_numpy(np.ascontiguousarray(v_local[rows], dtype=np.float64))
            sends.append(t)
            reqs.append(dist.isend(t, dst=q))
        for r in reqs:
            r.wait()
        ext = np.empty(len(v_local) + len(p.halo), dtype=self.dtype)
        ext[:len(v_local)] = v_local
        if p.halo.size:
            for q, cols in p.recv.items():
                ext[len(v_local) + np.searchsorted(p.halo, cols)] = bufs[q].numpy()
        return ext


def allreduce_sum(values) -> np.ndarray:
    import torch
    import torch.distributed as dist

    t = torch.tensor(np.asarray(values, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def distributed_sparse_chain(apply_local, extend, b_local: np.ndarray, dinv_local: np.ndarray, depth: int,
                             nests: int, residual_local=None, allreduce=allreduce_sum):
    """Host loop of the sharded sparse NN chain.

    apply_local(v_ext) returns the strip of P v = v - A D^-1 v from the extended vector;
    extend(v_local) performs the halo exchange. Returns (x_local, relative residual or None).
    """
    z = np.array(b_local, copy=True)
    for j in range(nests):
        t = (depth + 1) ** j
        acc = z.copy()
        u = z
        for _blk in range(depth):
            for _ in range(t):
                u = apply_local(extend(u))
            acc = acc + u
        z = acc
    rel = None
    if residual_local is not None:
        r = residual_local(extend(z))
        sums = allreduce([float(np.sum(r * r)), float(np.sum(b_local * b_local))])
        rel = float(np.sqrt(sums[0] / sums[1])) if sums[1] > 0 else float(np.sqrt(sums[0]))
    return dinv_local * z, rel
