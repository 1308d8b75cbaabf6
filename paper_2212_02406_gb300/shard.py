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

``sharded_sparse_chain`` runs the chain over strips through the library's row-strip entry
points (``CudaStrip``) or a host stand-in with the same interface (``HostStrip``, for CPU tests);
the exchange and reductions go through ``torch.distributed`` (NCCL on GPUs, gloo on CPUs) or,
for several strips in one process, ``LocalExchange``. ``distributed_sparse_chain`` is the same
loop over NumPy callables.
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


# ---- the sharded sparse chain on the library's row-strip entry points ------------------------

class CudaStrip:
    """One strip of the sparse chain on this process's GPU, through the library's row-strip
    entry points (``nn_csr_strip_*``): the strip's CSR arrays in the extended local numbering of
    its ``HaloPlan``, D^-1 of its rows and, after ``setup_strips``, the scaled values A' = A D^-1
    (which need D^-1 on the halo columns, exchanged like a vector)."""

    def __init__(self, plan: HaloPlan, row_ptr: np.ndarray, val: np.ndarray, device, dtype=None):
        import torch

        from . import abi

        self.abi = abi
        self.plan = plan
        self.n = plan.r1 - plan.r0
        self.n_ext = self.n + len(plan.halo)
        self.dtype = dtype or (torch.float64 if val.dtype == np.float64 else torch.float32)
        self.device = device
        e0, e1 = int(row_ptr[plan.r0]), int(row_ptr[plan.r1])
        self.rp = torch.from_numpy(plan.row_ptr.astype(np.int32)).to(device)
        self.col = torch.from_numpy(plan.col_local.astype(np.int32)).to(device)
        self.raw = torch.from_numpy(np.ascontiguousarray(val[e0:e1])).to(device=device, dtype=self.dtype)
        self.ws = torch.empty(abi.nn_csr_strip_workspace_bytes(self.n), dtype=torch.uint8, device=device)
        self.dinv = torch.empty(self.n, dtype=self.dtype, device=device)
        st = abi.nn_csr_strip_diag_inv(self.rp, self.col, self.raw, self.dinv, self.ws)
        if st != abi.NN_OK:
            raise ValueError(f"strip rows without a usable diagonal (status {st})")
        self.vals = None

    def new_ext(self):
        import torch

        return torch.zeros(self.n_ext, dtype=self.dtype, device=self.device)

    def scale(self, dinv_ext):
        import torch

        self.vals = torch.empty_like(self.raw)
        if self.abi.nn_csr_strip_scale(self.col, self.raw, dinv_ext, self.vals) != self.abi.NN_OK:
            raise RuntimeError("nn_csr_strip_scale failed")

    def product(self, src_ext, dst_ext, acc_in=None, acc_out=None):
        y = None if dst_ext is None else dst_ext[:self.n]
        st = self.abi.nn_csr_strip_product(self.rp, self.col, self.vals, src_ext, y, self.ws, acc_in, acc_out)
        if st != self.abi.NN_OK:
            raise RuntimeError(f"nn_csr_strip_product: status {st}")

    def residual(self, z_ext, b_local):
        st, sums = self.abi.nn_csr_strip_residual(self.rp, self.col, self.vals, z_ext, b_local, self.ws)
        if st != self.abi.NN_OK:
            raise RuntimeError(f"nn_csr_strip_residual: status {st}")
        return sums

    def finish(self, z_local):
        import torch

        x = torch.empty_like(z_local)
        if self.abi.nn_csr_strip_finish(z_local, self.dinv, x) != self.abi.NN_OK:
            raise RuntimeError("nn_csr_strip_finish failed")
        return x


class HostStrip:
    """The same strip interface on the host (SciPy CSR, torch CPU tensors): it stands in for
    ``CudaStrip`` where the host logic runs without a GPU (gloo ranks in the CPU tests)."""

    def __init__(self, plan: HaloPlan, row_ptr: np.ndarray, val: np.ndarray, device="cpu", dtype=None):
        import scipy.sparse as sp
        import torch

        self.plan = plan
        self.n = plan.r1 - plan.r0
        self.n_ext = self.n + len(plan.halo)
        self.dtype = torch.float64
        e0, e1 = int(row_ptr[plan.r0]), int(row_ptr[plan.r1])
        self.raw = np.asarray(val[e0:e1], dtype=np.float64)
        loc = sp.csr_matrix((self.raw, plan.col_local, plan.row_ptr), shape=(self.n, self.n_ext))
        diag = np.asarray(loc[:, :self.n].diagonal())
        if np.any(diag == 0):
            raise ValueError("strip rows without a usable diagonal")
        self.dinv = torch.from_numpy(1.0 / diag)
        self.a = None

    def new_ext(self):
        import torch

        return torch.zeros(self.n_ext, dtype=torch.float64)

    def scale(self, dinv_ext):
        import scipy.sparse as sp

        vals = self.raw * dinv_ext.numpy()[self.plan.col_local]
        self.a = sp.csr_matrix((vals, self.plan.col_local, self.plan.row_ptr), shape=(self.n, self.n_ext))

    def product(self, src_ext, dst_ext, acc_in=None, acc_out=None):
        import torch

        v = src_ext.numpy()
        y = torch.from_numpy(v[:self.n] - self.a @ v)
        if dst_ext is not None:
            dst_ext[:self.n] = y
        if acc_out is not None:
            acc_out.copy_(acc_in + y)

    def residual(self, z_ext, b_local):
        r = b_local.numpy() - self.a @ z_ext.numpy()
        return [float(np.sum(r * r)), float(np.sum(b_local.numpy() ** 2))]

    def finish(self, z_local):
        return self.dinv * z_local


def setup_strips(strips, exchange):
    """Second setup step of the strips this process holds: D^-1 extended over the halo columns
    (one exchange), then the scaled values A' = A D^-1."""
    exts = []
    for s in strips:
        e = s.new_ext()
        e[:s.n] = s.dinv
        exts.append(e)
    exchange(exts)
    for s, e in zip(strips, exts):
        s.scale(e)


class LocalExchange:
    """Halo exchange among strips held by one process (one device): each halo entry is copied from
    the owning strip's extended vector. Call with the strips' extended vectors in plan order."""

    def __init__(self, plans: list[HaloPlan], device):
        import torch

        starts = np.asarray([p.r0 for p in plans])
        self.moves = []
        for k, p in enumerate(plans):
            moves = []
            if p.halo.size:
                owners = np.searchsorted(starts, p.halo, side="right") - 1
                n = p.r1 - p.r0
                for q in np.unique(owners):
                    sel = np.nonzero(owners == q)[0]
                    src = torch.from_numpy(p.halo[sel] - plans[q].r0).to(device)
                    dst = torch.from_numpy(n + sel).to(device)
                    moves.append((int(q), src, dst))
            self.moves.append(moves)

    def __call__(self, exts):
        for k, moves in enumerate(self.moves):
            for q, src, dst in moves:
                exts[k][dst] = exts[q][src]


class DistExchange:
    """Halo exchange of this rank's strip with its neighbours through torch.distributed
    point-to-point operations (NCCL for device tensors, gloo for host tensors)."""

    def __init__(self, plan: HaloPlan, device):
        import torch

        self.plan = plan
        n = plan.r1 - plan.r0
        self.recv = {q: torch.from_numpy(n + np.searchsorted(plan.halo, cols)).to(device)
                     for q, cols in plan.recv.items()}
        self.send = {q: torch.from_numpy(np.asarray(rows, dtype=np.int64)).to(device) for q, rows in plan.send.items()}

    def __call__(self, exts):
        import torch
        import torch.distributed as dist

        ext = exts[0]
        ops, bufs = [], {}
        for q, idx in self.recv.items():
            bufs[q] = torch.empty(idx.numel(), dtype=ext.dtype, device=ext.device)
            ops.append(dist.P2POp(dist.irecv, bufs[q], q))
        for q, idx in self.send.items():
            ops.append(dist.P2POp(dist.isend, ext[idx].contiguous(), q))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        for q, idx in self.recv.items():
            ext[idx] = bufs[q]


def sharded_sparse_chain(strips, exchange, b_locals, depths, allreduce=None):
    """The explicit NN form X = D^-1 prod_j sum_{n=0}^{L_j} P^{n m_j} B over row strips (Corollary 1
    applied per strip; Corollary 6 for a depth per factor), in the order of the single-GPU chain:
    factor j applies its L_j blocks of m_j products, the last product of each block adds its
    result into the factor's accumulator, and the accumulator becomes z. Every product reads an
    extended vector whose halo was just exchanged. ``strips``: the strips this process holds (all
    of them in one process, or its own under torch.distributed), ``exchange``: fills the halos of
    their extended vectors, ``allreduce``: sums a list of floats over processes (None: one
    process). Returns (x_local per strip, relative residual ||B - A X||_F / ||B||_F)."""
    z = [s.new_ext() for s in strips]
    znew = [s.new_ext() for s in strips]
    u = [[s.new_ext(), s.new_ext()] for s in strips]
    for s, zz, b in zip(strips, z, b_locals):
        zz[:s.n] = b
    m = 1
    for j, depth in enumerate(depths):
        if j > 0:
            m *= depths[j - 1] + 1
        src = list(z)
        ping = 0
        for blk in range(1, depth + 1):
            for p in range(1, m + 1):
                last_of_block = p == m
                last_of_factor = last_of_block and blk == depth
                exchange(src)
                dst = [uu[ping] for uu in u]
                for k, s in enumerate(strips):
                    if last_of_block:
                        acc_in = (z[k] if blk == 1 else znew[k])[:s.n]
                        s.product(src[k], None if last_of_factor else dst[k], acc_in, znew[k][:s.n])
                    else:
                        s.product(src[k], dst[k])
                src = dst
                ping ^= 1
        z, znew = znew, z
    exchange(z)
    sums = [0.0, 0.0]
    for s, zz, b in zip(strips, z, b_locals):
        r2, b2 = s.residual(zz, b)
        sums[0] += r2
        sums[1] += b2
    if allreduce is not None:
        sums = list(allreduce(sums))
    rel = float(np.sqrt(sums[0] / sums[1])) if sums[1] > 0 else float(np.sqrt(sums[0]))
    return [s.finish(zz[:s.n]) for s, zz in zip(strips, z)], rel
