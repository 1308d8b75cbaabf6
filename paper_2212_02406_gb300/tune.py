"""Autotuner for the batched small-matrix kernel's thread tiling.

For every matrix size U it times nn_invert_batched_c64 on a homogeneous batch under each
configuration (0: CUDA cores, 8 x 8 threads per matrix, up to four matrices per CTA; 1: CUDA
cores, 16 x 16 threads per matrix; 2: tensor cores, U in {48, 64}; 3: CUDA cores, one warp
per matrix, U in {8, 16, 24, 32}) and keeps the
fastest. The result is a table U -> configuration, written
as JSON and passed to nn_batched_plan by callers (bench.py reads
``paper_2212_02406_gb300/batched_tuning.json``).

Usage on a GPU: ``python -m paper_2212_02406_gb300.tune --out batched_tuning.json``.
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def time_config(abi, torch, u: int, cfg: int, count: int, depth: int, nests: int, reps: int, seed: int) -> float:
    import numpy as np

    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.full(count, u, dtype=np.int32)
    offsets = np.arange(count, dtype=np.int64) * u * u
    # well-conditioned Hermitian test matrices: the timing does not depend on the values
    h = (rng.standard_normal((count, 2 * u, u)) + 1j * rng.standard_normal((count, 2 * u, u))) / np.sqrt(2.0)
    a = np.einsum("bki,bkj->bij", h.conj(), h) + 0.1 * np.eye(u)[None]
    A = torch.from_numpy(a.astype(np.complex64).reshape(-1)).cuda()
    X = torch.empty_like(A)
    offs = torch.from_numpy(offsets).cuda()
    sz = torch.from_numpy(sizes).cuda()
    plan_host = abi.nn_batched_plan(sizes, {u: cfg})
    classes = abi.nn_batched_plan_classes(plan_host)
    plan = torch.from_numpy(plan_host).cuda()
    res = torch.empty(count, dtype=torch.float32, device="cuda")
    st = torch.empty(count, dtype=torch.int32, device="cuda")
    ws = torch.empty(abi.nn_batched_workspace_bytes(count), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        abi.nn_invert_batched_c64(A, offs, sz, plan, depth, nests, 1.0 / 128, X, res, st, ws, classes=classes)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        abi.nn_invert_batched_c64(A, offs, sz, plan, depth, nests, 1.0 / 128, X, res, st, ws, classes=classes)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(sizes=(8, 16, 24, 32, 48, 64), count=4096, depth=2, nests=3, reps=5):
    import torch

    from . import abi, build

    build.build()
    abi.lib()
    table, timings = {}, {}
    for u in sizes:
        best = None
        for cfg in (0, 1, 2, 3):
            if cfg == 1 and (u + 15) // 16 > 4:
                continue
            if cfg == 2 and u not in (48, 64):
                continue
            if cfg == 3 and u not in (8, 16, 24, 32):
                continue
            ms = time_config(abi, torch, u, cfg, count, depth, nests, reps, seed=u)
            timings[f"{u}:{cfg}"] = ms
            if best is None or ms < best[1]:
                best = (cfg, ms)
        table[u] = best[0]
    return table, timings


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "batched_tuning.json"))
    ap.add_argument("--count", type=int, default=4096)
    args = ap.parse_args(argv)
    table, timings = tune(count=args.count)
    with open(args.out, "w") as f:
        json.dump({"cfg_by_u": {str(k): v for k, v in table.items()}, "ms_per_batch": timings,
                   "batch": args.count, "depth": 2, "nests": 3}, f, indent=1)
    print(json.dumps({"cfg_by_u": table, "ms": timings}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
