"""CPU-side checks of the C ABI: the library builds, loads, and exports every entry point
the headers in include/ declare; argument errors come back as status codes before any
device work (so these run without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2212_02406_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(nn_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.lib()


def test_every_declared_symbol_is_exported_and_bound(lib):
    declared = _declared()
    assert declared, "no declarations found in include/"
    for name in declared:
        assert hasattr(lib, name), f"{name} declared but not exported"
    assert declared == set(abi.exported_symbols())


def test_opts_struct_matches_header(lib):
    # NNOpts mirrors nn_opts field for field (the C struct gained x0_scalar at the end)
    text = open(os.path.join(ROOT, "include", "nn.h")).read()
    body = re.search(r"typedef struct nn_opts \{(.*?)\} nn_opts;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)\s*;", body)
    assert fields == [f for f, _ in abi.NNOpts._fields_]


def test_result_struct_matches_header(lib):
    # NNResult mirrors nn_result field for field (array members included)
    text = open(os.path.join(ROOT, "include", "nn.h")).read()
    body = re.search(r"typedef struct nn_result \{(.*?)\} nn_result;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)\s*(?:\[\w+\])?\s*;", body)
    assert fields == [f for f, _ in abi.NNResult._fields_]


def test_workspace_sizes(lib):
    assert abi.nn_workspace_bytes(0, "f64") == 0
    assert abi.nn_workspace_bytes(16, 99) == 0
    for dt in ("f64", "f32", "mixed_bf16", "mixed_f16"):
        a = abi.nn_workspace_bytes(100, dt)
        b = abi.nn_workspace_bytes(1000, dt)
        assert 0 < a < b
        assert abi.nn_workspace_bytes_host(1000, dt) >= b + 3 * 1000 * 1000 * 8
    # the mixed path pads to multiples of 128; FP16 and BF16 pieces share one layout
    assert abi.nn_workspace_bytes(129, "mixed_bf16") == abi.nn_workspace_bytes(256, "mixed_bf16")
    assert abi.nn_workspace_bytes(1000, "mixed_f16") == abi.nn_workspace_bytes(1000, "mixed_bf16")


def test_argument_errors_are_status_codes(lib):
    res = abi.NNResult()
    opts = abi.make_opts(depth=0)
    st = lib.nn_invert(None, 16, 16, None, 16, ctypes.byref(opts), None, 16, ctypes.byref(res), None, 0, None)
    assert st == abi.NN_ERR_ARG and res.status == abi.NN_ERR_ARG
    opts = abi.make_opts(depth=2, max_nests=65)
    assert lib.nn_invert(None, 16, 16, None, 16, ctypes.byref(opts), None, 16, ctypes.byref(res), None, 0,
                         None) == abi.NN_ERR_ARG
    opts = abi.make_opts(depth=2)
    assert lib.nn_invert(None, 16, 16, None, 16, ctypes.byref(opts), None, 16, None, None, 0, None) == abi.NN_ERR_ARG
    for bad in (-1.0, float("nan"), float("inf")):  # the X_0 = x0_scalar I hint must be >= 0 and finite
        opts = abi.make_opts(depth=2, dtype="mixed_bf16", x0_scalar=bad)
        assert lib.nn_invert(None, 16, 16, None, 16, ctypes.byref(opts), None, 16, ctypes.byref(res), None, 0,
                             None) == abi.NN_ERR_ARG
    for bad in (-1e-6, float("nan"), float("inf")):  # the forward-error target must be >= 0 and finite
        opts = abi.make_opts(depth=2, dtype="mixed_emu", fwd_tol=bad)
        assert lib.nn_invert(None, 16, 16, None, 16, ctypes.byref(opts), None, 16, ctypes.byref(res), None, 0,
                             None) == abi.NN_ERR_ARG
    out = ctypes.c_double()
    assert lib.nn_residual(None, 4, None, 4, 4, abi.NN_F64, ctypes.byref(out), None, 0, None) == abi.NN_ERR_ARG
    assert lib.nn_init_precond(None, 4, 4, 0, 0.0, None, 4, None, 0, None) == abi.NN_ERR_ARG


def test_solve_and_batched_interface_names(lib):
    # The solve (A X = B, the problem statement; Algorithm 2) and batched (Corollary 4's mMIMO use)
    # entry points in the interface's argument order: each is called through ctypes and answers a
    # bad argument with NN_ERR_ARG before any device work.
    res = abi.NNResult()
    opts = abi.make_opts(depth=2, max_nests=3, dtype="f64")
    assert lib.nn_solve(None, None, None, 16, 48, None, 16, 1, 2, 0.0, ctypes.byref(opts), None, 16,
                        ctypes.byref(res), None, 0, None) == abi.NN_ERR_ARG
    assert res.status == abi.NN_ERR_ARG
    assert lib.nn_solve(None, None, None, 16, 48, None, 16, 1, 2, 0.0, None, None, 16, ctypes.byref(res), None, 0,
                        None) == abi.NN_ERR_ARG
    sched = abi.make_opts(depth=2, max_nests=3, dtype="f64", depth_schedule=[2, 0])  # depth 0 is invalid
    assert lib.nn_solve(None, None, None, 16, 48, None, 16, 1, 2, 0.0, ctypes.byref(sched), None, 16,
                        ctypes.byref(res), None, 0, None) == abi.NN_ERR_ARG
    assert lib.nn_invert_batched(None, None, None, 4, 2, 3, 0.0, None, 1, None, None, None, None, 0,
                                 None) == abi.NN_ERR_ARG
    # the normal-equation solve of Corollary 3, too
    assert lib.nn_solve_normal(None, 4, 4, 0, None, 4, 1, ctypes.byref(opts), None, 1, ctypes.byref(res), None, 0,
                               None) == abi.NN_ERR_ARG


def _header_int(name):
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", open(h).read())
        if m:
            return int(m.group(1))
    raise AssertionError(f"{name} not defined in include/")


def _plan_class(cfg, u):
    """Tile class of an item as the header defines it: 0, 1 = tensor cores for U = 64, 48;
    CUDA-core classes ordered by threads per matrix (16 x 16 first), tile (4 down to 1), exact
    U first."""
    if cfg == 3:
        return 18 + (4 - u // 8)
    if cfg == 2:
        return 0 if u == 64 else 1
    tg = 8 if cfg == 0 else 16
    t = -(-u // tg)
    return 2 + (8 if cfg == 0 else 0) + (4 - t) * 2 + (0 if u % tg == 0 else 1)


@pytest.mark.parametrize("cfg_by_u", [None, {u: 0 for u in range(1, 33)}, {16: 2, 32: 2, 48: 2, 64: 2, 40: 2},
                                      {u: 3 for u in range(1, 65)}])
def test_batched_plan_layout(lib, cfg_by_u):
    """nn_batched_plan (host only): every matrix appears once, sizes within an item are equal,
    items of a tile class are contiguous and largest first, and the class table brackets them."""
    import numpy as np

    assert abi.NN_BATCHED_KERNELS == _header_int("NN_BATCHED_KERNELS")
    ncls = abi.NN_BATCHED_KERNELS
    rng = np.random.default_rng(7)
    sizes = rng.integers(1, 65, size=3000).astype(np.int32)
    sizes[:50] = 64
    plan = abi.nn_batched_plan(sizes, cfg_by_u)
    n_items, count, n_tc = int(plan[0]), int(plan[1]), int(plan[2])
    class_first = plan[3:3 + ncls + 1]
    hdr = 3 + ncls + 1
    order = plan[hdr:hdr + count]
    items = plan[hdr + count:hdr + count + 4 * n_items].reshape(n_items, 4)
    assert count == len(sizes) and len(plan) == hdr + 5 * count
    assert sorted(order.tolist()) == list(range(count))
    assert np.all(np.diff(sizes[order]) <= 0)
    assert class_first[0] == 0 and class_first[-1] == n_items and n_tc == class_first[2]
    assert np.all(np.diff(class_first) >= 0)
    covered = np.zeros(count, dtype=bool)
    for c in range(ncls):
        prev_u = 65
        for it in range(class_first[c], class_first[c + 1]):
            u, start, cnt, cfg = (int(v) for v in items[it])
            assert _plan_class(cfg, u) == c
            assert u <= prev_u
            prev_u = u
            assert 1 <= cnt and (cfg == 0 or cnt == 1) and cnt <= 4
            assert cfg != 2 or u in (48, 64)
            assert cfg != 3 or u in (8, 16, 24, 32)
            assert cfg != 0 or u <= 32
            assert np.all(sizes[order[start:start + cnt]] == u)
            assert not covered[start:start + cnt].any()
            covered[start:start + cnt] = True
    assert covered.all()
    mask = abi.nn_batched_plan_classes(plan)
    assert mask == sum(1 << c for c in range(ncls) if class_first[c + 1] > class_first[c])
    if cfg_by_u and cfg_by_u.get(64) == 2:
        assert n_tc > 0 and all(int(items[i, 0]) in (48, 64) for i in range(n_tc))


def test_dtype_constants_match_header():
    # the binding's dtype numbers are the header's enum values
    import os
    import re

    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "nn.h")).read()
    block = hdr[hdr.index("typedef enum nn_dtype"):]
    block = block[:block.index("} nn_dtype;")]
    block = re.sub(r"/\*.*?\*/", "", block, flags=re.S)
    values = {name: int(v) for name, v in re.findall(r"(NN_\w+)\s*=\s*(\d+)", block)}
    assert values["NN_MIXED_F16"] == abi.NN_MIXED_F16 == abi.DTYPES["mixed_f16"]
    for name, key in (("NN_F64", "f64"), ("NN_F32", "f32"), ("NN_MIXED_BF16", "mixed_bf16"),
                      ("NN_F64_DF", "f64_df"), ("NN_F64_EMU", "f64_emu"), ("NN_MIXED_EMU", "mixed_emu")):
        assert values[name] == abi.DTYPES[key], name
