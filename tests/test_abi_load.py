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


def test_workspace_sizes(lib):
    assert abi.nn_workspace_bytes(0, "f64") == 0
    assert abi.nn_workspace_bytes(16, 99) == 0
    for dt in ("f64", "f32", "mixed_bf16"):
        a = abi.nn_workspace_bytes(100, dt)
        b = abi.nn_workspace_bytes(1000, dt)
        assert 0 < a < b
        assert abi.nn_workspace_bytes_host(1000, dt) >= b + 3 * 1000 * 1000 * 8
    # the mixed path pads to multiples of 128
    assert abi.nn_workspace_bytes(129, "mixed_bf16") == abi.nn_workspace_bytes(256, "mixed_bf16")


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
    out = ctypes.c_double()
    assert lib.nn_residual(None, 4, None, 4, 4, abi.NN_F64, ctypes.byref(out), None, 0, None) == abi.NN_ERR_ARG
    assert lib.nn_init_precond(None, 4, 4, 0, 0.0, None, 4, None, 0, None) == abi.NN_ERR_ARG
