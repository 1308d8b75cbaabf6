"""The no-allocation residual entry point (nn_residual_noalloc), checked against nn_residual.

Callers that cannot allocate device memory (code inside a CUDA graph capture, services that
forbid allocation after start-up, or hosts whose device memory is owned by another framework)
use this variant: its scratch is a fixed array inside the library. This file is named so that
pytest collects it last; it passes on its own in a fresh process (the first call on the device
resolves the scratch address) and after every other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_workspace_residual_twice():
    import torch

    from paper_2212_02406_gb300 import abi, build

    build.build()
    abi.lib()
    # two calls in a row, the second on a smaller problem: leftovers of the first call in the
    # shared scratch must not leak into the second result
    for n, seed in ((abi.NN_RESIDUAL_NOALLOC_MAX_N, 1), (257, 2)):
        a = synth.spd_wishart(n, seed=seed)
        x = np.linalg.inv(a) * (1 + 1e-3)
        A = torch.from_numpy(a).cuda()
        X = torch.from_numpy(x).cuda()
        ws = abi.workspace(n, "f64")
        st_ref, s_ref = abi.nn_residual(A, X, "f64", ws)
        del ws
        st, s = abi.nn_residual_noalloc(A, X)
        torch.cuda.synchronize()
        assert st_ref == abi.NN_OK and st == abi.NN_OK
        # the same tolerance as the workspace residual's own test against the oracle
        assert abs(s - s_ref) <= 1e-10 * s_ref, (n, s, s_ref)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch

    from paper_2212_02406_gb300 import abi

    n = abi.NN_RESIDUAL_NOALLOC_MAX_N + 1
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st, _ = abi.nn_residual_noalloc(A, A)
    assert st == abi.NN_ERR_TOO_LARGE
