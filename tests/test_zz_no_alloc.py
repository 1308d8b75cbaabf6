"""The no-allocation residual entry point (nn_residual_noalloc), checked against the FP64
oracle and against nn_residual.

Services that forbid device allocation after start-up, and plug-ins whose host framework owns
all device memory and hands them only the operands, cannot pass a workspace: this variant keeps
its scratch in a fixed array inside the library. This file is named so that pytest collects it
last; it passes on its own in a fresh process (the first call on the device resolves the
scratch address) and after every other test.
"""
import numpy as np
import pytest

import synth
from oracle import dense

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_oracle_and_workspace_residual_twice():
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
        # the FP64 oracle's s = ||I - A X||_F / N (Section II error measure); the GPU sums the
        # same N-term products in another order, so the difference is a few units of 2^-53
        # times N ||A|| ||X|| / ||R||: 1e-10 relative covers it with a wide margin here
        s_ora = dense.rms_frob(dense.residual(a, x))
        assert abs(s - s_ora) <= 1e-10 * s_ora, (n, s, s_ora)
        # and the workspace entry point's value, to the same tolerance
        assert abs(s - s_ref) <= 1e-10 * s_ref, (n, s, s_ref)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch

    from paper_2212_02406_gb300 import abi

    n = abi.NN_RESIDUAL_NOALLOC_MAX_N + 1
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st, _ = abi.nn_residual_noalloc(A, A)
    assert st == abi.NN_ERR_TOO_LARGE
