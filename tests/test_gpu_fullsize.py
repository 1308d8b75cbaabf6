"""Full-size parity of the dense mixed path at the benchmarked configuration, through the
benchmark's own call.

Both mixed forms (BF16 and FP16 operand pieces) at N = 8192, A = Q diag(lambda) Q^T (Q from
QR of an N(0,1) matrix, lambda log-uniform on [1, 1e2]), X_0 = 2/(lambda_min + lambda_max) I
passed as the x0_scalar hint (the first nest element-wise), depth 2, tol 1e-6: the call bench.py
times. The oracle cannot run N = 8192 nests
in a test, so the checks use what holds at any size and is computable one output at a time:
* the nest count equals the first k where the spectral closed form
  sqrt(sum_j (1 - alpha lambda_j)^(2 3^k)) / N drops below tol (Appendix 2: R_k = R_0^(3^k));
* sampled rows of R = I - A X, recomputed in FP64, give ||R||_F / N < tol, under the call's
  certified residual;
* sampled entries X_ij against the closed form (A^-1)_ij = sum_m Q_im Q_jm / lambda_m, element
  by element: X - A^-1 = -A^-1 R, so |X_ij - (A^-1)_ij| <= ||(A^-1)_{i,:}||_2 ||R_{:,j}||_2
  (Cauchy-Schwarz), with both norms computed in FP64 for the sampled i and j.
A second case runs N = 2048 through the same hinted call and compares every entry of X with
the FP64 oracle's iterate after the same number of nests (Algorithm 1), with the same
element-wise bound built from both iterates' residual columns.
"""
import math

import numpy as np
import pytest

import synth
from oracle import dense

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["mixed_bf16", "mixed_f16"])
def test_mixed_n8192_kappa1e2_depth2_bench_call(dtype):
    import torch

    from paper_2212_02406_gb300 import abi, build

    build.build()
    n, kappa, depth, tol = 8192, 1e2, 2, 1e-6
    A, Q, lam = synth.spd_spectrum_torch(n, kappa, seed=0, device="cuda")
    alpha = 2.0 / (lam[0] + lam[-1])
    X0 = torch.empty_like(A)
    ws = abi.workspace(n, dtype)
    assert abi.nn_init_precond(A, "scalar", alpha, X0, ws) == abi.NN_OK
    X = torch.empty_like(A)
    opts = abi.make_opts(depth, tol, 64, dtype, x0_scalar=alpha)  # the bench's call
    st, res = abi.nn_invert(A, X0, opts, X, ws)
    torch.cuda.synchronize()
    assert st == abi.NN_OK, res
    assert res["residual_est"] < tol

    pred = [math.sqrt(float(np.sum((1.0 - alpha * lam) ** (2 * (depth + 1) ** k)))) / n for k in range(20)]
    k_pred = next(k for k, p in enumerate(pred) if p < tol)
    assert res["nests"] == k_pred, (res["history"], pred[:k_pred + 1])

    r = synth.rng(123)
    rows = torch.from_numpy(r.choice(n, size=48, replace=False)).cuda()
    r_rows = -(A[rows] @ X)
    r_rows[torch.arange(48, device="cuda"), rows] += 1.0
    s_est = float(torch.linalg.norm(r_rows)) / math.sqrt(48 * n)
    assert s_est < tol, s_est
    assert s_est <= 1.5 * res["residual_est"], (s_est, res["residual_est"])

    # element-wise against the spectral closed form of the inverse
    lam_t = torch.as_tensor(lam, device="cuda")
    ii = torch.from_numpy(r.integers(0, n, size=256)).cuda()
    jj = torch.from_numpy(r.integers(0, n, size=256)).cuda()
    qi = Q[ii] / lam_t[None, :]                       # rows i of Q diag(1/lambda)
    inv_ij = torch.einsum("km,km->k", qi, Q[jj])      # (A^-1)_ij
    inv_row_norm = torch.linalg.norm(qi, dim=1)       # ||(A^-1)_{i,:}||_2 (Q orthogonal)
    xj = X[:, jj]                                     # columns j of X
    rcol = -(A @ xj)
    rcol[jj, torch.arange(256, device="cuda")] += 1.0
    rcol_norm = torch.linalg.norm(rcol, dim=0)        # ||R_{:,j}||_2
    x_ij = X[ii, jj]
    bound = inv_row_norm * rcol_norm * (1 + 1e-10) + 1e-14
    diff = (x_ij - inv_ij).abs()
    assert bool(torch.all(diff <= bound)), float(torch.max(diff / bound))
    # and the sampled relative error is small in aggregate
    rel = float(torch.linalg.norm(x_ij - inv_ij) / torch.linalg.norm(inv_ij))
    assert rel <= 2 * math.sqrt(n) * s_est, rel


@pytest.mark.parametrize("dtype", ["mixed_bf16", "mixed_f16"])
def test_mixed_n2048_hinted_equals_oracle_nests(dtype):
    import torch

    from paper_2212_02406_gb300 import abi, build

    build.build()
    n, kappa, depth, tol = 2048, 1e2, 2, 1e-6
    a, q, lam = synth.spd_spectrum(n, kappa, seed=41)
    alpha = 2.0 / (lam[0] + lam[-1])
    x0 = dense.precond_scalar(n, alpha)
    A = torch.from_numpy(a).cuda()
    X0 = torch.from_numpy(x0).cuda()
    X = torch.empty_like(A)
    ws = abi.workspace(n, dtype)
    st, res = abi.nn_invert(A, X0, abi.make_opts(depth, tol, 40, dtype, x0_scalar=alpha), X, ws)
    torch.cuda.synchronize()
    assert st == abi.NN_OK, res
    x = X.cpu().numpy()
    # the FP64 oracle after the same number of nests
    ora = dense.nn_invert(a, x0, depth, tol=0.0, max_nests=res["nests"])
    assert ora.nests == res["nests"]
    r_gpu = dense.residual(a, x)
    r_ora = dense.residual(a, ora.x)
    assert dense.rms_frob(r_gpu) < tol
    # X - X_ora = A^-1 (R_ora - R_gpu): element-wise Cauchy-Schwarz with A^-1 = Q diag(1/lam) Q^T
    inv_rows = np.linalg.norm(q / lam[None, :], axis=1)
    dcol = np.linalg.norm(r_ora - r_gpu, axis=0)
    bound = np.outer(inv_rows, dcol) * (1 + 1e-10) + 1e-14
    assert np.all(np.abs(x - ora.x) <= bound), float(np.max(np.abs(x - ora.x) / bound))
