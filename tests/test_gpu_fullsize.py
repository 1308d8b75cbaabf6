"""Full-size parity of the dense mixed path at the benchmarked configuration.

N = 8192, A = Q diag(lambda) Q^T (Q from QR of an N(0,1) matrix, lambda log-uniform on
[1, 1e2]), X_0 = 2/(lambda_min + lambda_max) I, depth 2, tol 1e-6: the same call bench.py
times. The oracle cannot run N = 8192 nests in a test, so the check uses what holds at
any size and is computable one output at a time:
* the nest count equals the first k where the spectral closed form
  sqrt(sum_j (1 - alpha lambda_j)^(2 3^k)) / N drops below tol (Appendix 2: R_k = R_0^(3^k));
* sampled rows of R = I - A X, recomputed in FP64 on the host, give ||R||_F / N < tol;
* sampled entries of X against (A^-1)_ij = sum_m Q_im Q_jm / lambda_m, within the forward
  error bound 2 sqrt(N) s + 16 kappa u32.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_mixed_bf16_n8192_kappa1e2_depth2():
    import torch

    from paper_2212_02406_gb300 import abi, build

    build.build()
    n, kappa, depth, tol = 8192, 1e2, 2, 1e-6
    A, Q, lam = synth.spd_spectrum_torch(n, kappa, seed=0, device="cuda")
    alpha = 2.0 / (lam[0] + lam[-1])
    X0 = torch.empty_like(A)
    ws = abi.workspace(n, "mixed_bf16")
    assert abi.nn_init_precond(A, "scalar", alpha, X0, ws) == abi.NN_OK
    X = torch.empty_like(A)
    st, res = abi.nn_invert(A, X0, abi.make_opts(depth, tol, 64, "mixed_bf16"), X, ws)
    torch.cuda.synchronize()
    assert st == abi.NN_OK, res

    pred = [math.sqrt(float(np.sum((1.0 - alpha * lam) ** (2 * (depth + 1) ** k)))) / n for k in range(20)]
    k_pred = next(k for k, p in enumerate(pred) if p < tol)
    assert res["nests"] == k_pred, (res["history"], pred[:k_pred + 1])

    r = synth.rng(123)
    rows = r.choice(n, size=48, replace=False)
    x_host = X.cpu().numpy()
    a_rows = A[torch.from_numpy(rows).cuda()].cpu().numpy()
    r_rows = -a_rows @ x_host
    r_rows[np.arange(len(rows)), rows] += 1.0
    s_est = math.sqrt(float(np.mean(np.sum(r_rows ** 2, axis=1)))) / math.sqrt(n)
    assert s_est < tol, s_est

    q_host = Q.cpu().numpy()
    ii = r.integers(0, n, size=256)
    jj = r.integers(0, n, size=256)
    inv_ij = np.einsum("km,km->k", q_host[ii] / lam[None, :], q_host[jj])
    x_ij = x_host[ii, jj]
    rel = math.sqrt(float(np.sum((x_ij - inv_ij) ** 2) / np.sum(inv_ij ** 2)))
    assert rel <= 2 * math.sqrt(n) * s_est + 16 * kappa * 2.0 ** -24, (rel, s_est)
