"""The batched GPU tolerance, c G sqrt(U) u32 with c = 3, pinned on the CPU.

The tensor-core classes form each complex product P Q of order U from three BF16 pieces of every
real operand (24 significant bits: FP32 inputs exactly up to 2^-24, dropped piece pairs under
2^-25) accumulated in FP32, the CUDA-core classes from FP32 FMA chains; either way one product
carries about sqrt(U) u32 of relative rounding (U terms of random sign). A nest of depth L maps a
perturbation of X by the factor (L+1) r^L along an eigenvalue r of its residual (X p(AX) with
p(z) = sum_n (1-z)^n has derivative p(z) + z p'(z) = (L+1) r^L at z = 1 - r), so rounding made
in nest j reaches X_nests multiplied by prod_{i>j} (L+1) rho_i^L, rho_i = rho_0^((L+1)^i) the
residual's spectral radius after i nests (R_i = R_0^((L+1)^i), Appendix 2). With
G = sum_j prod_{i>j} (L+1) rho_i^L the GPU tests accept c G sqrt(U) u32, c = 2, against the
complex128 oracle's iterate (Corollary 4's mMIMO use of Algorithm 1).

This file checks, on the CPU, that the bound separates what it must: a model of the loop with
three-piece products stays well inside it for every matrix, while a model with two pieces per
operand (relative error 2^-17 per product, what a kernel that dropped a piece would compute)
falls outside it for most matrices of a batch, so a batch test catches it. The model is test
code for the tolerance only; the oracle stays the plain complex128 loop.
"""
import math

import numpy as np
import pytest

import synth
from oracle import batched

from batched_bounds import C_BATCHED, U32, amplification


def _bf16(x):
    """Round float32 values to BF16 (nearest, ties to even), returned as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _pieces(x, p):
    out, rem = [], np.asarray(x, dtype=np.float32)
    for _ in range(p):
        h = _bf16(rem)
        out.append(h)
        rem = (rem - h).astype(np.float32)
    return out


def _real_product(a, b, p):
    """sum over piece pairs (i, j), i + j < p, of A_i B_j: each pair exact, K chunks of 16 summed
    exactly, chunks and pairs accumulated in FP32 (the tensor core's FP32 accumulator)."""
    ap, bp = _pieces(a, p), _pieces(b, p)
    acc = np.zeros((a.shape[0], b.shape[1]), dtype=np.float32)
    k = a.shape[1]
    for d in range(p - 1, -1, -1):
        for i in range(d, -1, -1):
            j = d - i
            for k0 in range(0, k, 16):
                part = ap[i][:, k0:k0 + 16].astype(np.float64) @ bp[j][k0:k0 + 16, :].astype(np.float64)
                acc = (acc + part.astype(np.float32)).astype(np.float32)
    return acc


def _cproduct(p_, q_, pieces):
    pr, pi = p_.real.astype(np.float32), p_.imag.astype(np.float32)
    qr, qi = q_.real.astype(np.float32), q_.imag.astype(np.float32)
    cr = _real_product(pr, qr, pieces) - _real_product(pi, qi, pieces)
    ci = _real_product(pi, qr, pieces) + _real_product(pr, qi, pieces)
    return (cr.astype(np.float32) + 1j * ci.astype(np.float32)).astype(np.complex64)


def _model_loop(a, depth, nests, damping, pieces):
    """The batched kernel's loop in complex64 with piece products: X_0 = diag(A)^-1 / (1 + damping U),
    the first nest element-wise (X_0 diagonal), then R = I - A X, T = R, T = R + R T, X = X + X T."""
    u = a.shape[0]
    a = a.astype(np.complex64)
    d = (1.0 / (1.0 + damping * u)) / np.diag(a)
    eye = np.eye(u, dtype=np.complex64)
    r = (eye - a * d[None, :]).astype(np.complex64)            # R_0 = I - A X_0 (column scaling)
    t = r
    for _ in range(depth - 1):
        t = (r + _cproduct(r, t, pieces)).astype(np.complex64)
    x = (d[:, None] * (eye + t)).astype(np.complex64)           # X_1 = X_0 (I + T) (row scaling)
    for _ in range(1, nests):
        r = (eye - _cproduct(a, x, pieces)).astype(np.complex64)
        t = r
        for _ in range(depth - 1):
            t = (r + _cproduct(r, t, pieces)).astype(np.complex64)
        x = (x + _cproduct(x, t, pieces)).astype(np.complex64)
    return x


@pytest.mark.parametrize("damping,depth,nests", [(1.0 / 128.0, 2, 3), (1.0 / 128.0, 1, 3), (1.0 / 128.0, 3, 3),
                                                  (1.0 / 128.0, 2, 4), (0.0, 2, 3)])
def test_three_pieces_inside_two_pieces_outside(damping, depth, nests):
    bt = synth.mimo_gram_batch(36, seed=depth + 7 * nests, sizes=(8, 16, 24, 32, 48, 64))
    inside, outside, total = 0.0, 0, 0
    for k in range(bt.count):
        a = bt.matrix(k).astype(np.complex128)
        u = a.shape[0]
        run = batched.nn_batched([a], depth, nests, damping=lambda n: 1.0 / (1.0 + damping * n))[0]
        if run.status != 0:
            continue
        total += 1
        bound = C_BATCHED * amplification(a, depth, nests, damping) * math.sqrt(u) * U32
        e3 = np.linalg.norm(_model_loop(a, depth, nests, damping, 3) - run.x) / np.linalg.norm(run.x)
        e2 = np.linalg.norm(_model_loop(a, depth, nests, damping, 2) - run.x) / np.linalg.norm(run.x)
        inside = max(inside, e3 / bound)
        outside += int(e2 > bound)
    assert total >= 12
    assert inside <= 0.5, inside             # three pieces: at most half the bound
    assert outside >= total // 2, (outside, total)  # two pieces: most matrices exceed it
