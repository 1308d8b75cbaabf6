"""Seeded synthetic inputs for the Nested Neumann (NN) inversion workloads.

This module only draws and assembles inputs (matrices, right-hand sides, request
streams). It holds none of the NN method's arithmetic: no residuals, no Neumann
sums, no preconditioner scalings. Both the CPU oracle (``oracle/``) and the CUDA
path (``paper_2212_02406_gb300``) consume what it returns; neither is imported
here.

Every generator takes an explicit integer seed and uses NumPy's PCG64, so the
same call gives the same bytes on x86_64 and aarch64.

Workloads (all synthetic, shaped after the paper's problem classes: dense
positive-definite inversion, Section II-D Theorem; sparse systems, Algorithm 2
and Corollary 6; small complex Gram matrices from massive MIMO, Corollary 4):

* ``spd_wishart``       A = B B^T / N + 0.5 I, B ~ N(0,1)              (dense SPD, N=256 order check)
* ``spd_spectrum``      A = Q diag(lambda) Q^T, Q from QR of N(0,1),
                        lambda log-uniform on [1, kappa], ends pinned   (dense SPD precision sweep)
* ``mimo_gram_batch``   A = H^H H + sigma^2 I, H 128 x U ~ CN(0,1),
                        U uniform over {8,16,24,32,48,64}              (batched complex64)
* ``laplacian_5pt``     2-D 5-point Dirichlet Laplacian + shift I, CSR (sparse SpMV chain)
* ``gaussian_rhs``      N(0,1) right-hand sides
* ``request_stream``    Poisson arrivals of dense SPD requests          (served stream)
* ``rational_spd``      small integer SPD matrices for exact arithmetic
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MIMO_SIZES = (8, 16, 24, 32, 48, 64)
MIMO_ANTENNAS = 128


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def spd_wishart(n: int, seed: int = 0, shift: float = 0.5) -> np.ndarray:
    """A = B B^T / n + shift*I with B_ij ~ N(0,1); FP64, exactly symmetric."""
    b = rng(seed).standard_normal((n, n))
    a = b @ b.T / n
    a = 0.5 * (a + a.T)
    a[np.diag_indices(n)] += shift
    return a


def log_uniform_spectrum(n: int, kappa: float, seed: int) -> np.ndarray:
    """n eigenvalues exp(U[0, ln kappa]) with the ends pinned to 1 and kappa, sorted."""
    r = rng(seed + 7919)
    lam = np.exp(r.uniform(0.0, math.log(kappa), size=n))
    if n >= 1:
        lam[0] = 1.0
    if n >= 2:
        lam[-1] = kappa
    return np.sort(lam)


def haar_orthogonal(n: int, seed: int) -> np.ndarray:
    """Q from the QR factorisation of an N(0,1) matrix, signs fixed so diag(R) > 0."""
    g = rng(seed).standard_normal((n, n))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    return q


def spd_spectrum(n: int, kappa: float, seed: int = 0):
    """A = Q diag(lambda) Q^T with known spectrum; returns (A, Q, lambda), FP64.

    A is symmetrised after the product so it is exactly symmetric.
    """
    lam = log_uniform_spectrum(n, kappa, seed)
    q = haar_orthogonal(n, seed)
    a = (q * lam[None, :]) @ q.T
    a = 0.5 * (a + a.T)
    return a, q, lam


def spd_spectrum_torch(n: int, kappa: float, seed: int = 0, device="cuda"):
    """Same recipe as ``spd_spectrum`` for large n: the Gaussian draw and the spectrum
    come from PCG64 on the host, the QR and the product Q diag(lambda) Q^T run in FP64
    through PyTorch on ``device``. Returns (A, Q, lambda) as FP64 torch tensors on
    ``device`` (lambda as a NumPy array too). Bytes differ from ``spd_spectrum`` only
    by the library QR's rounding; every consumer gets the same returned tensors.
    """
    import torch

    lam = log_uniform_spectrum(n, kappa, seed)
    g = torch.from_numpy(rng(seed).standard_normal((n, n))).to(device)
    q, r = torch.linalg.qr(g)
    q = q * torch.sign(torch.diagonal(r))[None, :]
    del g, r
    lam_t = torch.from_numpy(lam).to(device)
    a = (q * lam_t[None, :]) @ q.T
    a = 0.5 * (a + a.T)
    return a, q, lam


def haar_unitary(n: int, seed: int) -> np.ndarray:
    """Complex Q from the QR factorisation of a CN(0,1) matrix, phases fixed so diag(R) > 0."""
    r = rng(seed)
    g = (r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))) / np.sqrt(2.0)
    q, rr = np.linalg.qr(g)
    d = np.diag(rr)
    return q * (d / np.abs(d))[None, :].conj()


def general_svd(n: int, cond: float, seed: int = 0, complex_: bool = False):
    """A = U diag(sigma) V^H, a general (non-Hermitian) matrix with geometric singular values
    from 1 down to 1/cond and Haar U, V; returns (A, sigma)."""
    sig = np.geomspace(1.0, 1.0 / cond, n)
    if complex_:
        u = haar_unitary(n, seed)
        v = haar_unitary(n, seed + 7919)
    else:
        u = haar_orthogonal(n, seed)
        v = haar_orthogonal(n, seed + 7919)
    return (u * sig[None, :]) @ v.conj().T, sig


def gaussian_rhs(n: int, k: int = 1, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """N x k right-hand sides with N(0,1) entries, column-major (Fortran order)."""
    return np.asfortranarray(rng(seed + 104729).standard_normal((n, k)).astype(dtype))


@dataclass
class MimoBatch:
    """Packed batch of Hermitian Gram matrices A_b = H_b^H H_b + sigma2 I.

    ``data`` holds the matrices back to back, each U_b x U_b row-major complex;
    ``offsets[b]`` is the element offset of matrix b and ``sizes[b]`` its U_b.
    """

    data: np.ndarray
    offsets: np.ndarray
    sizes: np.ndarray

    def matrix(self, b: int) -> np.ndarray:
        u = int(self.sizes[b])
        o = int(self.offsets[b])
        return self.data[o:o + u * u].reshape(u, u)

    @property
    def count(self) -> int:
        return int(self.sizes.shape[0])


def mimo_gram_batch(count: int, seed: int = 0, sigma2: float = 0.1,
                    sizes=MIMO_SIZES, antennas: int = MIMO_ANTENNAS,
                    dtype=np.complex64) -> MimoBatch:
    """``count`` Gram matrices with U_b uniform over ``sizes`` and H entries CN(0,1).

    The Gram product is formed in complex128 and rounded once to ``dtype``; the
    result is made exactly Hermitian with a real diagonal.
    """
    r = rng(seed)
    us = r.choice(np.asarray(sizes, dtype=np.int64), size=count)
    offs = np.zeros(count, dtype=np.int64)
    if count > 1:
        offs[1:] = np.cumsum(us[:-1] * us[:-1])
    total = int(np.sum(us * us))
    out = np.empty(total, dtype=dtype)
    for b in range(count):
        u = int(us[b])
        h = (r.standard_normal((antennas, u)) + 1j * r.standard_normal((antennas, u))) / math.sqrt(2.0)
        a = h.conj().T @ h
        a = 0.5 * (a + a.conj().T)
        a[np.diag_indices(u)] = a[np.diag_indices(u)].real + sigma2
        out[offs[b]:offs[b] + u * u] = a.astype(dtype).reshape(-1)
    return MimoBatch(out, offs, us)


def mimo_sizes(count: int, seed: int = 0, sizes=MIMO_SIZES) -> np.ndarray:
    """The U_b of a batch of ``count`` matrices drawn uniformly over ``sizes`` (first draw of the
    indexed recipe below)."""
    return rng(seed).choice(np.asarray(sizes, dtype=np.int64), size=count)


def mimo_gram_indexed(indices, sizes_all: np.ndarray, seed: int = 0, sigma2: float = 0.1,
                      antennas: int = MIMO_ANTENNAS, dtype=np.complex64) -> MimoBatch:
    """The matrices ``indices`` of a batch whose sizes are ``sizes_all``, each from its own stream
    PCG64([seed, b]) (so any subset is generated alone, e.g. one rank's share of a sharded batch):
    H_b with CN(0,1) entries, A_b = H_b^H H_b + sigma2 I in complex128, rounded once."""
    idx = np.asarray(indices, dtype=np.int64)
    us = np.asarray(sizes_all)[idx].astype(np.int64)
    offs = np.zeros(len(idx), dtype=np.int64)
    if len(idx) > 1:
        offs[1:] = np.cumsum(us[:-1] * us[:-1])
    out = np.empty(int(np.sum(us * us)), dtype=dtype)
    for k, b in enumerate(idx):
        u = int(us[k])
        r = np.random.Generator(np.random.PCG64([seed, int(b)]))
        h = (r.standard_normal((antennas, u)) + 1j * r.standard_normal((antennas, u))) / math.sqrt(2.0)
        a = h.conj().T @ h
        a = 0.5 * (a + a.conj().T)
        a[np.diag_indices(u)] = a[np.diag_indices(u)].real + sigma2
        out[offs[k]:offs[k] + u * u] = a.astype(dtype).reshape(-1)
    return MimoBatch(out, offs, us)


@dataclass
class Csr:
    """Compressed sparse row matrix with int32 indices (n rows, n columns)."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))


def laplacian_5pt(nx: int, ny: int | None = None, shift: float = 0.5,
                  dtype=np.float64) -> Csr:
    """5-point Dirichlet Laplacian on an nx x ny grid plus shift*I, CSR.

    Row r = iy*nx + ix has diagonal 4 + shift and -1 for each in-grid neighbour,
    columns sorted ascending. No randomness.
    """
    ny = nx if ny is None else ny
    n = nx * ny
    ix = np.arange(n, dtype=np.int64) % nx
    iy = np.arange(n, dtype=np.int64) // nx
    has_s = iy > 0
    has_w = ix > 0
    has_e = ix < nx - 1
    has_n = iy < ny - 1
    deg = 1 + has_s.astype(np.int64) + has_w + has_e + has_n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int64)
    val = np.empty(nnz, dtype=np.float64)
    pos = row_ptr[:-1].copy()
    r = np.arange(n, dtype=np.int64)
    # Column order: south (r-nx) < west (r-1) < diagonal < east (r+1) < north (r+nx).
    for mask, off, v in ((has_s, -nx, -1.0), (has_w, -1, -1.0), (None, 0, 4.0 + shift),
                         (has_e, 1, -1.0), (has_n, nx, -1.0)):
        rows = r if mask is None else r[mask]
        p = pos[rows]
        col[p] = rows + off
        val[p] = v
        pos[rows] += 1
    return Csr(n, row_ptr.astype(np.int32), col.astype(np.int32), val.astype(dtype))


def random_sparse_spd(n: int, per_row: int = 6, seed: int = 0, dtype=np.float64) -> Csr:
    """Symmetric, strictly diagonally dominant sparse matrix with ragged row lengths."""
    import scipy.sparse as sp

    r = rng(seed)
    rows = np.repeat(np.arange(n), per_row)
    cols = r.integers(0, n, size=n * per_row)
    vals = r.uniform(-1.0, 1.0, size=n * per_row)
    m = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    m = m + m.T
    m.setdiag(0.0)
    m.eliminate_zeros()
    d = np.asarray(abs(m).sum(axis=1)).ravel() + 1.0 + r.uniform(0.0, 1.0, size=n)
    m = (m + sp.diags(d)).tocsr()
    m.sort_indices()
    return Csr(n, m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(dtype))


@dataclass
class Request:
    rid: int
    arrival_s: float
    n: int
    kappa: float
    nrhs: int
    dtype: str  # "f32" or "bf16"
    seed: int


def request_stream(count: int, rate_per_s: float, seed: int = 0,
                   n_min: int = 16, n_max: int = 2048,
                   kappa_min: float = 10.0, kappa_max: float = 1e3,
                   max_rhs: int = 64) -> list[Request]:
    """Poisson arrivals; N log-uniform in [n_min, n_max], kappa log-uniform in
    [kappa_min, kappa_max], 1..max_rhs right-hand sides, dtype FP32/BF16 at 50/50."""
    r = rng(seed)
    gaps = r.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    ns = np.rint(np.exp(r.uniform(math.log(n_min), math.log(n_max), size=count))).astype(int)
    ks = np.exp(r.uniform(math.log(kappa_min), math.log(kappa_max), size=count))
    nr = r.integers(1, max_rhs + 1, size=count)
    dt = np.where(r.uniform(size=count) < 0.5, "f32", "bf16")
    seeds = r.integers(0, 2**31 - 1, size=count)
    return [Request(i, float(t[i]), int(ns[i]), float(ks[i]), int(nr[i]), str(dt[i]), int(seeds[i]))
            for i in range(count)]


def rational_spd(n: int, seed: int = 0, lo: int = -3, hi: int = 3):
    """Small integer SPD matrix B B^T + n I as nested Python int lists (exact input)."""
    r = rng(seed)
    b = r.integers(lo, hi + 1, size=(n, n))
    a = b @ b.T + n * np.eye(n, dtype=np.int64)
    return [[int(a[i, j]) for j in range(n)] for i in range(n)]
