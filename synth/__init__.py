"""Seeded synthetic test matrices for PbP-QLP (inputs only).

This module holds none of the factorization's arithmetic.  It builds the
matrix families of the paper's experiments (Section V-B: Haar-random U and V
with a prescribed spectrum; low-rank plus noise) and of the benchmark
workloads, from numpy's PCG64 stream (CPU) or torch's generator (device).
Both the CUDA path's tests and the CPU oracle take their inputs from here;
the Gaussian test matrix Phi of the method itself is NOT drawn here (each
side draws it from the counter-based Philox stream, or it is passed in).
"""
import math

import numpy as np


# ---------------------------------------------------------------- numpy (CPU)
def haar_columns(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """First ``cols`` columns of a Haar-distributed rows x rows orthogonal matrix.

    QR of a rows x cols standard Gaussian matrix with the column signs fixed so
    that diag(R) > 0 (Mezzadri 2007); the leading columns of a Haar matrix
    have exactly this distribution.
    """
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s


def spectrum(kind: str, count: int, param: float) -> np.ndarray:
    """Singular values sigma_1..sigma_count (1-based i).

    kind 'poly': i^-param; 'exp': exp(-i/param); 'linear_lowrank': the paper's
    Matrix 1 values, linspace(1, 1e-25, n)[:param] then zeros (param = k).
    """
    i = np.arange(1, count + 1, dtype=np.float64)
    if kind == "poly":
        return i ** (-float(param))
    if kind == "exp":
        return np.exp(-i / float(param))
    raise ValueError(kind)


def svd_matrix(seed: int, m: int, n: int, sigma: np.ndarray) -> np.ndarray:
    """A = U diag(sigma) V^T with Haar U (m x r), V (n x r), r = len(sigma)."""
    rng = np.random.default_rng(seed)
    r = len(sigma)
    U = haar_columns(rng, m, r)
    V = haar_columns(rng, n, r)
    return (U * sigma) @ V.T


def poly_decay(seed: int, m: int, n: int, alpha: float, rank: int = None) -> np.ndarray:
    """Haar U, V with sigma_i = i^-alpha (the paper's Matrix 4 for alpha = 2)."""
    r = min(m, n) if rank is None else rank
    return svd_matrix(seed, m, n, spectrum("poly", r, alpha))


def exp_decay(seed: int, m: int, n: int, scale: float, rank: int = None) -> np.ndarray:
    """Haar U, V with sigma_i = exp(-i/scale) (the paper's Matrix 3 for scale = 6)."""
    r = min(m, n) if rank is None else rank
    return svd_matrix(seed, m, n, spectrum("exp", r, scale))


def low_rank_plus_noise(seed: int, n: int, k: int, mu: float) -> np.ndarray:
    """The paper's Matrix 1: U diag(linspace(1,1e-25,n)[:k]) V^T + mu sigma_k N,
    N a Gaussian matrix normalised to ||N||_2 = 1."""
    rng = np.random.default_rng(seed)
    sig = np.linspace(1.0, 1e-25, n)[:k]
    U = haar_columns(rng, n, k)
    V = haar_columns(rng, n, k)
    N = rng.standard_normal((n, n))
    N /= np.linalg.norm(N, 2)
    return (U * sig) @ V.T + mu * sig[-1] * N


def rank_r(seed: int, m: int, n: int, r: int) -> np.ndarray:
    """Exactly rank-r Gaussian product X Y^T / sqrt(r)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) / math.sqrt(r)


def xyt_plus_noise(seed: int, m: int, n: int, r: int, eps: float, dtype=np.float32) -> np.ndarray:
    """A = X Y^T + eps E with X (m x r), Y (n x r), E (m x n) N(0,1) in ``dtype``."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, r)).astype(dtype)
    Y = rng.standard_normal((n, r)).astype(dtype)
    E = rng.standard_normal((m, n)).astype(dtype)
    return (X @ Y.T + dtype(eps) * E).astype(dtype)


def sparse_csr(seed: int, m: int, n: int, nnz_per_row: float, *, rank: int = 0, support: int = 0,
               decay: float = 20.0, dup_frac: float = 0.0, shuffle: bool = False, empty_rows: int = 0,
               empty_cols: int = 0):
    """Seeded sparse m x n matrix in CSR form: (rowptr int64, colind int32, values FP64).

    Noise part: about ``nnz_per_row`` N(0,1) entries per row at uniform
    columns.  Optional low-rank part: ``rank`` terms s_i u_i v_i^T with
    s_i = exp(-i / decay) * sqrt(m n) and u_i, v_i unit vectors supported on
    ``support`` random rows / columns.  ``dup_frac`` of the entries are split
    into two repeated (row, column) pairs that add up to the value;
    ``shuffle`` permutes the entries within each row; the first
    ``empty_rows`` rows and the last ``empty_cols`` columns hold nothing.
    """
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    live_r = np.arange(empty_rows, m)
    ncols_live = n - empty_cols
    cnt = rng.poisson(nnz_per_row, size=live_r.size)
    rows.append(np.repeat(live_r, cnt))
    cols.append(rng.integers(0, ncols_live, size=int(cnt.sum())))
    vals.append(rng.standard_normal(int(cnt.sum())))
    for i in range(rank):
        su = min(support, live_r.size)
        sv = min(support, ncols_live)
        ri = rng.choice(live_r, size=su, replace=False)
        cj = rng.choice(ncols_live, size=sv, replace=False)
        u = rng.standard_normal(su)
        v = rng.standard_normal(sv)
        u /= np.linalg.norm(u)
        v /= np.linalg.norm(v)
        s_i = math.exp(-i / decay) * math.sqrt(m * n)
        rows.append(np.repeat(ri, sv))
        cols.append(np.tile(cj, su))
        vals.append((s_i * np.outer(u, v)).ravel())
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    if dup_frac > 0 and r.size:
        pick = rng.random(r.size) < dup_frac
        part = rng.random(int(pick.sum()))
        base = v.copy()
        base[pick] *= 1.0 - part          # the two copies add up to the value
        r = np.concatenate([r, r[pick]])
        c = np.concatenate([c, c[pick]])
        v = np.concatenate([base, v[pick] * part])
    order = np.lexsort((rng.random(r.size) if shuffle else c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, c.astype(np.int32), v.astype(np.float64)


def csr_to_dense(rowptr, colind, values, m: int, n: int) -> np.ndarray:
    """Dense FP64 copy of a CSR matrix (repeated pairs add)."""
    A = np.zeros((m, n))
    r = np.repeat(np.arange(m), np.diff(rowptr))
    np.add.at(A, (r, colind.astype(np.int64)), values)
    return A


def batched_shapes(seed: int, count: int = 512, m_range=(256, 4096), n_lo: int = 128,
                   n_hi: int = 2048, k_range=(8, 64), alpha_range=(1.0, 3.0)):
    """Shapes and spectra of the uneven batch: m ~ U[256,4096],
    n ~ U[128, min(m,2048)], k ~ U[8,64], alpha ~ U[1,3] (integers inclusive)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        n = int(rng.integers(n_lo, min(m, n_hi) + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        a = float(rng.uniform(alpha_range[0], alpha_range[1]))
        out.append({"m": m, "n": n, "k": k, "alpha": a})
    return out


# ------------------------------------------------------------- torch (device)
def torch_svd_matrix(seed: int, m: int, n: int, sigma, device="cuda", dtype=None):
    """Device version of :func:`svd_matrix`: the Haar factors come from the same
    numpy stream (QR on the host, LAPACK), the product U diag(sigma) V^T is
    formed on the device in FP64."""
    import torch
    dtype = dtype or torch.float64
    rng = np.random.default_rng(seed)
    s = np.asarray(sigma, dtype=np.float64)
    r = len(s)
    U = torch.from_numpy(haar_columns(rng, m, r)).to(device)
    V = torch.from_numpy(haar_columns(rng, n, r)).to(device)
    sd = torch.from_numpy(s).to(device)
    return ((U * sd) @ V.T).to(dtype).contiguous()


def torch_xyt_plus_noise(seed: int, m: int, n: int, r: int, eps: float, device="cuda"):
    """Device FP32 X Y^T + eps E, the product in true FP32 (no TF32)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    X = torch.randn(m, r, generator=gen, device=device, dtype=torch.float32)
    Y = torch.randn(n, r, generator=gen, device=device, dtype=torch.float32)
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        A = X @ Y.T
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    A.add_(torch.randn(m, n, generator=gen, device=device, dtype=torch.float32), alpha=eps)
    return A


def _preload_torch_linalg():
    """Load torch's lazily opened CUDA linear-algebra library by absolute path
    (some profilers' environments break its lookup by name)."""
    import ctypes
    import os
    import torch
    lib = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(lib):
        try:
            ctypes.CDLL(lib, mode=ctypes.RTLD_GLOBAL)
        except OSError:
            pass


def torch_svd_matrix_device(seed: int, m: int, n: int, sigma, device="cuda"):
    """U diag(sigma) V^T with Haar U (m x r), V (n x r) drawn and orthonormalised
    on the device (torch QR with the sign fix); FP64."""
    import torch
    _preload_torch_linalg()
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    s = torch.as_tensor(np.asarray(sigma), device=device, dtype=torch.float64)
    r = s.numel()

    def haar(rows):
        g = torch.randn(rows, r, generator=gen, device=device, dtype=torch.float64)
        q, rr = torch.linalg.qr(g)
        sg = torch.sign(torch.diagonal(rr))
        sg[sg == 0] = 1.0
        return q * sg

    U = haar(m)
    V = haar(n)
    return ((U * s) @ V.T).contiguous()
