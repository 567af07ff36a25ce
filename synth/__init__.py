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
