"""FP64 CPU oracle for PbP-QLP — TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package.  The library's product path never loads it.
It shares no code with the CUDA sources.

The arithmetic lives in ``pbpqlp_oracle.c`` (plain C, FP64): Philox4x32-10 +
Box-Muller Gaussians, plain GEMM loops, a plain CSR product for sparse A
(Section III-C), Householder QR with diag(R) >= 0, and Algorithm 3 of the
paper executed step by step (dense or CSR A).  This module only marshals
numpy arrays to it and adds the plain numpy formulas for the reconstruction
and error of Eq. 8.  The learned-proposer MLP reference lives in
``oracle/mlp.py``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library.

    PBPQLP_ORACLE_LIB names another build of the same source to load instead
    (the mutation tests load copies with a planted mistake this way)."""
    global _lib
    if _lib is None:
        path = os.environ.get("PBPQLP_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_uint32)]
        L.orc_philox4x32_10.restype = None
        L.orc_gaussian.argtypes = [ctypes.c_uint64, i64, i64, d]
        L.orc_gaussian.restype = None
        L.orc_gemm.argtypes = [ctypes.c_int, i64, i64, i64, d, i64, d, i64, d, i64]
        L.orc_gemm.restype = None
        L.orc_qr.argtypes = [i64, i64, d, i64, d, i64, d]
        L.orc_qr.restype = ctypes.c_int
        L.orc_pbpqlp.argtypes = [i64, i64, d, i64, i64, ctypes.c_int, d, d, d, d, d, d, d]
        L.orc_pbpqlp.restype = ctypes.c_int
        pi64 = ctypes.POINTER(ctypes.c_int64)
        pi32 = ctypes.POINTER(ctypes.c_int32)
        L.orc_csr_mult.argtypes = [ctypes.c_int, i64, i64, pi64, pi32, d, i64, d, i64, d, i64]
        L.orc_csr_mult.restype = None
        L.orc_pbpqlp_csr.argtypes = [i64, i64, pi64, pi32, d, i64, ctypes.c_int, d, d, d, d, d, d, d]
        L.orc_pbpqlp_csr.restype = ctypes.c_int
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    """Host threads the oracle's OpenMP regions use."""
    return int(lib().orc_num_threads())


def philox4x32_10(counter, key):
    """Philox4x32-10 block: four 32-bit counter words, two key words -> four words."""
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in counter])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def gaussian(seed: int, shape, offset: int = 0) -> np.ndarray:
    """Standard normals for linear (row-major) indices offset.. of an array of ``shape``."""
    count = int(np.prod(shape))
    out = np.empty(count, dtype=np.float64)
    lib().orc_gaussian(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), offset, count, _dp(out))
    return out.reshape(shape)


def gemm(a, b, trans_a: bool = False) -> np.ndarray:
    """op(a) @ b with plain loops (op = transpose when ``trans_a``)."""
    a = _f64c(a)
    b = _f64c(b)
    M = a.shape[1] if trans_a else a.shape[0]
    K = a.shape[0] if trans_a else a.shape[1]
    assert b.shape[0] == K
    N = b.shape[1]
    c = np.empty((M, N), dtype=np.float64)
    lib().orc_gemm(1 if trans_a else 0, M, N, K, _dp(a), a.shape[1], _dp(b), N, _dp(c), N)
    return c


def qr(x):
    """Unpivoted thin Householder QR with diag(R) >= 0: returns (Q, R)."""
    x = _f64c(x)
    rows, cols = x.shape
    q = np.empty((rows, cols), dtype=np.float64)
    r = np.empty((cols, cols), dtype=np.float64)
    rc = lib().orc_qr(rows, cols, _dp(x), cols, _dp(q), cols, _dp(r))
    if rc != 0:
        raise ValueError("orc_qr failed (rows < cols?)")
    return q, r


def pbpqlp(A, ell: int, q: int, phi=None, seed: int = None):
    """Algorithm 3 of the paper in FP64 (paper orientation).

    ``phi`` is the m x ell Gaussian test matrix; if None it is drawn from
    ``seed`` with the same Philox/Box-Muller stream the library uses.
    Returns a dict with Q (m x ell), L (ell x ell, lower), P (n x ell),
    R (first-stage upper factor, Eq. 6), Pbar (n x ell), D (m x ell), Phi.
    """
    A = _f64c(A)
    m, n = A.shape
    if phi is None:
        if seed is None:
            raise ValueError("give phi or seed")
        phi = gaussian(seed, (m, ell))
    phi = _f64c(phi)
    assert phi.shape == (m, ell)
    Q = np.empty((m, ell))
    L = np.empty((ell, ell))
    P = np.empty((n, ell))
    R = np.empty((ell, ell))
    Pbar = np.empty((n, ell))
    D = np.empty((m, ell))
    rc = lib().orc_pbpqlp(m, n, _dp(A), n, ell, q, _dp(phi), _dp(Q), _dp(L), _dp(P),
                          _dp(R), _dp(Pbar), _dp(D))
    if rc != 0:
        raise ValueError("orc_pbpqlp failed: need 1 <= ell <= min(m, n), q >= 0")
    return {"Q": Q, "L": L, "P": P, "R": R, "Pbar": Pbar, "D": D, "Phi": phi}


def _csr_arrays(rowptr, colind, values):
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    va = _f64c(values)
    assert ci.shape == va.shape and rp[-1] == ci.size
    return rp, ci, va


def csr_mult(rowptr, colind, values, shape, B, trans: bool = False) -> np.ndarray:
    """A @ B (or A.T @ B) for A (shape m x n) in CSR form, with plain loops."""
    m, n = shape
    rp, ci, va = _csr_arrays(rowptr, colind, values)
    B = _f64c(B)
    N = B.shape[1]
    assert B.shape[0] == (m if trans else n)
    C = np.empty((n if trans else m, N), dtype=np.float64)
    lib().orc_csr_mult(1 if trans else 0, m, n, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                       ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(va), N, _dp(B), N, _dp(C), N)
    return C


def pbpqlp_csr(rowptr, colind, values, shape, ell: int, q: int, phi=None, seed: int = None):
    """Algorithm 3 for a sparse A (m x n) in CSR form; same outputs as ``pbpqlp``."""
    m, n = shape
    rp, ci, va = _csr_arrays(rowptr, colind, values)
    if phi is None:
        if seed is None:
            raise ValueError("give phi or seed")
        phi = gaussian(seed, (m, ell))
    phi = _f64c(phi)
    out = {k: np.empty(s) for k, s in (("Q", (m, ell)), ("L", (ell, ell)), ("P", (n, ell)), ("R", (ell, ell)),
                                        ("Pbar", (n, ell)), ("D", (m, ell)))}
    rc = lib().orc_pbpqlp_csr(m, n, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(va), ell, q, _dp(phi),
                              _dp(out["Q"]), _dp(out["L"]), _dp(out["P"]), _dp(out["R"]), _dp(out["Pbar"]),
                              _dp(out["D"]))
    if rc != 0:
        raise ValueError("orc_pbpqlp_csr failed: need 1 <= ell <= min(m, n), q >= 0")
    out["Phi"] = phi
    return out


def reconstruct(Q, L, P, r: int) -> np.ndarray:
    """Rank-r truncation Q[:, :r] L[:r, :r] P[:, :r]^T of Eq. 8 (r = ell gives QLP^T)."""
    return (Q[:, :r] @ L[:r, :r]) @ P[:, :r].T


def rel_fro_error(A, Q, L, P, r: int) -> float:
    """||A - Q_r L_r P_r^T||_F / ||A||_F, formed explicitly in FP64."""
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm(A - reconstruct(Q, L, P, r)) / np.linalg.norm(A))


def probe_error_estimate(A, Q, L, P, r: int, probes) -> float:
    """Randomized a-posteriori estimate of ||A - A_r||_F / ||A||_F.

    With Gaussian probes W (n x s), E||(A - A_r) w||^2 = ||A - A_r||_F^2 and
    E||A w||^2 = ||A||_F^2 for w ~ N(0, I); the estimator is the ratio of the
    two sample means (Halko, Martinsson, Tropp 2011, Section 4.3 idea).
    """
    A = np.asarray(A, dtype=np.float64)
    W = np.asarray(probes, dtype=np.float64)
    AW = A @ W
    EW = AW - Q[:, :r] @ (L[:r, :r] @ (P[:, :r].T @ W))
    return float(np.sqrt(np.sum(EW * EW) / np.sum(AW * AW)))
