"""FP64-accurate tensor-core products (digit form) against exact results and the oracle.

The products C = A Y and C = A^T Y of MODE_FP64_EMU go through the BF16
tensor cores as sums of exact integer digit products.  Pins, each independent
of the CUDA path: integer-valued operands, whose FP64 products are exact, must
come out bit-identical to numpy; Gaussian operands must sit within the FP64
error bound of the oracle's index-order sum; the factorization must meet the
same parity bar as the FP64 path (||Ak_gpu - Ak_cpu||_F / ||A||_F <= 1e-11).
The Grams of CholeskyQR use the same kernel in every mode, so every FP64
parity test covers it; here it is also compared with the FP64 FMA Grams.
"""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-11
U = 2.0 ** -53


@pytest.fixture(scope="module")
def pq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2103_07245_gb300 as pq
    pq.load(build_if_missing=True)
    return pq


def _sketch(pq, A_np, Y_np, trans, l=None):
    import torch
    m, n = A_np.shape
    l = Y_np.shape[1] if l is None else l
    plan = pq.Plan(m, n, l, 0, 0, seed=1, mode=pq.PBPQLP_MODE_FP64_EMU)
    A = torch.from_numpy(np.ascontiguousarray(A_np)).cuda()
    Y = torch.from_numpy(np.ascontiguousarray(Y_np)).cuda()
    C = plan.sketch(A, Y, trans=trans)
    rc, flags = plan.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    return C.cpu().numpy()


@pytest.mark.parametrize("m,n,N,trans", [
    (300, 257, 20, False),    # 3 row tiles, ragged contraction (9 windows), one column tile
    (300, 257, 20, True),
    (129, 1000, 70, False),   # ragged row tile, two column tiles
    (1000, 129, 70, True),
    (64, 33, 1, False),       # one column, contraction shorter than two windows
])
def test_integer_operands_are_exact(pq, m, n, N, trans):
    """Integer entries below 2^10: every FP64 product and partial sum is exact,
    so the digit-form product must equal numpy bit for bit."""
    rng = np.random.default_rng(m + n + N)
    A = rng.integers(-1023, 1024, size=(m, n)).astype(np.float64)
    Y = rng.integers(-1023, 1024, size=((m if trans else n), N)).astype(np.float64)
    C = _sketch(pq, A, Y, trans)
    ref = (A.T if trans else A) @ Y
    assert np.array_equal(C, ref)


def test_wide_dynamic_range_rows(pq):
    """Rows of A and columns of Y scaled from 2^-250 to 2^250 (products stay in
    range): the per-row exponents keep every output at full relative precision."""
    rng = np.random.default_rng(5)
    m, n, N = 200, 300, 24
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-250, 250, size=(m, 1)))
    Y = rng.standard_normal((n, N)) * np.exp2(rng.integers(-250, 250, size=(1, N)))
    C = _sketch(pq, A, Y, False)
    ref = oracle.gemm(A, Y)
    bound = 4 * n * U * (np.abs(A) @ np.abs(Y))
    assert np.all(np.abs(C - ref) <= bound)


@pytest.mark.parametrize("trans", [False, True])
def test_gaussian_within_fp64_bound(pq, trans):
    """|C_emu - C_oracle| <= 2 gamma_K |A||Y| elementwise (both sides hold the
    FP64 dot-product bound), and the normwise difference is at the FP64 level."""
    rng = np.random.default_rng(11)
    m, n, N = 700, 900, 110
    A = rng.standard_normal((m, n))
    Y = rng.standard_normal(((m if trans else n), N))
    C = _sketch(pq, A, Y, trans)
    At = A.T if trans else A
    ref = oracle.gemm(np.ascontiguousarray(At), Y)
    K = At.shape[1]
    assert np.all(np.abs(C - ref) <= 2 * K * U / (1 - K * U) * (np.abs(At) @ np.abs(Y)))
    assert np.linalg.norm(C - ref) <= 1e-15 * np.sqrt(K) * np.linalg.norm(ref)


def test_nonfinite_rows_give_nan(pq):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((150, 90))
    A[17, 40] = np.inf
    Y = rng.standard_normal((90, 8))
    C = _sketch(pq, A, Y, False)
    assert np.all(np.isnan(C[17])) and np.all(np.isfinite(np.delete(C, 17, axis=0)))


def _factor(pq, A_np, k, p, q, seed, mode):
    import torch
    m, n = A_np.shape
    plan = pq.Plan(m, n, k, p, q, seed, mode=mode)
    A = torch.from_numpy(np.ascontiguousarray(A_np)).cuda()
    out = plan.factor(A)
    rc, flags = plan.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    return [t.cpu().numpy() for t in out]


def _parity(A_np, g, ref, k):
    Ag = oracle.reconstruct(*g, k)
    Ac = oracle.reconstruct(ref["Q"], ref["L"], ref["P"], k)
    return np.linalg.norm(Ag - Ac) / np.linalg.norm(A_np)


@pytest.mark.parametrize("m,n,k,p,q", [
    (1000, 1000, 20, 5, 1),   # the 1000 x 1000 parity workload
    (333, 217, 15, 4, 2),     # ragged
    (700, 650, 200, 24, 1),   # l = 224
    (1200, 90, 7, 3, 0),      # q = 0
])
def test_emu_factorization_parity(pq, m, n, k, p, q):
    A_np = synth.poly_decay(m + n, m, n, 2.0) if m == n else synth.exp_decay(m + 7 * n, m, n, max(2.0, (k + p) / 3.0))
    g = _factor(pq, A_np, k, p, q, 9, pq.PBPQLP_MODE_FP64_EMU)
    ref = oracle.pbpqlp(A_np, k + p, q, seed=9)
    assert _parity(A_np, g, ref, k) <= TOL
    assert _parity(A_np, g, ref, k + p) <= TOL
    Qa, L, Qb = g
    assert np.array_equal(L, np.tril(L)) and np.all(np.diag(L) >= 0)
    assert np.allclose(Qa.T @ Qa, np.eye(k + p), atol=1e-13)


def test_emu_rank_deficient_recovery(pq):
    A_np = synth.rank_r(21, 200, 150, 8)
    Qa, L, Qb = _factor(pq, A_np, 10, 5, 1, 4, pq.PBPQLP_MODE_FP64_EMU)
    assert oracle.rel_fro_error(A_np, Qa, L, Qb, 10) < 1e-12


def test_digit_grams_match_fma_grams(pq, monkeypatch):
    """The same FP64 factorization with the digit-form Grams (default) and
    with the FP64 FMA Grams (PBPQLP_NO_OZ_GRAM=1 at plan creation)."""
    A_np = synth.exp_decay(3, 900, 800, 40.0)
    g1 = _factor(pq, A_np, 100, 10, 2, 5, pq.PBPQLP_MODE_FP64)
    monkeypatch.setenv("PBPQLP_NO_OZ_GRAM", "1")
    g2 = _factor(pq, A_np, 100, 10, 2, 5, pq.PBPQLP_MODE_FP64)
    a1, a2 = oracle.reconstruct(*g1, 100), oracle.reconstruct(*g2, 100)
    assert np.linalg.norm(a1 - a2) <= 1e-13 * np.linalg.norm(A_np)
    assert np.max(np.abs(g1[1] - g2[1])) <= 1e-12 * np.max(np.abs(g2[1]))


def test_emu_bitwise_repeatable(pq):
    """Exact integer digit sums make every product independent of the
    stream-K split and of timing: two runs agree bit for bit."""
    A_np = synth.exp_decay(8, 1500, 1300, 30.0)
    g1 = _factor(pq, A_np, 40, 10, 2, 3, pq.PBPQLP_MODE_FP64_EMU)
    g2 = _factor(pq, A_np, 40, 10, 2, 3, pq.PBPQLP_MODE_FP64_EMU)
    for a, b in zip(g1, g2):
        assert np.array_equal(a, b)


def test_digit_grams_match_fma_grams_l220(pq, monkeypatch):
    """l = 220 (16-CTA Cholesky with T = R^-T, cluster QR): digit-form orth
    products against the FP64 FMA path, and both against the oracle."""
    A_np = synth.exp_decay(4, 700, 650, 60.0)
    g1 = _factor(pq, A_np, 200, 20, 1, 6, pq.PBPQLP_MODE_FP64)
    monkeypatch.setenv("PBPQLP_NO_OZ_GRAM", "1")
    g2 = _factor(pq, A_np, 200, 20, 1, 6, pq.PBPQLP_MODE_FP64)
    ref = oracle.pbpqlp(A_np, 220, 1, seed=6)
    assert _parity(A_np, g1, ref, 200) <= TOL
    assert _parity(A_np, g2, ref, 200) <= TOL
