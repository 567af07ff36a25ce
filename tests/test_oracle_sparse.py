"""Pins of the oracle's sparse form (Section III-C: the same Algorithm 3 with
the products taken over the nonzeros of a CSR A) against numpy's dense
arithmetic and against the dense oracle, whose own pins are in
test_oracle_pins.py."""
import numpy as np
import pytest

import oracle
import synth


def _mat(seed, m, n, **kw):
    rp, ci, va = synth.sparse_csr(seed, m, n, **kw)
    return rp, ci, va, synth.csr_to_dense(rp, ci, va, m, n)


@pytest.mark.parametrize("kw", [dict(nnz_per_row=6.0),
                                dict(nnz_per_row=3.0, dup_frac=0.3, shuffle=True, empty_rows=9, empty_cols=11),
                                dict(nnz_per_row=0.5, rank=4, support=20)])
def test_csr_product_matches_dense_library_product(kw):
    m, n = 130, 97
    rp, ci, va, A = _mat(3, m, n, **kw)
    rng = np.random.default_rng(5)
    B = rng.standard_normal((n, 13))
    Bt = rng.standard_normal((m, 13))
    C = oracle.csr_mult(rp, ci, va, (m, n), B)
    Ct = oracle.csr_mult(rp, ci, va, (m, n), Bt, trans=True)
    assert np.allclose(C, A @ B, rtol=0, atol=1e-13 * np.abs(A).sum(1).max() * np.abs(B).max())
    assert np.allclose(Ct, A.T @ Bt, rtol=0, atol=1e-13 * np.abs(A).sum(0).max() * np.abs(Bt).max())


def test_csr_form_equals_dense_form():
    """Same Phi, same steps: the sparse and dense oracles agree to rounding."""
    m, n, k, p, q = 240, 170, 12, 5, 2
    rp, ci, va, A = _mat(7, m, n, nnz_per_row=4.0, rank=20, support=40, dup_frac=0.1, shuffle=True,
                         empty_rows=3, empty_cols=4)
    ref = oracle.pbpqlp(A, k + p, q, seed=21)
    sp = oracle.pbpqlp_csr(rp, ci, va, (m, n), k + p, q, seed=21)
    d = np.linalg.norm(oracle.reconstruct(sp["Q"], sp["L"], sp["P"], k) -
                       oracle.reconstruct(ref["Q"], ref["L"], ref["P"], k))
    assert d <= 1e-12 * np.linalg.norm(A)
    assert np.array_equal(sp["L"], np.tril(sp["L"]))


def test_csr_exact_recovery_at_rank_k():
    """rank(A) <= k: the sparse factorization reproduces A to roundoff."""
    m, n, r = 300, 260, 6
    rp, ci, va, A = _mat(11, m, n, nnz_per_row=0.0, rank=r, support=50)
    assert np.linalg.matrix_rank(A) == r
    out = oracle.pbpqlp_csr(rp, ci, va, (m, n), r + 4, 1, seed=3)
    assert oracle.rel_fro_error(A, out["Q"], out["L"], out["P"], r) <= 1e-12
