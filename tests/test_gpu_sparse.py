"""Sparse A (Section III-C): the CSR entry point against the oracle's CSR
form, against the dense GPU path on the same matrix, run to run, and on CSR
structures the device check must reject."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module")
def pq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2103_07245_gb300 as pq
    pq.load(build_if_missing=True)
    return pq


def _dev(rp, ci, va):
    import torch
    return (torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), torch.from_numpy(va).cuda())


def _factor_csr(pq, plan, rp, ci, va):
    out = plan.factor_csr(*_dev(rp, ci, va))
    rc, flags = plan.sync_status()
    return rc, flags, [t.cpu().numpy() for t in out]


# l chosen so that the SpMM's last 32-column chunk takes 1, 2 or 4 nonzeros per instruction
@pytest.mark.parametrize("m,n,k,p,q,kw", [
    (1000, 1000, 20, 5, 1, dict(nnz_per_row=8.0, rank=30, support=120)),          # l = 25: one chunk
    (700, 333, 8, 4, 2, dict(nnz_per_row=3.0, rank=20, support=60, dup_frac=0.2, shuffle=True, empty_rows=17,
                             empty_cols=9)),                                      # l = 12: 2 per chunk
    (500, 400, 3, 3, 1, dict(nnz_per_row=5.0, rank=6, support=50)),               # l = 6: 4 per chunk
    (300, 1100, 32, 8, 1, dict(nnz_per_row=25.0, rank=60, support=80)),           # l = 40: 1 + 8 columns
    (2500, 1800, 100, 10, 2, dict(nnz_per_row=12.0, rank=150, support=200)),      # l = 110: 3 + 14 columns
    (1200, 900, 100, 20, 1, dict(nnz_per_row=9.0, rank=130, support=120)),        # l = 120: 3 + 24 columns
    (260, 240, 200, 24, 0, dict(nnz_per_row=40.0)),                               # l = 224, q = 0
])
def test_csr_parity_with_oracle(pq, m, n, k, p, q, kw):
    rp, ci, va = synth.sparse_csr(100 + m, m, n, **kw)
    A = synth.csr_to_dense(rp, ci, va, m, n)
    plan = pq.Plan(m, n, k, p, q, seed=7)
    rc, flags, g = _factor_csr(pq, plan, rp, ci, va)
    assert rc == pq.PBPQLP_OK, flags
    ref = oracle.pbpqlp_csr(rp, ci, va, (m, n), k + p, q, seed=7)
    for r in (k, k + p):
        d = np.linalg.norm(oracle.reconstruct(*g, r) - oracle.reconstruct(ref["Q"], ref["L"], ref["P"], r))
        assert d / np.linalg.norm(A) <= TOL, (r, d)
    assert np.array_equal(g[1], np.tril(g[1]))


def test_csr_equals_dense_path_and_repeats_bitwise(pq):
    import torch
    m, n, k, p, q = 900, 650, 30, 8, 2
    rp, ci, va = synth.sparse_csr(5, m, n, nnz_per_row=6.0, rank=40, support=90, dup_frac=0.1, shuffle=True)
    A = synth.csr_to_dense(rp, ci, va, m, n)
    plan = pq.Plan(m, n, k, p, q, seed=11)
    rc1, _, g1 = _factor_csr(pq, plan, rp, ci, va)
    rc2, _, g2 = _factor_csr(pq, plan, rp, ci, va)
    assert rc1 == rc2 == pq.PBPQLP_OK
    for a, b in zip(g1, g2):
        assert np.array_equal(a, b)
    Qa, L, Qb = plan.factor(torch.from_numpy(A).cuda())
    rc, _ = plan.sync_status()
    assert rc == pq.PBPQLP_OK
    gd = [t.cpu().numpy() for t in (Qa, L, Qb)]
    d = np.linalg.norm(oracle.reconstruct(*g1, k) - oracle.reconstruct(*gd, k))
    assert d <= 1e-12 * np.linalg.norm(A)


def test_csr_exact_recovery_and_empty_matrix(pq):
    m, n, r = 800, 600, 8
    rp, ci, va = synth.sparse_csr(9, m, n, nnz_per_row=0.0, rank=r, support=100)
    A = synth.csr_to_dense(rp, ci, va, m, n)
    plan = pq.Plan(m, n, r, 4, 1, seed=2)
    rc, flags, g = _factor_csr(pq, plan, rp, ci, va)
    assert rc == pq.PBPQLP_OK, flags
    assert oracle.rel_fro_error(A, *g, r) <= 1e-12
    # no nonzeros at all: a finite factorization of the zero matrix
    import torch
    plan0 = pq.Plan(64, 48, 4, 2, 1, seed=1)
    rp0 = np.zeros(65, dtype=np.int64)
    out = plan0.factor_csr(torch.from_numpy(rp0).cuda(), torch.empty(0, dtype=torch.int32, device="cuda"),
                           torch.empty(0, dtype=torch.float64, device="cuda"))
    rc0, flags0 = plan0.sync_status()
    assert rc0 == pq.PBPQLP_OK and not (flags0 & ~1), flags0
    assert all(np.isfinite(t.cpu().numpy()).all() for t in out)
    assert np.abs(out[1].cpu().numpy()).max() == 0.0


@pytest.mark.parametrize("defect", ["col_out_of_range", "negative_col", "rowptr_decreasing", "rowptr_end"])
def test_csr_bad_structure_is_rejected_on_device(pq, defect):
    """Every defect is caught by the device check before any kernel indexes
    through the structure; the call after it, on a valid matrix, is clean."""
    m, n, k, p = 120, 90, 6, 4
    rp, ci, va = synth.sparse_csr(4, m, n, nnz_per_row=5.0)
    rp, ci = rp.copy(), ci.copy()
    if defect == "col_out_of_range":
        ci[len(ci) // 2] = n + 1000
    elif defect == "negative_col":
        ci[3] = -5
    elif defect == "rowptr_decreasing":
        rp[40] = rp[41] + 3 if rp[41] + 3 <= rp[-1] else rp[-1]
        rp[41] = max(rp[40] - 2, 0)
    else:
        rp[-1] = rp[-1] - 1
    plan = pq.Plan(m, n, k, p, 1, seed=3)
    rc, flags, g = _factor_csr(pq, plan, rp, ci, va)
    assert rc == pq.PBPQLP_EINVAL and flags & 16, (rc, flags)
    rp2, ci2, va2 = synth.sparse_csr(4, m, n, nnz_per_row=5.0)
    rc2, flags2, _ = _factor_csr(pq, plan, rp2, ci2, va2)
    assert rc2 == pq.PBPQLP_OK, flags2
