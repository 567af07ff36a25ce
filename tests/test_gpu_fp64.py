"""GPU parity of the plain FP64 path (MODE_FP64) against the CPU oracle.

The contract: on the same seeded A and Phi, the rank-k truncations agree to
||Ak_gpu - Ak_cpu||_F / ||A||_F <= 1e-11.  Phi is drawn on each side from the
same Philox4x32-10 stream (or passed in), so it is shared exactly up to the
last-bit differences of the two math libraries' log/cos/sin.
"""
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


def _run(pq, A_np, k, p, q, seed, omega=None):
    import torch
    m, n = A_np.shape
    A = torch.from_numpy(np.ascontiguousarray(A_np)).cuda()
    plan = pq.Plan(m, n, k, p, q, seed)
    om = None if omega is None else torch.from_numpy(omega).cuda()
    Qa, L, Qb = plan.factor(A, omega=om)
    rc, flags = plan.sync_status()
    return plan, A, (Qa, L, Qb), rc, flags


def _np(*ts):
    return [t.cpu().numpy() for t in ts]


def _parity(A_np, gpu, ref, k):
    Qa, L, Qb = gpu
    Ag = oracle.reconstruct(Qa, L, Qb, k)
    Ac = oracle.reconstruct(ref["Q"], ref["L"], ref["P"], k)
    return np.linalg.norm(Ag - Ac) / np.linalg.norm(A_np)


def test_omega_matches_oracle_stream(pq):
    import torch
    plan = pq.Plan(333, 217, 15, 4, 1, seed=987654321)
    om = plan.omega().cpu().numpy()
    ref = oracle.gaussian(987654321, (333, 19))
    assert np.max(np.abs(om - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_config1_parity(pq):
    """1000 x 1000, sigma_i = i^-2, Haar U, V; k = 20, p = 5, q = 1."""
    A_np = synth.poly_decay(1, 1000, 1000, 2.0)
    plan, A, out, rc, flags = _run(pq, A_np, 20, 5, 1, seed=2)
    assert rc == pq.PBPQLP_OK, flags
    ref = oracle.pbpqlp(A_np, 25, 1, seed=2)
    g = _np(*out)
    assert _parity(A_np, g, ref, 20) <= TOL
    assert _parity(A_np, g, ref, 25) <= TOL
    Qa, L, Qb = g
    assert np.array_equal(L, np.tril(L)) and np.all(np.diag(L) >= 0)
    assert np.allclose(Qa.T @ Qa, np.eye(25), atol=1e-13)
    assert np.allclose(Qb.T @ Qb, np.eye(25), atol=1e-13)
    # factor-wise parity (unique under diag >= 0 for full-rank panels)
    assert np.max(np.abs(L - ref["L"])) <= 1e-10 * np.max(np.abs(ref["L"]))
    assert np.max(np.abs(Qa[:, :20] - ref["Q"][:, :20])) <= 1e-9


@pytest.mark.parametrize("m,n,k,p,q", [
    (333, 217, 15, 4, 1),     # ragged, several tiles
    (217, 333, 15, 4, 2),     # m < n
    (1200, 90, 7, 3, 0),      # tall, basic form q = 0
    (97, 1500, 30, 10, 1),    # wide
    (64, 64, 1, 0, 1),        # l = 1
    (130, 70, 60, 10, 1),     # l = min(m, n) = 70
    (700, 650, 200, 24, 1),   # l = 224 (largest; cluster Cholesky and QR)
    (600, 500, 120, 11, 1),   # l = 131: cluster kernels, uneven rows per CTA
    (900, 800, 200, 17, 2),   # l = 217: cluster kernels, uneven rows per CTA
    (2049, 1031, 100, 17, 2), # l = 117, ragged tails everywhere
])
def test_parity_shapes(pq, m, n, k, p, q):
    A_np = synth.exp_decay(m + 7 * n, m, n, max(2.0, (k + p) / 3.0))
    plan, A, out, rc, flags = _run(pq, A_np, k, p, q, seed=m * n + k)
    assert rc == pq.PBPQLP_OK, flags
    ref = oracle.pbpqlp(A_np, k + p, q, seed=m * n + k)
    g = _np(*out)
    assert _parity(A_np, g, ref, k) <= TOL
    assert _parity(A_np, g, ref, k + p) <= TOL


def test_passed_omega_equals_seeded(pq):
    A_np = synth.poly_decay(3, 400, 300, 1.5)
    om = oracle.gaussian(5, (400, 20))
    _, _, out1, rc1, _ = _run(pq, A_np, 16, 4, 1, seed=5)
    _, _, out2, rc2, _ = _run(pq, A_np, 16, 4, 1, seed=999, omega=om)
    assert rc1 == rc2 == pq.PBPQLP_OK
    ref = oracle.pbpqlp(A_np, 20, 1, phi=om)
    assert _parity(A_np, _np(*out2), ref, 16) <= TOL
    assert _parity(A_np, _np(*out1), ref, 16) <= TOL


def test_bitwise_repeatable(pq):
    A_np = synth.poly_decay(4, 500, 400, 1.0)
    _, _, o1, _, _ = _run(pq, A_np, 10, 6, 2, seed=8)
    _, _, o2, _, _ = _run(pq, A_np, 10, 6, 2, seed=8)
    for a, b in zip(_np(*o1), _np(*o2)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_exact_recovery_rank_deficient(pq, q):
    """rank(A) = 8 < l = 15: the sketch panels are rank deficient, CholeskyQR
    breaks down and the shifted retry pairs take over; A is still recovered."""
    A_np = synth.rank_r(21, 200, 150, 8)
    plan, A, out, rc, flags = _run(pq, A_np, 10, 5, q, seed=4)
    assert rc == pq.PBPQLP_OK, flags
    assert flags & 1, "expected the shifted retry to be used"
    Qa, L, Qb = _np(*out)
    assert oracle.rel_fro_error(A_np, Qa, L, Qb, 10) < 1e-12
    assert np.array_equal(L, np.tril(L))


def test_zero_matrix(pq):
    A_np = np.zeros((120, 80))
    plan, A, out, rc, flags = _run(pq, A_np, 5, 3, 1, seed=1)
    assert rc == pq.PBPQLP_OK
    Qa, L, Qb = _np(*out)
    assert np.all(np.isfinite(Qa)) and np.all(L == 0) and np.all(np.isfinite(Qb))


def test_nonfinite_input_is_reported(pq):
    A_np = synth.poly_decay(9, 100, 80, 1.0)
    A_np[17, 33] = np.nan
    plan, A, out, rc, flags = _run(pq, A_np, 5, 3, 1, seed=1)
    assert rc == pq.PBPQLP_ENONFINITE and (flags & 4)


def test_reconstruct_and_error_methods(pq):
    A_np = synth.poly_decay(12, 600, 500, 1.5)
    k, p, q = 20, 10, 2
    plan, A, out, rc, _ = _run(pq, A_np, k, p, q, seed=3)
    Qa, L, Qb = out
    Ahat = plan.reconstruct(Qa, L, Qb, k).cpu().numpy()
    g = _np(Qa, L, Qb)
    assert np.linalg.norm(Ahat - oracle.reconstruct(*g, k)) <= 1e-13 * np.linalg.norm(A_np)
    e_true = oracle.rel_fro_error(A_np, *g, k)
    e_res = plan.error(A, Qa, L, Qb, k, method=pq.PBPQLP_ERR_RESIDUAL)
    e_id = plan.error(A, Qa, L, Qb, k, method=pq.PBPQLP_ERR_IDENTITY)
    assert abs(e_res - e_true) <= 1e-10 * e_true
    assert abs(e_id - e_true) <= 1e-6 * e_true
    e_pr = plan.error(A, Qa, L, Qb, k, method=pq.PBPQLP_ERR_PROBES, nprobes=16, probe_seed=77)
    W = oracle.gaussian(77, (500, 16))
    assert abs(e_pr - oracle.probe_error_estimate(A_np, *g, k, W)) <= 1e-10 * e_pr
    assert 0.5 * e_true < e_pr < 2.0 * e_true


@pytest.mark.slow
def test_config2_full_size_parity(pq):
    """The benchmark workload: 8000 x 8000, sigma_i = exp(-i/40), k = 100,
    p = 10, q = 2, compared in full against the oracle."""
    import torch
    sig = synth.spectrum("exp", 1500, 40.0)
    A = synth.torch_svd_matrix(2, 8000, 8000, sig)
    A_np = A.cpu().numpy()
    plan = pq.Plan(8000, 8000, 100, 10, 2, seed=3)
    Qa, L, Qb = plan.factor(A)
    rc, flags = plan.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    ref = oracle.pbpqlp(A_np, 110, 2, seed=3)
    g = _np(Qa, L, Qb)
    assert _parity(A_np, g, ref, 100) <= TOL


def test_rank_revealing_outputs(pq):
    """L-values, ||A||_2 estimate and numerical rank (Sections IV-C, V-D)."""
    import torch
    # norm estimate on a decaying spectrum: below sigma_1, and within 1e-3 of it with q = 2
    A_np = synth.poly_decay(12, 400, 300, 1.0)
    plan, A, out, rc, flags = _run(pq, A_np, 10, 5, 2, seed=6)
    assert rc == pq.PBPQLP_OK
    Qa, L, Qb = out
    lv, nrm, rk = plan.rank_revealing(L, tol=1e-6)
    s = np.linalg.svd(A_np, compute_uv=False)
    assert np.array_equal(lv.cpu().numpy(), np.abs(np.diag(L.cpu().numpy())))
    ref = oracle.pbpqlp(A_np, 15, 2, seed=6)
    assert abs(nrm - abs(ref["L"][0, 0])) <= 1e-12 * s[0]      # the estimate the algorithm defines
    assert nrm <= s[0] * (1 + 1e-12) and nrm >= 0.98 * s[0]
    # numerical rank of a rank-13 matrix plus 1e-10 noise
    rng = np.random.default_rng(3)
    B_np = synth.rank_r(8, 400, 300, 13) + 1e-10 * rng.standard_normal((400, 300))
    plan, B, out, rc, flags = _run(pq, B_np, 20, 5, 2, seed=6)
    lv, nrm, rk = plan.rank_revealing(out[1], tol=1e-6)
    assert rk == 13
    assert nrm <= np.linalg.svd(B_np, compute_uv=False)[0] * (1 + 1e-12)


def test_out_of_core_A_in_pinned_host_memory(pq):
    """A left in pinned host memory: the passes read it over the host link and
    the factors are bitwise those of a device-resident A."""
    import torch
    A_np = synth.poly_decay(17, 900, 700, 1.5)
    A_host = torch.from_numpy(A_np).pin_memory()
    A_dev = A_host.cuda()
    for mode in (pq.PBPQLP_MODE_FP64, pq.PBPQLP_MODE_BF16X3):
        plan = pq.Plan(900, 700, 20, 8, 2, seed=4, mode=mode)
        ref = [t.cpu() for t in plan.factor(A_dev)]
        got = [t.cpu() for t in plan.factor(A_host)]
        rc, flags = plan.sync_status()
        assert rc == pq.PBPQLP_OK, flags
        for a, b in zip(ref, got):
            assert torch.equal(a, b)


def test_pageable_host_A_is_rejected_before_any_launch(pq):
    import torch
    A = torch.from_numpy(synth.poly_decay(1, 200, 150, 1.0))      # pageable host memory
    plan = pq.Plan(200, 150, 10, 5, 1, seed=1)
    with pytest.raises(pq.PbpqlpError) as e:
        plan.factor(A)
    assert e.value.status == pq.PBPQLP_EINVAL
