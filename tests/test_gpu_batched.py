"""Batched factorization (many uneven matrices, work-list launches captured in
one CUDA graph) against the oracle, matrix by matrix."""
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


def _batch(seed, count):
    shapes = synth.batched_shapes(seed, count, m_range=(130, 900), n_lo=70, n_hi=600, k_range=(4, 40))
    mats = [synth.poly_decay(seed * 1000 + i, s["m"], s["n"], s["alpha"]) for i, s in enumerate(shapes)]
    return shapes, mats


def test_batched_matches_oracle_per_matrix(pq):
    import torch
    shapes, mats = _batch(3, 12)
    p, q, seed = 8, 1, 41
    B = pq.Batch([s["m"] for s in shapes], [s["n"] for s in shapes], [s["k"] for s in shapes], p, q, seed)
    As = [torch.from_numpy(a).cuda() for a in mats]
    Qa, L, Qb = B.factor(As)
    rc, flags = B.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    for i, (s, A) in enumerate(zip(shapes, mats)):
        ref = oracle.pbpqlp(A, s["k"] + p, q, seed=seed + i)
        g = [Qa[i].cpu().numpy(), L[i].cpu().numpy(), Qb[i].cpu().numpy()]
        for r in (s["k"], s["k"] + p):
            d = np.linalg.norm(oracle.reconstruct(*g, r) - oracle.reconstruct(ref["Q"], ref["L"], ref["P"], r))
            assert d / np.linalg.norm(A) <= TOL, (i, r, d)
        assert np.array_equal(g[1], np.tril(g[1]))


def test_batched_equals_single_and_replays_bitwise(pq):
    import torch
    shapes, mats = _batch(5, 6)
    p, q, seed = 6, 2, 9
    B = pq.Batch([s["m"] for s in shapes], [s["n"] for s in shapes], [s["k"] for s in shapes], p, q, seed)
    As = [torch.from_numpy(a).cuda() for a in mats]
    outs = B.outputs()
    B.factor(As, out=outs)
    first = [[t.clone() for t in ts] for ts in outs]
    B.factor(As, out=outs)      # graph replay
    rc, _ = B.sync_status()
    assert rc == pq.PBPQLP_OK
    for ts0, ts1 in zip(first, outs):
        for a, b in zip(ts0, ts1):
            assert torch.equal(a, b)
    for i, (s, A) in enumerate(zip(shapes, mats)):
        plan = pq.Plan(s["m"], s["n"], s["k"], p, q, seed=seed + i)
        Qa, L, Qb = plan.factor(As[i])
        g1 = [t.cpu().numpy() for t in (Qa, L, Qb)]
        g2 = [outs[0][i].cpu().numpy(), outs[1][i].cpu().numpy(), outs[2][i].cpu().numpy()]
        d = np.linalg.norm(oracle.reconstruct(*g1, s["k"]) - oracle.reconstruct(*g2, s["k"]))
        assert d / np.linalg.norm(A) <= TOL


def test_batched_status_is_per_matrix(pq):
    import torch
    shapes = [dict(m=200, n=150, k=10), dict(m=300, n=120, k=8), dict(m=180, n=180, k=12)]
    mats = [synth.rank_r(1, 200, 150, 5), synth.poly_decay(2, 300, 120, 1.0), synth.poly_decay(3, 180, 180, 2.0)]
    mats[1] = mats[1].copy()
    mats[1][7, 9] = np.nan
    B = pq.Batch([s["m"] for s in shapes], [s["n"] for s in shapes], [s["k"] for s in shapes], 5, 1, 3)
    Qa, L, Qb = B.factor([torch.from_numpy(a).cuda() for a in mats])
    rc, flags = B.sync_status()
    assert rc == pq.PBPQLP_ENONFINITE
    assert flags[1] & 4 and not (flags[0] & 4) and not (flags[2] & 4)
    assert flags[0] & 1      # rank 5 < l = 15: shifted retry used
    g0 = [Qa[0].cpu().numpy(), L[0].cpu().numpy(), Qb[0].cpu().numpy()]
    assert oracle.rel_fro_error(mats[0], *g0, 10) < 1e-12
    ref2 = oracle.pbpqlp(mats[2], 17, 1, seed=3 + 2)
    g2 = [Qa[2].cpu().numpy(), L[2].cpu().numpy(), Qb[2].cpu().numpy()]
    d = np.linalg.norm(oracle.reconstruct(*g2, 12) - oracle.reconstruct(ref2["Q"], ref2["L"], ref2["P"], 12))
    assert d / np.linalg.norm(mats[2]) <= TOL


def _errors(A64, g, ref, k):
    e_gpu = oracle.rel_fro_error(A64, *g, k)
    e_orc = oracle.rel_fro_error(A64, ref["Q"], ref["L"], ref["P"], k)
    return e_gpu, e_orc


@pytest.mark.parametrize("a32", [True, False])
def test_batched_split_tf32_within_1p1_of_oracle(pq, a32):
    """TF32 x3 tensor-core products, FP64 Gram / Cholesky / small QR: each
    matrix's rank-k error is within 1.1x of the oracle's on the same data."""
    import torch
    shapes = synth.batched_shapes(11, 10, m_range=(200, 1200), n_lo=100, n_hi=700, k_range=(8, 48))
    mats = [synth.poly_decay(500 + i, s["m"], s["n"], s["alpha"]).astype(np.float32).astype(np.float64)
            for i, s in enumerate(shapes)]
    p, q, seed = 8, 1, 77
    B = pq.Batch([s["m"] for s in shapes], [s["n"] for s in shapes], [s["k"] for s in shapes], p, q, seed,
                 mode=pq.PBPQLP_MODE_TF32X3)
    As = [torch.from_numpy(a.astype(np.float32) if a32 else a).cuda() for a in mats]
    Qa, L, Qb = B.factor(As)
    rc, flags = B.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    for i, (s, A) in enumerate(zip(shapes, mats)):
        ref = oracle.pbpqlp(A, s["k"] + p, q, seed=seed + i)
        g = [Qa[i].cpu().numpy(), L[i].cpu().numpy(), Qb[i].cpu().numpy()]
        e_gpu, e_orc = _errors(A, g, ref, s["k"])
        assert e_gpu <= 1.1 * e_orc, (i, s, e_gpu, e_orc)
        assert np.array_equal(g[1], np.tril(g[1]))


def test_batched_tf32_single_term_runs(pq):
    import torch
    shapes = synth.batched_shapes(12, 6, m_range=(200, 900), n_lo=100, n_hi=600, k_range=(8, 32))
    mats = [synth.poly_decay(700 + i, s["m"], s["n"], 1.0).astype(np.float32) for i, s in enumerate(shapes)]
    B = pq.Batch([s["m"] for s in shapes], [s["n"] for s in shapes], [s["k"] for s in shapes], 8, 1, 5,
                 mode=pq.PBPQLP_MODE_TF32)
    Qa, L, Qb = B.factor([torch.from_numpy(a).cuda() for a in mats])
    rc, flags = B.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    for i, (s, A) in enumerate(zip(shapes, mats)):
        A64 = A.astype(np.float64)
        ref = oracle.pbpqlp(A64, s["k"] + 8, 1, seed=5 + i)
        g = [Qa[i].cpu().numpy(), L[i].cpu().numpy(), Qb[i].cpu().numpy()]
        e_gpu, e_orc = _errors(A64, g, ref, s["k"])
        assert np.isfinite(e_gpu) and e_gpu <= 2.0 * e_orc, (i, e_gpu, e_orc)


def test_batched_autotune_keeps_results(pq, tmp_path):
    import json
    import torch
    shapes, mats = _batch(7, 5)
    p, q, seed = 8, 1, 21
    B = pq.Batch([s["m"] for s in shapes], [s["n"] for s in shapes], [s["k"] for s in shapes], p, q, seed)
    As = [torch.from_numpy(a).cuda() for a in mats]
    outs = B.outputs()
    table = str(tmp_path / "tune.jsonl")
    best = B.autotune(As, outs, table_path=table)
    assert best > 0
    rec = json.loads(open(table).read().strip().splitlines()[-1])
    assert rec["gram_chunk"] in (256, 512, 1024, 2048) and rec["trsm_rows"] in (64, 128, 256)
    B.factor(As, out=outs)
    rc, _ = B.sync_status()
    assert rc == pq.PBPQLP_OK
    for i, (s, A) in enumerate(zip(shapes, mats)):
        ref = oracle.pbpqlp(A, s["k"] + p, q, seed=seed + i)
        g = [outs[0][i].cpu().numpy(), outs[1][i].cpu().numpy(), outs[2][i].cpu().numpy()]
        d = np.linalg.norm(oracle.reconstruct(*g, s["k"]) - oracle.reconstruct(ref["Q"], ref["L"], ref["P"], s["k"]))
        assert d / np.linalg.norm(A) <= TOL


@pytest.mark.parametrize("mode", ["FP64", "TF32X3"])
def test_batched_digit_grams_match_fma_grams(pq, monkeypatch, mode):
    """Grouped exact-digit Grams (default) against the FP64 FMA Grams
    (PBPQLP_NO_OZ_GRAM=1 at plan creation) on the same batch; in FP64 mode
    the batch includes l > 128 (two 128-row tiles per Gram column)."""
    import torch
    md = getattr(pq, "PBPQLP_MODE_" + mode)
    if mode == "FP64":
        shapes = [dict(m=700, n=500, k=150), dict(m=400, n=300, k=60), dict(m=260, n=240, k=200),
                  dict(m=1500, n=180, k=20)]
        mats = [synth.poly_decay(900 + i, s["m"], s["n"], 1.5) for i, s in enumerate(shapes)]
    else:
        shapes = synth.batched_shapes(13, 8, m_range=(200, 1500), n_lo=100, n_hi=700, k_range=(8, 64))
        mats = [synth.poly_decay(950 + i, s["m"], s["n"], s["alpha"]) for i, s in enumerate(shapes)]
    p, q, seed = 8, 1, 15
    As = [torch.from_numpy(a).cuda() for a in mats]
    out = []
    for no_oz in (False, True):
        if no_oz:
            monkeypatch.setenv("PBPQLP_NO_OZ_GRAM", "1")
        B = pq.Batch([s["m"] for s in shapes], [s["n"] for s in shapes], [s["k"] for s in shapes], p, q, seed,
                     mode=md)
        Qa, L, Qb = B.factor(As)
        rc, flags = B.sync_status()
        assert rc == pq.PBPQLP_OK, flags
        out.append([[t.cpu().numpy() for t in (Qa[i], L[i], Qb[i])] for i in range(len(shapes))])
    for i, (s, A) in enumerate(zip(shapes, mats)):
        a1 = oracle.reconstruct(*out[0][i], s["k"])
        a2 = oracle.reconstruct(*out[1][i], s["k"])
        ref = oracle.pbpqlp(A, s["k"] + p, q, seed=seed + i)
        if mode == "FP64":
            assert np.linalg.norm(a1 - a2) <= 1e-12 * np.linalg.norm(A), (i, s)
            d = np.linalg.norm(a1 - oracle.reconstruct(ref["Q"], ref["L"], ref["P"], s["k"]))
            assert d / np.linalg.norm(A) <= TOL, (i, s, d)
        else:
            # the FP32 triangular solves of this mode round any last-bit Gram
            # difference at FP32 level: compare against the mode's error bar
            e_gpu, e_orc = _errors(A, out[0][i], ref, s["k"])
            assert e_gpu <= 1.1 * e_orc, (i, s, e_gpu, e_orc)
            assert np.linalg.norm(a1 - a2) <= 1e-2 * e_orc * np.linalg.norm(A), (i, s)


def test_batched_host_producer_fault_is_reported_without_launches(pq, monkeypatch):
    """Failure detection on the host: with PBPQLP_FAULT=batch_producer (read
    at plan creation) the work-list producer gives up half-way, the call
    returns an error having launched nothing, and a plan without the hook
    factors the same batch cleanly."""
    import torch
    shapes, mats = _batch(8, 3)
    args = ([s["m"] for s in shapes], [s["n"] for s in shapes], [s["k"] for s in shapes], 8, 1, 4)
    monkeypatch.setenv("PBPQLP_FAULT", "batch_producer")
    Bf = pq.Batch(*args)
    monkeypatch.delenv("PBPQLP_FAULT")
    As = [torch.from_numpy(a).cuda() for a in mats]
    torch.cuda.synchronize()
    n0 = pq.pbpqlp_kernel_launch_count()
    with pytest.raises(pq.PbpqlpError) as ei:
        Bf.factor(As)
    assert ei.value.status == pq.PBPQLP_ECUDA
    assert pq.pbpqlp_kernel_launch_count() == n0
    B = pq.Batch(*args)
    Qa, L, Qb = B.factor(As)
    rc, flags = B.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    for i, (s, A) in enumerate(zip(shapes, mats)):
        ref = oracle.pbpqlp(A, s["k"] + 8, 1, seed=4 + i)
        g = [Qa[i].cpu().numpy(), L[i].cpu().numpy(), Qb[i].cpu().numpy()]
        d = np.linalg.norm(oracle.reconstruct(*g, s["k"]) - oracle.reconstruct(ref["Q"], ref["L"], ref["P"], s["k"]))
        assert d / np.linalg.norm(A) <= TOL
