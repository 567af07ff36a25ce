"""Streamed A in the mixed and emulated modes (PBPQLP_STREAM_A; the
pass-efficient setting of Section III-C): A stays in pinned host memory and
every pass splits or digitises one block of its rows at a time, so no whole
converted copy of A is ever held on the device.  Against the oracle on the
same A and Phi: FP64-accurate emulated products to the FP64 parity bar
(1e-11), the split modes within 1.1x of the oracle's error."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2103_07245_gb300 as pq
    pq.load(build_if_missing=True)
    return pq


def _host(A_np, f32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(A_np.astype(np.float32) if f32 else A_np)).pin_memory()


def _run(pq, A, m, n, k, p, q, mode, seed):
    plan = pq.Plan(m, n, k, p, q, seed, mode=mode)
    Qa, L, Qb = plan.factor(A)
    rc, flags = plan.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    return plan, [t.cpu().numpy() for t in (Qa, L, Qb)]


@pytest.mark.parametrize("rows", ["256", "1000"])
def test_streamed_emulated_fp64_matches_oracle(pq, monkeypatch, rows):
    monkeypatch.setenv("PBPQLP_STREAM_ROWS", rows)
    m, n, k, p, q = 1100, 800, 40, 10, 2
    A_np = synth.poly_decay(61, m, n, 1.5)
    plan, g = _run(pq, _host(A_np, False), m, n, k, p, q, pq.PBPQLP_MODE_FP64_EMU | pq.PBPQLP_STREAM_A, 5)
    ref = oracle.pbpqlp(A_np, k + p, q, seed=5)
    for r in (k, k + p):
        d = np.linalg.norm(oracle.reconstruct(*g, r) - oracle.reconstruct(ref["Q"], ref["L"], ref["P"], r))
        assert d / np.linalg.norm(A_np) <= 1e-11, (r, d)
    # deterministic: a second run is bitwise the first
    Qa, L, Qb = plan.factor(_host(A_np, False))
    assert plan.sync_status()[0] == pq.PBPQLP_OK
    assert np.array_equal(L.cpu().numpy(), g[1]) and np.array_equal(Qb.cpu().numpy(), g[2])


@pytest.mark.parametrize("mode", ["BF16X3", "TF32X3"])
def test_streamed_split_modes_within_1p1_of_oracle(pq, monkeypatch, mode):
    monkeypatch.setenv("PBPQLP_STREAM_ROWS", "320")
    m, n, k, p, q = 1300, 900, 60, 10, 2
    rng = np.random.default_rng(7)
    X = rng.standard_normal((m, 80)).astype(np.float32)
    Y = rng.standard_normal((n, 80)).astype(np.float32)
    A32 = (X @ Y.T + np.float32(1e-3) * rng.standard_normal((m, n)).astype(np.float32)).astype(np.float32)
    A_np = A32.astype(np.float64)
    _, g = _run(pq, _host(A32, True), m, n, k, p, q, getattr(pq, "PBPQLP_MODE_" + mode) | pq.PBPQLP_STREAM_A, 8)
    ref = oracle.pbpqlp(A_np, k + p, q, seed=8)
    e_gpu = oracle.rel_fro_error(A_np, *g, k)
    e_orc = oracle.rel_fro_error(A_np, ref["Q"], ref["L"], ref["P"], k)
    assert e_gpu <= 1.1 * e_orc, (e_gpu, e_orc)


def test_streamed_blocked_width(pq, monkeypatch):
    """l = 260 > 224 with streamed digit products (column chunks do not apply: any width)."""
    monkeypatch.setenv("PBPQLP_STREAM_ROWS", "512")
    m, n, k, p, q = 1200, 1000, 250, 10, 1
    A_np = synth.exp_decay(62, m, n, 120.0)
    _, g = _run(pq, _host(A_np, False), m, n, k, p, q, pq.PBPQLP_MODE_FP64_EMU | pq.PBPQLP_STREAM_A, 3)
    ref = oracle.pbpqlp(A_np, k + p, q, seed=3)
    d = np.linalg.norm(oracle.reconstruct(*g, k) - oracle.reconstruct(ref["Q"], ref["L"], ref["P"], k))
    assert d / np.linalg.norm(A_np) <= 1e-11
