"""Mixed-precision modes (BF16 and split BF16 x3 tcgen05 products, FP64
Gram / Cholesky / small QR) against the FP64 oracle.

Kernel level: pbpqlp_sketch's tensor-core product equals the exact product of
the same BF16-rounded operands within the FP32 summation bound.
Method level: the rank-k error of the split mode is within 1.1x of the
oracle's error on the same A (the accuracy bar for the mixed modes)."""
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


def bf16_rn(x):
    """Round FP64 values to the nearest BF16 (8 significant bits, ties to even)."""
    x = np.asarray(x, dtype=np.float64)
    mant, ex = np.frexp(x)
    return np.ldexp(np.round(mant * 256.0), ex - 8)


def split(x):
    hi = bf16_rn(x)
    return hi, bf16_rn(x - hi)


def tf32_rna(x):
    """FP64 -> FP32 (nearest) -> TF32 (11 significant bits, ties away from zero)."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
    mant, ex = np.frexp(f)
    return np.ldexp(np.sign(mant) * np.floor(np.abs(mant) * 2048.0 + 0.5), ex - 11)


def split_tf32(x):
    hi = tf32_rna(x)
    return hi, tf32_rna(x - hi)


@pytest.mark.parametrize("mode_name", ["BF16", "BF16X3", "TF32", "TF32X3"])
@pytest.mark.parametrize("m,n,ncols,trans", [
    (300, 200, 20, False), (300, 200, 20, True),      # ragged row tiles and k-blocks
    (1000, 777, 224, False), (777, 1000, 224, True),  # widest N, several tiles
    (129, 4100, 17, False),                           # long contraction, one row past a tile
])
def test_tensor_core_product(pq, mode_name, m, n, ncols, trans):
    import torch
    mode = getattr(pq, "PBPQLP_MODE_" + mode_name)
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n)).astype(np.float32).astype(np.float64)
    rowsY = m if trans else n
    Y = rng.standard_normal((rowsY, ncols)) / np.sqrt(rowsY)
    plan = pq.Plan(m, n, max(1, ncols - 1), 1, 0, seed=1, mode=mode)
    C = plan.sketch(torch.from_numpy(A.astype(np.float32)).cuda(), torch.from_numpy(Y).cuda(), trans=trans)
    rc, flags = plan.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    C = C.cpu().numpy()
    Aop = A.T if trans else A
    sp = split_tf32 if mode_name.startswith("TF32") else split
    ah, al = sp(Aop)
    yh, yl = sp(Y)
    if mode_name in ("BF16", "TF32"):
        ref = ah @ yh
        mag = np.abs(ah) @ np.abs(yh)
    else:
        ref = ah @ yh + al @ yh + ah @ yl
        mag = np.abs(ah) @ np.abs(yh) + np.abs(al) @ np.abs(yh) + np.abs(ah) @ np.abs(yl)
    K = Aop.shape[1]
    assert np.all(np.abs(C - ref) <= (K + 2) * 2.0 ** -23 * mag + 1e-300)
    # typical error of FP32 accumulation, far below the dropped-term size
    rms = np.sqrt(np.mean((C - ref) ** 2)) / np.sqrt(np.mean(mag ** 2))
    assert rms < 64 * np.sqrt(K) * 2.0 ** -24


def _mixed_errors(pq, A32, k, p, q, seed, mode):
    import torch
    m, n = A32.shape
    A64 = A32.astype(np.float64)
    plan = pq.Plan(m, n, k, p, q, seed=seed, mode=mode)
    Qa, L, Qb = plan.factor(torch.from_numpy(A32).cuda())
    rc, flags = plan.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    g = [t.cpu().numpy() for t in (Qa, L, Qb)]
    ref = oracle.pbpqlp(A64, k + p, q, seed=seed)
    e_mixed = oracle.rel_fro_error(A64, *g, k)
    e_orc = oracle.rel_fro_error(A64, ref["Q"], ref["L"], ref["P"], k)
    return e_mixed, e_orc, g


def test_split_bf16_factorization_within_1p1_of_oracle(pq):
    A32 = synth.xyt_plus_noise(3, 2000, 1800, 20, 1e-3)
    e_mixed, e_orc, (Qa, L, Qb) = _mixed_errors(pq, A32, 20, 5, 2, 11, pq.PBPQLP_MODE_BF16X3)
    assert e_mixed <= 1.1 * e_orc, (e_mixed, e_orc)
    assert np.array_equal(L, np.tril(L))
    # the mixed modes apply the triangular factors in FP32: orthonormal to ~1e-7
    assert np.allclose(Qa.T @ Qa, np.eye(25), atol=1e-6)
    assert np.allclose(Qb.T @ Qb, np.eye(25), atol=1e-6)


def test_split_tf32_factorization_within_1p1_of_oracle(pq):
    A32 = synth.xyt_plus_noise(6, 1700, 1500, 24, 1e-3)
    e_mixed, e_orc, (Qa, L, Qb) = _mixed_errors(pq, A32, 24, 8, 2, 21, pq.PBPQLP_MODE_TF32X3)
    assert e_mixed <= 1.1 * e_orc, (e_mixed, e_orc)
    assert np.array_equal(L, np.tril(L))


def test_bf16_single_term_factorization_runs(pq):
    """One BF16 product per step: reported, not held to the 1.1x bar."""
    A32 = synth.xyt_plus_noise(4, 1500, 1500, 20, 1e-3)
    e_mixed, e_orc, _ = _mixed_errors(pq, A32, 20, 5, 2, 12, pq.PBPQLP_MODE_BF16)
    assert np.isfinite(e_mixed) and e_mixed >= e_orc * (1 - 1e-6)


def test_split_bf16_poly_decay(pq):
    A32 = synth.poly_decay(5, 1200, 1000, 1.0).astype(np.float32)
    e_mixed, e_orc, _ = _mixed_errors(pq, A32, 30, 10, 1, 13, pq.PBPQLP_MODE_BF16X3)
    assert e_mixed <= 1.1 * e_orc, (e_mixed, e_orc)


@pytest.mark.slow
def test_config3_full_size_within_1p1(pq):
    """20000 x 20000, A = X Y^T + 1e-3 E (FP32), k = 200, p = 20, q = 2."""
    import torch
    A = synth.torch_xyt_plus_noise(3, 20000, 20000, 200, 1e-3)
    A32 = A.cpu().numpy()
    e_mixed, e_orc, _ = _mixed_errors(pq, A32, 200, 20, 2, 17, pq.PBPQLP_MODE_BF16X3)
    assert e_mixed <= 1.1 * e_orc, (e_mixed, e_orc)


def test_bounded_wait_timeout_is_reported_and_context_survives(pq, monkeypatch):
    """Failure detection without a GPU fault: with PBPQLP_FAULT=tc_stall the
    tensor-core producer issues nothing, the consumers' bounded waits expire
    (50 ms), the kernel frees its TMEM and returns, and the status reads
    PBPQLP_ETIMEOUT; the next plan on the same context works."""
    import torch
    rng = np.random.default_rng(0)
    A = torch.from_numpy(rng.standard_normal((300, 200)).astype(np.float32)).cuda()
    Y = torch.from_numpy(rng.standard_normal((200, 16))).cuda()
    monkeypatch.setenv("PBPQLP_FAULT", "tc_stall")
    bad = pq.Plan(300, 200, 12, 4, 0, seed=1, mode=pq.PBPQLP_MODE_BF16X3)
    monkeypatch.delenv("PBPQLP_FAULT")
    bad.sketch(A, Y)
    rc, flags = bad.sync_status()
    assert rc == pq.PBPQLP_ETIMEOUT and (flags & 8), (rc, flags)
    good = pq.Plan(300, 200, 12, 4, 0, seed=1, mode=pq.PBPQLP_MODE_BF16X3)
    C = good.sketch(A, Y).cpu().numpy()
    rc, flags = good.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    ref = A.double().cpu().numpy() @ Y.cpu().numpy()
    assert np.max(np.abs(C - ref)) <= 1e-3 * np.max(np.abs(ref))
