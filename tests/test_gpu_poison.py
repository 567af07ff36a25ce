"""Reads of unwritten workspace memory: every path runs once on a zeroed
workspace and once on a workspace filled with 0xFF bytes (NaN as FP64 and
FP32, -1 as integers); the factors must be bitwise equal."""
import numpy as np
import pytest

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


def _twice(pq, ws, run, status):
    ws.fill_(0)
    a = [t.clone() for t in run()]
    rc, flags = status()
    assert rc == pq.PBPQLP_OK, flags
    ws.fill_(255)
    b = run()
    rc, flags = status()
    assert rc == pq.PBPQLP_OK, flags
    for x, y in zip(a, b):
        assert bool(np.isfinite(y.cpu().numpy()).all())
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


@pytest.mark.parametrize("mode", ["FP64", "FP64_EMU", "BF16X3", "TF32X3"])
def test_single_matrix_ignores_workspace_contents(pq, mode):
    import torch
    m, n, k, p, q = 700, 530, 40, 10, 1
    A = torch.from_numpy(synth.exp_decay(21, m, n, 15.0)).cuda()
    plan = pq.Plan(m, n, k, p, q, seed=3, mode=getattr(pq, "PBPQLP_MODE_" + mode))
    out = plan.outputs()
    _twice(pq, plan.workspace, lambda: plan.factor(A, out=out), plan.sync_status)


@pytest.mark.parametrize("mode", ["FP64", "TF32X3"])
def test_batched_ignores_workspace_contents(pq, mode):
    import torch
    shapes = synth.batched_shapes(17, 5, m_range=(200, 800), n_lo=100, n_hi=500, k_range=(8, 40))
    As = [torch.from_numpy(synth.poly_decay(40 + i, s["m"], s["n"], s["alpha"])).cuda() for i, s in enumerate(shapes)]
    B = pq.Batch([s["m"] for s in shapes], [s["n"] for s in shapes], [s["k"] for s in shapes], 8, 1, 6,
                 mode=getattr(pq, "PBPQLP_MODE_" + mode))
    out = B.outputs()

    def run():
        B.factor(As, out=out)
        return [t for ts in out for t in ts]
    _twice(pq, B.workspace, run, lambda: B.sync_status())


def test_sparse_ignores_workspace_contents(pq):
    import torch
    m, n = 900, 700
    rp, ci, va = synth.sparse_csr(23, m, n, 6.0, rank=30, support=80, dup_frac=0.1, shuffle=True)
    d = [torch.from_numpy(x).cuda() for x in (rp, ci, va)]
    plan = pq.Plan(m, n, 30, 10, 1, seed=8)
    out = plan.outputs()
    plan.factor_csr(*d, out=out)   # allocates the CSR workspace
    _twice(pq, plan._csr_ws, lambda: plan.factor_csr(*d, out=out), plan.sync_status)
