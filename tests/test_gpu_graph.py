"""Launch-sequence replay of pbpqlp_factor / pbpqlp_factor_from.

After two calls in a row with the same arguments a plan records its launch
sequence once into a CUDA graph and replays it while the arguments stay the
same.  A replay runs the same kernels on the same data, so every replayed
result must be bitwise the eagerly launched one (a plan made with
PBPQLP_NO_GRAPH=1), for every mode, for the blocked l, for A streamed from
pinned host memory and for a run continued from a basis; a replay reads A at
replay time (new contents in the same buffer give the new factors), and the
launch counter counts the replayed kernels."""
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


def _plans(pq, monkeypatch, m, n, k, p, q, mode, seed):
    monkeypatch.setenv("PBPQLP_NO_GRAPH", "1")
    eager = pq.Plan(m, n, k, p, q, seed, mode=mode)
    monkeypatch.delenv("PBPQLP_NO_GRAPH")
    return eager, pq.Plan(m, n, k, p, q, seed, mode=mode)


def _check(pq, plan, call, ref, launches_ref):
    import torch
    n0 = pq.pbpqlp_kernel_launch_count()
    got = call()
    torch.cuda.synchronize()
    rc, flags = plan.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    assert pq.pbpqlp_kernel_launch_count() - n0 == launches_ref


CASES = [
    ("FP64", 1000, 800, 40, 10, 2, False, False),
    ("FP64_EMU", 1100, 700, 50, 10, 2, False, False),
    ("BF16X3", 1300, 900, 60, 10, 2, True, False),
    ("TF32", 900, 1000, 30, 10, 1, True, False),
    ("FP64", 1200, 900, 290, 10, 1, False, False),     # l = 300: blocked Cholesky and QR
    ("FP64_EMU", 1100, 800, 40, 10, 2, False, True),   # A streamed from pinned host memory
]


@pytest.mark.parametrize("mode,m,n,k,p,q,f32,stream", CASES)
def test_replays_are_bitwise_the_eager_run(pq, monkeypatch, mode, m, n, k, p, q, f32, stream):
    import torch
    if stream:
        monkeypatch.setenv("PBPQLP_STREAM_ROWS", "256")
    md = getattr(pq, "PBPQLP_MODE_" + mode) | (pq.PBPQLP_STREAM_A if stream else 0)
    eager, plan = _plans(pq, monkeypatch, m, n, k, p, q, md, 11)
    A_np = synth.poly_decay(m + 3 * n, m, n, 1.5)
    A2_np = synth.exp_decay(m + n, m, n, 25.0)
    dt = torch.float32 if f32 else torch.float64

    def place(x):
        t = torch.from_numpy(np.ascontiguousarray(x)).to(dt)
        return t.pin_memory() if stream else t.cuda()

    A = place(A_np)
    n0 = pq.pbpqlp_kernel_launch_count()
    ref = [t.clone() for t in eager.factor(A)]
    torch.cuda.synchronize()
    launches = pq.pbpqlp_kernel_launch_count() - n0
    assert eager.sync_status()[0] == pq.PBPQLP_OK
    out = plan.outputs()
    for _ in range(4):      # eager, recorded + replayed, then replays
        _check(pq, plan, lambda: plan.factor(A, out=out), ref, launches)
    # new contents of the same A buffer: the replay reads them
    A.copy_(place(A2_np))
    ref2 = [t.clone() for t in eager.factor(A)]
    _check(pq, plan, lambda: plan.factor(A, out=out), ref2, launches)
    # other output buffers: eager again, then a new recording
    out2 = plan.outputs()
    for _ in range(3):
        _check(pq, plan, lambda: plan.factor(A, out=out2), ref2, launches)
    _check(pq, plan, lambda: plan.factor(A, out=out), ref2, launches)


def test_continued_runs_replay_bitwise(pq, monkeypatch):
    import torch
    m, n, k, p = 900, 700, 30, 10
    A = torch.from_numpy(synth.poly_decay(5, m, n, 1.5)).cuda()
    sketch = pq.Plan(m, n, k, 20, 0, 17)
    _, _, _, P0 = sketch.factor_from(A, pbar_out=True)
    P0 = P0[:, :k + p].contiguous()
    eager, plan = _plans(pq, monkeypatch, m, n, k, p, 2, pq.PBPQLP_MODE_FP64, 999)
    n0 = pq.pbpqlp_kernel_launch_count()
    ref = [t.clone() for t in eager.factor_from(A, pbar0=P0, pbar_out=True)]
    torch.cuda.synchronize()
    launches = pq.pbpqlp_kernel_launch_count() - n0
    out = plan.outputs()
    pb = torch.empty(n, k + p, dtype=torch.float64, device="cuda")

    def call():
        pq.pbpqlp_factor_from(plan.handle, A, A.stride(0), pq.PBPQLP_F64, plan.workspace, plan.ws_bytes, P0,
                              P0.stride(0), pb, *out)
        return (*out, pb)

    for _ in range(4):
        _check(pq, plan, call, ref, launches)
