"""pbpqlp_factor_static: the factorization entry point for callers that cannot
allocate device memory (their host framework owns every device allocation, or
they must not pay cudaMalloc's implicit synchronisation).  It runs in the
library's fixed device scratch array; its results must equal, bit for bit,
those of pbpqlp_factor with a caller workspace (the same deterministic
kernels), match the oracle to the parity bar, and leave free device memory
unchanged once the first call on the device has made its one-time set-up.

This file is collected last on purpose, and passes both alone in a fresh
process and after the rest of the suite."""
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


def test_static_scratch_matches_workspace_entry_point(pq):
    import torch
    m, n, k, p, q = 1000, 1000, 20, 5, 1
    plan = pq.Plan(m, n, k, p, q, seed=2)
    assert plan.ws_bytes <= pq.PBPQLP_STATIC_SCRATCH_BYTES
    # a warm-up call makes the one-time per-device set-up (the array's address
    # lookup, which may load the module and reserve the array) before anything
    # is measured
    A0 = torch.from_numpy(synth.poly_decay(9, m, n, 2.0)).cuda()
    Qa, L, Qb = plan.outputs()
    pq.pbpqlp_factor_static(plan.handle, A0, A0.stride(0), pq.PBPQLP_F64, None, Qa, L, Qb)
    assert plan.sync_status()[0] == pq.PBPQLP_OK
    # two calls in a row, on two different matrices, each against the workspace
    # entry point (the same deterministic kernels: bitwise equal) and the oracle
    for call, seed in enumerate((1, 5)):
        A_np = synth.poly_decay(seed, m, n, 2.0)
        A = torch.from_numpy(A_np).cuda()
        Qa_w, L_w, Qb_w = plan.factor(A)
        rc, flags = plan.sync_status()
        assert rc == pq.PBPQLP_OK, flags
        Qa, L, Qb = plan.outputs()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        launches0 = pq.pbpqlp_kernel_launch_count()
        pq.pbpqlp_factor_static(plan.handle, A, A.stride(0), pq.PBPQLP_F64, None, Qa, L, Qb)
        rc, flags = plan.sync_status()
        assert rc == pq.PBPQLP_OK, (call, flags)
        assert torch.cuda.mem_get_info()[0] == free0, "the static entry point changed free device memory"
        assert pq.pbpqlp_kernel_launch_count() > launches0
        for got, ref in ((Qa, Qa_w), (L, L_w), (Qb, Qb_w)):
            assert torch.equal(got, ref), call
        ref = oracle.pbpqlp(A_np, k + p, q, seed=2)
        got = [t.cpu().numpy() for t in (Qa, L, Qb)]
        diff = np.linalg.norm(oracle.reconstruct(*got, k) - oracle.reconstruct(ref["Q"], ref["L"], ref["P"], k)) \
            / np.linalg.norm(A_np)
        assert diff <= TOL, (call, diff)


def test_static_scratch_rejects_plans_above_its_size(pq):
    h = pq.pbpqlp_plan(8000, 8000, 100, 10, 2, seed=1, mode=pq.PBPQLP_MODE_FP64)
    try:
        assert pq.pbpqlp_workspace_bytes(h) > pq.PBPQLP_STATIC_SCRATCH_BYTES
        with pytest.raises(pq.PbpqlpError) as e:
            pq.pbpqlp_factor_static(h, 256, 8000, pq.PBPQLP_F64, None, 256, 256, 256)
        assert e.value.status == pq.PBPQLP_EWORKSPACE
    finally:
        pq.pbpqlp_plan_destroy(h)
