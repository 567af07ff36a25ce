"""pbpqlp_factor_from: Algorithm 3 continued from a basis.

The thin-QR prefix property makes the first l' columns of a wider run's basis
the basis of the l'-column run with Phi's first l' columns, at every power
iteration; a continued run must therefore match the oracle run with that
Phi prefix (parity bar 1e-11), and splitting a run at any iteration must give
bitwise the same factors as the unsplit run (the same kernels)."""
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


def _diff(A_np, g, ref, r):
    return np.linalg.norm(oracle.reconstruct(*g, r) - oracle.reconstruct(ref["Q"], ref["L"], ref["P"], r)) \
        / np.linalg.norm(A_np)


@pytest.mark.parametrize("m,n,k,p,q", [(900, 700, 30, 10, 2), (600, 1100, 50, 5, 1), (1300, 1000, 240, 10, 1)])
def test_continuing_a_wider_sketch_matches_the_oracle_with_the_phi_prefix(pq, m, n, k, p, q):
    import torch
    A_np = synth.poly_decay(m + n, m, n, 1.5)
    A = torch.from_numpy(A_np).cuda()
    l0, seed = k + 20, 17
    sketch = pq.Plan(m, n, k, 20, 0, seed)
    Qa0, L0, Qb0, P0 = sketch.factor_from(A, pbar_out=True)
    assert sketch.sync_status()[0] == pq.PBPQLP_OK
    # the sketch itself is the plain q = 0 run
    phi = oracle.gaussian(seed, (m, l0))
    ref0 = oracle.pbpqlp(A_np, l0, 0, phi=phi)
    assert _diff(A_np, [t.cpu().numpy() for t in (Qa0, L0, Qb0)], ref0, k) <= TOL
    assert np.max(np.abs(P0.cpu().numpy() - ref0["Pbar"])) <= 1e-9
    # continue its first k + p columns with q power iterations
    plan = pq.Plan(m, n, k, p, q, seed=999)     # the seed is unused when starting from a basis
    Qa, L, Qb, Pq = plan.factor_from(A, pbar0=P0[:, :k + p], pbar_out=True)
    rc, flags = plan.sync_status()
    assert rc == pq.PBPQLP_OK, flags
    ref = oracle.pbpqlp(A_np, k + p, q, phi=np.ascontiguousarray(phi[:, :k + p]))
    g = [t.cpu().numpy() for t in (Qa, L, Qb)]
    assert _diff(A_np, g, ref, k) <= TOL
    assert _diff(A_np, g, ref, k + p) <= TOL
    assert np.max(np.abs(Pq.cpu().numpy() - ref["Pbar"])) <= 1e-9


def test_split_runs_are_bitwise_the_unsplit_run(pq):
    import torch
    m, n, k, p = 800, 650, 40, 10
    A = torch.from_numpy(synth.exp_decay(5, m, n, 30.0)).cuda()
    full = pq.Plan(m, n, k, p, 2, seed=3)
    ref = [t.clone() for t in full.factor_from(A, pbar_out=True)]
    # the first iteration only, then the rest from its basis
    one = pq.Plan(m, n, k, p, 1, seed=3)
    _, _, _, P1 = one.factor_from(A, iterations_only=True)
    rest = pq.Plan(m, n, k, p, 1, seed=3)
    got = rest.factor_from(A, pbar0=P1, pbar_out=True)
    assert rest.sync_status()[0] == pq.PBPQLP_OK
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    # and the plain entry point gives the same factors
    Qa, L, Qb = full.factor(A)
    for a, b in zip(ref[:3], (Qa, L, Qb)):
        assert torch.equal(a, b)


def test_argument_checks(pq):
    import torch
    m, n, k, p = 300, 200, 10, 5
    A = torch.from_numpy(synth.exp_decay(6, m, n, 10.0)).cuda()
    plan = pq.Plan(m, n, k, p, 1, seed=1)
    narrow = torch.zeros(n, k + p - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(pq.PbpqlpError) as e:
        pq.pbpqlp_factor_from(plan.handle, A, n, pq.PBPQLP_F64, plan.workspace, plan.ws_bytes, narrow, k + p - 1,
                              None, *plan.outputs())
    assert e.value.status == pq.PBPQLP_EINVAL
    with pytest.raises(pq.PbpqlpError) as e:   # nothing to write
        pq.pbpqlp_factor_from(plan.handle, A, n, pq.PBPQLP_F64, plan.workspace, plan.ws_bytes, None, 0, None,
                              None, None, None)
    assert e.value.status == pq.PBPQLP_EINVAL
