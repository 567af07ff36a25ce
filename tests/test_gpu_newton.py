"""The Newton-refined FP64 reciprocal and reciprocal square root, and the
one-step Goldschmidt reciprocal, that the Cholesky and QR kernels use on
their pivot chains, against correctly rounded
results (numpy's IEEE division, and 1/sqrt taken in extended precision), over
every exponent of the double format and its edge cases.

Bound: 2 ulp of the correctly rounded result for positive normal inputs;
the inputs the helpers hand to CUDA's own division / square root (zero,
subnormal, negative, Inf, NaN, d >= 2^1023 for the reciprocal) must match
IEEE results exactly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ULP_BOUND = 2.0


@pytest.fixture(scope="module")
def pq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2103_07245_gb300 as pq
    pq.load(build_if_missing=True)
    return pq


def _inputs():
    rng = np.random.default_rng(17)
    # every biased exponent 1..2046, eight random mantissas each, plus the mantissa ends
    e = np.repeat(np.arange(1, 2047, dtype=np.int64), 10)
    mant = rng.integers(0, 1 << 52, e.size, dtype=np.int64)
    mant[0::10] = 0
    mant[1::10] = (1 << 52) - 1
    bits = (e << 52) | mant
    normal = bits.view(np.float64)
    tiny = np.finfo(np.float64).tiny
    edges = np.array([1.0, 2.0, 0.5, 3.0, 4.0, 1.0 - 2.0 ** -53, 2.0 - 2.0 ** -52, tiny, tiny * (1 + 2.0 ** -52),
                      2.0 ** 1023, 1.5 * 2.0 ** 1023, np.finfo(np.float64).max, 2.0 ** 1022, 2.0 ** -1022 * 3,
                      2.0 ** 1000, 2.0 ** -1000])
    special = np.array([0.0, -0.0, tiny / 2, tiny / 2 ** 30, 5e-324, -1.0, -tiny, np.inf, -np.inf, np.nan])
    return normal, edges, special


def _ulps(got, ref):
    ref = ref.astype(np.float64)
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_newton_helpers_within_ulp_bound(pq):
    import torch
    normal, edges, special = _inputs()
    d = np.concatenate([normal, edges, special])
    td = torch.from_numpy(d).cuda()
    rcp = torch.empty_like(td)
    rsq = torch.empty_like(td)
    rgs = torch.empty_like(td)
    pq.pbpqlp_newton_check(td, td.numel(), rcp, rsq, rgs)
    torch.cuda.synchronize()
    rcp, rsq, rgs = rcp.cpu().numpy(), rsq.cpu().numpy(), rgs.cpu().numpy()
    npos = normal.size + edges.size
    x = d[:npos]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore", under="ignore"):
        ref_rcp = 1.0 / x
        ref_rsq = (np.longdouble(1.0) / np.sqrt(x.astype(np.longdouble))).astype(np.float64)
    # reciprocal: results that are normal doubles within the bound; d >= 2^1023
    # (subnormal results) goes to the IEEE division and must match it exactly
    big = x >= 2.0 ** 1023
    u = _ulps(rcp[:npos][~big], ref_rcp[~big])
    assert np.max(u) <= ULP_BOUND, (np.max(u), x[~big][np.argmax(u)])
    assert np.array_equal(rcp[:npos][big], ref_rcp[big])
    # the Goldschmidt reciprocal: every positive normal input, including d >= 2^1023
    u = _ulps(rgs[:npos], ref_rcp)
    assert np.max(u) <= ULP_BOUND, (np.max(u), x[np.argmax(u)])
    u = _ulps(rsq[:npos], ref_rsq)
    assert np.max(u) <= ULP_BOUND, (np.max(u), x[np.argmax(u)])
    # the rest takes IEEE division and square root: bit-identical (NaN as NaN)
    with np.errstate(divide="ignore", invalid="ignore"):
        s_rcp = 1.0 / special
        s_rsq = 1.0 / np.sqrt(special)
    got_r, got_s = rcp[npos:], rsq[npos:]
    assert np.array_equal(np.isnan(got_r), np.isnan(s_rcp)) and np.array_equal(np.isnan(got_s), np.isnan(s_rsq))
    ok = ~np.isnan(s_rcp)
    assert np.array_equal(got_r[ok].view(np.int64), s_rcp[ok].view(np.int64)), (got_r, s_rcp)
    ok = ~np.isnan(s_rsq)
    assert np.array_equal(got_s[ok].view(np.int64), s_rsq[ok].view(np.int64)), (got_s, s_rsq)
