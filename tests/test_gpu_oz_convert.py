"""The conversion that ends every FP64-accurate digit product: each output is
accumulated as two exact 64-bit integer sums hi and lo worth
(hi 2^28 + lo) 2^e, and must come out as that value rounded once to the
nearest double, ties to even.  The kernels' form (64-bit operations and one
hardware integer-to-double conversion) must agree bit for bit with the
reference form (92-bit integer normalisation), and both with Python's
correctly rounded int-to-float conversion wherever the result is a normal
double (there a power-of-two scale is exact)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2103_07245_gb300 as pq
    pq.load(build_if_missing=True)
    return pq


def _cases():
    rng = np.random.default_rng(23)
    n = 200000
    kh = rng.integers(0, 62, n)
    kl = rng.integers(0, 63, n)
    hi = (rng.integers(0, 1 << 62, n, dtype=np.int64) >> (62 - kh)) * rng.choice([-1, 1], n)
    lo = (rng.integers(0, 1 << 62, n, dtype=np.int64) >> (62 - np.minimum(kl, 62))) * rng.choice([-1, 1], n)
    e = rng.integers(-300, 300, n)
    his, los, es = [hi], [lo], [e]
    # halfway cases of the 53-bit rounding at every shift, both signs, odd and even mantissas
    hw_h, hw_l = [], []
    for t in range(1, 36):
        for m in ((1 << 52) + 1, (1 << 52) + 2, (1 << 53) - 1, (1 << 52) | 0x5555):
            N = m * (1 << t) + (1 << (t - 1))
            for sgn in (1, -1):
                v = sgn * N
                for d in (0, 5, -3):              # the same value with lo carrying past 2^28 either way
                    h = (v >> 28) - d
                    hw_h.append(h)
                    hw_l.append(v - h * (1 << 28))
    # the H < 2^35 boundary, zero, lo-only values, L = 0 negatives
    for H in ((1 << 35) - 1, 1 << 35, (1 << 35) + 1, (1 << 61) + 12345, 0, 1, -1):
        for L in (0, 1, (1 << 27), (1 << 28) - 1):
            for sgn in (1, -1):
                hw_h.append(sgn * H)
                hw_l.append(sgn * L)
    for v in (0, 1, -1, (1 << 62) - 1, -(1 << 62) + 1, 12345678901234567):
        hw_h.append(0)
        hw_l.append(v)
    his.append(np.array(hw_h, dtype=np.int64))
    los.append(np.array(hw_l, dtype=np.int64))
    es.append(rng.integers(-200, 200, len(hw_h)))
    # scales that leave the normal range (the fallback)
    k = 4000
    his.append(rng.integers(-(1 << 50), 1 << 50, k, dtype=np.int64))
    los.append(rng.integers(-(1 << 60), 1 << 60, k, dtype=np.int64))
    es.append(np.concatenate([rng.integers(-1200, -1000, k // 2), rng.integers(950, 1000, k - k // 2)]))
    return np.concatenate(his), np.concatenate(los), np.concatenate(es).astype(np.int32)


def test_fast_conversion_is_the_correctly_rounded_value(pq):
    import torch
    hi, lo, e = _cases()
    n = hi.size
    th, tl, te = (torch.from_numpy(x).cuda() for x in (hi, lo, e))
    fast = torch.empty(n, dtype=torch.float64, device="cuda")
    exact = torch.empty_like(fast)
    pq.pbpqlp_oz_convert_check(th, tl, te, n, fast, exact)
    torch.cuda.synchronize()
    f, x = fast.cpu().numpy(), exact.cpu().numpy()
    assert np.array_equal(f.view(np.int64), x.view(np.int64)), np.flatnonzero(f.view(np.int64) != x.view(np.int64))[:5]
    checked = 0
    for i in range(n):
        N = int(hi[i]) * (1 << 28) + int(lo[i])
        if N == 0:
            assert f[i] == 0.0
            continue
        r = float(N)                        # correctly rounded, ties to even
        m, ex = math.frexp(r)
        if not (-1021 <= ex + int(e[i]) <= 1024):
            continue                        # outside the normal range: bitwise against the reference above
        want = math.ldexp(r, int(e[i]))
        assert f[i] == want, (i, int(hi[i]), int(lo[i]), int(e[i]), f[i], want)
        checked += 1
    assert checked > n * 0.95
