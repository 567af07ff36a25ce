"""Host-side checks of the C ABI: the library loads, exports every function
include/*.h declares, and validates arguments without touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for mt in re.finditer(r"\b(pbpqlp_\w+)\s*\(", src):
            names.add(mt.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def pq():
    import paper_2103_07245_gb300 as pq
    pq.load(build_if_missing=True)
    return pq


def test_library_exports_every_declared_symbol(pq):
    names = _declared_functions()
    assert "pbpqlp_factor" in names and "pbpqlp_plan" in names
    lib = ctypes.CDLL(pq.lib_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_strerror(pq):
    assert pq.pbpqlp_version() >= 10000
    for code in range(0, 9):
        assert isinstance(pq.strerror(code), str) and pq.strerror(code)


@pytest.mark.parametrize("args", [
    (0, 10, 2, 1, 1),      # m < 1
    (10, 10, 0, 1, 1),     # k < 1
    (10, 10, 8, 3, 1),     # l > min(m, n)
    (10, 10, 2, -1, 1),    # p < 0
    (10, 10, 2, 1, -1),    # q < 0
    (5000, 5000, 4090, 10, 1),  # l > 4096
])
def test_plan_rejects_bad_sizes(pq, args):
    with pytest.raises(pq.PbpqlpError) as e:
        pq.pbpqlp_plan(*args, seed=1, mode=pq.PBPQLP_MODE_FP64, stream=0)
    assert e.value.status == pq.PBPQLP_EINVAL


def test_plan_rejects_bad_mode(pq):
    with pytest.raises(pq.PbpqlpError) as e:
        pq.pbpqlp_plan(100, 100, 5, 5, 1, seed=1, mode=99, stream=0)
    assert e.value.status == pq.PBPQLP_EINVAL


def test_plan_workspace_is_sized_and_factor_validates(pq):
    h = pq.pbpqlp_plan(1000, 1000, 20, 5, 1, seed=1, mode=pq.PBPQLP_MODE_FP64, stream=0)
    try:
        ws = pq.pbpqlp_workspace_bytes(h)
        # at least the five panels m x l / n x l in FP64
        assert ws >= 5 * 1000 * 25 * 8
        # null pointers / small workspace are rejected before any launch
        with pytest.raises(pq.PbpqlpError) as e:
            pq.pbpqlp_factor(h, 0, 1000, pq.PBPQLP_F64, 0, ws, None, 0, 0, 0)
        assert e.value.status == pq.PBPQLP_EINVAL
        with pytest.raises(pq.PbpqlpError) as e:
            pq.pbpqlp_factor(h, 256, 1000, pq.PBPQLP_F64, 512, ws - 1, None, 256, 256, 256)
        assert e.value.status == pq.PBPQLP_EWORKSPACE
        with pytest.raises(pq.PbpqlpError) as e:
            pq.pbpqlp_factor(h, 256, 999, pq.PBPQLP_F64, 512, ws, None, 256, 256, 256)
        assert e.value.status == pq.PBPQLP_EINVAL
    finally:
        pq.pbpqlp_plan_destroy(h)


def test_batched_plan_validates(pq):
    with pytest.raises(pq.PbpqlpError) as e:
        pq.pbpqlp_plan_batched([100, 50], [80, 60], [10, 60], 5, 1, seed=1, stream=0)
    assert e.value.status == pq.PBPQLP_EINVAL
    h = pq.pbpqlp_plan_batched([100, 500], [80, 300], [10, 20], 5, 1, seed=1, stream=0)
    try:
        assert pq.pbpqlp_batch_workspace_bytes(h) > 8 * (100 + 500) * 32
    finally:
        pq.pbpqlp_batch_destroy(h)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library every entry point raises."""
    import paper_2103_07245_gb300 as pq
    monkeypatch.setattr(pq._build, "LIB", str(tmp_path / "absent" / "libpbpqlp.so"))
    monkeypatch.setattr(pq, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        pq.load()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        pq.pbpqlp_version()


def test_plan_accepts_blocked_widths_and_rejects_them_without_digit_products(pq, monkeypatch):
    # l > 224 takes the blocked l x l steps, which need the digit-form products
    h = pq.pbpqlp_plan(2000, 2000, 990, 10, 1, seed=1, mode=pq.PBPQLP_MODE_FP64, stream=0)
    assert pq.pbpqlp_workspace_bytes(h) > 3 * 1000 * 1000 * 8
    pq.pbpqlp_plan_destroy(h)
    monkeypatch.setenv("PBPQLP_NO_OZ_GRAM", "1")
    with pytest.raises(pq.PbpqlpError) as e:
        pq.pbpqlp_plan(2000, 2000, 990, 10, 1, seed=1, mode=pq.PBPQLP_MODE_FP64, stream=0)
    assert e.value.status == pq.PBPQLP_EUNSUPPORTED


def test_streamed_plans_hold_no_copy_of_A(pq):
    """PBPQLP_STREAM_A: the mixed and emulated plans keep one row block of A, not A."""
    m = n = 20000
    h0 = pq.pbpqlp_plan(m, n, 200, 20, 2, seed=1, mode=pq.PBPQLP_MODE_BF16X3, stream=0)
    h1 = pq.pbpqlp_plan(m, n, 200, 20, 2, seed=1, mode=pq.PBPQLP_MODE_BF16X3 | pq.PBPQLP_STREAM_A, stream=0)
    h2 = pq.pbpqlp_plan(m, n, 200, 20, 2, seed=1, mode=pq.PBPQLP_MODE_FP64_EMU, stream=0)
    h3 = pq.pbpqlp_plan(m, n, 200, 20, 2, seed=1, mode=pq.PBPQLP_MODE_FP64_EMU | pq.PBPQLP_STREAM_A, stream=0)
    try:
        w0, w1, w2, w3 = (pq.pbpqlp_workspace_bytes(h) for h in (h0, h1, h2, h3))
        assert w0 > 8 * m * n > w1          # split copies of A and A^T: 8 bytes per element
        assert w2 > 32 * m * n > w3         # digits of A and A^T: 32 bytes per element
        assert w1 < 2 << 30 and w3 < 2 << 30
    finally:
        for h in (h0, h1, h2, h3):
            pq.pbpqlp_plan_destroy(h)
