"""The benchmark's reference arm (the oracle timed on the host cores) prints
one JSON line with the keys the measurement contract names; run here on
small dense and CSR workloads so it needs no GPU."""
import argparse
import contextlib
import io
import json

import pytest

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(fn, w):
    import bench
    args = argparse.Namespace(steps=1, warmup=0)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert fn(args, w, 1, 0) == 0
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    return json.loads(lines[0])


def _check(line):
    import bench
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_line_dense():
    pytest.importorskip("torch")
    import bench
    w = dict(m=120, n=90, k=6, p=4, q=1, gen="svd", spectrum="exp", scale=10.0, rank_cap=60, mode="FP64",
             desc="small dense check")
    _check(_run(bench.run_reference, w))


def test_reference_arm_line_sparse():
    import bench
    w = dict(sparse=True, m=300, n=200, k=8, p=4, q=1, nnz_per_row=6.0, rank=5, support=30, mode="FP64",
             desc="small CSR check")
    line = _run(bench.run_reference, w)
    _check(line)
    assert line["config"]["nnz"] > 0
