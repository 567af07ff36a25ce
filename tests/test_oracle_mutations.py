"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of the oracle's C source, builds it, and runs the CPU pins against
that copy in a subprocess: at least one pin must fail.  (The Philox stream and
the Box-Muller mapping are pinned by known-answer vectors and by the GPU
parity tests, which draw the same stream independently.)"""
import os
import subprocess
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pbpqlp_oracle.c")

MUTANTS = {
    "gemm_sign": ("c[j] += a * b[j];", "c[j] -= a * b[j];"),
    "qr_no_sign_fix": ("sgn[j] = (W[j * cols + j] < 0.0) ? -1.0 : 1.0;", "sgn[j] = 1.0;"),
    "L_not_transposed": ("L[i * l + j] = Rt[j * l + i];", "L[i * l + j] = Rt[i * l + j];"),
    "P_without_Ptil": ("orc_gemm(0, n, l, l, Pb, l, Pt, l, P, l);",
                       "memcpy(P, Pb, sizeof(double) * (size_t)n * (size_t)l);"),
    "csr_skips_first_entry": ("for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {",
                              "for (int64_t e = rowptr[i] + 1; e < rowptr[i + 1]; ++e) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mut = tmp_path / "oracle_mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", str(so), str(mut), "-lm"],
                   check=True)
    env = dict(os.environ, PBPQLP_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-k", "not paper",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_sparse.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "mistake %r passed every pin:\n%s" % (name, r.stdout[-2000:])
    assert "failed" in r.stdout, r.stdout[-2000:]


# Planted mistakes in the Python parts of the oracle: AdamW (oracle/mlp.py)
# and the probe estimator (oracle/__init__.py).  Each copy is loaded as a
# module of its own and must fail the closed-form pins of test_oracle_aux_pins.
PY_MUTANTS = {
    "adamw_no_bias_correction": ("mlp.py", "(m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)",
                                 "m / (np.sqrt(v) + eps)"),
    "adamw_coupled_l2": ("mlp.py", "    m = b1 * m + (1 - b1) * g\n",
                         "    g = g + wd * p\n    m = b1 * m + (1 - b1) * g\n"),
    "adamw_bias_exponent_off_by_one": ("mlp.py", "(1 - b1 ** t)", "(1 - b1 ** (t + 1))"),
    "probe_no_sqrt": ("__init__.py", "np.sqrt(np.sum(EW * EW) / np.sum(AW * AW))",
                      "np.sum(EW * EW) / np.sum(AW * AW)"),
    "probe_sign_of_reconstruction": ("__init__.py", "EW = AW - Q[:, :r]", "EW = AW + Q[:, :r]"),
}


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_python_pins_catch_planted_mistake(name, tmp_path, orc):
    import importlib.util
    import types

    fname, old, new = PY_MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    assert src.count(old) == 1, name
    path = tmp_path / ("mutant_" + fname)
    path.write_text(src.replace(old, new))
    import test_oracle_aux_pins as pins
    if fname == "mlp.py":
        spec = importlib.util.spec_from_file_location("mlp_mutant", str(path))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        with pytest.raises(AssertionError):
            pins.check_adamw(mod)
    else:
        # only the estimator is taken from the mutant; the factorization stays the oracle's
        ns = {}
        code = src.replace(old, new)
        start = code.index("def probe_error_estimate")
        exec(compile("import numpy as np\n" + code[start:], str(path), "exec"), ns)
        mod = types.SimpleNamespace(pbpqlp=orc.pbpqlp, probe_error_estimate=ns["probe_error_estimate"])
        with pytest.raises(AssertionError):
            pins.check_probe_estimate(mod)
