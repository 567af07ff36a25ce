"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of the oracle's C source, builds it, and runs the CPU pins against
that copy in a subprocess: at least one pin must fail.  (The Philox stream and
the Box-Muller mapping are pinned by known-answer vectors and by the GPU
parity tests, which draw the same stream independently.)"""
import os
import subprocess
import sys

import pytest

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
