"""Pins for the FP64 CPU oracle against what the paper and the mathematics fix.

Each test would catch a plausible slip in the oracle (a dropped term, a wrong
sign or index, a transposed operand): known-answer vectors for the generator,
library cross-checks for GEMM/QR, the closed forms of Eqs. 3-8 (Q L P^T =
A Pbar Pbar^T, L = Q^T A P, the Pythagorean identity), exact recovery, the
Eckart-Young bound, the deterministic inequalities of Theorems 5-7 and the
bands printed in the paper's Section V-B figures.
"""
import math

import numpy as np
import pytest

import synth


def _sv(x):
    return np.linalg.svd(x, compute_uv=False)


def _np_orth(x):
    q, r = np.linalg.qr(x)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s


# ------------------------------------------------------------------ Philox
def test_philox_known_answer_vectors(orc):
    # Known-answer vectors published with Random123 (Salmon et al., SC'11).
    assert orc.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert orc.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert orc.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]) == \
        [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_gaussian_is_standard_normal(orc):
    from scipy import stats
    n = 400_000
    z = orc.gaussian(20240611, (n,))
    assert abs(z.mean()) < 5.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 0.05
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # even (cos) and odd (sin) samples of one pair are independent normals
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 5.0 / math.sqrt(n / 2)
    assert stats.kstest(z[1::2], "norm").pvalue > 1e-4
    # a pair's squared radius is chi^2 with 2 dof, i.e. Exp(1/2)
    r2 = z[0::2] ** 2 + z[1::2] ** 2
    assert stats.kstest(r2, "expon", args=(0, 2.0)).pvalue > 1e-4


def test_gaussian_counter_addressing(orc):
    full = orc.gaussian(7, (64,))
    part = orc.gaussian(7, (11,), offset=13)
    assert np.array_equal(full[13:24], part)
    assert not np.allclose(orc.gaussian(8, (64,)), full)


# ------------------------------------------------------------- GEMM and QR
@pytest.mark.parametrize("trans", [False, True])
def test_gemm_matches_library(orc, trans):
    rng = np.random.default_rng(0)
    a = rng.standard_normal((37, 23))
    b = rng.standard_normal((23 if not trans else 37, 9))
    ref = (a.T if trans else a) @ b
    assert np.allclose(orc.gemm(a, b, trans_a=trans), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape", [(50, 20), (20, 20), (300, 7), (5, 1)])
def test_qr_matches_lapack(orc, shape):
    rng = np.random.default_rng(shape[0] * 31 + shape[1])
    x = rng.standard_normal(shape)
    q, r = orc.qr(x)
    qn = _np_orth(x)
    rn = qn.T @ x
    assert np.allclose(q, qn, atol=1e-13)
    assert np.allclose(r, np.triu(rn), atol=1e-12)
    assert np.all(np.diag(r) >= 0) and np.array_equal(r, np.triu(r))
    assert np.allclose(q.T @ q, np.eye(shape[1]), atol=1e-14)


def test_qr_rank_deficient_still_factors(orc):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((40, 3)) @ rng.standard_normal((3, 6))
    q, r = orc.qr(x)
    assert np.allclose(q @ r, x, atol=1e-12)
    assert np.allclose(q.T @ q, np.eye(6), atol=1e-13)


# --------------------------------------------------------- the factorization
@pytest.fixture(scope="module")
def small_run(orc):
    A = synth.poly_decay(11, 120, 90, 1.5)
    out = orc.pbpqlp(A, 12, 1, seed=3)
    return A, out


def test_output_structure(small_run):
    A, o = small_run
    Q, L, P, R, Pb = o["Q"], o["L"], o["P"], o["R"], o["Pbar"]
    assert np.array_equal(L, np.tril(L)) and np.array_equal(R, np.triu(R))
    assert np.all(np.diag(L) >= 0) and np.all(np.diag(R) >= 0)
    for B in (Q, P, Pb):
        assert np.allclose(B.T @ B, np.eye(B.shape[1]), atol=1e-13)


def test_steps_follow_algorithm(small_run):
    A, o = small_run
    Q, L, P, R, Pb, D, Phi = (o[k] for k in ("Q", "L", "P", "R", "Pbar", "D", "Phi"))
    # Eq. 3 / Eq. 4 with one power iteration, orth after every product
    p0 = _np_orth(A.T @ Phi)
    pm = _np_orth(A @ p0)
    p1 = _np_orth(A.T @ pm)
    assert np.allclose(Pb, p1, atol=1e-11)
    assert np.allclose(D, A @ Pb, atol=1e-13)            # Eq. 5
    assert np.allclose(Q @ R, D, atol=1e-13)             # Eq. 6
    # Eq. 7-8: P = Pbar Ptil with R^T = Ptil Rtil, L = Rtil^T  <=>  R = L Ptil^T
    Ptil = Pb.T @ P
    assert np.allclose(Ptil.T @ Ptil, np.eye(12), atol=1e-13)
    assert np.allclose(L @ Ptil.T, R, atol=1e-13)


def test_closed_forms(small_run):
    A, o = small_run
    Q, L, P, Pb = o["Q"], o["L"], o["P"], o["Pbar"]
    nA = np.linalg.norm(A)
    Ahat = Q @ L @ P.T
    assert np.linalg.norm(Ahat - A @ Pb @ Pb.T) / nA < 1e-13          # QLP^T = A Pbar Pbar^T
    assert np.allclose(L, Q.T @ A @ P, atol=1e-13)                     # L = Q^T A P
    assert abs(np.linalg.norm(A - Ahat) ** 2 - (nA ** 2 - np.linalg.norm(L) ** 2)) < 1e-12 * nA ** 2
    k = 7
    Ak = Q[:, :k] @ L[:k, :k] @ P[:, :k].T
    Q1 = Q[:, :k]
    assert np.linalg.norm(Ak - Q1 @ Q1.T @ A @ Pb @ Pb.T) / nA < 1e-13
    assert abs(np.linalg.norm(A - Ak) ** 2 - (nA ** 2 - np.linalg.norm(L[:k, :k]) ** 2)) < 1e-12 * nA ** 2


@pytest.mark.parametrize("q", [0, 1, 2])
def test_exact_recovery_when_rank_at_most_k(orc, q):
    A = synth.rank_r(21, 200, 150, 8)
    o = orc.pbpqlp(A, 15, q, seed=4)
    for k in (8, 10):
        assert orc.rel_fro_error(A, o["Q"], o["L"], o["P"], k) < 1e-13


def test_full_sampling_gives_exact_singular_values(orc):
    A = synth.poly_decay(5, 40, 30, 1.0)
    o = orc.pbpqlp(A, 30, 0, seed=9)
    assert np.allclose(_sv(o["L"]), _sv(A), rtol=1e-12, atol=1e-15)
    assert orc.rel_fro_error(A, o["Q"], o["L"], o["P"], 30) < 1e-13


def test_rank_one_closed_form(orc):
    rng = np.random.default_rng(2)
    u = rng.standard_normal(50); u /= np.linalg.norm(u)
    v = rng.standard_normal(30); v /= np.linalg.norm(v)
    A = 3.5 * np.outer(u, v)
    o = orc.pbpqlp(A, 4, 1, seed=10)
    assert abs(o["L"][0, 0] - 3.5) < 1e-13
    assert abs(abs(o["Q"][:, 0] @ u) - 1) < 1e-13 and abs(abs(o["P"][:, 0] @ v) - 1) < 1e-13
    assert np.allclose(o["L"][1:, :], 0, atol=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_eckart_young_and_diag_tracks_sigma(orc, seed):
    A = synth.poly_decay(100 + seed, 80, 60, 2.0)
    s = _sv(A)
    k, p = 6, 4
    o = orc.pbpqlp(A, k + p, 2, seed=seed)
    err = np.linalg.norm(A - orc.reconstruct(o["Q"], o["L"], o["P"], k))
    tail = np.linalg.norm(s[k:])
    assert err >= tail * (1 - 1e-12)
    assert err <= 1.5 * tail
    dL = np.abs(np.diag(o["L"]))[:k]
    ratio = dL / s[:k]
    assert np.all(ratio > 0.8) and np.all(ratio < 1.25), ratio
    # L[:j,:j] = Q_j^T A P_j is a compression of A, so |det L[:j,:j]| <= sigma_1...sigma_j
    assert np.all(np.cumprod(dL) <= np.cumprod(s[:k]) * (1 + 1e-12))


@pytest.mark.parametrize("seed,k", [(0, 5), (1, 10), (2, 3), (3, 12)])
def test_rank_revealing_inequalities(orc, seed, k):
    """Theorem 5 (left side), Theorem 6 (Mathias-Stewart) and Theorem 7 (left side)."""
    A = synth.exp_decay(200 + seed, 90, 70, 4.0)
    s = _sv(A)
    ell = 16
    o = orc.pbpqlp(A, ell, 1, seed=seed)
    L, R, D = o["L"], o["R"], o["D"]
    tol = 1 + 1e-12
    assert np.all(_sv(L) <= s[:ell] * tol + 1e-15)
    assert np.all(_sv(D) <= s[:ell] * tol + 1e-15)
    assert _sv(L[:k, :k])[-1] >= _sv(R[:k, :k])[-1] / tol
    assert _sv(L[k:, k:])[0] <= _sv(R[k:, k:])[0] * tol
    assert _sv(L[:k, :k])[-1] <= s[k - 1] * tol


def test_nested_sampling_prefix(orc):
    """Unpivoted QR keeps nested spans: a run with l' < l columns of Phi is the prefix of the l run."""
    A = synth.exp_decay(31, 100, 80, 8.0)
    m, ell, ellp = 100, 16, 10
    phi = orc.gaussian(77, (m, ell))
    big = orc.pbpqlp(A, ell, 1, phi=phi)
    small = orc.pbpqlp(A, ellp, 1, phi=phi[:, :ellp].copy())
    assert np.allclose(small["Pbar"], big["Pbar"][:, :ellp], atol=1e-11)
    assert np.allclose(small["Q"], big["Q"][:, :ellp], atol=1e-11)
    assert np.allclose(small["R"], big["R"][:ellp, :ellp], atol=1e-11)


def test_power_iteration_prefix(orc):
    """The run for q+1 is the run for q followed by one more A / A^T product pair."""
    A = synth.poly_decay(41, 90, 70, 1.2)
    r1 = orc.pbpqlp(A, 9, 1, seed=5)
    r2 = orc.pbpqlp(A, 9, 2, seed=5)
    pm = _np_orth(A @ r1["Pbar"])
    pb = _np_orth(A.T @ pm)
    assert np.allclose(pb, r2["Pbar"], atol=1e-10)


def test_transposed_orientation_is_sketch_of_AAT(orc):
    """Factoring A^T with Phi = Omega (n x l) gives the sketch range of Y = (A A^T)^q A Omega,
    and D = A^T Pbar = B^T with B = Pbar^T A."""
    A = synth.poly_decay(51, 70, 50, 1.0)
    ell, q = 8, 1
    omega = orc.gaussian(12, (50, ell))
    o = orc.pbpqlp(A.T.copy(), ell, q, phi=omega)
    Y = A @ A.T @ A @ omega
    Qy = _np_orth(Y)
    assert np.allclose(o["Pbar"] @ o["Pbar"].T, Qy @ Qy.T, atol=1e-10)
    assert np.allclose(o["D"], (o["Pbar"].T @ A).T, atol=1e-13)


# ------------------------------------------------------- generators + paper
def test_generator_spectra_match_paper_closed_forms(golden):
    s4 = _sv(synth.poly_decay(1, 200, 200, 2.0))
    g4 = golden["matrix4_svd_closed_form"]
    assert abs(s4[9] - g4["sigma_10"]) < 1e-14 and abs(s4[10] - g4["sigma_11"]) < 1e-14
    s3 = _sv(synth.exp_decay(2, 200, 200, 6.0))
    g3 = golden["matrix3_svd_closed_form"]
    assert abs(s3[0] - g3["sigma_1"]) < 1e-14 and abs(s3[1] - g3["sigma_2"]) < 1e-14


@pytest.mark.slow
def test_paper_matrix4_q2_bands(orc, golden):
    """Section V-B, Matrix 4 with q = 2: |L_ii| and spectral errors against the printed curves,
    as ratios to the closed-form optimum (the paper's RNG differs, so medians over seeds)."""
    gL = golden["matrix4_q2_L_values"]
    gE = golden["matrix4_q2_spectral_error"]
    n = gL["n"]
    lv, er = [], []
    for seed in range(3):
        A = synth.poly_decay(1000 + seed, n, n, 2.0)
        o = orc.pbpqlp(A, gL["d"], 2, seed=seed)
        lv.append([abs(o["L"][i - 1, i - 1]) / s for i, s in zip(gL["i"], gL["sigma_i"])])
        row = []
        for d, opt in zip(gE["d"], gE["optimum_sigma_d_plus_1"]):
            od = orc.pbpqlp(A, d, 2, seed=seed)
            E = A - orc.reconstruct(od["Q"], od["L"], od["P"], d)
            row.append(_sv(E)[0] / opt)
        er.append(row)
    lv = np.median(np.array(lv), axis=0)
    er = np.median(np.array(er), axis=0)
    paper_lv = np.array(gL["paper_abs_L_ii"]) / np.array(gL["sigma_i"])
    paper_er = np.array(gE["paper_error"]) / np.array(gE["optimum_sigma_d_plus_1"])
    assert np.all(np.abs(lv - paper_lv) <= np.array([1e-4, 0.1, 0.1])), (lv, paper_lv)
    assert np.all(np.abs(er - paper_er) <= 0.15 * paper_er), (er, paper_er)
    assert np.all(er >= 1 - 1e-9)


@pytest.mark.slow
def test_paper_low_rank_small_gap_q2(orc, golden):
    g = golden["matrix1_smallgap_q2_spectral_error"]
    ratios = []
    for seed in range(3):
        A = synth.low_rank_plus_noise(2000 + seed, g["n"], g["k"], g["mu"])
        o = orc.pbpqlp(A, g["d"], g["q"], seed=seed)
        E = A - orc.reconstruct(o["Q"], o["L"], o["P"], g["d"])
        ratios.append(_sv(E)[0] / _sv(A)[g["d"]])
    paper_ratio = g["paper_error"] / g["paper_svd"]
    assert abs(np.median(ratios) - paper_ratio) < 0.05, (ratios, paper_ratio)


# ------------------------------------------------------- proposer MLP (oracle)
def test_oracle_mlp_gradient_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    p = rng.standard_normal(mlp.PARAMS) * 0.2
    X = rng.standard_normal((7, mlp.IN))
    yq = rng.integers(0, mlp.NQ, 7)
    yp = rng.integers(0, mlp.NP, 7)
    loss, g = mlp.loss_grad(p, X, yq, yp)
    assert mlp.PARAMS == 21768 and g.shape == (mlp.PARAMS,)
    idx = rng.choice(mlp.PARAMS, 40, replace=False)
    for i in idx:
        h = 1e-6
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (mlp.loss_grad(pp, X, yq, yp)[0] - mlp.loss_grad(pm, X, yq, yp)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_oracle_mlp_closed_forms():
    from oracle import mlp
    # GELU(0) = 0, GELU'(0) = 1/2, GELU(x) - GELU(-x) = x
    assert mlp.gelu(np.array([0.0]))[0] == 0.0 and abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    x = np.linspace(-3, 3, 13)
    assert np.allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-14)
    # zero weights: uniform heads, loss = log 5 + log 3 for any labels
    p = np.zeros(mlp.PARAMS)
    loss, _ = mlp.loss_grad(p, np.ones((4, mlp.IN)), [0, 1, 2, 3], [0, 1, 2, 0])
    assert abs(loss - (np.log(5) + np.log(3))) < 1e-12


def test_l11_estimates_two_norm_from_below(orc):
    """Section V-D: |L_11| estimates ||A||_2; it can never exceed it
    (|L_11| <= sigma_1(L) <= sigma_1(A)) and with q = 2 it is within 1e-3."""
    for seed in range(3):
        A = synth.poly_decay(300 + seed, 200, 150, 1.0)
        s1 = _sv(A)[0]
        for q in (0, 1, 2):
            o = orc.pbpqlp(A, 12, q, seed=seed)
            assert abs(o["L"][0, 0]) <= s1 * (1 + 1e-13)
        assert abs(o["L"][0, 0]) >= (1 - 1e-3) * s1
