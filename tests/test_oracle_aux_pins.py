"""Pins for the oracle's two auxiliary functions, against closed forms.

- ``oracle.mlp.adamw``: AdamW as Loshchilov & Hutter define it ("Decoupled
  Weight Decay Regularization", ICLR 2019, Algorithm 2): bias-corrected first
  and second moments, and a weight decay applied to the parameters directly,
  not added to the gradient.  The pins use the facts that fix it:
    * at t = 1 the bias-corrected moments are g and g^2 for any beta1, beta2,
      so the step is lr * (g / (|g| + eps) + wd * p);
    * under a constant gradient the corrected moments stay g and g^2 at
      every t, so seven steps follow a geometric closed form;
    * a zero gradient with wd > 0 shrinks p by exactly (1 - lr wd)
      (L2 decay folded into the gradient would move p by about lr sign(p));
    * with beta1 = 0 the step is g_t / (sqrt(vhat_t) + eps), where vhat_t is
      the normalised exponentially weighted mean of the squared gradients.
- ``oracle.probe_error_estimate``: with the identity as probes (W = I_n) the
  ratio of the probe sums is exactly ||A - A_r||_F^2 / ||A||_F^2, for any
  orthogonal W as well; it is 0 when A has rank r and the factors recover it.

The check functions take the module under test, so that the mutation tests
can run them against copies of the oracle with one planted mistake.  A last
pin fixes the rotation invariance that lets the proposer train on A = Sigma.
"""
import numpy as np


def check_adamw(mlp):
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    p0 = np.array([0.5, -1.25, 2.0])
    g = np.array([0.3, -0.02, 4.0])
    z = np.zeros(3)
    # t = 1, wd = 0: the move is lr * g / (|g| + eps), whatever beta1, beta2
    for bb1, bb2 in ((0.9, 0.999), (0.5, 0.9), (0.0, 0.99)):
        p1, m1, v1 = mlp.adamw(p0, z, z, g, 1, lr, bb1, bb2, eps, 0.0)
        assert np.allclose(p1, p0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15), (bb1, bb2, p1)
        assert np.allclose(m1, (1 - bb1) * g, rtol=1e-15, atol=0)
        assert np.allclose(v1, (1 - bb2) * g * g, rtol=1e-15, atol=0)
    # t = 1, wd > 0: decoupled decay adds lr * wd * p to the move
    wd = 0.1
    p1, _, _ = mlp.adamw(p0, z, z, g, 1, lr, b1, b2, eps, wd)
    assert np.allclose(p1, p0 - lr * (g / (np.abs(g) + eps) + wd * p0), rtol=0, atol=1e-15), p1
    # zero gradient: p shrinks by exactly (1 - lr wd); coupled L2 decay would not
    p1, _, _ = mlp.adamw(p0, z, z, z, 1, lr, b1, b2, eps, wd)
    assert np.allclose(p1, p0 * (1 - lr * wd), rtol=1e-15, atol=0), p1
    # a constant gradient for seven steps: corrected moments stay g and g^2,
    # so p_t = (1 - lr wd) p_{t-1} - lr s with s = g / (|g| + eps)
    p, m, v = p0.copy(), z.copy(), z.copy()
    for t in range(1, 8):
        p, m, v = mlp.adamw(p, m, v, g, t, lr, b1, b2, eps, wd)
    c = 1.0 - lr * wd
    s = g / (np.abs(g) + eps)
    closed = c ** 7 * p0 - lr * s * sum(c ** j for j in range(7))
    assert np.allclose(p, closed, rtol=1e-13, atol=1e-15), (p, closed)
    assert np.allclose(m, (1 - b1 ** 7) * g, rtol=1e-13, atol=0)
    assert np.allclose(v, (1 - b2 ** 7) * g * g, rtol=1e-13, atol=0)
    # beta1 = 0, changing gradients, wd = 0: the step is g_t / (sqrt(vhat_t) + eps)
    # with vhat_t = sum_j b2^(t-j) g_j^2 / sum_j b2^(t-j)
    gs = [np.array([0.3, -0.02, 4.0]), np.array([-1.0, 0.5, 0.25]), np.array([0.05, 0.05, -2.0]),
          np.array([2.0, -3.0, 1.0]), np.array([0.7, 0.1, -0.4]), np.array([-0.2, 0.9, 3.0]),
          np.array([1.5, -0.6, 0.02])]
    p, m, v = p0.copy(), z.copy(), z.copy()
    expect = p0.copy()
    for t, gt in enumerate(gs, start=1):
        p, m, v = mlp.adamw(p, m, v, gt, t, lr, 0.0, b2, eps, 0.0)
        w = np.array([b2 ** (t - j) for j in range(1, t + 1)])
        vhat = sum(wj * gj * gj for wj, gj in zip(w, gs[:t])) / w.sum()
        expect = expect - lr * gt / (np.sqrt(vhat) + eps)
    assert np.allclose(p, expect, rtol=1e-13, atol=1e-15), (p, expect)


def check_probe_estimate(orc):
    rng = np.random.default_rng(3)
    m, n, ell, r = 60, 40, 12, 8
    U = np.linalg.qr(rng.standard_normal((m, n)))[0]
    V = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = (U * (0.7 ** np.arange(n))) @ V.T
    o = orc.pbpqlp(A, ell, 1, seed=4)
    Q, L, P = o["Q"], o["L"], o["P"]
    exact = np.linalg.norm(A - Q[:, :r] @ L[:r, :r] @ P[:, :r].T) / np.linalg.norm(A)
    # W = I_n and W orthogonal: the estimate is the exact ratio
    for W in (np.eye(n), np.linalg.qr(rng.standard_normal((n, n)))[0]):
        est = orc.probe_error_estimate(A, Q, L, P, r, W)
        assert abs(est - exact) <= 1e-12 * exact, (est, exact)
    # exact recovery: rank(A) = r <= ell gives 0 for any probes
    B = (U[:, :r] * (2.0 ** -np.arange(r))) @ V[:, :r].T
    ob = orc.pbpqlp(B, ell, 1, seed=5)
    est = orc.probe_error_estimate(B, ob["Q"], ob["L"], ob["P"], r, rng.standard_normal((n, 16)))
    assert est <= 1e-13, est


def test_adamw_against_closed_forms():
    from oracle import mlp
    check_adamw(mlp)


def test_probe_estimate_against_closed_forms(orc):
    check_probe_estimate(orc)


def test_factorization_depends_on_the_spectrum_only(orc):
    """The reading behind the proposer's diagonal training matrices: for
    A = U Sigma V^T and any Phi, Algorithm 3 on (A, Phi) and on (Sigma, U^T Phi)
    give the same L and the same errors (every orth is a thin QR, and
    qr(W X) = W qr(X) for orthogonal W), and U^T Phi is Gaussian when Phi is."""
    rng = np.random.default_rng(11)
    m, n, ell, k = 70, 50, 12, 8
    U = np.linalg.qr(rng.standard_normal((m, m)))[0]
    V = np.linalg.qr(rng.standard_normal((n, n)))[0]
    sig = 0.8 ** np.arange(n)
    S = np.zeros((m, n))
    S[np.arange(n), np.arange(n)] = sig
    A = U @ S @ V.T
    phi = rng.standard_normal((m, ell))
    for q in (0, 1, 2):
        a = orc.pbpqlp(A, ell, q, phi=phi)
        b = orc.pbpqlp(S, ell, q, phi=U.T @ phi)
        assert np.allclose(a["L"], b["L"], rtol=0, atol=1e-12 * sig[0]), q
        ea = orc.rel_fro_error(A, a["Q"], a["L"], a["P"], k)
        eb = orc.rel_fro_error(S, b["Q"], b["L"], b["P"], k)
        assert abs(ea - eb) <= 1e-12, (q, ea, eb)
