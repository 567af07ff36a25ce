"""The learned (q, p) proposer: BF16 tensor-core MLP kernels against the FP64
oracle MLP, the AdamW step, the feature kernel against its definition, and
training on the GPU."""
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


def _blocks(g):
    from oracle import mlp
    o, out = 0, {}
    for name, shape in mlp.SHAPES:
        nn = int(np.prod(shape))
        out[name] = g[o:o + nn]
        o += nn
    return out


def test_forward_and_gradients_match_oracle(pq):
    import torch
    from oracle import mlp
    from paper_2103_07245_gb300.proposer import Proposer
    prop = Proposer(seed=3)
    rng = np.random.default_rng(1)
    B = 300
    X = rng.standard_normal((B, 32)).astype(np.float32)
    yq = rng.integers(0, 5, B).astype(np.int32)
    yp = rng.integers(0, 3, B).astype(np.int32)
    Xt = torch.from_numpy(X).cuda()
    loss = prop.loss_grad(Xt, torch.from_numpy(yq).cuda(), torch.from_numpy(yp).cuda())
    p = prop.params.cpu().numpy().astype(np.float64)
    ref_loss, ref_g = mlp.loss_grad(p, X.astype(np.float64), yq, yp)
    assert abs(float(loss) - ref_loss) <= 1e-2 * abs(ref_loss)
    g = prop.grad.cpu().numpy().astype(np.float64)
    gb, rb = _blocks(g), _blocks(ref_g)
    for name in rb:
        rel = np.linalg.norm(gb[name] - rb[name]) / np.linalg.norm(rb[name])
        assert rel <= 3e-2, (name, rel)
    logits = prop.logits(Xt).cpu().numpy()
    ref_logits, _ = mlp.forward(p, X.astype(np.float64))
    assert np.max(np.abs(logits - ref_logits)) <= 2e-2 * np.max(np.abs(ref_logits)) + 1e-3


def test_adamw_step_matches_formula(pq):
    import torch
    from oracle import mlp
    rng = np.random.default_rng(2)
    n = pq.pbpqlp_mlp_param_count()
    p0, m0, v0, g = (rng.standard_normal(n).astype(np.float32) for _ in range(4))
    v0 = np.abs(v0)
    tp, tm, tv, tg = (torch.from_numpy(x.copy()).cuda() for x in (p0, m0, v0, g))
    pq.pbpqlp_mlp_adamw(tp, tm, tv, tg, 7, 1e-3, 0.9, 0.999, 1e-8, 1e-2)
    rp, rm, rv = mlp.adamw(p0.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64),
                           g.astype(np.float64), 7, 1e-3, 0.9, 0.999, 1e-8, 1e-2)
    assert np.allclose(tp.cpu().numpy(), rp, rtol=1e-5, atol=1e-6)
    assert np.allclose(tm.cpu().numpy(), rm, rtol=1e-5, atol=1e-6)
    assert np.allclose(tv.cpu().numpy(), rv, rtol=1e-5, atol=1e-6)


def test_features_follow_definition(pq):
    import torch
    from paper_2103_07245_gb300.proposer import features
    k, l, m, n = 20, 40, 1500, 900
    d = np.arange(1, l + 1, dtype=np.float64) ** -2.0
    Lm = np.tril(np.random.default_rng(0).standard_normal((l, l))) * 0.01
    np.fill_diagonal(Lm, d * np.where(np.arange(l) % 2, -1.0, 1.0))    # signs must not matter
    Lt = torch.from_numpy(Lm).cuda()
    F = features([Lt], [l], [k], [m], [n]).cpu().numpy()[0]
    D = lambda j: d[min(max(j, 1), l) - 1]
    assert abs(F[0] - math.log(m) / 8) < 1e-6 and abs(F[1] - math.log(n) / 8) < 1e-6
    assert abs(F[2] - math.log(k) / 4) < 1e-6 and abs(F[3] - 10 * k / min(m, n)) < 1e-6
    assert abs(F[4] - math.log10(D(round(0.1 * k)) / D(1)) / 4) < 1e-6
    assert abs(F[13] - math.log10(D(k) / D(1)) / 4) < 1e-6
    assert abs(F[14] - math.log10(D(k + 1) / D(1)) / 4) < 1e-6
    assert abs(F[20] - math.log10(D(k) / D(k + 1))) < 1e-5
    tail = 0.5 * math.log10(np.sum(d[k:] ** 2) / np.sum(d[:k] ** 2)) / 4
    assert abs(F[25] - tail) < 1e-5
    # slope of log10(j^-2) is -2 / (j ln 10): the fitted slope times k is near -2 k / (j ln 10) averaged
    assert F[26] < 0 and F[27] < 0
    assert F[31] == 1.0


def test_training_on_gpu_fits_a_rule(pq):
    import torch
    from paper_2103_07245_gb300.proposer import Proposer, train
    rng = np.random.default_rng(4)
    X = rng.standard_normal((2048, 32)).astype(np.float32)
    W = rng.standard_normal((32, 2))
    yq = np.digitize(X @ W[:, 0], [-1.0, -0.3, 0.3, 1.0]).astype(np.int32)
    yp = np.digitize(X @ W[:, 1], [-0.5, 0.5]).astype(np.int32)
    prop = Proposer(seed=5)
    hist = train(prop, torch.from_numpy(X).cuda(), yq, yp, epochs=40, batch=256, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0], hist[::10]
    qs, ps = prop.propose(torch.from_numpy(X).cuda())
    acc_q = np.mean(np.array(qs) == yq)
    acc_p = np.mean(np.array([{5: 0, 10: 1, 20: 2}[x] for x in ps]) == yp)
    assert acc_q > 0.8 and acc_p > 0.85, (acc_q, acc_p)


@pytest.mark.slow
def test_trained_proposer_gains_over_fixed_q2_p10(pq):
    """Train on labelled matrices the method generates (one trajectory each),
    then compare the guarded proposal (the sketch's trajectory continued) with
    the plain fixed (q = 2, p = 10) method on held-out 2048 x 2048 matrices
    (k = 64, polynomial or exponential decay): at least the same share meets
    1.5 x the optimal tail, with fewer passes over A and less GPU time."""
    import torch
    from paper_2103_07245_gb300 import proposer as P
    F_all, yq_all, yp_all = [], [], []
    for chunk in range(4):
        As, ks, tails = P.make_matrices(100 + chunk, 96, m_range=(512, 2048))
        F, err, yq, yp = P.label(As, ks, tails, seed=chunk)
        F_all.append(F)
        yq_all.append(yq)
        yp_all.append(yp)
        del As
    F = torch.cat(F_all)
    prop = P.Proposer(seed=1)
    hist = P.train(prop, F, np.concatenate(yq_all), np.concatenate(yp_all), epochs=200, batch=128, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    As, ks, tails = P.make_matrices(999, 32, fixed=(2048, 2048, 64), eval_mix=True)
    res = P.evaluate(prop, As, ks, tails)
    res.pop("proposals")
    print(res)
    assert res["proposer_success"] >= res["fixed_success"], res
    assert res["proposer_passes"] < res["fixed_passes"], res
    assert res["proposer_ms"] < res["fixed_ms"], res
