"""Learned (q, p) proposer for PbP-QLP: data, training and the guarded proposal.

Every numerical step runs in the library's kernels (factorizations, feature
extraction, MLP forward / backward / AdamW, the a-posteriori estimator); this
module only moves torch tensors between those calls.

- Labels come from the method itself, one trajectory per training matrix:
  the (q = 0, p = 20) sketch's basis is iterated to q = 4 with
  pbpqlp_factor_from, and every (q, p), q in {0..4}, p in {5, 10, 20},
  projects the first k + p columns of the q-th basis (the thin-QR prefix
  property makes that the (q, p) run with the sketch's Phi prefix).  The
  label is the cheapest pair whose relative Frobenius error is <= 1.5 x the
  optimal tail ||sigma_{k+1:}|| / ||A||_F (with a 10% margin).  Cost is what
  the guarded proposal pays after its sketch: nothing for (0, 20) itself,
  else (2q + 1)(k + p), passes over A times panel width.  Errors through the
  identity ||A - A_k||^2 = ||A||^2 - ||L_k||^2 of Eq. 8 (pbpqlp_error).
- Features: pbpqlp_features on the L-values of the (q = 0, p = 20) sketch.
- Guarded proposal: the sketch's trajectory is continued to the proposed
  (q, p) from the first k + p columns of its basis, the result's error is
  taken a posteriori (pbpqlp_error: the identity of Eq. 8 by default, or
  Gaussian probes) and, when it misses the caller's tolerance, the plain
  method with fixed (q = 2, p = 10) is run instead.
"""
import math
import os

import numpy as np

import paper_2103_07245_gb300 as pq

Q_CHOICES = (0, 1, 2, 3, 4)
P_CHOICES = (5, 10, 20)
FIXED = (2, 10)


class Proposer:
    """The MLP's parameters and AdamW state on the device."""

    def __init__(self, seed=0, device="cuda"):
        import torch
        self.device = device
        self.n = pq.pbpqlp_mlp_param_count()
        self.params = torch.empty(self.n, dtype=torch.float32, device=device)
        pq.pbpqlp_mlp_init(self.params, seed)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.t = 0
        self._ws = {}

    def _workspace(self, batch):
        import torch
        if batch not in self._ws:
            nb = pq.pbpqlp_mlp_workspace_bytes(batch)
            self._ws[batch] = (torch.empty(nb, dtype=torch.uint8, device=self.device), nb)
        return self._ws[batch]

    def loss_grad(self, X, yq, yp):
        import torch
        ws, nb = self._workspace(X.shape[0])
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        pq.pbpqlp_mlp_loss_grad(self.params, X, yq, yp, X.shape[0], self.grad, loss, ws, nb)
        return loss

    def step(self, X, yq, yp, lr=2e-3, weight_decay=1e-4):
        loss = self.loss_grad(X, yq, yp)
        self.t += 1
        pq.pbpqlp_mlp_adamw(self.params, self.m, self.v, self.grad, self.t, lr, 0.9, 0.999, 1e-8, weight_decay)
        return loss

    def logits(self, X):
        import torch
        ws, nb = self._workspace(X.shape[0])
        out = torch.empty(X.shape[0], 8, dtype=torch.float32, device=self.device)
        pq.pbpqlp_mlp_forward(self.params, X, X.shape[0], out, ws, nb)
        return out

    def propose(self, X):
        """(q, p) per row of the feature matrix X (count x 32, FP32 device)."""
        import torch
        ws, nb = self._workspace(X.shape[0])
        qi = torch.empty(X.shape[0], dtype=torch.int32, device=self.device)
        pi = torch.empty_like(qi)
        pq.pbpqlp_propose(X, X.shape[0], self.params, qi, pi, ws, nb)
        qs = [Q_CHOICES[int(x)] for x in qi.cpu()]
        ps = [P_CHOICES[int(x)] for x in pi.cpu()]
        return qs, ps

    def save(self, path):
        np.savez(path, params=self.params.cpu().numpy(), m=self.m.cpu().numpy(), v=self.v.cpu().numpy(), t=self.t)

    def load(self, path):
        import torch
        d = np.load(path)
        self.params.copy_(torch.from_numpy(d["params"]))
        self.m.copy_(torch.from_numpy(d["m"]))
        self.v.copy_(torch.from_numpy(d["v"]))
        self.t = int(d["t"])


def features(Ls, ls, ks, ms, ns, device="cuda"):
    import torch
    cnt = len(Ls)
    F = torch.empty(cnt, 32, dtype=torch.float32, device=device)
    nb = pq.pbpqlp_features_workspace_bytes(cnt)
    ws = torch.empty(nb, dtype=torch.uint8, device=device)
    pq.pbpqlp_features(Ls, ls, ks, ms, ns, F, ws, nb)
    return F


MARGIN = 1.1   # labels and the estimator check keep 10% below the tolerance
P_SKETCH = 20  # oversampling of the q = 0 sketch the features come from


def sketch(A, k, seed):
    """The (q = 0, p = 20) sketch: its factors and its basis Pbar (n x (k + 20)),
    the start of every trajectory below (2 passes over A)."""
    plan = pq.Plan(A.shape[0], A.shape[1], k, P_SKETCH, 0, seed)
    Qa, L, Qb, Pbar = plan.factor_from(A, pbar_out=True)
    return plan, (Qa, L, Qb), Pbar


def trajectory_errors(A, k, seed):
    """Rank-k relative errors err[q][p] for q in Q_CHOICES, p in P_CHOICES from
    ONE trajectory: the sketch's basis is iterated to q = 4 (two passes per
    iteration), and (q, p) projects the first k + p columns of the q-th basis
    (one pass each).  By the thin-QR prefix property this is, up to rounding,
    the (q, p) run with the first k + p columns of the sketch's Phi.  Errors
    through the identity of Eq. 8 (pbpqlp_error, PBPQLP_ERR_IDENTITY).
    Returns (err, L of the sketch, passes over A)."""
    m, n = A.shape
    plan0, (Qa, L0, Qb), P0 = sketch(A, k, seed)
    err = np.zeros((len(Q_CHOICES), len(P_CHOICES)))
    err[0, P_CHOICES.index(P_SKETCH)] = plan0.error(A, Qa, L0, Qb, k, method=pq.PBPQLP_ERR_IDENTITY)
    step = pq.Plan(m, n, k, P_SKETCH, 1, seed)
    bases = [P0]
    for _ in Q_CHOICES[1:]:
        bases.append(step.factor_from(A, pbar0=bases[-1], iterations_only=True)[3])
    proj = {p: (plan0 if p == P_SKETCH else pq.Plan(m, n, k, p, 0, seed)) for p in P_CHOICES}
    passes = 2 + 2 * (len(Q_CHOICES) - 1)
    for qi in range(len(Q_CHOICES)):
        for pi, p in enumerate(P_CHOICES):
            if qi == 0 and p == P_SKETCH:
                continue
            plan = proj[p]
            Qa, L, Qb, _ = plan.factor_from(A, pbar0=bases[qi][:, :k + p])
            err[qi, pi] = plan.error(A, Qa, L, Qb, k, method=pq.PBPQLP_ERR_IDENTITY)
            passes += 1
    return err, L0, passes


def label(As, ks, tails, seed=0, workers=1):
    """Features of the (0, 20) sketch, the error table err[i][q][p] (one
    trajectory per matrix) and the labels: the cheapest pair with error <=
    1.5 x tail / MARGIN.  Cost is what the guarded proposal pays after its
    sketch: nothing for (0, 20) itself, else (2q + 1)(k + p) (the continued
    trajectory: q iterations and the projection, times the panel width)."""
    import torch
    cnt = len(As)
    err = np.zeros((cnt, len(Q_CHOICES), len(P_CHOICES)))
    Ls = [None] * cnt
    if workers <= 1:
        for i, (A, k) in enumerate(zip(As, ks)):
            err[i], Ls[i], _ = trajectory_errors(A, k, seed + i)
    else:
        # one CUDA stream per worker thread: the trajectories are independent and
        # latency-bound, so several run at once (the library calls release the GIL)
        import concurrent.futures as cf
        torch.cuda.synchronize()
        streams = [torch.cuda.Stream() for _ in range(workers)]

        def run(wid):
            with torch.cuda.stream(streams[wid]):
                for i in range(wid, cnt, workers):
                    err[i], Ls[i], _ = trajectory_errors(As[i], ks[i], seed + i)
            streams[wid].synchronize()

        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(run, range(workers)))
        torch.cuda.synchronize()
    F = features(Ls, [k + P_SKETCH for k in ks], ks, [a.shape[0] for a in As], [a.shape[1] for a in As])
    yq, yp = [], []
    for i, k in enumerate(ks):
        best, bc = None, None
        for qi, q in enumerate(Q_CHOICES):
            for pi, p in enumerate(P_CHOICES):
                if err[i, qi, pi] <= 1.5 * tails[i] / MARGIN:
                    c = 0 if (q, p) == (0, P_SKETCH) else (2 * q + 1) * (k + p)
                    if bc is None or c < bc:
                        best, bc = (qi, pi), c
        if best is None:
            best = (len(Q_CHOICES) - 1, len(P_CHOICES) - 1)
        yq.append(best[0])
        yp.append(best[1])
    return F, err, np.array(yq), np.array(yp)


def random_family(rng, m, n):
    """Spectrum of a training / evaluation matrix: polynomial, exponential or low rank plus noise."""
    r = min(m, n)
    i = np.arange(1, r + 1, dtype=np.float64)
    fam = rng.integers(0, 3)
    if fam == 0:
        return i ** (-rng.uniform(0.5, 3.0))
    if fam == 1:
        return np.exp(-i * rng.uniform(1 / 80, 1 / 10))
    rank = int(rng.integers(8, 96))
    mu = 10 ** rng.uniform(-4, -1)
    s = np.full(r, mu)
    s[:rank] = np.linspace(1.0, 0.5, rank)
    return s


def make_matrices(seed, count, m_range=(512, 2048), k_range=(8, 64), fixed=None, eval_mix=False, device="cuda",
                  diagonal=False):
    """Seeded matrices, their k and their optimal relative tails ||sigma_{k+1:}|| / ||sigma||.

    With diagonal, A = Sigma (m x n, the singular values on the diagonal) instead
    of U Sigma V^T with Haar U, V.  For a Gaussian Phi the factorization's
    output distribution depends on Sigma only (U^T Phi is again Gaussian, and
    V^T is undone by the basis), so the errors, the L-values and hence the
    features and labels have the same distribution at no generation cost;
    the held-out evaluation keeps Haar factors."""
    import torch
    import synth
    rng = np.random.default_rng(seed)
    As, ks, tails = [], [], []
    for j in range(count):
        if fixed:
            m, n, k = fixed
        else:
            m = int(rng.integers(m_range[0], m_range[1] + 1))
            n = int(rng.integers(m_range[0], m_range[1] + 1))
            k = int(rng.integers(k_range[0], k_range[1] + 1))
        if eval_mix or rng.random() < 0.5:
            i = np.arange(1, min(m, n) + 1, dtype=np.float64)
            sig = i ** (-rng.uniform(0.5, 3.0)) if rng.random() < 0.5 else np.exp(-i * rng.uniform(1 / 80, 1 / 10))
        else:
            sig = random_family(rng, m, n)
        sseed = int(rng.integers(1 << 30))
        if diagonal:
            A = torch.zeros(m, n, dtype=torch.float64, device=device)
            r = min(m, n)
            A[torch.arange(r, device=device), torch.arange(r, device=device)] = torch.as_tensor(sig[:r], device=device)
            As.append(A)
        else:
            As.append(synth.torch_svd_matrix_device(sseed, m, n, sig, device=device))
        ks.append(k)
        tails.append(float(np.linalg.norm(sig[k:]) / np.linalg.norm(sig)))
    return As, ks, tails


def labelled_chunks(chunks, make_chunk, shard_dir=None):
    """Features and labels of `chunks` chunks, make_chunk(c) -> (F, yq, yp).

    With shard_dir, chunk c is kept in shard_dir/chunk_<c>.npz once made and
    read back instead of being made again, so an interrupted label run
    resumes where it stopped (a shard is written whole through a temporary
    file, never half).  Returns lists of numpy arrays."""
    F_all, yq_all, yp_all = [], [], []
    for c in range(chunks):
        path = os.path.join(shard_dir, "chunk_%05d.npz" % c) if shard_dir else None
        if path and os.path.exists(path):
            d = np.load(path)
            F, yq, yp = d["F"], d["yq"], d["yp"]
        else:
            F, yq, yp = make_chunk(c)
            F = F.cpu().numpy() if hasattr(F, "cpu") else np.asarray(F)
            yq, yp = np.asarray(yq), np.asarray(yp)
            if path:
                os.makedirs(shard_dir, exist_ok=True)
                tmp = path + ".tmp.npz"
                np.savez(tmp, F=F, yq=yq, yp=yp)
                os.replace(tmp, path)
        F_all.append(F)
        yq_all.append(yq)
        yp_all.append(yp)
    return F_all, yq_all, yp_all


def train(prop, F, yq, yp, epochs=300, batch=256, lr=2e-3, seed=0, ckpt=None, ckpt_every=0):
    """Minibatch AdamW on the labelled features; returns the loss history.

    With ckpt (a path) the weights, AdamW state, epoch and loss history are
    saved every ckpt_every epochs and at the end; a run started with an
    existing checkpoint continues from it and reaches exactly the weights of
    an uninterrupted run (the epoch permutations of the skipped epochs are
    drawn and discarded)."""
    import torch
    rng = np.random.default_rng(seed)
    n = F.shape[0]
    yq_t = torch.as_tensor(yq, dtype=torch.int32, device=F.device)
    yp_t = torch.as_tensor(yp, dtype=torch.int32, device=F.device)
    hist, start = [], 0
    if ckpt and os.path.exists(ckpt):
        prop.load(ckpt)
        d = np.load(ckpt)
        start = int(d["epoch"])
        hist = [float(x) for x in d["hist"]]
        for _ in range(start):
            rng.permutation(n)

    def save(ep):
        tmp = ckpt + ".tmp.npz"
        prop.save(tmp)
        d = dict(np.load(tmp))
        np.savez(tmp, epoch=ep, hist=np.asarray(hist, dtype=np.float64), **d)
        os.replace(tmp, ckpt)

    for ep in range(start, epochs):
        perm = torch.as_tensor(rng.permutation(n), device=F.device)
        tot = 0.0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            loss = prop.step(F[idx].contiguous(), yq_t[idx].contiguous(), yp_t[idx].contiguous(), lr=lr)
            tot += float(loss)
        hist.append(tot / max(1, n // batch))
        if ckpt and ckpt_every and (ep + 1) % ckpt_every == 0:
            save(ep + 1)
    if ckpt:
        save(epochs)
    return hist


def evaluate(prop, As, ks, tails, seed=0, nprobes=24, guard="identity"):
    """Fixed (2, 10) against the guarded proposal on the same matrices, with
    GPU time (CUDA events on the current stream) and passes over A.

    Guarded proposal per matrix: the (0, 20) sketch with its basis (2 passes),
    the network's (q, p) from the sketch's features (one batched launch for
    all matrices, its time shared out), the sketch's trajectory continued from
    the first k + p columns of its basis (2q + 1 passes; none when the
    proposal is (0, 20) itself), the a-posteriori error of the result (1
    pass: with guard "identity" the exact sqrt(||A||^2 - ||L_k||^2) / ||A||
    of Eq. 8, which reads A once for ||A||_F; with guard "probes" the
    Gaussian-probe estimate), and fixed (2, 10) (6 passes) when it misses the
    caller's tolerance (1.5 x the optimal tail) / MARGIN."""
    import torch

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        return out, (e0, e1)

    cnt = len(As)
    t_fixed, e_fixed = [], []
    for i, (A, k) in enumerate(zip(As, ks)):
        plan = pq.Plan(A.shape[0], A.shape[1], k, FIXED[1], FIXED[0], seed + i)   # host set-up, not timed
        (Qa, L, Qb), ev = timed(lambda: plan.factor(A))
        t_fixed.append(ev)
        e_fixed.append(plan.error(A, Qa, L, Qb, k, method=pq.PBPQLP_ERR_IDENTITY))
        del plan
    sk, t_sketch = [], []
    for i, (A, k) in enumerate(zip(As, ks)):
        plan0 = pq.Plan(A.shape[0], A.shape[1], k, P_SKETCH, 0, seed + i)
        out, ev = timed(lambda: plan0.factor_from(A, pbar_out=True))
        sk.append((plan0, out[:3], out[3]))
        t_sketch.append(ev)
    (F, (qs, ps)), ev_prop = timed(lambda: (lambda F: (F, prop.propose(F)))(
        features([o[1][1] for o in sk], [k + P_SKETCH for k in ks], ks, [a.shape[0] for a in As],
                 [a.shape[1] for a in As])))
    e_prop, passes, fallback, t_rest = [], [], [], []
    for i, (A, k) in enumerate(zip(As, ks)):
        q, p = qs[i], ps[i]
        plan0, (Qa0, L0, Qb0), P0 = sk[i]
        # host set-up of the plans this matrix may use, outside the timed region
        cont = None if (q, p) == (0, P_SKETCH) else pq.Plan(A.shape[0], A.shape[1], k, p, q, seed + i)
        fixed = pq.Plan(A.shape[0], A.shape[1], k, FIXED[1], FIXED[0], seed + i)
        fixed_out = fixed.outputs()

        def run(i=i, A=A, k=k, q=q, p=p, plan0=plan0, Qa0=Qa0, L0=L0, Qb0=Qb0, P0=P0, cont=cont, fixed=fixed,
                fixed_out=fixed_out):
            if cont is None:
                plan, Qa, L, Qb = plan0, Qa0, L0, Qb0
            else:
                plan = cont
                Qa, L, Qb, _ = plan.factor_from(A, pbar0=P0[:, :k + p])
            if guard == "probes":
                est = plan.error(A, Qa, L, Qb, k, method=pq.PBPQLP_ERR_PROBES, nprobes=nprobes, probe_seed=99 + i)
            else:
                est = plan.error(A, Qa, L, Qb, k, method=pq.PBPQLP_ERR_IDENTITY)
            fb = est > 1.5 * tails[i] / MARGIN
            if fb:
                plan = fixed
                Qa, L, Qb = plan.factor(A, out=fixed_out)
            return plan, Qa, L, Qb, fb

        (plan, Qa, L, Qb, fb), ev = timed(run)
        t_rest.append(ev)
        e = plan.error(A, Qa, L, Qb, k, method=pq.PBPQLP_ERR_IDENTITY)   # bookkeeping, after the timed region
        n_pass = 2 + (0 if (q, p) == (0, P_SKETCH) else 2 * q + 1) + 1 + (2 * FIXED[0] + 2 if fb else 0)
        e_prop.append(e)
        passes.append(n_pass)
        fallback.append(fb)
    torch.cuda.synchronize()
    ms = lambda ev: ev[0].elapsed_time(ev[1])
    ms_fixed = np.array([ms(ev) for ev in t_fixed])
    ms_prop = np.array([ms(a) + ms(b) for a, b in zip(t_sketch, t_rest)]) + ms(ev_prop) / cnt
    ok_fixed = np.array(e_fixed) <= 1.5 * np.array(tails)
    ok_prop = np.array(e_prop) <= 1.5 * np.array(tails)
    return {"fixed_success": float(ok_fixed.mean()), "proposer_success": float(ok_prop.mean()),
            "fixed_passes": float(2 * FIXED[0] + 2), "proposer_passes": float(np.mean(passes)),
            "fixed_ms": float(ms_fixed.mean()), "proposer_ms": float(ms_prop.mean()),
            "sketch_ms": float(np.mean([ms(ev) for ev in t_sketch])), "propose_ms": ms(ev_prop) / cnt,
            "continue_ms": float(np.mean([ms(ev) for ev in t_rest])),
            "time_saved": float(1.0 - ms_prop.mean() / ms_fixed.mean()),
            "fallback_rate": float(np.mean(fallback)), "proposals": list(zip(qs, ps))}


def main(argv=None):
    """Generate labelled matrices, train on the GPU, evaluate against fixed (2, 10).

    python -m paper_2103_07245_gb300.proposer --chunks 16 --chunk 128 --eval 128 \
        --save weights.npz --json summary.json
    """
    import argparse
    import json
    import time
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--chunks", type=int, default=8)
    ap.add_argument("--chunk", type=int, default=96)
    ap.add_argument("--max-dim", type=int, default=2048)
    ap.add_argument("--eval", type=int, default=64)
    ap.add_argument("--eval-chunk", type=int, default=128)
    ap.add_argument("--workers", type=int, default=1, help="concurrent label trajectories (one stream each)")
    ap.add_argument("--diagonal", action="store_true",
                    help="training matrices A = Sigma (same label distribution as Haar U Sigma V^T)")
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--save", default=None)
    ap.add_argument("--json", default=None)
    ap.add_argument("--shards", default=None, help="directory of label shards (resumable label generation)")
    ap.add_argument("--ckpt", default=None, help="training checkpoint (resumable training)")
    ap.add_argument("--ckpt-every", type=int, default=20)
    args = ap.parse_args(argv)
    pq.load(build_if_missing=True)
    t0 = time.time()

    def make_chunk(c):
        As, ks, tails = make_matrices(1000 * args.seed + c, args.chunk, m_range=(512, args.max_dim),
                                      diagonal=args.diagonal)
        F, err, yq, yp = label(As, ks, tails, seed=c, workers=args.workers)
        return F, yq, yp

    F_all, yq_all, yp_all = labelled_chunks(args.chunks, make_chunk, args.shards)
    t_label = time.time() - t0
    F = torch.from_numpy(np.concatenate(F_all)).to("cuda")
    yq = np.concatenate(yq_all)
    yp = np.concatenate(yp_all)
    prop = Proposer(seed=args.seed + 1)
    hist = train(prop, F, yq, yp, epochs=args.epochs, batch=128, lr=2e-3, seed=args.seed, ckpt=args.ckpt,
                 ckpt_every=args.ckpt_every)
    t_train = time.time() - t0 - t_label
    if args.save:
        prop.save(args.save)
    # held-out 2048 x 2048 matrices, k = 64, evaluated in chunks (each chunk's matrices held at once)
    parts, props = [], []
    for c0 in range(0, args.eval, args.eval_chunk):
        cnt = min(args.eval_chunk, args.eval - c0)
        As, ks, tails = make_matrices(999_000 + 7919 * args.seed + c0, cnt, fixed=(2048, 2048, 64), eval_mix=True)
        r = evaluate(prop, As, ks, tails, seed=c0)
        props += r.pop("proposals")
        parts.append((cnt, r))
        del As
    tot = sum(c for c, _ in parts)
    res = {key: sum(c * r[key] for c, r in parts) / tot for key in parts[0][1] if key != "time_saved"}
    res["time_saved"] = 1.0 - res["proposer_ms"] / res["fixed_ms"]
    res.update({"train_matrices": int(F.shape[0]), "eval_matrices": args.eval, "loss_first": hist[0],
                "loss_last": hist[-1], "label_q_hist": np.bincount(yq, minlength=5).tolist(),
                "label_p_hist": np.bincount(yp, minlength=3).tolist(),
                "proposed_q_hist": np.bincount([q for q, _ in props], minlength=5).tolist(),
                "seconds_label": t_label, "seconds_train": t_train, "seconds_total": time.time() - t0})
    out = json.dumps(res)
    print(out, flush=True)
    if args.json:
        with open(args.json, "w") as f:
            f.write(out + "\n")
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
