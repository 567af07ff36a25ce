"""Checkpoint and resume of the learned part, on CPU: label shards make an
interrupted label run resume where it stopped, and a training run resumed
from its checkpoint reaches exactly the state of an uninterrupted one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2103_07245_gb300 import proposer as P   # noqa: E402


def test_label_shards_resume(tmp_path):
    calls = []

    def make_chunk(c):
        calls.append(c)
        rng = np.random.default_rng(c)
        return torch.from_numpy(rng.standard_normal((5, 32)).astype(np.float32)), rng.integers(0, 5, 5), \
            rng.integers(0, 3, 5)

    d = str(tmp_path / "shards")
    first = P.labelled_chunks(4, make_chunk, d)
    assert calls == [0, 1, 2, 3]
    calls.clear()
    again = P.labelled_chunks(4, make_chunk, d)
    assert calls == []
    (tmp_path / "shards" / "chunk_00002.npz").unlink()     # the run that was interrupted
    resumed = P.labelled_chunks(4, make_chunk, d)
    assert calls == [2]
    for a, b, c in zip(first, again, resumed):
        for x, y, z in zip(a, b, c):
            assert np.array_equal(x, y) and np.array_equal(x, z)


class _FakeProp:
    """The Proposer's step / save / load interface with a deterministic CPU update."""

    def __init__(self):
        self.params = torch.zeros(6, dtype=torch.float64)
        self.m = torch.zeros(6, dtype=torch.float64)
        self.v = torch.zeros(6, dtype=torch.float64)
        self.t = 0

    def step(self, X, yq, yp, lr):
        self.t += 1
        g = X.double().mean(0)[:6] * (1.0 + yq.double().mean()) - 0.1 * self.params
        self.m = 0.9 * self.m + g
        self.params = self.params + lr * self.m
        return torch.tensor(float((self.params ** 2).sum()) + float(yp.double().mean()))

    def save(self, path):
        np.savez(path, params=self.params.numpy(), m=self.m.numpy(), v=self.v.numpy(), t=self.t)

    def load(self, path):
        d = np.load(path)
        self.params = torch.from_numpy(d["params"]).clone()
        self.m = torch.from_numpy(d["m"]).clone()
        self.v = torch.from_numpy(d["v"]).clone()
        self.t = int(d["t"])


def test_training_resumes_from_checkpoint_exactly(tmp_path):
    rng = np.random.default_rng(0)
    F = torch.from_numpy(rng.standard_normal((64, 32)).astype(np.float32))
    yq = rng.integers(0, 5, 64)
    yp = rng.integers(0, 3, 64)
    straight = _FakeProp()
    h_straight = P.train(straight, F, yq, yp, epochs=7, batch=16, lr=0.05, seed=3)
    ck = str(tmp_path / "ckpt.npz")
    part = _FakeProp()
    P.train(part, F, yq, yp, epochs=4, batch=16, lr=0.05, seed=3, ckpt=ck, ckpt_every=2)   # stopped after 4
    resumed = _FakeProp()
    h_resumed = P.train(resumed, F, yq, yp, epochs=7, batch=16, lr=0.05, seed=3, ckpt=ck, ckpt_every=2)
    assert np.array_equal(resumed.params.numpy(), straight.params.numpy())
    assert resumed.t == straight.t
    assert h_resumed == h_straight
