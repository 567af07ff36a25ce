"""FP64 reference of the (q, p) proposer MLP — TEST INFRASTRUCTURE ONLY.

The exact function the library's BF16 kernels approximate: 32 -> 128 -> 128
-> 8 with GELU(x) = x Phi(x) (erf form), logits 0..4 for q and 5..7 for p,
loss = mean over the batch of the two heads' cross-entropies, AdamW with bias
correction and decoupled weight decay.  Plain numpy in FP64; no rounding to
BF16.  Parameters are the flat vector W1 (128 x 32), b1, W2 (128 x 128), b2,
W3 (8 x 128), b3.
"""
import numpy as np
from scipy.special import erf

IN, HID, NQ, NP = 32, 128, 5, 3
OUT = NQ + NP
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)), ("b3", (OUT,))]
PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(p, X):
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ w["W1"].T + w["b1"]
    h1 = gelu(z1)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = gelu(z2)
    logits = h2 @ w["W3"].T + w["b3"]
    return logits, (X, z1, h1, z2, h2)


def _softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss_grad(p, X, yq, yp):
    """Mean cross-entropy of both heads and its gradient (flat, FP64)."""
    w = unpack(p)
    logits, (X, z1, h1, z2, h2) = forward(p, X)
    B = X.shape[0]
    yq = np.asarray(yq)
    yp = np.asarray(yp)
    pq = _softmax(logits[:, :NQ])
    pp = _softmax(logits[:, NQ:])
    loss = -np.mean(np.log(pq[np.arange(B), yq]) + np.log(pp[np.arange(B), yp]))
    dlog = np.zeros_like(logits)
    dlog[:, :NQ] = pq
    dlog[:, NQ:] = pp
    dlog[np.arange(B), yq] -= 1.0
    dlog[np.arange(B), NQ + yp] -= 1.0
    dlog /= B
    g = {"W3": dlog.T @ h2, "b3": dlog.sum(axis=0)}
    dz2 = (dlog @ w["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ w["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return float(loss), pack(g)


def adamw(p, m, v, g, t, lr, b1, b2, eps, wd):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * ((m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps) + wd * p)
    return p, m, v
