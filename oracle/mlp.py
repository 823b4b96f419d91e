"""CPU reference of the threshold-predicting MLP -- TEST INFRASTRUCTURE ONLY.

Not part of the paper: the learned filter predicts a query's k-th-nearest
distance so the scan can keep only records at or under it (an exact fallback
covers wrong predictions).  Architecture and numerics, written plainly in
float64 NumPy:

  x  = [166 query bits, popc(q) / 166]              (167 features)
  h1 = relu(W1 x + b1)      W1: 256 x 167
  h2 = relu(W2 h1 + b2)     W2: 256 x 256
  y  = w3 . h2 + b3         w3: 256

BF16 weights: every matrix/vector product uses bf16-rounded weights and
bf16-rounded layer inputs (x, h1, h2); sums are exact here (float64) and FP32
on the GPU.  Loss: pinball (quantile) loss, mean over the batch,
  L = mean(max(q (t - y), (q - 1)(t - y))).
Optimizer: Adam with bias correction on float32 master parameters.

Only tests, the smoke check and the benchmark's CPU legs may use this module.
"""
from __future__ import annotations

import numpy as np

IN, H = 167, 256
SHAPES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(flat):
    out, i = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[i: i + n], dtype=np.float64).reshape(shape)
        i += n
    return out


def flatten(params):
    return np.concatenate([np.asarray(params[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def features(packed):
    """packed: uint64[B, 3] queries (key j = word j // 64, bit j % 64) -> float64[B, 167], bf16-rounded."""
    packed = np.asarray(packed, dtype=np.uint64).reshape(-1, 3)
    bits = np.unpackbits(packed.view(np.uint8), axis=1, bitorder="little")[:, :166].astype(np.float64)
    pc = bits.sum(1, keepdims=True) / 166.0
    return bf16(np.concatenate([bits, pc], axis=1))


def forward(params, X, round_bf16=True):
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, w3 = r(params["W1"]), r(params["W2"]), r(params["w3"])
    z1 = X @ W1.T + params["b1"]
    h1 = np.maximum(z1, 0.0)
    h1r = r(h1)
    z2 = h1r @ W2.T + params["b2"]
    h2 = np.maximum(z2, 0.0)
    h2r = r(h2)
    y = h2r @ w3 + params["b3"][0]
    cache = dict(X=X, z1=z1, h1r=h1r, z2=z2, h2r=h2r, W2=W2, w3=w3)
    return y, cache


def pinball(y, t, q):
    r = np.asarray(t, np.float64) - y
    return float(np.mean(np.maximum(q * r, (q - 1.0) * r)))


def pinball_grad(y, t, q):
    """dL/dy of the mean pinball loss: -q/B where t > y, (1 - q)/B otherwise."""
    r = np.asarray(t, np.float64) - y
    return np.where(r > 0, -q, 1.0 - q) / y.shape[0]


def backward(cache, dy):
    """Gradients of every parameter given dL/dy (chain rule through both ReLUs)."""
    X, z1, h1r, z2, h2r, W2, w3 = (cache[k] for k in ("X", "z1", "h1r", "z2", "h2r", "W2", "w3"))
    g = {}
    g["w3"] = h2r.T @ dy
    g["b3"] = np.array([dy.sum()])
    dh2 = np.outer(dy, w3) * (z2 > 0)
    g["W2"] = dh2.T @ h1r
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(0)
    return g


def loss_and_grad(flat, packed, targets, q, round_bf16=True):
    params = unflatten(flat)
    X = features(packed) if round_bf16 else features(packed)
    y, cache = forward(params, X, round_bf16)
    loss = pinball(y, targets, q)
    g = backward(cache, pinball_grad(y, targets, q))
    return loss, flatten(g), y


def adam(flat, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns new (params, m, v) in float32 like the GPU master copy."""
    f32 = np.float32
    flat, grad, m, v = (np.asarray(a, np.float32) for a in (flat, grad, m, v))
    m = f32(b1) * m + f32(1 - b1) * grad
    v = f32(b2) * v + f32(1 - b2) * grad * grad
    mh = m / f32(1 - b1 ** step)
    vh = v / f32(1 - b2 ** step)
    return flat - f32(lr) * mh / (np.sqrt(vh) + f32(eps)), m, v


def init_params(seed=0):
    """He-normal weights, zero biases (host-side, seeded), float32."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.standard_normal((H, IN)) * np.sqrt(2.0 / IN), "b1": np.zeros(H),
         "W2": rng.standard_normal((H, H)) * np.sqrt(2.0 / H), "b2": np.zeros(H),
         "w3": rng.standard_normal(H) * np.sqrt(1.0 / H), "b3": np.array([20.0])}
    return flatten(p).astype(np.float32)
