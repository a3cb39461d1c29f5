"""FP64 reference of the learned radius proposer's network and of its loss
gradient (numpy).

TEST INFRASTRUCTURE ONLY (imported by tests/), independent of the CUDA
sources.  The network is 12 -> 64 -> 64 -> 2 with ReLU hidden layers and
this arithmetic: BF16 weights, FP32 biases, and the input of every layer
(the features, h1, h2) rounded to BF16 (round to nearest even) -- the
operand precision of the GPU's tensor-core products.  The reference decodes
the same BF16 weight bits, applies the same rounding to the layer inputs
and evaluates everything else in FP64.  The gradient treats the rounding
as the identity (straight-through), as the GPU's training kernel does.
Loss per sample: 0.5 m0 (o0 - y0)^2 + m1 BCE(o1, y1), BCE(z, y) =
max(z, 0) - z y + log(1 + exp(-|z|)), times a common scale.
Pinned in tests/test_mlp_oracle.py: the rounding against torch's bfloat16
conversion; the unrounded network's gradient, and the straight-through
gradient (rounding offsets frozen at the evaluation point), by central
finite differences.

Also the two update rules around the network: one Adam step (Kingma & Ba,
"Adam: A Method for Stochastic Optimization", 2015, Algorithm 1, with its
bias-corrected moments), pinned by the closed forms of its first step and
of a constant gradient; and the proposer's radius rule as the library's
interface states it (a hit point the F-test kept, called doomed, gets a
smaller radius clipped by Eq. radiusupdate's bound and a cleared window),
pinned by its invariants and hand cases.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 12, 64, 2
SHAPES = [("W1", (N_H, N_IN)), ("W2", (N_H, N_H)), ("W3", (N_OUT, N_H)),
          ("b1", (N_H,)), ("b2", (N_H,)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
N_WEIGHTS = N_H * N_IN + N_H * N_H + N_OUT * N_H
BLOB_BYTES = 2 * N_WEIGHTS + 4 * (N_H + N_H + N_OUT)


def split(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + k], np.float64).reshape(shape)
        o += k
    return out


def from_blob(blob: bytes | np.ndarray) -> dict:
    """Decode the device blob layout (bf16 W1, W2, W3; f32 b1, b2, b3)."""
    raw = np.frombuffer(bytes(blob), dtype=np.uint8)
    w16 = raw[:2 * N_WEIGHTS].view(np.uint16).astype(np.uint32) << 16
    weights = w16.view(np.float32).astype(np.float64)
    biases = raw[2 * N_WEIGHTS:BLOB_BYTES].view(np.float32).astype(np.float64)
    return split(np.concatenate([weights, biases]))


def bf16_round(x) -> np.ndarray:
    """x rounded to the nearest BF16 value (ties to even) via float32, as
    float64; no NaN or infinity inputs."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _layer_input_bf16(layer: int, v: np.ndarray) -> np.ndarray:
    return bf16_round(v)


def forward(p: dict, X: np.ndarray, act=_layer_input_bf16):
    """Outputs and intermediates.  act(layer, v) maps the input v of layer
    0, 1, 2 (the features, h1, h2) to what the layer multiplies: BF16
    rounding by default (the network's definition); identity for the exact
    real-valued network."""
    X = np.asarray(X, np.float64)
    xb = act(0, X)
    z1 = xb @ p["W1"].T + p["b1"]
    h1 = act(1, np.maximum(z1, 0.0))
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = act(2, np.maximum(z2, 0.0))
    out = h2 @ p["W3"].T + p["b3"]
    return out, (xb, z1, h1, z2, h2)


def loss_and_grad(p: dict, X, Y, M, scale: float, act=_layer_input_bf16):
    """Loss and its gradient w.r.t. every parameter, flattened in the order
    W1, W2, W3, b1, b2, b3 (the master-parameter order).  act as in
    forward; its effect is differentiated as the identity."""
    out, (xb, z1, h1, z2, h2) = forward(p, X, act)
    Y = np.asarray(Y, np.float64)
    M = np.asarray(M, np.float64)
    e = out[:, 0] - Y[:, 0]
    z = out[:, 1]
    bce = np.maximum(z, 0) - z * Y[:, 1] + np.log1p(np.exp(-np.abs(z)))
    loss = scale * np.sum(0.5 * M[:, 0] * e * e + M[:, 1] * bce)
    sig = 1.0 / (1.0 + np.exp(-z))
    dout = scale * np.stack([M[:, 0] * e, M[:, 1] * (sig - Y[:, 1])], 1)
    dW3 = dout.T @ h2
    db3 = dout.sum(0)
    dh2 = (dout @ p["W3"]) * (z2 > 0)
    dW2 = dh2.T @ h1
    db2 = dh2.sum(0)
    dh1 = (dh2 @ p["W2"]) * (z1 > 0)
    dW1 = dh1.T @ xb
    db1 = dh1.sum(0)
    grad = np.concatenate([dW1.ravel(), dW2.ravel(), dW3.ravel(), db1, db2, db3])
    return loss, grad


def loss_only(flat: np.ndarray, X, Y, M, scale: float, act=_layer_input_bf16) -> float:
    return loss_and_grad(split(flat), X, Y, M, scale, act)[0]


def adam_step(master, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in FP64 (Kingma & Ba 2015, Algorithm 1): the moment
    estimates m <- beta1 m + (1 - beta1) g and v <- beta2 v + (1 - beta2) g^2,
    their bias corrections m / (1 - beta1^t) and v / (1 - beta2^t) at step
    t >= 1, and theta <- theta - lr * mhat / (sqrt(vhat) + eps).  Returns
    (theta, m, v) as new arrays."""
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    theta = np.asarray(master, np.float64) - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def propose(r, t, out, bound: float, threshold: float, min_ratio: float):
    """The proposer's rule after an iteration's F-test update, per hit point:
    one the test has just rejected (t == 0) is left alone; otherwise, when
    the network calls it doomed (sigmoid(o1) > threshold) and predicts a
    smaller radius (o0 < 0), the radius becomes
    max(r * max(exp(o0), min_ratio), bound) -- never below the bound of
    Eq. radiusupdate -- and, if that is smaller than r, its window is cleared
    (t = 0).  FP64.  Returns (new radii, new t, mask of the hit points
    shrunk); the caller clears the counts and sums of the masked ones."""
    r = np.asarray(r, np.float64)
    t = np.asarray(t)
    o = np.asarray(out, np.float64)
    doomed = (1.0 / (1.0 + np.exp(-o[:, 1])) > threshold) & (o[:, 0] < 0.0) & (t > 0)
    rn = np.maximum(r * np.maximum(np.exp(np.minimum(o[:, 0], 0.0)), min_ratio), bound)
    shrunk = doomed & (rn < r)
    return np.where(shrunk, rn, r), np.where(shrunk, 0, t), shrunk
