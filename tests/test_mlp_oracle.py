"""Pins of the FP64 network oracle: the BF16 rounding of the layer inputs
against torch's bfloat16 conversion; the gradient of the exact network and
the straight-through gradient of the BF16 network against central finite
differences; blob decoding against numpy's float conversion (CPU only)."""
import numpy as np
import torch

from oracle import mlp_oracle as MO


def _identity(layer, v):
    return v


def _net(seed, n=40):
    rng = np.random.default_rng(seed)
    flat = rng.normal(0, 0.3, MO.N_PARAMS)
    X = rng.normal(0, 1, (n, MO.N_IN))
    Y = np.stack([rng.normal(-1, 1, n), rng.integers(0, 2, n)], 1).astype(float)
    M = rng.uniform(0, 1, (n, 2))
    return rng, flat, X, Y, M


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-30, 100), rng.normal(0, 1e30, 100),
                        [0.0, -0.0, 1.0, -2.5, 3.0e38]]).astype(np.float32)
    # exact ties: low half 0x8000 on even and odd upper halves
    ties = (rng.integers(0x3F00, 0x4100, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32)
    x = np.concatenate([x, ties, -ties])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(MO.bf16_round(x), want)


def test_exact_network_gradient_matches_finite_differences():
    rng, flat, X, Y, M = _net(0)
    loss, g = MO.loss_and_grad(MO.split(flat), X, Y, M, 1 / 40, act=_identity)
    idx = rng.choice(MO.N_PARAMS, 200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat); e[i] = h
        fd = (MO.loss_only(flat + e, X, Y, M, 1 / 40, act=_identity) -
              MO.loss_only(flat - e, X, Y, M, 1 / 40, act=_identity)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_straight_through_gradient_is_the_frozen_rounding_gradient():
    """With each layer input's rounding offset frozen at the evaluation
    point, the network is smooth in the parameters; its finite-difference
    gradient is what the BF16 network's gradient must be."""
    rng, flat, X, Y, M = _net(6)
    p = MO.split(flat)
    loss, g = MO.loss_and_grad(p, X, Y, M, 1 / 40)
    _, (xb, z1, h1, z2, h2) = MO.forward(p, X)
    E = [xb - X, h1 - np.maximum(z1, 0.0), h2 - np.maximum(z2, 0.0)]
    assert max(np.abs(e).max() for e in E) > 0          # the rounding is active

    def frozen(layer, v):
        return v + E[layer]

    assert MO.loss_only(flat, X, Y, M, 1 / 40, act=frozen) == loss
    idx = rng.choice(MO.N_PARAMS, 200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat); e[i] = h
        fd = (MO.loss_only(flat + e, X, Y, M, 1 / 40, act=frozen) -
              MO.loss_only(flat - e, X, Y, M, 1 / 40, act=frozen)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_blob_decoding():
    rng = np.random.default_rng(1)
    w = rng.normal(0, 1, MO.N_WEIGHTS).astype(np.float32)
    b = rng.normal(0, 1, MO.N_PARAMS - MO.N_WEIGHTS).astype(np.float32)
    bf = (w.view(np.uint32) >> 16).astype(np.uint16)          # truncation: exact bf16 values
    blob = bf.tobytes() + b.tobytes()
    assert len(blob) == MO.BLOB_BYTES
    p = MO.from_blob(blob)
    want = (bf.astype(np.uint32) << 16).view(np.float32)
    assert np.array_equal(p["W1"].ravel(), want[:768])
    assert np.array_equal(p["b3"], b[-2:].astype(np.float64))
