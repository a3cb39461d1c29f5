"""Pins of the FP64 network oracle: analytic gradient against central finite
differences; blob decoding against numpy's float conversion (CPU only)."""
import numpy as np

from oracle import mlp_oracle as MO


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    flat = rng.normal(0, 0.3, MO.N_PARAMS)
    X = rng.normal(0, 1, (40, MO.N_IN))
    Y = np.stack([rng.normal(-1, 1, 40), rng.integers(0, 2, 40)], 1).astype(float)
    M = rng.uniform(0, 1, (40, 2))
    loss, g = MO.loss_and_grad(MO.split(flat), X, Y, M, 1 / 40)
    idx = rng.choice(MO.N_PARAMS, 200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat); e[i] = h
        fd = (MO.loss_only(flat + e, X, Y, M, 1 / 40) - MO.loss_only(flat - e, X, Y, M, 1 / 40)) / (2 * h)
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
