"""Pins of the FP64 network oracle: the BF16 rounding of the layer inputs
against torch's bfloat16 conversion; the gradient of the exact network and
the straight-through gradient of the BF16 network against central finite
differences; blob decoding against numpy's float conversion; the Adam step
against the closed forms of its first step and of a constant gradient; the
proposer's rule against its invariants and hand cases (CPU only)."""
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


def test_adam_first_step_is_lr_times_sign():
    # at t = 1 from zero moments the bias corrections give mhat = g and
    # vhat = g^2, so every parameter moves by lr * g / (|g| + eps)
    rng = np.random.default_rng(21)
    theta = rng.normal(0, 1, 500)
    g = rng.normal(0, 1, 500) * 10.0 ** rng.uniform(-6, 2, 500)
    lr = 3e-3
    th, m, v = MO.adam_step(theta, g, np.zeros(500), np.zeros(500), 1, lr)
    assert np.allclose(th, theta - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g, rtol=1e-15) and np.allclose(v, 0.001 * g * g, rtol=1e-15)


def test_adam_constant_gradient_moves_lr_per_step():
    # with one gradient g at every step, m_t = (1 - beta1^t) g and
    # v_t = (1 - beta2^t) g^2: the corrected moments are g and g^2 at every
    # t, and theta moves by the same lr * g / (|g| + eps) each step
    g = np.array([2.0, -0.5, 1e-3, -7.0])
    theta = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    lr = 1e-2
    for step in range(1, 8):
        theta, m, v = MO.adam_step(theta, g, m, v, step, lr)
        assert np.allclose(m, (1 - 0.9 ** step) * g, rtol=1e-13)
        assert np.allclose(v, (1 - 0.999 ** step) * g * g, rtol=1e-12)
    assert np.allclose(theta, -7 * lr * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # a zero gradient leaves a zero-moment parameter where it is
    th, _, _ = MO.adam_step(np.ones(3), np.zeros(3), np.zeros(3), np.zeros(3), 5, 0.1)
    assert np.array_equal(th, np.ones(3))


def test_propose_rule_hand_cases_and_invariants():
    bound, thr, mr = 0.01, 0.5, 0.1
    r = np.array([0.04, 0.04, 0.04, 0.04, 0.04, 0.011, 0.04])
    t = np.array([3, 0, 3, 3, 3, 3, 5])
    out = np.array([[np.log(0.5), 5.0],     # doomed, halve
                    [np.log(0.5), 5.0],     # just rejected by the test: untouched
                    [np.log(0.5), -5.0],    # not doomed
                    [0.3, 5.0],             # doomed but asks for a larger radius
                    [-10.0, 5.0],           # clamp at min_ratio
                    [np.log(0.5), 5.0],     # clamp at the bound
                    [np.log(0.9999), 0.001]])   # sigmoid just above the threshold
    rn, tn, sh = MO.propose(r, t, out, bound, thr, mr)
    assert np.allclose(rn, [0.02, 0.04, 0.04, 0.04, 0.004 if 0.004 > bound else bound, bound, 0.04 * 0.9999])
    assert list(sh) == [True, False, False, False, True, True, True]
    assert list(tn) == [0, 0, 3, 3, 0, 0, 0]
    # invariants on random inputs: never larger, never below the bound
    # (unless it already was), cleared windows exactly where shrunk
    rng = np.random.default_rng(3)
    r = rng.uniform(0.005, 0.05, 2000)
    t = rng.integers(0, 6, 2000)
    out = rng.normal(0, 2, (2000, 2))
    rn, tn, sh = MO.propose(r, t, out, bound, 0.7, 0.2)
    assert np.all(rn <= r) and np.all((rn >= bound) | (rn == r))
    assert np.array_equal(sh, rn < r) and np.all(tn[sh] == 0) and np.array_equal(tn[~sh], t[~sh])
    assert np.all(rn[sh] >= np.maximum(0.2 * r[sh], bound) * (1 - 1e-15))
