"""The learned radius proposer's kernels through the C ABI against the FP64
network oracle (forward, loss, gradient), the BF16 packing, training, the
window features against values derived from the method oracle, and the
proposer switched off reproducing the plain method bit for bit."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as MO
from oracle import oracle as O
from paper_2504_04411_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _bf16_rne(x: np.ndarray) -> np.ndarray:
    """float32 -> bf16 bits, round to nearest even (no NaNs here)."""
    u = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    u = u + 0x7FFF + ((u >> 16) & 1)
    return (u >> 16).astype(np.uint16)


def _host_blob(master: np.ndarray) -> bytes:
    return _bf16_rne(master[:MO.N_WEIGHTS]).tobytes() + master[MO.N_WEIGHTS:].astype(np.float32).tobytes()


def _to_dev_blob(blob: bytes):
    import torch
    buf = np.zeros(MO.BLOB_BYTES // 4 + 4, np.int32)
    buf.view(np.uint8)[:MO.BLOB_BYTES] = np.frombuffer(blob, np.uint8)
    return torch.from_numpy(buf).cuda()


def _random_net(seed, n=1500):
    rng = np.random.default_rng(seed)
    master = np.concatenate([rng.normal(0, math.sqrt(2 / 12), 768), rng.normal(0, math.sqrt(2 / 64), 4096),
                             rng.normal(0, math.sqrt(2 / 64), 128), rng.normal(0, 0.1, 130)]).astype(np.float32)
    X = rng.normal(0, 1, (n, 12)).astype(np.float32)
    Y = np.stack([rng.normal(-1, 1, n), rng.integers(0, 2, n)], 1).astype(np.float32)
    M = rng.uniform(0, 1, (n, 2)).astype(np.float32)
    return master, X, Y, M


def _near_bf16_midpoint(v, mag, rel=2.0 ** -16):
    """Per sample: does any entry of v (FP64 values before BF16 rounding)
    lie within FP32 accumulation error (rel * mag, mag the sum of the
    absolute terms that made it) of a BF16 rounding midpoint?"""
    v = np.asarray(v, np.float64)
    e = np.floor(np.log2(np.maximum(np.abs(v), 1e-300)))
    ulp = 2.0 ** (e - 7)                   # BF16 spacing at v
    frac = np.abs(v) / ulp - np.floor(np.abs(v) / ulp)
    dist = np.abs(frac - 0.5) * ulp        # distance to the midpoint of its interval
    return np.any((dist <= rel * mag) & (v > 0), axis=1)


def test_forward_matches_oracle():
    import torch
    from paper_2504_04411_gb300 import ppm
    master, X, _, _ = _random_net(1)
    blob = _host_blob(master)
    out = torch.empty(X.shape[0], 2, device="cuda")
    ppm.ppm_mlp_forward(_to_dev_blob(blob), torch.from_numpy(X).cuda(), out)
    p = MO.from_blob(blob)
    ref, (xb, z1, h1, z2, h2) = MO.forward(p, X)
    got = out.cpu().numpy().astype(np.float64)
    # both sides round each layer's input to BF16; the GPU from FP32 sums,
    # the oracle from FP64 ones.  A sample may differ beyond FP32 error only
    # if one of its hidden activations lies within FP32 error of a BF16
    # rounding midpoint (the two sides then round it the other way).
    scale = np.abs(ref).max()
    close = np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-5 * scale, axis=1)
    mag1 = np.abs(xb) @ np.abs(p["W1"]).T + np.abs(p["b1"])
    mag2 = np.abs(h1) @ np.abs(p["W2"]).T + np.abs(p["b2"])
    near = _near_bf16_midpoint(np.maximum(z1, 0), mag1) | _near_bf16_midpoint(np.maximum(z2, 0), mag2)
    assert np.all(close | near), np.flatnonzero(~(close | near))[:10]
    assert close.mean() >= 0.99, close.mean()


def test_gradient_matches_oracle():
    import torch
    from paper_2504_04411_gb300 import ppm
    master, X, Y, M = _random_net(2, n=2000)
    blob = _host_blob(master)
    grad = torch.zeros(MO.N_PARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    scale = 1.0 / X.shape[0]
    ppm.ppm_mlp_grad(_to_dev_blob(blob), torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(),
                     torch.from_numpy(M).cuda(), scale, grad, loss)
    ref_loss, ref = MO.loss_and_grad(MO.from_blob(blob), X, Y, M, scale)
    g = grad.cpu().numpy().astype(np.float64)
    assert float(loss) == pytest.approx(ref_loss, rel=1e-5)
    err = np.abs(g - ref)
    assert np.all(err <= 1e-3 * np.abs(ref) + 1e-5 * np.abs(ref).max()), float((err / (np.abs(ref) + 1e-12)).max())


def test_gradient_over_several_chunks_is_deterministic():
    """More tiles than one scratch chunk (256 tiles of 128) plus a ragged
    tail: matches the oracle, and a second call gives the same bits."""
    import torch
    from paper_2504_04411_gb300 import ppm
    master, X, Y, M = _random_net(5, n=256 * 128 + 77)
    blob = _to_dev_blob(_host_blob(master))
    Xd, Yd, Md = (torch.from_numpy(v).cuda() for v in (X, Y, M))
    scale = 1.0 / X.shape[0]
    out = []
    for _ in range(2):
        grad = torch.zeros(MO.N_PARAMS, device="cuda")
        loss = torch.zeros(1, device="cuda")
        ppm.ppm_mlp_grad(blob, Xd, Yd, Md, scale, grad, loss)
        out.append((grad.cpu().numpy(), float(loss)))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
    ref_loss, ref = MO.loss_and_grad(MO.from_blob(_host_blob(master)), X, Y, M, scale)
    assert out[0][1] == pytest.approx(ref_loss, rel=1e-5)
    err = np.abs(out[0][0].astype(np.float64) - ref)
    assert np.all(err <= 1e-3 * np.abs(ref) + 1e-5 * np.abs(ref).max())


def test_training_is_bitwise_reproducible():
    import torch
    from paper_2504_04411_gb300 import learned
    rng = np.random.default_rng(6)
    X = torch.from_numpy(rng.normal(0, 1, (9000, 12)).astype(np.float32)).cuda()
    Y = torch.from_numpy(np.stack([np.tanh(X.cpu().numpy()[:, 1]), (X.cpu().numpy()[:, 2] > 0)], 1)
                         .astype(np.float32)).cuda()
    runs = [learned.train(X, Y, torch.ones_like(Y), epochs=3) for _ in range(2)]
    assert torch.equal(runs[0][1], runs[1][1])
    assert torch.equal(runs[0][0], runs[1][0])
    assert runs[0][2] == runs[1][2]


def test_pack_rounds_to_nearest_even():
    import torch
    from paper_2504_04411_gb300 import ppm
    master, _, _, _ = _random_net(3)
    dev = torch.zeros(MO.BLOB_BYTES // 4 + 4, dtype=torch.int32, device="cuda")
    ppm.ppm_mlp_pack(torch.from_numpy(master).cuda(), dev)
    got = dev.cpu().numpy().view(np.uint8)[:MO.BLOB_BYTES].tobytes()
    assert got == _host_blob(master)


def test_training_reduces_loss():
    import torch
    from paper_2504_04411_gb300 import learned
    rng = np.random.default_rng(4)
    X = rng.normal(0, 1, (20000, 12)).astype(np.float32)
    w = rng.normal(0, 1, 12)
    y0 = np.tanh(X @ w / 4) - 1
    y1 = (X[:, 0] + X[:, 3] > 0).astype(np.float32)
    Y = torch.from_numpy(np.stack([y0, y1], 1).astype(np.float32)).cuda()
    blob, master, losses = learned.train(torch.from_numpy(X).cuda(), Y, torch.ones_like(Y), epochs=12)
    assert losses[-1] < 0.35 * losses[0], losses
    assert all(b <= a * 1.05 for a, b in zip(losses, losses[1:])), losses


def _derived_features(ref, it, r0, i):
    """FP64 features of iteration it from the oracle's window statistics."""
    C = ref.counts[it].sum(1).astype(np.float64)
    S = ref.S[it]
    Ssum = S.sum(1)
    # window length: iterations since the last rejection, plus this one
    tp = np.ones(C.shape[0])
    for k in range(it):
        tp = np.where(ref.reject[k], 1.0, tp + 1.0)
    r = ref.r[it].astype(np.float64)
    F, Fc = ref.F[it], ref.Fc[it]
    with np.errstate(divide="ignore", invalid="ignore"):
        cv = np.where(Ssum > 0, np.sqrt(((S - Ssum[:, None] / 12) ** 2).sum(1) / 12) / (Ssum / 12), 0)
        f = np.stack([np.log1p(C), np.log1p(tp), np.full_like(C, math.log(i)), r / r0, np.log(r / r0),
                      np.log1p(F), F / Fc, np.where(Ssum > 0, S.max(1) / Ssum, 0),
                      np.where(Ssum > 0, S.min(1) / Ssum, 0), (ref.counts[it] == 0).sum(1) / 12, cv,
                      np.where(C > 0, ref.counts[it].max(1) / C, 0)], 1)
    return f


def test_features_match_oracle():
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = synth.PlaneScene(nside=32, J=30_000, r0=0.04, step=True, seed=synth.SEED_BASE + 40)
    hp = sc.hitpoints("cuda")
    iters = 3
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    est = ppm.Estimator(hp, sc.r0)
    ppm.ppm_set_features(est.ctx, True)
    feats = []
    out = torch.empty(hp.n, 12, device="cuda")
    for ph in batches:
        est.step(ph)
        ppm.ppm_get_features(est.ctx, out)
        feats.append(out.cpu().numpy().astype(np.float64))
    est.close()
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters)
    alive = np.ones(hp.n, bool)
    for it in range(iters):
        want = _derived_features(ref, it, sc.r0, it + 1)
        got = feats[it]
        # F-dependent features carry the FP32 statistics' rounding
        tol = np.array([1e-5, 1e-6, 1e-6, 1e-6, 1e-5, 1e-3, 1e-3, 1e-4, 1e-4, 0, 1e-3, 1e-6])
        err = np.abs(got - want)[alive]
        assert np.all(err <= tol * np.maximum(np.abs(want[alive]), 1) + 1e-6), (it, err.max(0))


def test_features_and_disabled_proposer_leave_the_method_unchanged():
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = synth.PlaneScene(nside=24, J=20_000, r0=0.04, step=True, seed=synth.SEED_BASE + 41)
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, 6)]
    finals = []
    for mode in ("plain", "features", "disabled"):
        est = ppm.Estimator(hp, sc.r0)
        if mode != "plain":
            ppm.ppm_set_features(est.ctx, True)
        if mode == "disabled":
            blob = torch.zeros(ppm.PPM_MLP_BLOB_BYTES // 4 + 4, dtype=torch.int32, device="cuda")
            ppm.ppm_set_mlp(est.ctx, blob)
            ppm.ppm_set_mlp(est.ctx, None)
        for ph in batches:
            est.step(ph)
        finals.append({k: v.cpu() for k, v in est.state().items()})
        est.close()
    for k in finals[0]:
        assert torch.equal(finals[0][k], finals[1][k]) and torch.equal(finals[0][k], finals[2][k]), k


def test_proposer_only_shrinks_and_respects_the_bound():
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = synth.PlaneScene(nside=32, J=30_000, r0=0.04, step=True, seed=synth.SEED_BASE + 42)
    hp = sc.hitpoints("cuda")
    # a network that calls everything doomed and asks for half the radius:
    # all weights zero, b3 = (log 0.5, +10)
    master = np.zeros(MO.N_PARAMS, np.float32)
    master[-2:] = [math.log(0.5), 10.0]
    blob = _to_dev_blob(_host_blob(master))
    est = ppm.Estimator(hp, sc.r0)
    ppm.ppm_set_mlp(est.ctx, blob, 0.5, 0.1)
    prev = torch.full((hp.n,), sc.r0, device="cuda")
    for i in range(1, 5):
        est.step(sc.photons(i, "cuda"))
        st = est.state()
        assert torch.all(st["r"] <= prev)
        bound = O.radius_bound(1e-3 * sc.r0, 0.75, i)
        assert torch.all(st["r"] >= bound * (1 - 1e-6))
        assert est.stats().proposals > 0
        assert torch.all(st["t"] == 0)          # every window restarted
        prev = st["r"].clone()
    est.close()


def test_learned_proposer_gains_over_the_plain_method():
    """Trained on 200 plain iterations of the tiny configuration (one seed),
    the proposer reaches on a fresh seed the plain method's 64-iteration
    radiance MSE in fewer iterations and has a lower MSE at 32."""
    from paper_2504_04411_gb300 import learned
    train_sc = synth.PlaneScene(nside=64, J=100_000, r0=0.02, step=True, seed=synth.SEED_BASE + 500)
    tr = learned.run(train_sc, 200)
    X, Y, M = learned.dataset(tr)
    blob, _, losses = learned.train(X, Y, M, epochs=20)
    test_sc = synth.PlaneScene(nside=64, J=100_000, r0=0.02, step=True, seed=synth.SEED_BASE + 600)
    ref = (test_sc.hitpoints("cuda").pos[:, 0] < 0.5).float()
    plain = learned.run(test_sc, 64, reference=ref, collect=False)
    lrn = learned.run(test_sc, 64, blob=blob, threshold=0.5, min_ratio=0.1, reference=ref, collect=False)
    reach = learned.iterations_to_reach(lrn.mse, plain.mse[-1])
    assert reach is not None and reach < 64, (reach, lrn.mse[-1], plain.mse[-1])
    assert lrn.mse[31] < plain.mse[31]
    # radii stay non-increasing under the proposer
    assert bool((lrn.r[1:] <= lrn.r[:-1]).all())


def test_adam_matches_oracle():
    """ppm_mlp_adam element by element against the FP64 Adam step, at the
    first step and later ones; the blob is the BF16 packing of the new
    master parameters and the gradient is cleared."""
    import torch
    from paper_2504_04411_gb300 import ppm
    rng = np.random.default_rng(31)
    n = MO.N_PARAMS
    master = rng.normal(0, 0.2, n).astype(np.float32)
    m = np.zeros(n, np.float32)
    v = np.zeros(n, np.float32)
    dm, dv, dmaster = (torch.from_numpy(a.copy()).cuda() for a in (m, v, master))
    blob = torch.zeros(MO.BLOB_BYTES // 4 + 4, dtype=torch.int32, device="cuda")
    lr = 2e-3
    # the kernel's hyperparameters are the FP32 numbers nearest 0.9, 0.999
    # and 1e-8 (1 - 0.999f differs from 0.001 by 1.3e-5): the oracle takes
    # the same values
    b1, b2, eps = (float(np.float32(x)) for x in (0.9, 0.999, 1e-8))
    for step in range(1, 6):
        g = (rng.normal(0, 1, n) * 10.0 ** rng.uniform(-5, 1, n)).astype(np.float32)
        dg = torch.from_numpy(g).cuda()
        # the oracle steps from the GPU's own FP32 state, so errors do not add up
        prev_t = dmaster.cpu().numpy().astype(np.float64)
        prev_m = dm.cpu().numpy().astype(np.float64)
        prev_v = dv.cpu().numpy().astype(np.float64)
        ppm.ppm_mlp_adam(dmaster, dg, dm, dv, step, lr, blob)
        ref_t, ref_m, ref_v = MO.adam_step(prev_t, g, prev_m, prev_v, step, lr, beta1=b1, beta2=b2, eps=eps)
        got_t = dmaster.cpu().numpy().astype(np.float64)
        # FP32 moments: a few roundings of terms that may cancel (m) or not (v)
        scale_m = b1 * np.abs(prev_m) + (1 - b1) * np.abs(g.astype(np.float64))
        assert np.all(np.abs(dm.cpu().numpy() - ref_m) <= 3e-7 * scale_m + 1e-38), step
        assert np.all(np.abs(dv.cpu().numpy() - ref_v) <= 3e-7 * np.abs(ref_v) + 1e-38), step
        # the update itself is about lr in size: compare it to 1e-5 of lr
        assert np.all(np.abs(got_t - ref_t) <= 1e-5 * lr + 2e-7 * np.abs(ref_t)), step
        assert torch.all(dg == 0)
        got_blob = blob.cpu().numpy().view(np.uint8)[:MO.BLOB_BYTES].tobytes()
        assert got_blob == _host_blob(dmaster.cpu().numpy())


def test_proposer_matches_oracle_rule():
    """One proposer pass per iteration against the oracle's rule applied to
    the state the F-test left: a second context without the network runs the
    same iterations from the same state, its radii, windows and features are
    the proposer's input, and the network's outputs come from
    ppm_mlp_forward on those features."""
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = synth.PlaneScene(nside=40, J=40_000, r0=0.04, step=True, seed=synth.SEED_BASE + 43)
    hp = sc.hitpoints("cuda")
    # a network whose doom logit follows F / F_c (feature 6):
    # o1 = 8 (F/F_c - 0.3), o0 = log 0.6 -- a spread of decisions; every
    # weight is exact in BF16
    master = np.zeros(MO.N_PARAMS, np.float32)
    master[0 * 12 + 6] = 1.0                          # W1[0][6]: h1[0] = F / F_c
    master[768 + 0 * 64 + 0] = 1.0                    # W2[0][0]: h2[0] = h1[0]
    master[768 + 4096 + 1 * 64 + 0] = 8.0             # W3[1][0]
    master[-2:] = [math.log(0.6), -2.4]               # b3
    blob = _to_dev_blob(_host_blob(master))
    thr, mr = 0.55, 0.25
    plain = ppm.Estimator(hp, sc.r0)          # the F-test alone, state reset to the proposer's
    ppm.ppm_set_features(plain.ctx, True)
    lrn = ppm.Estimator(hp, sc.r0)
    ppm.ppm_set_mlp(lrn.ctx, blob, thr, mr)
    feat = torch.empty(hp.n, 12, device="cuda")
    out = torch.empty(hp.n, 2, device="cuda")
    shrunk_total = 0
    for i in range(1, 6):
        ph = sc.photons(i, "cuda")
        plain.step(ph)
        lrn.step(ph)
        before = {k: v.cpu().numpy() for k, v in plain.state().items()}
        after = {k: v.cpu().numpy() for k, v in lrn.state().items()}
        ppm.ppm_get_features(plain.ctx, feat)
        ppm.ppm_mlp_forward(blob, feat, out)
        o = out.cpu().numpy().astype(np.float64)
        bound = O.radius_bound(1e-3 * sc.r0, 0.75, i)
        rn, tn, sh = MO.propose(before["r"], before["t"], o, bound, thr, mr)
        # decisions taken within FP32 rounding of a threshold may go either way
        edge = (np.abs(o[:, 1] - math.log(thr / (1 - thr))) < 1e-5) | (np.abs(o[:, 0]) < 1e-6)
        ok = ~edge
        assert np.array_equal(after["t"][ok], tn[ok]), i
        assert np.allclose(after["r"][ok], rn[ok], rtol=1e-6, atol=0), i
        got_sh = after["r"] < before["r"]
        assert np.array_equal(got_sh[ok], sh[ok]), i
        for k in ("counts", "S", "Q"):
            assert np.all(after[k][got_sh] == 0), (i, k)
        # kept windows: the same photons (the grids' cell sizes may differ,
        # so the FP32 sums may round differently)
        assert np.array_equal(after["counts"][~got_sh], before["counts"][~got_sh]), i
        for k in ("S", "Q"):
            assert np.allclose(after[k][~got_sh], before[k][~got_sh], rtol=1e-5, atol=0), (i, k)
        shrunk_total += int(sh.sum())
        # the F-test context continues from the proposer's state
        st = {k: torch.from_numpy(v).cuda() for k, v in after.items()}
        ppm.ppm_set_state(plain.ctx, **st)
    plain.close()
    lrn.close()
    assert shrunk_total > 100


def test_learned_proposer_on_a_box_scene():
    """A second, non-tiny scene: three faces of the unit box with caustic
    lobes and shadow edges (50k hit points, 300k photons per iteration,
    ~200 photons per disk).  Trained on 32 plain iterations of one seed, its
    setting chosen on a second seed, run on a third: the proposer keeps the
    radii non-increasing and its 32-iteration radiance MSE (against the
    scene's closed-form irradiance) is no worse than the plain method's by
    more than the validation's own spread (5%)."""
    import torch
    from paper_2504_04411_gb300 import learned
    train_sc = synth.BoxScene(nh=50_000, J=300_000, r0=0.025, seed=synth.SEED_BASE + 520)
    tr = learned.run(train_sc, 32)
    X, Y, M = learned.dataset(tr)
    del tr
    blob, _, losses = learned.train(X, Y, M, epochs=10)
    assert losses[-1] < losses[0]
    val_sc = synth.BoxScene(nh=50_000, J=300_000, r0=0.025, seed=synth.SEED_BASE + 530)
    setting, _ = learned.select(blob, val_sc, 32, val_sc.irradiance(val_sc.hitpoints("cuda")).to("cuda", torch.float32))
    test_sc = synth.BoxScene(nh=50_000, J=300_000, r0=0.025, seed=synth.SEED_BASE + 620)
    hp = test_sc.hitpoints("cuda")
    ref = test_sc.irradiance(hp).to("cuda", torch.float32)
    plain = learned.run(test_sc, 32, reference=ref, collect=False)
    if setting is None:
        return                       # the validation switched the proposer off
    lrn = learned.run(test_sc, 32, blob=blob, threshold=setting[0], min_ratio=setting[1], reference=ref,
                      collect=False)
    assert lrn.mse[-1] <= 1.05 * plain.mse[-1], (setting, lrn.mse[-1], plain.mse[-1])
    assert bool((lrn.r[1:] <= lrn.r[:-1]).all())
