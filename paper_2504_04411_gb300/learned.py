"""The learned radius proposer: training data from the plain method, GPU
training with the library's own forward/backward/Adam kernels, and the
equal-MSE comparison with the plain method.

Samples: every (hit point, iteration i) of a plain run whose test did not
reject at i.  Features: the 12 window features the gather writes
(include/ppm.h).  Targets: y0 = log(r_final / r_{i+1}) (how far the radius
still has to go) and y1 = 1 if the radius is rejected within the next K
tests.  Inputs are standardized for training and the standardization is
folded into the first layer, so the network the kernels run takes the raw
features.  Host code here only orchestrates: every forward, backward and
update runs in libppm.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import ppm

LOOKAHEAD = 4


@dataclass
class Trajectory:
    X: torch.Tensor       # (iters, n, 12) features of each iteration's tests
    r: torch.Tensor       # (iters + 1, n) radius before each iteration, then final
    t: torch.Tensor       # (iters, n) window length after each iteration's update
    L: torch.Tensor       # (n,) final radiance
    mse: list             # per-iteration MSE against the reference, if given


def run(scene, iters: int, params=None, blob=None, threshold=0.5, min_ratio=0.1, seed_offset=0,
        reference=None, collect=True) -> Trajectory:
    """Run the method on scene for iters iterations (the proposer on when
    blob is given), recording features, radii and the MSE of the running
    estimate against reference (a tensor of the exact radiance)."""
    hp = scene.hitpoints("cuda")
    est = ppm.Estimator(hp, scene.r0, 0.75, params)
    n = est.n
    if collect or blob is not None:
        ppm.ppm_set_features(est.ctx, True)
    if blob is not None:
        ppm.ppm_set_mlp(est.ctx, blob, threshold, min_ratio)
    X, R, T, mse = [], [], [], []
    feat = torch.empty(n, 12, device="cuda")
    r = torch.empty(n, device="cuda")
    t = torch.empty(n, device="cuda", dtype=torch.int32)
    ppm.ppm_get_state(est.ctx, r=r)
    R.append(r.clone())
    for i in range(1, iters + 1):
        est.step(scene.photons(i + seed_offset, "cuda"))
        if collect:
            ppm.ppm_get_features(est.ctx, feat)
            X.append(feat.clone())
        ppm.ppm_get_state(est.ctx, r=r, t=t)
        R.append(r.clone())
        T.append(t.clone())
        if reference is not None:
            mse.append(float(((est.radiance() - reference) ** 2).mean()))
    L = est.radiance()
    est.close()
    return Trajectory(torch.stack(X) if X else None, torch.stack(R), torch.stack(T), L, mse)


def dataset(tr: Trajectory, K: int = LOOKAHEAD):
    """(X, Y, M) training tensors from a plain-method trajectory."""
    iters = tr.t.shape[0]
    r_final = tr.r[-1]
    rej = tr.t == 0                                    # rejected at iteration i
    Xs, Ys, Ms = [], [], []
    for i in range(iters - K):
        keep = ~rej[i]
        y0 = torch.log(r_final / tr.r[i + 1])
        y1 = rej[i + 1:i + 1 + K].any(0).float()
        Xs.append(tr.X[i][keep])
        Ys.append(torch.stack([y0, y1], 1)[keep])
        Ms.append(torch.ones_like(Ys[-1]))
    return torch.cat(Xs), torch.cat(Ys), torch.cat(Ms)


def train(X, Y, M, epochs: int = 20, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Train the network on the GPU with the library's kernels.  Returns
    (blob, master, losses per epoch)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    mu = X.mean(0)
    sd = X.std(0).clamp_min(1e-6)
    Xs = ((X - mu) / sd).contiguous()
    P = ppm.PPM_MLP_PARAMS
    master = torch.zeros(P, device="cuda")
    # He initialisation for the ReLU layers
    sizes = [(64, 12), (64, 64), (2, 64)]
    o = 0
    for fo, fi in sizes:
        master[o:o + fo * fi] = torch.randn(fo * fi, generator=g).cuda() * math.sqrt(2.0 / fi)
        o += fo * fi
    grad = torch.zeros(P, device="cuda")
    m = torch.zeros(P, device="cuda")
    v = torch.zeros(P, device="cuda")
    loss = torch.zeros(1, device="cuda")
    blob = torch.zeros(ppm.PPM_MLP_BLOB_BYTES // 4 + 4, device="cuda", dtype=torch.int32)
    ppm.ppm_mlp_pack(master, blob)
    n = Xs.shape[0]
    losses = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        loss.zero_()
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            xb, yb, mb = Xs[idx].contiguous(), Y[idx].contiguous(), M[idx].contiguous()
            ppm.ppm_mlp_grad(blob, xb, yb, mb, 1.0 / xb.shape[0], grad, loss)
            step += 1
            ppm.ppm_mlp_adam(master, grad, m, v, step, lr, blob)
        losses.append(float(loss) / math.ceil(n / batch))
    # fold the standardization into the first layer: W1 x' + b1 with
    # x' = (x - mu) / sd  ==  (W1 / sd) x + (b1 - W1 mu / sd)
    W1 = master[:768].view(64, 12)
    b1 = master[768 + 4096 + 128:768 + 4096 + 128 + 64]
    b1 -= (W1 * (mu / sd)).sum(1)
    W1 /= sd
    ppm.ppm_mlp_pack(master, blob)
    torch.cuda.synchronize()
    return blob, master, losses


# (doom threshold, smallest shrink ratio) settings the validation chooses from
SETTINGS = ((0.5, 0.1), (0.7, 0.25), (0.85, 0.5), (0.95, 0.5), (0.99, 0.7))


def select(blob, scene, iters: int, reference, params=None, settings=SETTINGS):
    """Choose the proposer's setting on a validation scene (a seed that is
    neither the training nor the test seed): the setting with the lowest
    radiance MSE after `iters` iterations, or None -- the proposer off --
    when none beats the plain method there.  Returns (setting, {setting or
    "plain": MSE})."""
    mses = {"plain": run(scene, iters, params=params, reference=reference, collect=False).mse[-1]}
    best, best_mse = None, mses["plain"]
    for thr, mr in settings:
        m = run(scene, iters, params=params, blob=blob, threshold=thr, min_ratio=mr, reference=reference,
                collect=False).mse[-1]
        mses[f"{thr},{mr}"] = m
        if m < best_mse:
            best, best_mse = (thr, mr), m
    return best, mses


def iterations_to_reach(mse: list, target: float) -> int | None:
    for i, v in enumerate(mse):
        if v <= target:
            return i + 1
    return None
