"""Helpers that run the CUDA path through the C ABI and compare it with the
CPU oracle on the same photons (imported by the gpu tests)."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Reject decisions are compared bit for bit wherever the oracle's FP64 F is
# farther than BAND * F_c from F_c.  Inside the band the GPU's F (FP32 window
# sums, FP32 F) may fall on the other side: both decisions are correct
# readings of the same data, and that hit point's later trajectory is
# excluded from the comparison (counted as "diverged").
BAND = 1e-3
S_RTOL = 2e-5      # FP32 window sums against FP64
L_RTOL = 1e-5      # radiance / estimate against FP64


@dataclass
class Report:
    iters: int = 0
    n: int = 0
    diverged: int = 0
    band_flips: list = field(default_factory=list)
    max_rel_S: float = 0.0
    max_rel_F: float = 0.0
    max_rel_L: float = 0.0
    pairs_checked: int = 0


def run_gpu(hp, batches, r0, alpha=0.75, params=None, J=None, hps=None):
    """hps: optional hit points traced anew for every iteration."""
    import torch

    from paper_2504_04411_gb300 import ppm
    est = ppm.Estimator(hp, r0, alpha, params)
    states, stats = [], []
    for i, ph in enumerate(batches):
        if hps is not None:
            est.retrace(hps[i])
        est.step(ph, J)
        st = est.state()
        states.append({k: v.cpu().numpy() for k, v in st.items()})
        s = est.stats()
        stats.append({"pairs": s.pairs, "candidates": s.candidates, "rejects": s.rejects,
                      "flags": s.flags, "r_max": s.r_max, "cell": s.cell})
    L = est.radiance().cpu().numpy()
    est.close()
    torch.cuda.synchronize()
    return states, stats, L


def compare(states, stats, L, ref, iters, ch_test=0, band=BAND, check_pairs=True) -> Report:
    rep = Report(iters=iters, n=states[0]["r"].shape[0])
    n = rep.n
    diverged = np.zeros(n, bool)
    for it in range(iters):
        g = states[it]
        rej_o = ref.reject[it]
        rej_g = g["t"] == 0
        Fo, Fc = ref.F[it], ref.Fc[it]
        alive = ~diverged
        # radius used in this iteration must agree for live hit points
        if it > 0:
            assert np.array_equal(states[it - 1]["r"][alive], ref.r[it][alive])
        in_band = np.abs(Fo - Fc) <= band * Fc
        bad = alive & ~in_band & (rej_g != rej_o)
        assert not bad.any(), (f"iteration {it + 1}: decisions differ outside the band at "
                               f"{np.flatnonzero(bad)[:10]} F={Fo[bad][:5]} Fc={Fc[bad][:5]} "
                               f"F_gpu={g['F'][bad][:5]}")
        flip = alive & in_band & (rej_g != rej_o)
        if flip.any():
            rep.band_flips += [(it + 1, int(i)) for i in np.flatnonzero(flip)]
        if check_pairs and not diverged.any() and not flip.any():
            assert stats[it]["pairs"] == int(ref.pairs[it].sum()), (it, stats[it]["pairs"], int(ref.pairs[it].sum()))
            rep.pairs_checked += 1
        assert stats[it]["flags"] == 0
        same = alive & ~flip
        assert np.array_equal(g["r"][same], ref.r[it + 1][same])
        keep = same & ~rej_o
        assert np.array_equal(g["counts"][keep], ref.counts[it][keep]), f"counts differ at iteration {it + 1}"
        assert np.all(g["counts"][same & rej_o] == 0)
        So = ref.S[it][keep]
        Sg = g["S"][keep][:, ch_test, :].astype(np.float64)
        scale = np.abs(So).sum(1, keepdims=True) + 1e-30
        relS = np.abs(Sg - So) / scale
        rep.max_rel_S = max(rep.max_rel_S, float(relS.max()) if relS.size else 0.0)
        assert rep.max_rel_S <= S_RTOL, rep.max_rel_S
        okF = keep & (Fo > 0)
        if okF.any():
            relF = np.abs(g["F"][okF].astype(np.float64) - Fo[okF]) / Fo[okF]
            rep.max_rel_F = max(rep.max_rel_F, float(relF.max()))
        diverged |= flip
    rep.diverged = int(diverged.sum())
    alive = ~diverged
    Lo = ref.tau / iters
    Lg = L.reshape(Lo.shape).astype(np.float64)
    scale = np.abs(Lo).max() + 1e-30
    relL = np.abs(Lg[alive] - Lo[alive]) / np.maximum(np.abs(Lo[alive]), 1e-3 * scale)
    rep.max_rel_L = float(relL.max()) if relL.size else 0.0
    assert rep.max_rel_L <= L_RTOL, rep.max_rel_L
    tau_g = states[-1]["tau"].reshape(ref.tau.shape)
    relT = np.abs(tau_g[alive] - ref.tau[alive]) / np.maximum(np.abs(ref.tau[alive]), 1e-3 * np.abs(ref.tau).max() + 1e-300)
    assert relT.max() <= L_RTOL if relT.size else True
    return rep
