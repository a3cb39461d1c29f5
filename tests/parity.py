"""Helpers that run the CUDA path through the C ABI and compare it with the
CPU oracle on the same photons (imported by the gpu tests)."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Reject decisions are compared bit for bit wherever the oracle's FP64 F is
# farther than BAND * F_c from F_c (the scope table's 1e-4).  Inside the
# band the GPU's F (FP32 window sums, FP32 F) may fall on the other side:
# both decisions are correct readings of the same data, and that hit
# point's later trajectory is excluded from the comparison (counted as
# "diverged").  The measured F error (<= 3e-6 relative) leaves a 30x margin.
BAND = 1e-4
S_RTOL = 2e-5      # FP32 window sums S_g, Q_g against FP64, per group
F_RTOL = 1e-5      # the F statistic of the last test, per hit point
L_RTOL = 1e-5      # radiance / estimate against FP64
# absolute floors, relative to the largest value of the compared array:
# only values that are zero (or within FP32 underflow of it) use them
FLOOR = 1e-9


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


def _close(got, want, rtol, what, it):
    """Element-wise |got - want| <= rtol |want| + FLOOR max|want|; returns
    the largest relative error over the nonzero entries."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    if want.size == 0:
        return 0.0
    floor = FLOOR * float(np.abs(want).max())
    err = np.abs(got - want)
    bad = err > rtol * np.abs(want) + floor
    assert not bad.any(), (f"{what} differs at iteration {it + 1}: {int(bad.sum())} entries, "
                           f"e.g. got {got[bad][:4]} want {want[bad][:4]}")
    nz = np.abs(want) > floor
    return float((err[nz] / np.abs(want[nz])).max()) if nz.any() else 0.0


def compare(states, stats, L, ref, iters, band=BAND, check_pairs=True) -> Report:
    """Every iteration's GPU state against the oracle's, element by element:
    radii, window lengths, per-group counts (exact); decisions (exact outside
    the band); per-group window sums S and Q of every tested channel, F of
    the last test, the iteration's estimate term (tau difference) of every
    hit point (within the tolerances above); the final radiance."""
    rep = Report(iters=iters, n=states[0]["r"].shape[0])
    n = rep.n
    diverged = np.zeros(n, bool)
    ntc = states[0]["S"].shape[1]
    Sc = ref.Sc if ref.Sc is not None else ref.S[:, :, None, :]
    Qc = ref.Qc if ref.Qc is not None else ref.Q[:, :, None, :]
    assert Sc.shape[2] == ntc, (Sc.shape, ntc)
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
        assert np.array_equal(g["t"][same & ~rej_o], (states[it - 1]["t"][same & ~rej_o] + 1) if it > 0
                              else np.ones(int((same & ~rej_o).sum()), np.int32))
        keep = same & ~rej_o
        assert np.array_equal(g["counts"][keep], ref.counts[it][keep]), f"counts differ at iteration {it + 1}"
        assert np.all(g["counts"][same & rej_o] == 0)
        assert np.all(g["S"][same & rej_o] == 0) and np.all(g["Q"][same & rej_o] == 0)
        # window sums of every tested channel, per group
        rep.max_rel_S = max(rep.max_rel_S, _close(g["S"][keep], Sc[it][keep], S_RTOL, "S", it))
        rep.max_rel_S = max(rep.max_rel_S, _close(g["Q"][keep], Qc[it][keep], S_RTOL, "Q", it))
        # F of this iteration's test (rejected hit points included)
        rep.max_rel_F = max(rep.max_rel_F, _close(g["F"][same], Fo[same], F_RTOL, "F", it))
        # this iteration's estimate term of every hit point (rejected included)
        if ref.est is not None:
            prev = states[it - 1]["tau"] if it > 0 else np.zeros_like(g["tau"])
            dtau = (g["tau"] - prev).reshape(ref.est[it].shape)
            rep.max_rel_L = max(rep.max_rel_L, _close(dtau[same], ref.est[it][same], L_RTOL, "estimate term", it))
        diverged |= flip
    rep.diverged = int(diverged.sum())
    alive = ~diverged
    Lo = ref.tau / iters
    Lg = L.reshape(Lo.shape).astype(np.float64)
    rep.max_rel_L = max(rep.max_rel_L, _close(Lg[alive], Lo[alive], L_RTOL, "radiance", iters - 1))
    tau_g = states[-1]["tau"].reshape(ref.tau.shape)
    _close(tau_g[alive], ref.tau[alive], L_RTOL, "tau", iters - 1)
    return rep
