"""Pins of the CPU oracle against things other than itself: values the paper
prints, closed forms, textbook routines (scipy), geometry in FP64, invariants
of the method, and statistics of the analytic test scenes.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2504_04411_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_constants.json")))
NG = GOLD["n_annuli"]["value"] * GOLD["n_sectors"]["value"]
ALPHA = GOLD["alpha_F"]["value"]


# ---------------------------------------------------------------- F_c ------
@pytest.mark.parametrize("d2", [1, 3, 10, 57, 1000, 123456])
def test_fcrit_d1_1_is_t_squared(d2):
    # F(1, d2) quantile = square of the two-sided t quantile
    t = stats.t.ppf(1 - ALPHA / 2, d2)
    assert O.f_crit(1, d2, ALPHA) == pytest.approx(t * t, rel=1e-10)


@pytest.mark.parametrize("d2", [1, 2, 7, 20, 500, 1e6])
@pytest.mark.parametrize("a", [0.01, 0.05, 0.1])
def test_fcrit_d1_2_closed_form(d2, a):
    # CDF of F(2, d2) is 1 - (1-x)^(d2/2): quantile = d2/2 (a^(-2/d2) - 1)
    want = d2 / 2 * (a ** (-2.0 / d2) - 1)
    assert O.f_crit(2, d2, a) == pytest.approx(want, rel=1e-10)


@pytest.mark.parametrize("d1", [1, 3, 11, 40])
def test_fcrit_d2_2_closed_form(d1):
    # CDF of F(d1, 2) is x^(d1/2): quantile = 2 y / (d1 (1 - y)), y = q^(2/d1)
    y = (1 - ALPHA) ** (2.0 / d1)
    assert O.f_crit(d1, 2, ALPHA) == pytest.approx(2 * y / (d1 * (1 - y)), rel=1e-9)


def test_fcrit_paper_limits():
    # Sec. 6.1.1 prints chi_c = 24.724 for 12 groups and F_c ~ 2.25 in the
    # limit m -> inf: F(11, inf) = chi2(11)/11.
    fc_inf = O.f_crit(NG - 1, 1e13, ALPHA)
    assert abs(11 * fc_inf - GOLD["chi_c"]["value"]) < 2e-3
    assert round(fc_inf, GOLD["F_c_limit"]["digits"]) == GOLD["F_c_limit"]["value"]
    # at one iteration of the tiny configuration (m = 1e5 samples per group)
    fc = O.f_crit(11, 12 * (1e5 - 1), ALPHA)
    assert fc == pytest.approx(2.2477393, abs=2e-7)
    assert fc > fc_inf


@pytest.mark.parametrize("d1,d2", [(11, 12), (11, 120), (11, 12 * 99999),
                                   (11, 12 * (64 * 2e6 - 1)), (5, 33), (30, 7)])
def test_fcrit_matches_scipy(d1, d2):
    assert O.f_crit(d1, d2, ALPHA) == pytest.approx(stats.f.ppf(1 - ALPHA, d1, d2), rel=1e-9)


@pytest.mark.parametrize("J", [2, 1000, 2_000_000, 16_000_000])
def test_fcrit_matches_high_precision_at_huge_d2(J):
    # 40-digit evaluation of the same quantile (mpmath, independent code):
    # d2 = 12 (t J - 1) reaches 6e10, where lgamma cancels in FP64
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for t in [1, 64, 300]:
        d2 = 12 * (t * J - 1)
        a, b = mp.mpf(11) / 2, mp.mpf(d2) / 2
        ex = mp.findroot(lambda F: mp.betainc(a, b, 0, 11 * F / (11 * F + d2), regularized=True)
                         - (1 - mp.mpf(ALPHA)), mp.mpf("2.5"))
        assert O.f_crit(11, d2, ALPHA) == pytest.approx(float(ex), rel=2e-12)


def test_betainc_matches_scipy():
    from scipy import special
    rng = np.random.default_rng(1)
    for _ in range(200):
        a, b = rng.uniform(0.5, 50, 2)
        x = rng.uniform(0, 1)
        assert O.betainc(a, b, x) == pytest.approx(special.betainc(a, b, x), rel=1e-9, abs=1e-14)


# ------------------------------------------------------------ ANOVA F ------
def _full_table(groups, m):
    return [np.concatenate([np.asarray(g, float), np.zeros(m - len(g))]) for g in groups]


def test_anova_matches_f_oneway():
    rng = np.random.default_rng(2)
    for trial in range(20):
        m = int(rng.integers(5, 60))
        groups = []
        for g in range(NG):
            c = int(rng.integers(0, m))
            groups.append(rng.exponential(1.0 + g * 0.1 * (trial % 3), c))
        F = O.anova_f(groups, m)
        ref = stats.f_oneway(*_full_table(groups, m)).statistic
        assert F == pytest.approx(ref, rel=1e-10)


def test_anova_single_nonzero_sample_is_one():
    # one nonzero sample among 12 m: SSB/11 = psi^2/(12 m), SSW/(12(m-1)) =
    # psi^2/(12 m), so F = 1 exactly, for any m and psi.
    for m in [2, 10, 1e5, 3e9]:
        for g in range(NG):
            groups = [[] for _ in range(NG)]
            groups[g] = [0.37]
            assert O.anova_f(groups, m) == pytest.approx(1.0, rel=1e-9)


def test_anova_balanced_and_scale_invariance():
    groups = [[0.5, 0.25]] * NG
    assert O.anova_f(groups, 100) == pytest.approx(0.0, abs=1e-12)
    rng = np.random.default_rng(3)
    groups = [rng.uniform(0, 1, rng.integers(0, 8)) for _ in range(NG)]
    f1 = O.anova_f(groups, 50)
    f2 = O.anova_f([np.asarray(g) * 1e-7 for g in groups], 50)
    assert f1 == pytest.approx(f2, rel=1e-9)


def test_anova_equal_flux_limit_is_pearson_chi2():
    # equal psi, m -> inf: 11 F -> sum (c_g - C/12)^2 / (C/12), the statistic
    # of the chi-square test of CPPM (Sec. 3.2.3)
    rng = np.random.default_rng(4)
    counts = rng.integers(3, 30, NG)
    groups = [np.ones(c) for c in counts]
    C = counts.sum()
    chi2 = ((counts - C / NG) ** 2 / (C / NG)).sum()
    assert 11 * O.anova_f(groups, 1e12) == pytest.approx(chi2, rel=1e-8)


# ---------------------------------------------- CPPM's chi-square test ------
@pytest.mark.parametrize("alpha", [0.5, 0.1, 0.05, 0.01, 1e-4])
def test_chi2_crit_two_dof_closed_form(alpha):
    # chi^2(2) is the exponential law with mean 2: quantile -2 ln(alpha)
    assert O.chi2_crit(2, alpha) == pytest.approx(-2.0 * math.log(alpha), rel=1e-12)


def test_chi2_crit_paper_value_and_scipy():
    # Sec. 6.1.1 prints chi_c = 24.724 for CPPM's 12 groups at alpha 0.01
    want = GOLD["chi_c"]["value"]
    got = O.chi2_crit(NG - 1, ALPHA)
    assert abs(got - want) < 10.0 ** -GOLD["chi_c"]["digits"], got
    for k in (1, 3, 11, 40):
        for a in (0.2, 0.01, 1e-3):
            assert O.chi2_crit(k, a) == pytest.approx(stats.chi2.ppf(1 - a, k), rel=1e-11)


def test_chi2_counts_matches_scipy_and_limits():
    rng = np.random.default_rng(7)
    for _ in range(20):
        c = rng.integers(0, 50, NG)
        if c.sum() == 0:
            continue
        assert O.chi2_counts(c) == pytest.approx(stats.chisquare(c).statistic, rel=1e-12)
    assert O.chi2_counts(np.full(NG, 9)) == 0.0                 # even spread
    one = np.zeros(NG, np.int64)
    one[5] = 40
    assert O.chi2_counts(one) == pytest.approx((NG - 1) * 40, rel=1e-14)   # all in one group: (n-1) C
    assert O.chi2_counts(np.zeros(NG, np.int64)) == 0.0         # no photons: no evidence


def test_cppm_rejection_rate_is_alpha():
    # under an even spread of photons, Pearson's X^2 of the counts follows
    # chi^2(11) closely (about nine photons per group here), so CPPM's first
    # test rejects with probability about alpha
    J, r0, seeds = 20000, 0.045, 10
    rej = n = 0
    for s in range(seeds):
        sc = synth.PlaneScene(nside=64, J=J, r0=r0, step=False, lo=-r0, hi=1 + r0,
                              seed=synth.SEED_BASE + 100 + s)
        hp = sc.hitpoints().numpy()
        res = O.run(hp, synth.stack_numpy([sc.photons(1)]), r0, 1, test=1)
        assert np.allclose(res.Fc, O.chi2_crit(NG - 1, ALPHA))
        rej += int(res.reject[0].sum())
        n += res.reject[0].size
    p = rej / n
    sigma = math.sqrt(ALPHA * (1 - ALPHA) / n)
    assert abs(p - ALPHA) < 5 * sigma, (p, sigma)


def test_cppm_is_blind_to_a_zero_flux_edge():
    # Sec. 3.2.3: the chi-square test sees where photons land, not what they
    # carry.  Photons keep landing evenly in a shadow (flux 0 for x > 0.5),
    # so CPPM keeps the radii at the edge that the F-test shrinks.
    sc = synth.PlaneScene(nside=32, J=20000, r0=0.04, step=True)
    hp = sc.hitpoints().numpy()
    iters = 10
    ph = synth.stack_numpy([sc.photons(i) for i in range(1, iters + 1)])
    f = O.run(hp, ph, sc.r0, iters)
    c = O.run(hp, ph, sc.r0, iters, test=1)
    x, y = hp["pos"][:, 0], hp["pos"][:, 1]
    near = (np.abs(x - 0.5) < 0.5 * sc.r0) & (y > 2 * sc.r0) & (y < 1 - 2 * sc.r0)
    assert np.all(f.r[-1][near] < sc.r0)
    assert np.mean(c.r[-1][near] < sc.r0) < 0.3
    # both take the same pairs and windows until their decisions differ
    assert np.array_equal(f.pairs[0], c.pairs[0]) and np.array_equal(f.counts[0], c.counts[0])
    for it in range(iters):
        assert np.allclose(c.F[it], [O.chi2_counts(k) for k in c.counts[it]], rtol=1e-12)


# ------------------------------------------------------ classification ------
def _geom_group(xh, u, v, r, xp):
    d = np.asarray(xh, float) - np.asarray(xp, float)
    yu, yv = d @ np.asarray(u, float), d @ np.asarray(v, float)
    if d @ d > r * r:
        return -1, None
    ang = math.atan2(yv, yu) % (2 * math.pi)
    sector = int(ang // (math.pi / 3)) % 6
    ring = 0 if 2 * (yu * yu + yv * yv) < r * r else 1
    # distance of the point to the nearest class boundary, for tolerance
    rho = math.hypot(yu, yv)
    bd = min(abs(rho - r / math.sqrt(2)), abs(rho - r),
             min(abs(ang - k * math.pi / 3) for k in range(7)) * rho)
    return ring * 6 + sector, bd


def test_classify_matches_fp64_geometry():
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(20000):
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        t = np.cross(n, [1.0, 0, 0] if abs(n[0]) < 0.9 else [0, 1.0, 0]); t /= np.linalg.norm(t)
        b = np.cross(n, t)
        xh = rng.uniform(-1, 1, 3)
        r = rng.uniform(1e-3, 0.1)
        off = rng.uniform(-1.2, 1.2, 2) * r
        xp = xh - off[0] * t - off[1] * b
        g = O.classify(xh.astype(np.float32), t.astype(np.float32), b.astype(np.float32), r,
                       xp.astype(np.float32))
        ref, bd = _geom_group(xh.astype(np.float32), t.astype(np.float32),
                              b.astype(np.float32), np.float32(r), xp.astype(np.float32))
        if bd is not None and bd < 1e-5 * r:
            continue  # within rounding of a class boundary
        if ref == -1 and abs(np.linalg.norm(off) - r) < 1e-5 * r:
            continue
        assert g == ref
        checked += 1
    assert checked > 19000


def test_classify_hand_cases():
    z3 = np.zeros(3, np.float32)
    u = np.array([1, 0, 0], np.float32); v = np.array([0, 1, 0], np.float32)
    r = np.float32(0.5)  # exactly representable: r^2 = 0.25 exactly
    # photon at distance exactly r on -u: y = x_h - x_p = (+r, 0): closed disk,
    # outer annulus, angle 0 -> sector 0 -> group 6
    assert O.classify(z3, u, v, r, np.array([-0.5, 0, 0], np.float32)) == 6
    # just outside
    assert O.classify(z3, u, v, r, np.array([-0.5000001, 0, 0], np.float32)) == -1
    # angle 90 degrees, inner: photon at (0,-0.1): y = (0, 0.1) -> sector 1
    assert O.classify(z3, u, v, r, np.array([0, -0.1, 0], np.float32)) == 1
    # angle 180, inner: y = (-0.1, 0) -> sector 3 (yv == 0, yu < 0)
    assert O.classify(z3, u, v, r, np.array([0.1, 0, 0], np.float32)) == 3
    # angle 270 outer: y = (0, -0.4) -> sector 4, ring 1
    assert O.classify(z3, u, v, r, np.array([0, 0.4, 0], np.float32)) == 10
    # equal-area annulus boundary: rho^2 = r^2/2 belongs to the outer ring
    x = np.float32(0.25); y = np.float32(0.25)  # rho^2 = 0.125 = r^2/2
    assert O.classify(z3, u, v, r, np.array([-x, -y, 0], np.float32)) == 6
    # same-surface filter: perpendicular normals are not gathered
    nz = int(synth.pack_snorm8(__import__("torch").tensor([0.0, 0, 1])).item()) & 0xffffffff
    nx = int(synth.pack_snorm8(__import__("torch").tensor([1.0, 0, 0])).item()) & 0xffffffff
    assert O.normal_dot(nz, nz) == 127 * 127
    assert O.classify(z3, u, v, r, np.array([0, -0.1, 0], np.float32), nz, nx) == -1
    assert O.classify(z3, u, v, r, np.array([0, -0.1, 0], np.float32), nz, nz) == 1


def test_groups_are_equi_areal():
    # uniform photons in the disk fall in the 12 groups with probability 1/12
    rng = np.random.default_rng(6)
    xh = np.array([0.3, 0.4, 0.0], np.float32)
    u = np.array([0.6, 0.8, 0], np.float32); v = np.array([-0.8, 0.6, 0], np.float32)
    r = np.float32(0.05)
    counts = np.zeros(NG, int)
    pts = xh[:2] + rng.uniform(-r, r, (60000, 2))
    for p in pts.astype(np.float32):
        g = O.classify(xh, u, v, r, np.array([p[0], p[1], 0], np.float32))
        if g >= 0:
            counts[g] += 1
    chi2 = ((counts - counts.sum() / NG) ** 2 / (counts.sum() / NG)).sum()
    assert chi2 < stats.chi2.ppf(0.999, NG - 1)


# ------------------------------------------------------ radius update ------
def test_radius_update_eq():
    r_min, a = 2e-5, 0.75
    for i in [1, 2, 10, 1000]:
        want = r_min * math.sqrt((i + 1) ** (a - 1))
        assert O.radius_bound(r_min, a, i) == pytest.approx(want, rel=1e-7)
    assert O.shrink(0.02, 0.7, 1e-5) == pytest.approx(0.014, rel=1e-7)
    assert O.shrink(1e-5, 0.7, 2e-5) == pytest.approx(2e-5, rel=1e-7)


# ---------------------------------------------------------- MIS weight ------
def test_mis_weight_limits():
    # no competing technique: weight 1 (plain photon mapping)
    assert O.mis_weight(0, 0, 0, 0, 0, 1e5, 0.01) == pytest.approx(1.0)
    # connections dominate: weight -> 0
    assert O.mis_weight(0, 1e12, 0, 1e12, 0, 1e5, 0.01) < 1e-6
    # p_VM grows with r^2 (Sec. 4.2): the weight increases with r
    ws = [O.mis_weight(0.5, 2.0, 0.7, 1.0, 9000, 1e5, r) for r in [1e-3, 3e-3, 1e-2]]
    assert ws[0] < ws[1] < ws[2]
    # balance heuristic with one connection pdf ratio R at eta = 1: w = 1/(1+R)
    assert O.mis_weight(0, 3.0, 0, 0, 0, 1 / math.pi, 1.0) == pytest.approx(0.25)


# ------------------------------------------------------ whole method ------
def _independent_in_disk(hp, ph, r):
    """In-disk counts from FP64 geometry, bracketing FP32 rounding."""
    d = hp["pos"][:, None, :2].astype(float) - ph["pos"][None, :, :2].astype(float)
    d2 = (d ** 2).sum(-1)
    return ((d2 <= (r * (1 - 1e-5)) ** 2).sum(1), (d2 <= (r * (1 + 1e-5)) ** 2).sum(1))


def _rec709_luminance_row():
    """Y row of the RGB -> XYZ matrix of ITU-R BT.709: the primaries'
    chromaticities (R 0.64/0.33, G 0.30/0.60, B 0.15/0.06) scaled so that
    R = G = B = 1 gives the D65 white point (x 0.3127, y 0.3290) with Y = 1."""
    prim = np.array([[0.64, 0.33], [0.30, 0.60], [0.15, 0.06]])
    xyz = np.array([[x / y, 1.0, (1 - x - y) / y] for x, y in prim]).T   # columns: R, G, B
    wx, wy = 0.3127, 0.3290
    white = np.array([wx / wy, 1.0, (1 - wx - wy) / wy])
    scale = np.linalg.solve(xyz, white)
    return xyz[1] * scale


def test_luminance_weights_are_rec709():
    # the weights follow from the BT.709 primaries and white point (to the
    # four decimals the standard quotes), not from a retyped table
    y = _rec709_luminance_row()
    assert y.sum() == pytest.approx(1.0, abs=1e-12)
    for rgb, want in (((1, 0, 0), y[0]), ((0, 1, 0), y[1]), ((0, 0, 1), y[2])):
        assert O.lum(*rgb) == pytest.approx(want, abs=5e-5)
    assert O.lum(1, 1, 1) == pytest.approx(1.0, abs=1e-12)
    # linear: scaling and adding fluxes
    assert O.lum(0.3, 2.0, 0.7) == pytest.approx(0.3 * O.lum(1, 0, 0) + 2 * O.lum(0, 1, 0) + 0.7 * O.lum(0, 0, 1),
                                                 rel=1e-14)


def test_run_tests_the_luminance_of_rgb_flux():
    # one hit point, one photon inside its disk: the tested value in the
    # window is the photon's luminance; the estimate keeps all three channels
    hp = {"pos": np.array([[0.5, 0.5, 0.0]], np.float32), "u": np.array([[1, 0, 0]], np.float32),
          "v": np.array([[0, 1, 0]], np.float32)}
    rgb = np.array([0.25, 0.5, 2.0], np.float32)
    ph = {"pos": np.array([[[0.505, 0.5, 0.0], [0.9, 0.9, 0.0]]], np.float32),
          "flux": np.array([[rgb, [1, 1, 1]]], np.float32)}
    res = O.run(hp, ph, 0.02, 1, alpha_f=1e-12)
    y = _rec709_luminance_row()
    assert res.S[0, 0].sum() == pytest.approx(float(y @ rgb.astype(np.float64)), rel=1e-4)
    assert res.S[0, 0].sum() == pytest.approx(O.lum(*rgb.astype(np.float64)), rel=1e-15)
    assert res.Q[0, 0].sum() == pytest.approx(O.lum(*rgb.astype(np.float64)) ** 2, rel=1e-15)
    area = math.pi * float(np.float32(0.02)) ** 2
    assert np.allclose(res.tau[0], rgb.astype(np.float64) / area, rtol=1e-12)
    # per-channel mode: three windows, one per channel
    res3 = O.run(hp, ph, 0.02, 1, alpha_f=1e-12, rgb_test=True)
    assert np.allclose(res3.Sc[0, 0].sum(axis=1), rgb, rtol=1e-12)


def test_run_counts_match_geometry():
    sc = synth.PlaneScene(nside=16, J=5000, r0=0.06, step=True)
    hp = sc.hitpoints().numpy()
    batches = [sc.photons(i) for i in range(1, 3)]
    ph = synth.stack_numpy(batches)
    res = O.run(hp, ph, sc.r0, 2)
    lo, hi = _independent_in_disk(hp, {"pos": ph["pos"][0]}, sc.r0)
    assert np.all(res.pairs[0] >= lo) and np.all(res.pairs[0] <= hi)
    # test counts after the first iteration equal the pairs of iteration 1
    assert np.array_equal(res.counts[0].sum(1), res.pairs[0])


def test_run_invariants_and_step_edge():
    sc = synth.PlaneScene(nside=32, J=20000, r0=0.04, step=True)
    hp = sc.hitpoints().numpy()
    iters = 10
    ph = synth.stack_numpy([sc.photons(i) for i in range(1, iters + 1)])
    res = O.run(hp, ph, sc.r0, iters, k=0.7, alpha=0.75)
    r = res.r
    assert np.all(np.diff(r, axis=0) <= 0)                       # non-increasing
    r_min = 1e-3 * sc.r0
    for it in range(iters):
        shr = res.reject[it]
        assert np.all(r[it + 1][~shr] == r[it][~shr])             # kept when not rejected
        bound = O.radius_bound(r_min, 0.75, it + 1)
        want = np.maximum((np.float32(0.7) * r[it][shr]).astype(np.float32), np.float32(bound))
        assert np.array_equal(r[it + 1][shr], want)
    # window counts restart after a rejection
    for it in range(1, iters):
        prev_rej = res.reject[it - 1]
        assert np.array_equal(res.counts[it][prev_rej].sum(1), res.pairs[it][prev_rej])
        keep = ~prev_rej
        assert np.array_equal(res.counts[it][keep].sum(1),
                              res.counts[it - 1][keep].sum(1) + res.pairs[it][keep])
    # step edge at x = 0.5: hit points whose disk straddles it shrink, far
    # ones keep (almost all) their radius (Sec. 6.1.1: small radii at
    # illumination discontinuities)
    x = hp["pos"][:, 0]
    near = np.abs(x - 0.5) < 0.5 * sc.r0
    far = (np.abs(x - 0.5) > 3 * sc.r0) & (x > 2 * sc.r0) & (x < 1 - 2 * sc.r0) \
        & (hp["pos"][:, 1] > 2 * sc.r0) & (hp["pos"][:, 1] < 1 - 2 * sc.r0)
    assert np.all(r[-1][near] < sc.r0)
    assert np.mean(r[-1][far] < sc.r0) < 0.2
    assert np.median(r[-1][near]) < np.median(r[-1][far])


def test_rejection_rate_is_alpha():
    # Sec. 5.1: on unbiased estimates the test wrongly rejects with
    # probability alpha_F.  Uniform photons with constant flux on a square
    # larger than every disk: the first test of every hit point is under H0.
    J, r0, seeds = 20000, 0.045, 10
    rej = 0
    n = 0
    for s in range(seeds):
        sc = synth.PlaneScene(nside=64, J=J, r0=r0, step=False, lo=-r0, hi=1 + r0,
                              seed=synth.SEED_BASE + 100 + s)
        hp = sc.hitpoints().numpy()
        ph = synth.stack_numpy([sc.photons(1)])
        res = O.run(hp, ph, r0, 1)
        rej += int(res.reject[0].sum())
        n += res.reject[0].size
    p = rej / n
    sigma = math.sqrt(ALPHA * (1 - ALPHA) / n)
    assert abs(p - ALPHA) < 4 * sigma, (p, sigma)


def test_unbiased_constant_plane():
    # constant irradiance: the estimate is unbiased for every radius, so the
    # mean of L over hit points and iterations equals the flux density
    sc = synth.PlaneScene(nside=32, J=20000, r0=0.04, step=False, lo=-0.05, hi=1.05)
    hp = sc.hitpoints().numpy()
    iters = 6
    ph = synth.stack_numpy([sc.photons(i) for i in range(1, iters + 1)])
    res = O.run(hp, ph, sc.r0, iters)
    L = res.tau[:, 0] / iters
    E = sc.irradiance_density()
    # per hit point and iteration ~ Poisson(J pi r^2 / A) photons
    lam = sc.J * math.pi * sc.r0 ** 2 / (sc.hi - sc.lo) ** 2
    se = E / math.sqrt(lam * iters * L.size)
    # neighbouring disks share photons: allow for the correlation
    assert abs(L.mean() - E) < 8 * se * math.sqrt(math.pi * (sc.r0 * 32) ** 2)


def test_step_edge_expected_estimate_closed_form():
    # E[per-iteration estimate] = density * |disk ∩ lit| / (pi r^2); check
    # the first-iteration estimate averaged over seeds for hit points at
    # several offsets from the edge x = 0.5 (circular segment area)
    r = 0.05
    offs = np.array([-0.04, -0.02, 0.0, 0.02, 0.04], np.float32)
    hp = {"pos": np.stack([0.5 + offs, np.full(5, 0.5, np.float32), np.zeros(5, np.float32)], 1),
          "u": np.tile(np.array([1, 0, 0], np.float32), (5, 1)),
          "v": np.tile(np.array([0, 1, 0], np.float32), (5, 1))}
    acc = np.zeros(5)
    runs = 30
    for s in range(runs):
        sc = synth.PlaneScene(nside=1, J=40000, r0=r, step=True, seed=synth.SEED_BASE + 500 + s)
        ph = synth.stack_numpy([sc.photons(1)])
        acc += O.run(hp, ph, r, 1).tau[:, 0]
    est = acc / runs
    def lit_fraction(d):  # fraction of the disk centred at 0.5 + d with x < 0.5
        h = -d  # signed distance from centre to the edge, lit side x < 0.5
        if h >= r: return 1.0
        if h <= -r: return 0.0
        seg = r * r * math.acos(abs(h) / r) - abs(h) * math.sqrt(r * r - h * h)
        frac = seg / (math.pi * r * r)
        return 1 - frac if h > 0 else frac
    want = np.array([lit_fraction(float(d)) for d in offs])
    lam = 40000 * math.pi * r * r
    assert np.all(np.abs(est - want) < 5 / math.sqrt(lam * runs) + 1e-3)


# ------------------------------------------ hit points traced anew ----------
def test_retrace_with_the_same_hit_points_equals_the_static_run():
    # one hit-point set per iteration, all equal: exactly the static method
    sc = synth.PlaneScene(nside=24, J=10000, r0=0.05, step=True)
    hp = sc.hitpoints().numpy()
    iters = 6
    ph = synth.stack_numpy([sc.photons(i) for i in range(1, iters + 1)])
    a = O.run(hp, ph, sc.r0, iters)
    b = O.run(hp, ph, sc.r0, iters, hp_iters=[hp] * iters)
    for f in ("r", "counts", "S", "Q", "F", "reject", "pairs", "t", "tau"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_retrace_uses_each_iterations_hit_points():
    # the pairs of iteration i are those of iteration i's positions (FP64
    # geometry brackets them), and the statistics of a pixel carry over
    sc = synth.PlaneScene(nside=16, J=5000, r0=0.06, step=True)
    iters = 4
    hps = [sc.hitpoints_jittered(i).numpy() for i in range(1, iters + 1)]
    batches = [sc.photons(i) for i in range(1, iters + 1)]
    ph = synth.stack_numpy(batches)
    res = O.run(hps[0], ph, sc.r0, iters, hp_iters=hps)
    for it in range(iters):
        r = res.r[it].astype(np.float64)
        d = hps[it]["pos"][:, None, :2].astype(np.float64) - ph["pos"][it][None, :, :2]
        d2 = (d ** 2).sum(-1)
        lo = (d2 <= (r[:, None] * (1 - 1e-6)) ** 2).sum(1)
        hi = (d2 <= (r[:, None] * (1 + 1e-6)) ** 2).sum(1)
        assert np.all(res.pairs[it] >= lo) and np.all(res.pairs[it] <= hi), it
    for it in range(1, iters):
        keep = ~res.reject[it - 1]
        assert np.array_equal(res.counts[it][keep].sum(1), res.counts[it - 1][keep].sum(1) + res.pairs[it][keep])
    # jitter moves the disks: a static run on the same photons differs
    static = O.run(hps[0], ph, sc.r0, iters)
    assert not np.array_equal(static.pairs[1:], res.pairs[1:])


def test_retrace_constant_plane_unbiased():
    # constant irradiance: each iteration's estimate is unbiased wherever its
    # hit point lands, so the mean over pixels and iterations is the density
    sc = synth.PlaneScene(nside=32, J=20000, r0=0.04, step=False, lo=-0.05, hi=1.05)
    iters = 6
    hps = [sc.hitpoints_jittered(i).numpy() for i in range(1, iters + 1)]
    ph = synth.stack_numpy([sc.photons(i) for i in range(1, iters + 1)])
    res = O.run(hps[0], ph, sc.r0, iters, hp_iters=hps)
    L = res.tau[:, 0] / iters
    E = sc.irradiance_density()
    lam = sc.J * math.pi * sc.r0 ** 2 / (sc.hi - sc.lo) ** 2
    se = E / math.sqrt(lam * iters * L.size)
    assert abs(L.mean() - E) < 8 * se * math.sqrt(math.pi * (sc.r0 * 32) ** 2)


@pytest.mark.parametrize("scene", ["plane", "box", "translated"])
def test_grid_form_equals_brute_force(scene):
    """The timed CPU form (photons sorted by grid cell, each disk's cells
    scanned) gathers exactly the brute force's pairs: counts, decisions,
    radii and window lengths bit for bit; sums, F and the estimate to FP64
    rounding (the sums add the same values in another order)."""
    if scene == "plane":
        sc = synth.PlaneScene(nside=24, J=12_000, r0=0.05, step=True, seed=synth.SEED_BASE + 70)
        hp = sc.hitpoints().numpy()
    else:
        sc = synth.BoxScene(nh=900, J=15_000, r0=0.05, rgb=True, vcm=True, seed=synth.SEED_BASE + 71)
        hp = sc.hitpoints().numpy()
    iters = 4
    ph = synth.stack_numpy([sc.photons(i) for i in range(1, iters + 1)])
    if scene == "translated":
        off = np.array([-37.25, 1000.5, 3.0], np.float32)
        hp = dict(hp, pos=(hp["pos"] + off).astype(np.float32))
        ph = dict(ph, pos=(ph["pos"] + off).astype(np.float32))
    kw = dict(k=0.9, vcm=True) if scene != "plane" else {}
    a = O.run(hp, ph, sc.r0, iters, **kw)
    b = O.run(hp, ph, sc.r0, iters, grid=True, **kw)
    assert a.pairs.sum() > 1000
    for f in ("r", "counts", "reject", "pairs", "t"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    for f in ("S", "Q", "F", "tau", "est"):
        assert np.allclose(getattr(a, f), getattr(b, f), rtol=1e-12, atol=1e-300), f
