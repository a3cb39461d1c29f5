"""CUDA path (through the C ABI) against the CPU oracle, element by element,
on the same seeded photons.  Counts, groups, radii and reject decisions are
compared exactly (decisions outside a 1e-3 band around F_c); window sums,
F and the estimate within the stated tolerances (tests/parity.py)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_04411_gb300 import synth

from parity import compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _params(**kw):
    from paper_2504_04411_gb300 import ppm
    p = ppm.ppm_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ------------------------------------------------------------------ F_c ----
@pytest.mark.parametrize("J", [2, 10, 1000, 100_000, 2_000_000, 16_000_000])
def test_fcrit_table_matches_oracle(J):
    import torch
    from paper_2504_04411_gb300 import ppm
    tmax = 300
    out = torch.empty(tmax + 1, device="cuda", dtype=torch.float64)
    ppm.ppm_f_critical(J, 0.01, tmax, out)
    got = out.cpu().numpy()
    assert got[0] == 0.0
    for t in [1, 2, 3, 7, 16, 64, 199, 256, 300]:
        want = O.f_crit(11, 12 * (t * J - 1), 0.01)
        assert got[t] == pytest.approx(want, rel=1e-11), (t, got[t], want)


def test_fcrit_other_alpha_and_monotone():
    import torch
    from paper_2504_04411_gb300 import ppm
    out = torch.empty(65, device="cuda", dtype=torch.float64)
    for a in [0.05, 0.1]:
        ppm.ppm_f_critical(5000, a, 64, out)
        got = out.cpu().numpy()
        assert np.all(np.diff(got[1:]) < 0)   # more samples: smaller F_c
        for t in [1, 9, 64]:
            assert got[t] == pytest.approx(O.f_crit(11, 12 * (t * 5000 - 1), a), rel=1e-11)


# ----------------------------------------------- CPPM's chi-square test ----
@pytest.mark.parametrize("dof", [1, 2, 11, 40])
def test_chi2_critical_matches_oracle(dof):
    import torch
    from paper_2504_04411_gb300 import ppm
    out = torch.empty(1, device="cuda", dtype=torch.float64)
    for a in (0.2, 0.01, 1e-3):
        ppm.ppm_chi2_critical(dof, a, out)
        assert float(out) == pytest.approx(O.chi2_crit(dof, a), rel=1e-12), (dof, a)


def _cppm_check(states, stats, L, ref, iters):
    """Decisions from exact integer counts: identical on both sides, so the
    whole trajectory must agree (no band, no divergence)."""
    rep = compare(states, stats, L, ref, iters)
    assert rep.diverged == 0 and not rep.band_flips, rep
    for it in range(iters):
        assert np.array_equal(states[it]["t"] == 0, ref.reject[it])
        X = states[it]["F"].astype(np.float64)
        assert np.allclose(X, ref.F[it], rtol=1e-7, atol=0), it      # X^2 stored as FP32
    return rep


def test_cppm_tiny_config_full_trajectory():
    """The tiny configuration (step edge at x = 0.5) with the count test:
    radii, windows, X^2 and estimate against the oracle, iteration by
    iteration."""
    sc = synth.PlaneScene(nside=64, J=100_000, r0=0.02, step=True)
    iters = 16
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    states, stats, L = run_gpu(hp, batches, sc.r0, params=_params(test=1))
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters, test=1)
    _cppm_check(states, stats, L, ref, iters)
    assert 0 < ref.reject.sum() < ref.reject.size


def test_cppm_box_scene_with_normals():
    """Three faces of the unit box (same-surface test), lobes and shadows."""
    sc = _box(seed=4)
    iters = 8
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    states, stats, L = run_gpu(hp, batches, sc.r0, params=_params(test=1, cell_factor=0.6))
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters, test=1)
    _cppm_check(states, stats, L, ref, iters)


def test_cppm_box_scene_rgb_vcm():
    """RGB flux with VCM+ weights: the counts decide, the weighted RGB
    estimate follows the radii."""
    sc = _box(rgb=True, vcm=True, seed=5)
    iters = 5
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    p = _params(channels=3, vcm=1, k=0.9, test=1)
    states, stats, L = run_gpu(hp, batches, sc.r0, params=p)
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters, k=0.9, vcm=True, test=1)
    _cppm_check(states, stats, L, ref, iters)


def test_cppm_argument_checks():
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = synth.PlaneScene(nside=8, J=1000, r0=0.1)
    hp = sc.hitpoints("cuda")
    for kw in ({"test": 2}, {"test": -1}, {"test": 1, "channels": 3, "rgb_test": 1}):
        with pytest.raises(ppm.PPMError) as e:
            ppm.Estimator(hp, sc.r0, 0.75, _params(**kw))
        assert e.value.code == ppm.PPM_EINVAL
    est = ppm.Estimator(hp, sc.r0, 0.75, _params(test=1))
    with pytest.raises(ppm.PPMError) as e:
        ppm.ppm_set_features(est.ctx, True)
    assert e.value.code == ppm.PPM_EINVAL
    est.close()
    out = torch.empty(1, device="cuda", dtype=torch.float64)
    for dof, a in ((0, 0.01), (1001, 0.01), (11, 0.0), (11, 1.0)):
        with pytest.raises(ppm.PPMError):
            ppm.ppm_chi2_critical(dof, a, out)


# ------------------------------------------ hit points traced anew ------
@pytest.mark.parametrize("mapping", [0, 1, 4])
def test_retraced_hit_points_full_trajectory(mapping):
    """SPPM-style pixels: each iteration's hit points land at a new random
    point of their pixel (ppm_set_hitpoints), statistics carried per pixel;
    the whole trajectory against the oracle on the same positions."""
    sc = synth.PlaneScene(nside=64, J=100_000, r0=0.02, step=True)
    iters = 12
    hps = [sc.hitpoints_jittered(i, "cuda") for i in range(1, iters + 1)]
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    states, stats, L = run_gpu(hps[0], batches, sc.r0, params=_params(mapping=mapping), hps=hps)
    ref = O.run(hps[0].numpy(), synth.stack_numpy(batches), sc.r0, iters,
                hp_iters=[h.numpy() for h in hps])
    rep = compare(states, stats, L, ref, iters)
    assert rep.diverged <= 4, rep
    assert ref.reject.sum() > 50


def test_retrace_with_the_same_hit_points_is_bit_identical():
    sc = synth.PlaneScene(nside=40, J=50_000, r0=0.03, step=True)
    iters = 6
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    a = run_gpu(hp, batches, sc.r0)
    b = run_gpu(hp, batches, sc.r0, hps=[sc.hitpoints("cuda") for _ in range(iters)])
    for sa, sb in zip(a[0], b[0]):
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(a[2], b[2])


def test_set_hitpoints_argument_checks():
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = synth.PlaneScene(nside=8, J=1000, r0=0.1)
    hp = sc.hitpoints("cuda")
    est = ppm.Estimator(hp, sc.r0, 0.75)
    small = synth.PlaneScene(nside=7).hitpoints("cuda")
    nq = torch.zeros(hp.n, dtype=torch.int32, device="cuda")
    for args, kw in (((small.pos, small.u, small.v), {}),            # another count
                     ((hp.pos, hp.u, hp.v), {"nq": nq})):           # normals the context lacks
        with pytest.raises(ppm.PPMError) as e:
            ppm.ppm_set_hitpoints(est.ctx, *args, **kw)
        assert e.value.code == ppm.PPM_EINVAL
    est.close()


# --------------------------------------------------------- plane scenes ----
MAPPINGS = [0, 1, 2, 3, 4]


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_tiny_config_full_trajectory(mapping):
    """64x64 hit points on z=0, r0=0.02, 16 iterations of 100k photons with
    a step edge at x=0.5: the whole trajectory against the oracle."""
    sc = synth.PlaneScene(nside=64, J=100_000, r0=0.02, step=True)
    iters = 16
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    states, stats, L = run_gpu(hp, batches, sc.r0, params=_params(mapping=mapping))
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters)
    rep = compare(states, stats, L, ref, iters)
    assert rep.diverged <= 4, rep
    assert rep.max_rel_F < 1e-3
    # the method really shrinks at the edge
    assert ref.reject.sum() > 50


def test_ragged_count_and_small_radius():
    """A hit-point count that is not a multiple of the block size, radii
    smaller than the cell, hit points outside the photon square."""
    sc = synth.PlaneScene(nside=37, J=30_000, r0=0.013, step=True, lo=0.1, hi=0.9,
                          seed=synth.SEED_BASE + 7)
    iters = 6
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    states, stats, L = run_gpu(hp, batches, sc.r0, params=_params(cell_factor=2.0))
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters)
    compare(states, stats, L, ref, iters)


@pytest.mark.parametrize("mapping", MAPPINGS)
@pytest.mark.parametrize("cf", [0.5, 1.0, 4.0])
def test_cell_factor_does_not_change_results(cf, mapping):
    sc = synth.PlaneScene(nside=20, J=20_000, r0=0.05, step=True, seed=synth.SEED_BASE + 8)
    iters = 4
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    states, stats, L = run_gpu(hp, batches, sc.r0, params=_params(cell_factor=cf, mapping=mapping))
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters)
    compare(states, stats, L, ref, iters)


# ------------------------------------------------------------ box scenes ---
def _box(nh=3001, J=30_000, rgb=False, vcm=False, seed=0):
    return synth.BoxScene(nh=nh, J=J, r0=0.04, rgb=rgb, vcm=vcm, seed=synth.SEED_BASE + 20 + seed)


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_box_scene_normals_lobes_shadows(mapping):
    sc = _box()
    iters = 8
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    states, stats, L = run_gpu(hp, batches, sc.r0, params=_params(mapping=mapping))
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters)
    rep = compare(states, stats, L, ref, iters)
    assert rep.diverged <= 3


def test_box_scene_rgb_luminance_test():
    sc = _box(rgb=True, seed=1)
    iters = 5
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    states, stats, L = run_gpu(hp, batches, sc.r0, params=_params(channels=3))
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters)
    compare(states, stats, L, ref, iters)


@pytest.mark.parametrize("mapping", [0, 1, 2, 3, 4])
def test_box_scene_rgb_per_channel_test(mapping):
    """One F-test per RGB channel, reject if any rejects: every channel's
    window sums against the oracle.  Traversal 3 tests one channel and
    traversal 4 gathers one flux channel: both are refused."""
    from paper_2504_04411_gb300 import ppm
    sc = _box(rgb=True, seed=2)
    iters = 5
    hp = sc.hitpoints("cuda")
    p = _params(channels=3, rgb_test=1, mapping=mapping)
    if mapping in (3, 4):
        with pytest.raises(ppm.PPMError) as e:
            ppm.Estimator(hp, sc.r0, params=p)
        assert e.value.code == ppm.PPM_EINVAL
        return
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    states, stats, L = run_gpu(hp, batches, sc.r0, params=p)
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters, rgb_test=True)
    compare(states, stats, L, ref, iters)


@pytest.mark.parametrize("mapping", MAPPINGS)
@pytest.mark.parametrize("rgb", [False, True])
def test_box_scene_vcm_merge_weights(rgb, mapping):
    sc = _box(rgb=rgb, vcm=True, seed=3)
    iters = 5
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    p = _params(channels=3 if rgb else 1, vcm=1, k=0.9, mapping=mapping)
    if rgb and mapping == 4:          # traversal 4 gathers one flux channel
        from paper_2504_04411_gb300 import ppm
        with pytest.raises(ppm.PPMError) as e:
            ppm.Estimator(hp, sc.r0, params=p)
        assert e.value.code == ppm.PPM_EINVAL
        return
    states, stats, L = run_gpu(hp, batches, sc.r0, params=p)
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters, k=0.9, vcm=True)
    compare(states, stats, L, ref, iters)


@pytest.mark.parametrize("mapping", MAPPINGS)
@pytest.mark.parametrize("offset", [(300.25, -512.5, 77.0), (-3000.0, 1500.0, 2000.0)])
def test_translated_box_scene(offset, mapping):
    """The box scene moved far from the origin: FP32 coordinates are coarse
    there (about 2.4e-4 apart at 3000), which the cell cull's margins and the
    trimmed row ranges must cover; every pair the disk test accepts is still
    found, as the oracle's brute force says."""
    import dataclasses
    import torch
    sc = _box(seed=4)
    iters = 4
    d = torch.tensor(offset, dtype=torch.float32, device="cuda")
    hp = sc.hitpoints("cuda")
    hp = dataclasses.replace(hp, pos=(hp.pos + d).contiguous())
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    batches = [dataclasses.replace(b, pos=(b.pos + d).contiguous()) for b in batches]
    states, stats, L = run_gpu(hp, batches, sc.r0, params=_params(mapping=mapping))
    ref = O.run(hp.numpy(), synth.stack_numpy(batches), sc.r0, iters)
    rep = compare(states, stats, L, ref, iters)
    assert rep.diverged <= 3


# hit point minus photon offsets with exact FP32 values around a disk of
# radius 1/4, and the group each one must land in (annulus * 6 + sector;
# inner iff 2 rho^2 < r^2, sector k = [60k, 60(k+1)) degrees of atan2(yv, yu),
# ties as the classification rule fixes them)
_TIES = [((0.25, 0.0), 6), ((-0.25, 0.0), 9), ((0.0, 0.25), 7), ((0.0, -0.25), 10),   # d^2 == r^2: inside
         ((0.125, 0.125), 6), ((-0.125, 0.125), 8), ((-0.125, -0.125), 9),            # 2 rho^2 == r^2: outer
         ((0.125, -0.125), 11),
         ((0.125, 0.0), 0), ((-0.125, 0.0), 3), ((0.0, 0.125), 1), ((0.0, -0.125), 4),  # yv == 0 / yu == 0
         ((0.0, 0.0), 1),                                                             # the centre
         ((0.25 + 2.0 ** -20, 0.0), None), ((0.0, -0.25 - 2.0 ** -20), None)]          # just outside


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_exact_boundary_photons(mapping):
    """Photons exactly on the disk edge, the annulus boundary and the sector
    edges: every traversal puts each in the group the rule fixes (closed
    disk, boundary to the outer annulus), as the oracle does."""
    import torch
    from paper_2504_04411_gb300 import ppm
    centres = [(0.5, 0.5), (0.125, 0.875)]          # disks 0.53 apart: no shared photons
    hp = synth.HitPoints(torch.tensor([[x, y, 0.0] for x, y in centres], dtype=torch.float32).cuda(),
                         torch.tensor([[1.0, 0.0, 0.0]] * 2).cuda(), torch.tensor([[0.0, 1.0, 0.0]] * 2).cuda(),
                         None, None)
    pos = [[x - dx, y - dy, 0.0] for x, y in centres for (dx, dy), _ in _TIES]
    J = len(pos)
    ph = synth.Photons(torch.tensor(pos, dtype=torch.float32).cuda(),
                       torch.full((J,), 1.0 / J, dtype=torch.float32).cuda(), None, None, None)
    want = np.zeros(12, np.int64)
    for _, g in _TIES:
        if g is not None:
            want[g] += 1
    params = _params(mapping=mapping, alpha_f=1e-12)     # no rejection: the window keeps the counts
    states, stats, L = run_gpu(hp, [ph], 0.25, params=params)
    ref = O.run(hp.numpy(), synth.stack_numpy([ph]), 0.25, 1, alpha_f=1e-12)
    assert np.array_equal(ref.counts[0], np.stack([want, want]))
    assert np.array_equal(states[0]["counts"], np.stack([want, want]).astype(np.int32))
    assert stats[0]["pairs"] == 2 * int(want.sum())
    compare(states, stats, L, ref, 1)


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_photons_on_cell_boundaries(mapping):
    """Photons on a lattice of step 1/64 with cells of edge 0.25 (0.125 along
    x, the split edge): many photons lie exactly on cell faces along every
    axis, on the half-cell faces along x, and exactly on disk edges.  Row
    trimming and the split x cells must keep every in-disk photon: counts
    equal the oracle's exactly for every traversal."""
    import torch
    centres = [(0.5, 0.5), (0.375, 0.625), (0.7, 0.25), (0.123, 0.871), (0.9375, 0.0625)]
    hp = synth.HitPoints(torch.tensor([[x, y, 0.0] for x, y in centres], dtype=torch.float32).cuda(),
                         torch.tensor([[1.0, 0.0, 0.0]] * len(centres)).cuda(),
                         torch.tensor([[0.0, 1.0, 0.0]] * len(centres)).cuda(), None, None)
    c = np.arange(65, dtype=np.float64) / 64.0
    xx, yy = np.meshgrid(c, c, indexing="ij")
    pos = np.stack([xx.ravel(), yy.ravel(), np.zeros(xx.size)], 1).astype(np.float32)
    J = pos.shape[0]
    ph = synth.Photons(torch.from_numpy(pos).cuda(), torch.full((J,), 1.0 / J, dtype=torch.float32).cuda(),
                       None, None, None)
    params = _params(mapping=mapping, cell_factor=1.0, alpha_f=1e-12)   # cell edge 0.25 = r0
    states, stats, L = run_gpu(hp, [ph], 0.25, params=params)
    assert stats[0]["cell"] == pytest.approx(0.25)
    ref = O.run(hp.numpy(), synth.stack_numpy([ph]), 0.25, 1, alpha_f=1e-12)
    # the tested counts of the iteration sum to its pairs; a hit point the
    # test kept holds them as its window (a rejected one starts a new one:
    # the disks cut by the lattice's edge are far from uniform)
    assert stats[0]["pairs"] == int(ref.counts[0].sum())
    kept = states[0]["t"] > 0
    assert kept.sum() >= 2
    assert np.array_equal(states[0]["counts"][kept], ref.counts[0][kept].astype(np.int32))
    compare(states, stats, L, ref, 1)


# ------------------------------------------------------------ edge cases ---
def test_empty_iterations_and_single_hit_point():
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = synth.PlaneScene(nside=1, J=5000, r0=0.3, step=False)
    hp = sc.hitpoints("cuda")
    est = ppm.Estimator(hp, sc.r0)
    empty_pos = torch.empty(0, 3, device="cuda")
    empty_flux = torch.empty(0, device="cuda")
    ppm.ppm_build_grid(est.ctx, empty_pos, empty_flux, J=5000)
    ppm.ppm_gather_test_update(est.ctx, 1)
    est.it = 1
    st = est.state()
    assert int(st["t"][0]) == 1 and float(st["r"][0]) == pytest.approx(0.3)
    assert est.stats().pairs == 0
    ph = sc.photons(2, "cuda")
    est.step(ph)
    s = est.stats()
    assert s.pairs > 0 and s.iter == 2
    L = est.radiance().cpu().numpy()
    ref = O.run(hp.numpy(), synth.stack_numpy([ph]), sc.r0, 1)
    assert L[0] == pytest.approx(ref.tau[0, 0] / 2, rel=1e-5)
    est.close()


def test_no_hit_points():
    import torch
    from paper_2504_04411_gb300 import ppm
    z = torch.empty(0, 3, device="cuda")
    ctx = ppm.ppm_create(z, z, z, 0.1)
    ph = synth.PlaneScene(J=1000).photons(1, "cuda")
    ppm.ppm_build_grid(ctx, ph.pos, ph.flux, J=1000)
    ppm.ppm_gather_test_update(ctx, 1)
    ppm.ppm_radiance(ctx, torch.empty(0, device="cuda"))
    assert ppm.ppm_stats(ctx).pairs == 0
    ppm.ppm_destroy(ctx)


def test_argument_and_sequence_errors():
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = synth.PlaneScene(nside=4, J=1000)
    hp = sc.hitpoints("cuda")
    with pytest.raises(ppm.PPMError) as e:
        ppm.ppm_create(hp.pos, hp.u, hp.v, -1.0)
    assert e.value.code == ppm.PPM_EINVAL
    with pytest.raises(ppm.PPMError):
        ppm.ppm_create(hp.pos, hp.u, hp.v, 0.1, alpha=1.5)
    with pytest.raises(ppm.PPMError):
        ppm.ppm_create(hp.pos, hp.u, hp.v, 0.1, params=_params(cell_factor=0.1))
    with pytest.raises(ppm.PPMError):
        ppm.ppm_create(hp.pos, hp.u, hp.v, 0.1, params=_params(vcm=1))   # no rho / normals
    est = ppm.Estimator(hp, 0.1)
    with pytest.raises(ppm.PPMError) as e:
        ppm.ppm_gather_test_update(est.ctx, 1)          # no grid yet
    assert e.value.code == ppm.PPM_ESTATE
    ph = sc.photons(1, "cuda")
    with pytest.raises(ppm.PPMError) as e:
        ppm.ppm_build_grid(est.ctx, ph.pos, ph.flux, J=1)   # J < 2
    assert e.value.code == ppm.PPM_EINVAL
    with pytest.raises(ppm.PPMError):
        ppm.ppm_build_grid(est.ctx, ph.pos, torch.zeros(1000, 3, device="cuda"), J=1000)  # channels
    ppm.ppm_build_grid(est.ctx, ph.pos, ph.flux, J=1000)
    with pytest.raises(ppm.PPMError) as e:
        ppm.ppm_gather_test_update(est.ctx, 2)          # skipped iteration 1
    assert e.value.code == ppm.PPM_ESTATE
    ppm.ppm_gather_test_update(est.ctx, 1)
    with pytest.raises(ppm.PPMError):
        ppm.ppm_build_grid(est.ctx, ph.pos, ph.flux, J=999)  # J changed
    est.close()


def test_size_limits_are_refused():
    """Sizes beyond the documented limits are refused with PPM_EINVAL before
    any memory is touched (small real arrays stand behind the pointers)."""
    import ctypes
    import torch
    from paper_2504_04411_gb300 import ppm
    L = ppm.load()
    buf = torch.zeros(64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    out = ctypes.c_void_p()
    hp = ppm.ppm_hitpoints(1 << 31, p, p, p, None, None)            # above 2^31 - 1 hit points
    assert L.ppm_create(ctypes.byref(hp), 0.1, 0.75, None, None, ctypes.byref(out)) == ppm.PPM_EINVAL
    assert not out.value
    sc = synth.PlaneScene(nside=4, J=1000)
    est = ppm.Estimator(sc.hitpoints("cuda"), 0.1)
    ph = ppm.ppm_photons(0xfffffff1, 0xfffffff1, p, p, 1, 0, None, None, None)   # above 2^32 - 16 photons
    assert L.ppm_build_grid(est.ctx, ctypes.byref(ph)) == ppm.PPM_EINVAL
    ph = ppm.ppm_photons(-1, 1000, p, p, 1, 0, None, None, None)
    assert L.ppm_build_grid(est.ctx, ctypes.byref(ph)) == ppm.PPM_EINVAL
    assert L.ppm_iterate_host(est.ctx, ctypes.byref(ph), 1) == ppm.PPM_EINVAL
    est.close()
    assert L.ppm_sort_pairs(p, p, p, p, 0xffffffff, 8, None) == ppm.PPM_EINVAL   # n >= 2^32 - 1
    assert L.ppm_sort_pairs_noalloc(p, p, p, p, ppm.PPM_NOALLOC_MAX_PAIRS + 1, 8, None) == ppm.PPM_EINVAL
    assert L.ppm_f_critical(1, 0.01, 10, p, None) == ppm.PPM_EINVAL               # J < 2
    assert L.ppm_mlp_forward(p, p, -1, p, None) == ppm.PPM_EINVAL


def test_deterministic_and_resumable():
    """Two runs give bitwise-identical state; a context resumed from a
    checkpoint continues exactly like the straight run."""
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = _box(nh=2000, J=20000, seed=5)
    hp = sc.hitpoints("cuda")
    batches = [sc.photons(i, "cuda") for i in range(1, 7)]
    runs = []
    for _ in range(2):
        est = ppm.Estimator(hp, sc.r0)
        for ph in batches:
            est.step(ph)
        runs.append({k: v.cpu() for k, v in est.state().items()})
        est.close()
    for k in runs[0]:
        assert torch.equal(runs[0][k], runs[1][k]), k
    est = ppm.Estimator(hp, sc.r0)
    for ph in batches[:3]:
        est.step(ph)
    ck = est.state()
    est.close()
    est2 = ppm.Estimator(hp, sc.r0)
    ppm.ppm_set_state(est2.ctx, **ck)
    ppm.ppm_set_iteration(est2.ctx, 3)
    est2.it = 3
    for ph in batches[3:]:
        est2.step(ph)
    fin = {k: v.cpu() for k, v in est2.state().items()}
    est2.close()
    for k in fin:
        assert torch.equal(fin[k], runs[0][k]), k


# -------------------------------------------- full size, sampled outputs ---
@pytest.mark.parametrize("mapping", MAPPINGS)
def test_frame_config_full_size_sampled(mapping):
    """1920x1080 hit points on three faces, 2M photons per iteration, the
    launch configuration the benchmark times; 2 iterations; 3000 random hit
    points checked against the oracle."""
    import torch
    sc = synth.BoxScene()
    hp = sc.hitpoints("cuda")
    iters = 2
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    from paper_2504_04411_gb300 import ppm
    est = ppm.Estimator(hp, sc.r0, params=_params(mapping=mapping))
    sts = []
    for ph in batches:
        est.step(ph)
        sts.append({k: v.cpu().numpy() for k, v in est.state().items()})
        assert est.stats().flags == 0
    L = est.radiance().cpu().numpy()
    est.close()
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(hp.n, 3000, replace=False))
    sub = {k: v[idx] for k, v in hp.numpy().items()}
    ref = O.run(sub, synth.stack_numpy(batches), sc.r0, iters)
    sub_states = [{k: v[idx] for k, v in s.items()} for s in sts]
    rep = compare(sub_states, [{"pairs": 0, "flags": 0}] * iters, L[idx], ref, iters,
                  check_pairs=False)
    assert rep.diverged <= 3
    torch.cuda.synchronize()


def test_vcm_merge_scale_full_size_sampled():
    """3840x2160 hit points on three faces, 16M RGB light vertices per
    iteration with log-normal MIS pdf ratios and cosine-distributed incoming
    directions, r0 = 0.0026 (0.3% of the scene's bounding radius), k = 0.9:
    the VCM+ merge configuration at full size, 2 iterations, 1000 random hit
    points against the oracle."""
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = synth.BoxScene(nh=3840 * 2160, J=16_000_000, r0=0.0026, rgb=True, vcm=True,
                        seed=synth.SEED_BASE + 5)
    hp = sc.hitpoints("cuda")
    iters = 2
    batches = [sc.photons(i, "cuda") for i in range(1, iters + 1)]
    p = _params(channels=3, vcm=1, k=0.9)
    est = ppm.Estimator(hp, sc.r0, params=p)
    sts = []
    for ph in batches:
        est.step(ph)
        sts.append({k: v.cpu().numpy() for k, v in est.state().items()})
        assert est.stats().flags == 0
    L = est.radiance().cpu().numpy()
    est.close()
    rng = np.random.default_rng(12)
    idx = np.sort(rng.choice(hp.n, 1000, replace=False))
    sub = {k: v[idx] for k, v in hp.numpy().items()}
    ref = O.run(sub, synth.stack_numpy(batches), sc.r0, iters, k=0.9, vcm=True)
    sub_states = [{k: v[idx] for k, v in s.items()} for s in sts]
    rep = compare(sub_states, [{"pairs": 0, "flags": 0}] * iters, L[idx], ref, iters, check_pairs=False)
    assert rep.diverged <= 3
    assert ref.pairs.sum() > 50_000
    torch.cuda.synchronize()
