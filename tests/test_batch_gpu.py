"""Batched persistent launch (many independent problems per iteration,
replayed as a CUDA graph) through the C ABI: every problem against the
oracle, and bit-identical to the same problem run as its own context."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_04411_gb300 import synth

from parity import compare

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


def _problems():
    sizes = [(1500, 12_000), (130, 4_000), (4100, 30_000), (700, 50_000), (2600, 9_000), (1, 2_000)]
    return [synth.SquaresScene(nh=nh, J=J, n_squares=1 + i % 3, seed=synth.SEED_BASE + 300 + i)
            for i, (nh, J) in enumerate(sizes)]


def _run_batch(scenes, iters, params, cfs=None):
    import torch
    from paper_2504_04411_gb300 import ppm
    hps = [s.hitpoints("cuda") for s in scenes]
    phs = [[s.photons(i, "cuda") for s in scenes] for i in range(1, iters + 1)]
    b = ppm.Batch(hps, [s.r0 for s in scenes], [s.J for s in scenes], params=params, cell_factors=cfs)
    states, stats = [], []
    graph = []
    for it in range(iters):
        b.step(phs[it])
        states.append([{k: v.cpu().numpy() for k, v in b.state(p).items()} for p in range(len(scenes))])
        stats.append(b.stats())
        graph.append(ppm.ppm_batch_graph_ready(b.b))
    L = [b.radiance(p).cpu().numpy() for p in range(len(scenes))]
    b.close()
    torch.cuda.synchronize()
    return hps, phs, states, stats, L, graph


@pytest.mark.parametrize("mapping", [0, 1, 3, 4])
def test_batch_matches_oracle_per_problem(mapping):
    scenes = _problems()
    iters = 4
    hps, phs, states, stats, L, graph = _run_batch(scenes, iters, _params(mapping=mapping))
    assert graph == [False, True, True, True]        # captured at the 2nd iteration
    for p, sc in enumerate(scenes):
        ref = O.run(hps[p].numpy(), synth.stack_numpy([phs[i][p] for i in range(iters)]), sc.r0, iters)
        st = [states[i][p] for i in range(iters)]
        ss = [{"pairs": stats[i][p].pairs, "flags": stats[i][p].flags} for i in range(iters)]
        rep = compare(st, ss, L[p], ref, iters)
        assert rep.diverged <= 2


@pytest.mark.parametrize("mapping", [0, 1, 3, 4])
def test_batch_bit_identical_to_single_contexts(mapping):
    """Traversals 0-3 visit a hit point's photons in the same order in a
    batch as in a context, so the state is bit-identical.  Traversal 4 splits
    a cell's photons over the lanes by position, and a batch's cells can
    also hold other problems' photons (skipped): the lanes' partial sums, and
    so the rounding of the window sums, can differ.  Counts, windows, radii
    and decisions stay identical."""
    from paper_2504_04411_gb300 import ppm
    scenes = _problems()
    iters = 4
    cfs = [0.5, 1.0, 2.0, 1.0, 0.5, 1.0]
    hps, phs, states, stats, L, _ = _run_batch(scenes, iters, _params(mapping=mapping), cfs)
    exact = ("r", "t", "counts")
    for p, sc in enumerate(scenes):
        est = ppm.Estimator(hps[p], sc.r0, params=_params(mapping=mapping, cell_factor=cfs[p]))
        for i in range(iters):
            est.step(phs[i][p])
            one = {k: v.cpu().numpy() for k, v in est.state().items()}
            for k in one:
                if mapping != 4 or k in exact:
                    assert np.array_equal(one[k], states[i][p][k]), (p, i, k)
                else:
                    assert np.allclose(one[k], states[i][p][k], rtol=1e-5, atol=1e-6 * np.abs(one[k]).max()), \
                        (p, i, k)
            assert est.stats().pairs == stats[i][p].pairs
        Lc = est.radiance().cpu().numpy()
        if mapping != 4:
            assert np.array_equal(Lc, L[p])
        else:
            assert np.allclose(Lc, L[p], rtol=1e-5, atol=1e-6 * np.abs(Lc).max())
        est.close()


@pytest.mark.parametrize("tile", [128, 192, 1024])
def test_batch_tile_size_does_not_change_results(tile):
    """Larger tiles (several 64-hit-point blocks in turn, ragged ends) give
    the same state and estimate as the default tiles, bit for bit."""
    scenes = _problems()
    iters = 3
    _, _, s64, st64, L64, _ = _run_batch(scenes, iters, _params(mapping=0))
    _, _, sT, stT, LT, _ = _run_batch(scenes, iters, _params(mapping=0, tile=tile))
    for p in range(len(scenes)):
        for i in range(iters):
            for k in s64[i][p]:
                assert np.array_equal(s64[i][p][k], sT[i][p][k]), (tile, p, i, k)
            assert stT[i][p].pairs == st64[i][p].pairs
        assert np.array_equal(L64[p], LT[p])


def test_batch_rejects_bad_tile_sizes():
    from paper_2504_04411_gb300 import ppm
    scenes = _problems()[:2]
    hps = [s.hitpoints("cuda") for s in scenes]
    for tile in (-64, 32, 100, 2048):
        with pytest.raises(ppm.PPMError):
            ppm.Batch(hps, [s.r0 for s in scenes], [s.J for s in scenes], params=_params(tile=tile))


def test_batch_rejects_bad_iterations():
    from paper_2504_04411_gb300 import ppm
    scenes = _problems()[:2]
    hps = [s.hitpoints("cuda") for s in scenes]
    b = ppm.Batch(hps, [s.r0 for s in scenes], [s.J for s in scenes])
    good = [s.photons(1, "cuda") for s in scenes]
    short = synth.Photons(good[0].pos[:-1].contiguous(), good[0].flux[:-1].contiguous(),
                          good[0].nq[:-1].contiguous(), None, None)
    with pytest.raises(ppm.PPMError) as e:
        ppm.ppm_batch_iterate(b.b, [short, good[1]], 1)
    assert e.value.code == ppm.PPM_EINVAL
    with pytest.raises(ppm.PPMError) as e:
        ppm.ppm_batch_iterate(b.b, good, 2)
    assert e.value.code == ppm.PPM_ESTATE
    b.step(good)
    assert b.stats()[0].iter == 1
    b.close()


def test_batch_windows_beyond_the_initial_critical_value_table():
    """Windows longer than the 1024 window lengths tabulated at create: the
    tables grow (the graph is captured again), no window is clamped to the
    table (flags bit 1 stays clear) and the F of windows past 1024 matches
    the oracle (within the FP32 drift of 1030-iteration window sums)."""
    import torch
    from paper_2504_04411_gb300 import ppm
    iters = 1030
    # uniform photons reaching well past every disk: the null hypothesis
    # holds, and at alpha_F = 1e-9 no test rejects, so windows grow to 1030
    scenes = [synth.PlaneScene(nside=6, J=900, r0=0.1, step=False, lo=-0.3, hi=1.3,
                               seed=synth.SEED_BASE + 500 + i) for i in range(2)]
    hps = [s.hitpoints("cuda") for s in scenes]
    phs = [[s.photons(i, "cuda") for s in scenes] for i in range(1, iters + 1)]
    b = ppm.Batch(hps, [s.r0 for s in scenes], [s.J for s in scenes], params=_params(alpha_f=1e-9))
    for it in range(iters):
        b.step(phs[it])
        if it == 2:
            assert ppm.ppm_batch_graph_ready(b.b)
    stats = b.stats()
    states = [{k: v.cpu().numpy() for k, v in b.state(p).items()} for p in range(len(scenes))]
    b.close()
    torch.cuda.synchronize()
    for p, sc in enumerate(scenes):
        assert stats[p].flags == 0 and stats[p].iter == iters
        ref = O.run(hps[p].numpy(), synth.stack_numpy([ph[p] for ph in phs]),
                    sc.r0, iters, alpha_f=1e-9)
        st = states[p]
        assert np.array_equal(st["t"], ref.t) and np.array_equal(st["r"], ref.r[-1])
        assert np.all(ref.t == iters)                 # windows past the initial table
        assert np.allclose(st["F"], ref.F[-1], rtol=1e-3, atol=1e-6)
        assert np.array_equal(st["counts"], ref.counts[-1])



@pytest.mark.parametrize("mode", ["rgb", "rgb_test", "vcm_rgb", "vcm"])
@pytest.mark.parametrize("mapping", [0, 1, 3, 4])
def test_batch_rgb_and_vcm_problems_match_oracle(mode, mapping):
    """Batches of RGB problems (luminance test or one test per channel) and
    VCM+ problems (merge weights; RGB or one channel): every problem against
    the oracle, element by element.  Traversal 3 with per-channel tests and
    traversal 4 with RGB flux are refused at create."""
    from paper_2504_04411_gb300 import ppm
    rgb = mode != "vcm"
    vcm = mode.startswith("vcm")
    sizes = [(900, 12_000, 0.05), (130, 5_000, 0.08), (2100, 20_000, 0.04), (1, 3_000, 0.1)]
    scenes = [synth.BoxScene(nh=nh, J=J, r0=r0, rgb=rgb, vcm=vcm, seed=synth.SEED_BASE + 600 + i)
              for i, (nh, J, r0) in enumerate(sizes)]
    p = _params(mapping=mapping, channels=3 if rgb else 1, rgb_test=int(mode == "rgb_test"), vcm=int(vcm),
                k=0.9 if vcm else 0.7)
    if (mapping == 3 and mode == "rgb_test") or (mapping == 4 and rgb):
        hps = [s.hitpoints("cuda") for s in scenes]
        with pytest.raises(ppm.PPMError) as e:
            ppm.Batch(hps, [s.r0 for s in scenes], [s.J for s in scenes], params=p)
        assert e.value.code == ppm.PPM_EINVAL
        return
    iters = 4
    hps, phs, states, stats, L, graph = _run_batch(scenes, iters, p)
    assert graph[-1]
    for q, sc in enumerate(scenes):
        st = [s[q] for s in states]
        ss = [{"pairs": s[q].pairs, "flags": s[q].flags} for s in stats]
        ref = O.run(hps[q].numpy(), synth.stack_numpy([ph[q] for ph in phs]), sc.r0, iters,
                    rgb_test=mode == "rgb_test", vcm=vcm, k=0.9 if vcm else 0.7)
        rep = compare(st, ss, L[q], ref, iters)
        assert rep.diverged <= 2
