"""Host-fed iterations (ppm_iterate_host / ppm_stats_host): the same
photons fed from host memory give bit-identical state, estimate and
counters to device-fed iterations (ppm_build_grid + ppm_gather_test_update),
with page-locked and pageable arrays, growing photon counts and the VCM+
inputs; counters of iterations older than the last two are refused."""
import dataclasses

import pytest
import torch

from paper_2504_04411_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _host(ph, pinned: bool):
    def h(t):
        if t is None:
            return None
        t = t.cpu().contiguous()
        return t.pin_memory() if pinned else t
    return dataclasses.replace(ph, pos=h(ph.pos), flux=h(ph.flux), nq=h(ph.nq), rho=h(ph.rho), wq=h(ph.wq))


def _same_state(a, b):
    for k in a:
        assert torch.equal(a[k], b[k]), k


def _run_pair(sc, batches, J, params):
    from paper_2504_04411_gb300 import ppm
    hp = sc.hitpoints("cuda")
    dev = ppm.Estimator(hp, sc.r0, 0.75, params)
    host = ppm.Estimator(hp, sc.r0, 0.75, params)
    dev_stats = []
    keep = []
    for i, ph in enumerate(batches):
        dev.step(ph, J=J)
        dev_stats.append(dev.stats())
        hph = _host(ph, pinned=(i % 3 != 2))      # every third iteration pageable
        keep.append(hph)
        it = host.step_host(hph, J=J)
        if it > 1:
            s = ppm.ppm_stats_host(host.ctx, it - 1)
            d = dev_stats[it - 2]
            assert (s.pairs, s.candidates, s.rejects, s.pairs_total, s.flags) == \
                (d.pairs, d.candidates, d.rejects, d.pairs_total, d.flags)
            assert s.r_max == d.r_max and s.cell == d.cell and s.iter == it - 1
    s = ppm.ppm_stats_host(host.ctx, host.it)
    d = dev_stats[-1]
    assert (s.pairs, s.candidates, s.rejects, s.pairs_total) == (d.pairs, d.candidates, d.rejects, d.pairs_total)
    torch.cuda.synchronize()
    _same_state(dev.state(), host.state())
    assert torch.equal(dev.radiance(), host.radiance())
    return dev, host


def test_host_fed_box_scene_bit_identical():
    from paper_2504_04411_gb300 import ppm
    sc = synth.BoxScene(nh=3001, J=30_000, r0=0.04, seed=synth.SEED_BASE + 40)
    batches = [sc.photons(i, "cuda") for i in range(1, 8)]
    dev, host = _run_pair(sc, batches, None, ppm.ppm_default_params())
    # only the last two iterations' counters are kept
    with pytest.raises(ppm.PPMError):
        ppm.ppm_stats_host(host.ctx, host.it - 2)
    with pytest.raises(ppm.PPMError):
        ppm.ppm_stats_host(host.ctx, host.it + 1)
    # out-of-sequence iteration
    with pytest.raises(ppm.PPMError):
        ph = _host(batches[0], pinned=True)
        ppm.ppm_iterate_host(host.ctx, host.it + 2, ph.pos, ph.flux, ph.pos.shape[0], nq=ph.nq)
    dev.close()
    host.close()


def test_host_fed_growing_photon_count():
    """Fewer photons than J in the first iterations, then all of them: the
    device buffers grow between iterations."""
    from paper_2504_04411_gb300 import ppm
    sc = synth.PlaneScene(nside=40, J=40_000, r0=0.03, step=True, seed=synth.SEED_BASE + 41)
    batches = []
    for i in range(1, 7):
        ph = sc.photons(i, "cuda")
        n = [5_000, 12_000, 0, 40_000, 20_000, 40_000][i - 1]
        batches.append(dataclasses.replace(ph, pos=ph.pos[:n].contiguous(), flux=ph.flux[:n].contiguous()))
    dev, host = _run_pair(sc, batches, sc.J, ppm.ppm_default_params())
    dev.close()
    host.close()


@pytest.mark.parametrize("rgb", [False, True])
def test_host_fed_vcm_inputs(rgb):
    from paper_2504_04411_gb300 import ppm
    sc = synth.BoxScene(nh=2000, J=20_000, r0=0.04, rgb=rgb, vcm=True, seed=synth.SEED_BASE + 42)
    p = ppm.ppm_default_params()
    p.channels = 3 if rgb else 1
    p.vcm = 1
    p.k = 0.9
    batches = [sc.photons(i, "cuda") for i in range(1, 5)]
    dev, host = _run_pair(sc, batches, None, p)
    dev.close()
    host.close()
