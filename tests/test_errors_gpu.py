"""Device-side problems reach the caller as error codes (through the C ABI):
a bounded wait that gives up (PPM_ETIMEOUT) and a gather that had to skip
cells (PPM_EINCOMPLETE).  Nothing here faults or hangs the GPU: the wait is
made to run out by a test-only poll limit, after which the sort's writes stay
inside their arrays and every kernel downstream of it does nothing."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_04411_gb300 import synth

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


def test_lookback_wait_that_gives_up_is_reported_as_timeout():
    """wait_limit = 1 poll: the blocks of the grid's sort stop waiting for
    their predecessors almost at once.  ppm_stats and ppm_get_state then
    return PPM_ETIMEOUT, the gather has left the state untouched, and the
    device still runs a fresh context correctly."""
    import torch
    from paper_2504_04411_gb300 import ppm
    sc = synth.PlaneScene(nside=64, J=2_000_000, r0=0.02, step=True, seed=synth.SEED_BASE + 40)
    hp = sc.hitpoints("cuda")
    ph = sc.photons(1, "cuda")
    est = ppm.Estimator(hp, sc.r0, params=_params(wait_limit=1))
    timed_out = False
    for _ in range(3):              # a wait runs out in (nearly) every build
        est.step(ph)
        try:
            est.stats()
        except ppm.PPMError as e:
            assert e.code == ppm.PPM_ETIMEOUT, e
            timed_out = True
            break
    assert timed_out, "no look-back wait ran out with a one-poll limit"
    s = ppm.ppm_iter_stats()
    rc = ppm.load().ppm_stats(est.ctx, ppm.ctypes.byref(s))
    assert rc == ppm.PPM_ETIMEOUT and (s.flags & 4)
    with pytest.raises(ppm.PPMError) as e:
        est.state()
    assert e.value.code == ppm.PPM_ETIMEOUT
    # the gather did nothing: radii and windows as created
    r = torch.empty(hp.n, device="cuda")
    t = torch.empty(hp.n, device="cuda", dtype=torch.int32)
    v = ppm.ppm_state_view(ppm._ptr(r), ppm._ptr(t), None, None, None, None, None)
    assert ppm.load().ppm_get_state(est.ctx, ppm.ctypes.byref(v)) == ppm.PPM_ETIMEOUT
    assert torch.all(r == np.float32(sc.r0)) and torch.all(t == 0)
    est.close()
    # the device and the library still work: a context with the default
    # limit gathers exactly what the oracle does
    small = synth.PlaneScene(nside=16, J=20_000, r0=0.05, step=True, seed=synth.SEED_BASE + 41)
    hp2 = small.hitpoints("cuda")
    ph2 = small.photons(1, "cuda")
    est2 = ppm.Estimator(hp2, small.r0)
    est2.step(ph2)
    st = est2.stats()
    est2.close()
    ref = O.run(hp2.numpy(), synth.stack_numpy([ph2]), small.r0, 1)
    assert st.flags == 0 and st.pairs == int(ref.pairs[0].sum())


def test_spheres_wider_than_a_hash_block_are_reported_as_incomplete():
    """Hit points 1e5 away from the origin: the cull sphere's rounding margin
    (proportional to the coordinates) spans more cells than a hash block, so
    the gather clamps the cell box and flags it; ppm_stats returns
    PPM_EINCOMPLETE with the counters filled in."""
    import torch
    from paper_2504_04411_gb300 import ppm
    n = 256
    g = torch.Generator().manual_seed(7)
    pos = torch.zeros(n, 3)
    pos[:, 0] = 1e5 + torch.rand(n, generator=g)
    pos[:, 1] = 1e5 + torch.rand(n, generator=g)
    u = torch.tensor([1.0, 0.0, 0.0]).expand(n, 3).contiguous()
    v = torch.tensor([0.0, 1.0, 0.0]).expand(n, 3).contiguous()
    hp = synth.HitPoints(pos.cuda(), u.cuda(), v.cuda(), None, None)
    J = 20_000
    ppos = torch.zeros(J, 3)
    ppos[:, 0] = 1e5 + torch.rand(J, generator=g)
    ppos[:, 1] = 1e5 + torch.rand(J, generator=g)
    ph = synth.Photons(ppos.cuda(), torch.full((J,), 1.0 / J).cuda(), None, None, None)
    est = ppm.Estimator(hp, 0.01, params=_params(cell_factor=1.0))
    est.step(ph)
    s = ppm.ppm_iter_stats()
    rc = ppm.load().ppm_stats(est.ctx, ppm.ctypes.byref(s))
    est.close()
    assert rc == ppm.PPM_EINCOMPLETE, rc
    assert s.flags & 1 and not s.flags & 4
    assert s.iter == 1 and s.candidates > 0
