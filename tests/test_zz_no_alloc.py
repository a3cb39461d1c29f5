"""ppm_sort_pairs_noalloc, the sort for callers that cannot call cudaMalloc
(real-time loops, device memory owned by another allocator): through the C
ABI its output must equal ppm_sort_pairs' exactly, on two calls in a row
(the fixed scratch array keeps the previous call's contents), and sizes
beyond its fixed capacity must be refused.  Runs last so a failure here
leaves every other test already run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _pair(n, bits, seed):
    import torch
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 1 << min(bits, 14), n, dtype=np.uint64).astype(np.uint32)
    vals = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    return (torch.from_numpy(keys.view(np.int32)).cuda(), torch.from_numpy(vals.view(np.int32)).cuda())


@pytest.mark.parametrize("n,bits", [(1 << 20, 22), (300_001, 17), (5, 8)])
def test_noalloc_sort_equals_allocating_sort_twice(n, bits):
    import torch
    from paper_2504_04411_gb300 import ppm
    for call, seed in enumerate((n + 1, n + 2)):        # two calls in a row
        k, v = _pair(n, bits, seed)
        k_ref, v_ref = torch.empty_like(k), torch.empty_like(v)
        ppm.ppm_sort_pairs(k, v, k_ref, v_ref, bits)
        k_na, v_na = torch.full_like(k, -1), torch.full_like(v, -1)
        ppm.ppm_sort_pairs_noalloc(k, v, k_na, v_na, bits)
        torch.cuda.synchronize()
        assert torch.equal(k_na, k_ref), f"keys differ on call {call + 1}"
        assert torch.equal(v_na, v_ref), f"values differ on call {call + 1}"


def test_noalloc_sort_in_place_and_limit():
    import torch
    from paper_2504_04411_gb300 import ppm
    k, v = _pair(70_000, 32, 9)
    k_ref, v_ref = torch.empty_like(k), torch.empty_like(v)
    ppm.ppm_sort_pairs(k, v, k_ref, v_ref, 32)
    ppm.ppm_sort_pairs_noalloc(k, v, k, v, 32)
    assert torch.equal(k, k_ref) and torch.equal(v, v_ref)
    big = torch.zeros(ppm.PPM_NOALLOC_MAX_PAIRS + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(ppm.PPMError) as e:
        ppm.ppm_sort_pairs_noalloc(big, big, big.clone(), big.clone(), 8)
    assert e.value.code == ppm.PPM_EINVAL
