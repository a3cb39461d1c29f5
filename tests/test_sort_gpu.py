"""The stable radix sort (the photon grid's cell sort) through the C ABI
against numpy's stable argsort: bit-exact keys and values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _sort(keys, vals, bits, inplace=False):
    import torch
    from paper_2504_04411_gb300 import ppm
    k = torch.from_numpy(keys.view(np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    if inplace:
        ppm.ppm_sort_pairs(k, v, k, v, bits)
        return k.cpu().numpy().view(np.uint32), v.cpu().numpy().view(np.uint32)
    ko, vo = torch.empty_like(k), torch.empty_like(v)
    ppm.ppm_sort_pairs(k, v, ko, vo, bits)
    assert torch.equal(k.cpu(), torch.from_numpy(keys.view(np.int32)))   # inputs untouched
    return ko.cpu().numpy().view(np.uint32), vo.cpu().numpy().view(np.uint32)


def _ref(keys, vals, bits):
    m = np.uint64((1 << bits) - 1)
    order = np.argsort(keys.astype(np.uint64) & m, kind="stable")
    return keys[order], vals[order]


@pytest.mark.parametrize("n", [0, 1, 2, 7, 2047, 2048, 2049, 100_003, 1 << 20, 3_000_001])
@pytest.mark.parametrize("bits", [8, 13, 22, 32])
def test_sort_pairs_matches_stable_argsort(n, bits):
    rng = np.random.default_rng(n * 31 + bits)
    # few distinct keys as well as random ones: stability matters
    hi = 1 << min(bits, 12) if n % 2 else (1 << bits)
    keys = rng.integers(0, hi, n, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    got_k, got_v = _sort(keys, vals, bits, inplace=(n % 3 == 0))
    ref_k, ref_v = _ref(keys, vals, bits)
    assert np.array_equal(got_k, ref_k)
    assert np.array_equal(got_v, ref_v)


def test_sort_pairs_many_tiles():
    """20M pairs, 27-bit keys (4 passes, ~9,800 tiles waiting on their
    predecessors' counts), few distinct high digits."""
    rng = np.random.default_rng(11)
    n, bits = 20_000_000, 27
    keys = (rng.integers(0, 1 << 15, n, dtype=np.uint64) << np.uint64(12)).astype(np.uint32)
    keys |= rng.integers(0, 1 << 12, n, dtype=np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    got_k, got_v = _sort(keys, vals, bits)
    ref_k, ref_v = _ref(keys, vals, bits)
    assert np.array_equal(got_k, ref_k) and np.array_equal(got_v, ref_v)


def test_sort_pairs_ignores_bits_above_width():
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 1 << 32, 50_000, dtype=np.uint64).astype(np.uint32)
    vals = rng.integers(0, 1 << 32, 50_000, dtype=np.uint64).astype(np.uint32)
    got_k, got_v = _sort(keys, vals, 10)
    ref_k, ref_v = _ref(keys, vals, 10)
    assert np.array_equal(got_k, ref_k) and np.array_equal(got_v, ref_v)


def test_sort_pairs_rejects_bad_arguments():
    import torch
    from paper_2504_04411_gb300 import ppm
    k = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(ppm.PPMError) as e:
        ppm.ppm_sort_pairs(k, k.clone(), k.clone(), k.clone(), 0)
    assert e.value.code == ppm.PPM_EINVAL
    with pytest.raises(ppm.PPMError):
        ppm.ppm_sort_pairs(k, k.clone(), k.clone(), k.clone(), 33)
