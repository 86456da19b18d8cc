"""The stable (key, value) sort of the spatial preparation (rbfd_sort_pairs)
against numpy's stable sort: the one-block register/shared-memory bitonic sort
up to 8,192 pairs and the LSD radix sort beyond, across the power-of-two and
warp boundaries, with many equal keys (the order of equal keys is part of the
result: input order) and with keys wider than key_bits (only the low bits
order; the whole key moves with its value)."""
import numpy as np
import pytest

from paper_2107_13887_gb300 import rbfd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [1, 2, 3, 31, 32, 33, 100, 1000, 1023, 1024, 1025, 2048, 4000, 4096, 4097, 8191, 8192, 8193, 100_000]


def run(keys, vals, key_bits):
    dev = torch.device("cuda", 0)
    k = torch.from_numpy(keys.view(np.int32)).to(dev)
    v = torch.from_numpy(vals.view(np.int32)).to(dev)
    rbfd.sort_pairs(k, v, key_bits)
    return k.cpu().numpy().view(np.uint32), v.cpu().numpy().view(np.uint32)


def expect(keys, vals, key_bits):
    mask = np.uint32(0xFFFFFFFF if key_bits == 32 else (1 << key_bits) - 1)
    perm = np.argsort(keys & mask, kind="stable")
    return keys[perm], vals[perm]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kind", ["wide", "few_distinct", "sorted_desc"])
def test_sort_pairs_matches_stable_sort(n, kind):
    rng = np.random.default_rng(n * 7 + len(kind))
    if kind == "wide":
        keys = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    elif kind == "few_distinct":
        keys = rng.integers(0, 5, n).astype(np.uint32)
    else:
        keys = np.arange(n, 0, -1, dtype=np.uint32) // 3  # descending runs of equal keys
    vals = rng.permutation(n).astype(np.uint32)
    for key_bits in (32, 24, 3):
        got_k, got_v = run(keys.copy(), vals.copy(), key_bits)
        want_k, want_v = expect(keys, vals, key_bits)
        assert np.array_equal(got_k, want_k), f"keys differ (n={n}, {kind}, key_bits={key_bits})"
        assert np.array_equal(got_v, want_v), f"values differ (n={n}, {kind}, key_bits={key_bits})"


def test_sort_pairs_edge_arguments():
    dev = torch.device("cuda", 0)
    e = torch.empty(0, dtype=torch.int32, device=dev)
    rbfd.sort_pairs(e, e.clone(), 32)  # nothing to do
    k = torch.zeros(4, dtype=torch.int32, device=dev)
    with pytest.raises(rbfd.RbfdError) as ei:
        rbfd.sort_pairs(k, k.clone(), 0)
    assert ei.value.status == rbfd.EINVAL
    with pytest.raises(rbfd.RbfdError) as ei:
        rbfd.sort_pairs(k, k.clone(), 33)
    assert ei.value.status == rbfd.EINVAL
    with pytest.raises(ValueError):
        rbfd.sort_pairs(k.cpu(), k.clone(), 32)
