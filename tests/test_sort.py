"""The builder's stable radix sort (multi-CTA onesweep passes and the one-CTA
sort) against numpy's stable argsort on the sorted bit range: ragged tile
tails, narrow last digits with junk above and below the range, skewed and
constant digits, odd and even pass counts."""
import numpy as np
import pytest

import paper_1809_04424_b300 as vr
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def expected(keys, lo, nb):
    field = (keys >> np.uint64(lo)) & np.uint64((1 << nb) - 1) if nb < 64 else keys
    return keys[np.argsort(field, kind="stable")]


def run(torch, fn, keys, lo, nb):
    dev = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    fn(dev, lo, nb)
    torch.cuda.synchronize()
    return dev.cpu().numpy().view(np.uint64)


def keyset(kind, n, seed):
    g = synth.rng(seed)
    k = g.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + g.integers(0, 2, size=n, dtype=np.uint64)
    if kind == "skew":      # 90% of keys share the low 16 bits
        m = g.random(n) < 0.9
        k[m] = (k[m] & ~np.uint64(0xffff)) | np.uint64(0x1234)
    elif kind == "const":   # one value on the sorted range: order must not move
        k = (k & ~np.uint64(0xfffff)) | np.uint64(0x5a5a5)
    elif kind == "sorted_desc":
        k = np.sort(k)[::-1].copy()
    return k


@pytest.mark.parametrize("n", [2, 4097, 8192, 8193, 50_001, 262_144, 262_145, 1_000_003])
@pytest.mark.parametrize("lo,nb", [(0, 1), (3, 5), (26, 12), (7, 17), (20, 24), (0, 64)])
def test_sort_matches_stable_argsort(torch, n, lo, nb):
    keys = keyset("random", n, 1000 + n % 97 + lo + nb)
    assert np.array_equal(run(torch, vr.vr_sort_keys, keys, lo, nb), expected(keys, lo, nb))


@pytest.mark.parametrize("n", [200_003, 300_007])   # 1024-key tiles below 2^18 keys, 4096-key above
@pytest.mark.parametrize("kind", ["skew", "const", "sorted_desc"])
@pytest.mark.parametrize("lo,nb", [(0, 16), (4, 13), (0, 20)])
def test_sort_structured_keys(torch, kind, lo, nb, n):
    keys = keyset(kind, n, 7)
    assert np.array_equal(run(torch, vr.vr_sort_keys, keys, lo, nb), expected(keys, lo, nb))


def test_sort_many_tiles(torch):
    """3.5M keys: about 850 tiles chained through the look-back, 3 passes."""
    keys = keyset("random", 3_500_000, 11)
    assert np.array_equal(run(torch, vr.vr_sort_keys, keys, 13, 21), expected(keys, 13, 21))


@pytest.mark.parametrize("n,lo,nb", [(10_000, 0, 5), (131_072, 9, 11), (70_000, 40, 24)])
def test_noalloc_sort_ignores_bits_outside_range(torch, n, lo, nb):
    keys = keyset("random", n, 5 + nb)
    assert np.array_equal(run(torch, vr.vr_sort_keys_noalloc, keys, lo, nb), expected(keys, lo, nb))


def test_sort_empty_and_single(torch):
    for n in (0, 1):
        keys = keyset("random", n, 3)
        assert np.array_equal(run(torch, vr.vr_sort_keys, keys, 0, 8), keys)
