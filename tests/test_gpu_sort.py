"""The library's own prefix sum and stable radix sort (the model set-up's
surfel sort by node set, the JᵀJ pattern build, appending's compactions and
new-set sort), against their plain definitions: numpy's cumulative sum and
numpy's stable argsort of the digits the sort looks at."""
import numpy as np
import pytest

import paper_1904_13073_gb300 as sw

pytestmark = pytest.mark.gpu

TILE = 4096


@pytest.mark.parametrize("n", [0, 1, 31, TILE - 1, TILE, TILE + 1, 3 * TILE + 17, (1 << 20) + 5,
                               TILE * TILE + 123])
@pytest.mark.parametrize("inclusive", [False, True])
def test_scan_matches_cumsum(n, inclusive):
    rng = np.random.default_rng(n + 7 * inclusive)
    v = rng.integers(-1000, 1001, size=n, dtype=np.int32)
    got = sw.sw_debug_scan(v, inclusive=inclusive)
    inc = np.cumsum(v, dtype=np.int64).astype(np.int32)
    want = inc if inclusive else np.concatenate([[0], inc[:-1]]).astype(np.int32) if n else inc
    np.testing.assert_array_equal(got, want)


def test_scan_in_flag_pattern():
    # the compaction's use: 0/1 flags, exclusive positions of the flagged items
    rng = np.random.default_rng(3)
    f = (rng.random(300_001) < 0.3).astype(np.int32)
    got = sw.sw_debug_scan(f)
    np.testing.assert_array_equal(got[f == 1], np.arange(int(f.sum()), dtype=np.int32))


def _keys(kind, n, dtype, rng):
    bits = 8 * np.dtype(dtype).itemsize
    if kind == "uniform":
        return rng.integers(0, np.iinfo(dtype).max, size=n, dtype=dtype, endpoint=True)
    if kind == "few":        # many equal keys: the order among them must be kept
        return rng.integers(0, 7, size=n).astype(dtype) << dtype(bits - 8)
    if kind == "equal":
        return np.full(n, 12345, dtype)
    if kind == "sentinel":   # the appending step's found surfels sort last with ~0
        k = rng.integers(0, 1 << 16, size=n).astype(dtype)
        k[rng.random(n) < 0.4] = np.iinfo(dtype).max
        return k
    if kind == "sorted":
        return np.sort(rng.integers(0, 1 << 20, size=n).astype(dtype))
    if kind == "reversed":
        return np.sort(rng.integers(0, 1 << 20, size=n).astype(dtype))[::-1].copy()
    raise ValueError(kind)


def _expect(k, v, begin, end):
    sk = (k >> k.dtype.type(begin)) if begin else k
    if end - begin < 8 * k.dtype.itemsize:
        sk = sk & k.dtype.type((1 << (end - begin)) - 1)
    order = np.argsort(sk, kind="stable")
    return k[order], (None if v is None else v[order])


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("n", [1, 2, 100, TILE, TILE + 1, 50_000, 300_001])
@pytest.mark.parametrize("kind", ["uniform", "few", "equal", "sentinel", "sorted", "reversed"])
def test_radix_sort_pairs(dtype, n, kind):
    rng = np.random.default_rng(hash((kind, n, np.dtype(dtype).itemsize)) % 2**32)
    k = _keys(kind, n, dtype, rng)
    v = np.arange(n, dtype=np.int32)
    gk, gv = sw.sw_debug_radix_sort(k, v)
    ek, ev = _expect(k, v, 0, 8 * k.dtype.itemsize)
    np.testing.assert_array_equal(gk, ek)
    np.testing.assert_array_equal(gv, ev)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("n", [TILE - 3, 70_001])
@pytest.mark.parametrize("bits", [(4, 20), (0, 5), (3, 3), (9, 32)])
def test_radix_sort_bit_range_keys_only(dtype, n, bits):
    rng = np.random.default_rng(n + bits[0] * 100 + bits[1])
    k = _keys("uniform", n, dtype, rng)
    gk, gv = sw.sw_debug_radix_sort(k, None, *bits)
    assert gv is None
    ek, _ = _expect(k, None, *bits)
    np.testing.assert_array_equal(gk, ek)


def test_radix_sort_rejects_bad_ranges():
    k = np.arange(10, dtype=np.uint32)
    with pytest.raises(sw.SwError):
        sw.sw_debug_radix_sort(k, None, 0, 33)
    with pytest.raises(sw.SwError):
        sw.sw_debug_radix_sort(k, None, 9, 3)
    gk, _ = sw.sw_debug_radix_sort(np.zeros(0, np.uint64))
    assert gk.size == 0
