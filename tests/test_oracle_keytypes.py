"""Pins of the oracle's Top-K for the key types beyond int64 and float32:
float64 (the paper's key column is a double, Sec. V-A), uint64, int32 and
uint32.  float64 is ordered by IEEE 754-2019 totalOrder; the fixture
``golden/f64_total_order.txt`` lists special values in that order, written by
hand from the standard's case list.  Integer keys are checked by brute force
on small alphabets that include each type's extremes, and on larger inputs
against numpy's own sort of the same values."""
import itertools
import os

import numpy as np
import pytest

import oracle
from tests.test_oracle_topk import brute_topk

HERE = os.path.dirname(os.path.abspath(__file__))


def f64_specials():
    bits, names = [], []
    with open(os.path.join(HERE, "golden", "f64_total_order.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            b, name = line.split(None, 1)
            bits.append(int(b, 16))
            names.append(name.strip())
    return np.array(bits, dtype=np.uint64), names


def test_f64_total_order_comparator():
    bits, names = f64_specials()
    for i, j in itertools.product(range(len(bits)), repeat=2):
        assert oracle.f64_total_below(int(bits[i]), int(bits[j])) == (i < j), (names[i], names[j])


def test_f64_specials_brute():
    bits, _ = f64_specials()
    rank = {int(b): i for i, b in enumerate(bits)}
    rng = np.random.default_rng(6)
    cases = [list(p) for p in itertools.product(range(len(bits)), repeat=2)]
    cases += [list(rng.integers(0, len(bits), size=int(rng.integers(3, 12)))) for _ in range(300)]
    for idx in cases:
        b = bits[idx]
        keys = b.view(np.float64)
        n = len(idx)
        for desc in (False, True):
            for k in (0, 1, 2, n // 2, n, n + 1):
                ok, orow = oracle.topk(keys, k, oracle.DESC if desc else oracle.ASC)
                want = brute_topk([rank[int(x)] for x in b], list(range(n)), k, desc)
                assert [int(x) for x in orow] == want
                assert ok.view(np.uint64).tolist() == [int(b[i]) for i in want]   # raw bits kept


def test_f64_finite_values_against_numeric_sort():
    # without NaN and -0, totalOrder is the numeric order: numpy's stable sort pins it
    rng = np.random.default_rng(7)
    keys = np.concatenate([rng.standard_normal(3000) * 1e300, rng.standard_normal(3000) * 1e-300,
                           np.array([np.inf, -np.inf, 0.0, 5e-324, -5e-324])])
    keys[::11] = keys[3]                                     # ties
    rng.shuffle(keys)
    for order, k in ((oracle.ASC, 100), (oracle.DESC, 2500), (oracle.DESC, keys.shape[0])):
        ok, orow = oracle.topk(keys, k, order)
        perm = np.lexsort((np.arange(keys.shape[0]), keys if order == oracle.ASC else -keys))
        np.testing.assert_array_equal(orow, perm[:k])
        np.testing.assert_array_equal(ok, keys[perm[:k]])


@pytest.mark.parametrize("dtype,alphabet", [
    (np.uint64, [0, 1, 2**63 - 1, 2**63, 2**64 - 1]),
    (np.int32, [-2**31, -1, 0, 1, 2**31 - 1]),
    (np.uint32, [0, 1, 2**31 - 1, 2**31, 2**32 - 1]),
])
def test_integer_types_brute(dtype, alphabet):
    vals = np.array(alphabet, dtype=dtype)
    ranks = {int(v): i for i, v in enumerate(vals)}          # alphabet listed in value order
    for n in range(0, 6):
        for idx in itertools.product(range(len(vals)), repeat=n):
            keys = vals[list(idx)] if n else np.empty(0, dtype=dtype)
            for desc in (False, True):
                for k in (0, 1, 3, n + 1):
                    ok, orow = oracle.topk(keys, k, oracle.DESC if desc else oracle.ASC)
                    want = brute_topk([ranks[int(x)] for x in keys], list(range(n)), k, desc)
                    assert [int(x) for x in orow] == want
                    assert [int(x) for x in ok] == [int(keys[i]) for i in want]


@pytest.mark.parametrize("dtype", [np.uint64, np.int32, np.uint32])
def test_integer_types_against_numpy(dtype):
    rng = np.random.default_rng(8)
    info = np.iinfo(dtype)
    keys = rng.integers(info.min, info.max, 20_000, dtype=dtype, endpoint=True)
    keys[::7] = keys[5]
    for order, k in ((oracle.ASC, 777), (oracle.DESC, 20_000)):
        ok, orow = oracle.topk(keys, k, order)
        key_sort = keys.astype(object) if dtype == np.uint64 else keys.astype(np.int64)
        rows = sorted(range(keys.shape[0]), key=lambda i: ((key_sort[i] if order == oracle.ASC
                                                            else -key_sort[i]), i))
        assert orow.tolist() == rows[:k]
