"""Pins for the Top-K oracle (Sec. III-A: LIMIT-based Top-K returning pointers).

The oracle is checked against things other than itself: exhaustive brute
force (repeated best-pick) on tiny inputs, IEEE totalOrder's listed special
values, invariants that define Top-K, closed forms of structured inputs, and
Python's own sort as a library special case.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import datagen

I64_MIN = -(1 << 63)
I64_MAX = (1 << 63) - 1
HERE = os.path.dirname(os.path.abspath(__file__))


def f32_specials():
    bits, names = [], []
    with open(os.path.join(HERE, "golden", "f32_total_order.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            b, name = line.split(None, 1)
            bits.append(int(b, 16))
            names.append(name.strip())
    return np.array(bits, dtype=np.uint32), names


def brute_topk(ranks, rowids, k, desc):
    """Repeated best-pick: O(n*k) selection on (rank, row-id) with Python ints."""
    rem = list(range(len(ranks)))
    out = []
    for _ in range(min(k, len(ranks))):
        best = rem[0]
        for i in rem[1:]:
            ki, kb = ranks[i], ranks[best]
            if (ki > kb if desc else ki < kb) or (ki == kb and rowids[i] < rowids[best]):
                best = i
        out.append(best)
        rem.remove(best)
    return out


@pytest.mark.parametrize("alphabet,nmax", [((-1, 0, 1), 6), ((I64_MIN, -1, 0, I64_MAX), 5)])
def test_exhaustive_small_i64(alphabet, nmax):
    for n in range(0, nmax + 1):
        for seq in itertools.product(alphabet, repeat=n):
            keys = np.array(seq, dtype=np.int64)
            for rowids in (None, np.arange(n, dtype=np.uint32)[::-1].copy() + 7):
                rid = list(range(n)) if rowids is None else [int(r) for r in rowids]
                for desc in (False, True):
                    for k in range(0, n + 2):
                        ok, orow = oracle.topk(keys, k, oracle.DESC if desc else oracle.ASC, rowids)
                        want = brute_topk(list(seq), rid, k, desc)
                        assert [int(x) for x in orow] == [rid[i] for i in want], (seq, k, desc)
                        assert [int(x) for x in ok] == [seq[i] for i in want]


def test_f32_total_order_comparator():
    bits, names = f32_specials()
    for i, j in itertools.product(range(len(bits)), repeat=2):
        assert oracle.f32_total_below(bits[i], bits[j]) == (i < j), (names[i], names[j])


def test_f32_specials_brute():
    bits, _ = f32_specials()
    rank = {int(b): i for i, b in enumerate(bits)}
    rng = np.random.default_rng(5)
    cases = [list(p) for p in itertools.product(range(len(bits)), repeat=2)]
    cases += [list(rng.integers(0, len(bits), size=int(rng.integers(3, 12)))) for _ in range(300)]
    for idx in cases:
        b = bits[idx]
        keys = b.view(np.float32)
        n = len(idx)
        for desc in (False, True):
            for k in (0, 1, 2, n // 2, n, n + 1):
                ok, orow = oracle.topk(keys, k, oracle.DESC if desc else oracle.ASC)
                want = brute_topk([rank[int(x)] for x in b], list(range(n)), k, desc)
                assert [int(x) for x in orow] == want
                assert ok.view(np.uint32).tolist() == [int(b[i]) for i in want]  # raw bits kept


def _check_invariants(keys, rowids, k, desc, ok, orow, rank_of):
    n = keys.shape[0]
    cnt = min(k, n)
    assert ok.shape[0] == cnt and orow.shape[0] == cnt
    rid = np.arange(n, dtype=np.uint32) if rowids is None else rowids
    sign = -1 if desc else 1
    comp = [(sign * rank_of(keys[i]), int(rid[i])) for i in range(n)]
    out = [(sign * rank_of(ok[j]), int(orow[j])) for j in range(cnt)]
    assert out == sorted(out)                                  # ordered
    if cnt:
        assert sum(1 for c in comp if c < out[-1]) == cnt - 1  # domination
    # multiset: selected + unselected = input
    from collections import Counter
    assert not (Counter(out) - Counter(comp))


@pytest.mark.parametrize("dist", ["uniform", "ascending", "dup1024"])
@pytest.mark.parametrize("key_type", ["i64", "f32"])
def test_invariants_medium(dist, key_type):
    n = 3000
    keys = datagen.topk_keys(n, dist, key_type, seed=1)
    if key_type == "i64":
        rank_of = int
    else:
        # rank by IEEE totalOrder through the comparator already pinned above
        import functools
        order = sorted(set(keys.view(np.uint32).tolist()),
                       key=functools.cmp_to_key(lambda a, b: -1 if oracle.f32_total_below(a, b)
                                                else (1 if oracle.f32_total_below(b, a) else 0)))
        pos = {b: i for i, b in enumerate(order)}
        rank_of = lambda x: pos[int(np.float32(x).view(np.uint32))]
    rowids = datagen.splitmix64(99, n).astype(np.uint32) >> np.uint32(20)   # duplicates allowed
    for k in (1, 10, 100, n, n + 5):
        for desc in (False, True):
            for rid in (None, rowids):
                ok, orow = oracle.topk(keys, k, oracle.DESC if desc else oracle.ASC, rid)
                _check_invariants(keys, rid, k, desc, ok, orow, rank_of)


def test_closed_form_ascending():
    for n in (1, 7, 1000, 1 << 16):
        for kt in ("i64", "f32"):
            keys = datagen.topk_keys(n, "ascending", kt)
            for k in (1, 10, 100, n):
                _, desc = oracle.topk(keys, k, oracle.DESC)
                _, asc = oracle.topk(keys, k, oracle.ASC)
                c = min(k, n)
                assert desc.tolist() == list(range(n - 1, n - 1 - c, -1))
                assert asc.tolist() == list(range(c))


def test_closed_form_heavy_duplicates():
    n = 1 << 15
    keys = datagen.topk_keys(n, "dup1024", "i64", seed=2)
    top = np.flatnonzero(keys == keys.max())
    bot = np.flatnonzero(keys == keys.min())
    for k in (1, 5, min(len(top), len(bot))):
        _, orow = oracle.topk(keys, k, oracle.DESC)
        assert orow.tolist() == top[:k].tolist()
        _, orow = oracle.topk(keys, k, oracle.ASC)
        assert orow.tolist() == bot[:k].tolist()


def test_library_sort_special_case():
    # K >= N reduces Top-K to a full ORDER BY; compare with Python's sort.
    n = 5000
    keys = datagen.topk_keys(n, "uniform", "i64", seed=3)
    keys[::7] = keys[3]                                      # ties
    rows = list(zip(keys.tolist(), range(n)))
    ok, orow = oracle.topk(keys, n, oracle.DESC)
    want = sorted(rows, key=lambda t: (-t[0], t[1]))
    assert orow.tolist() == [r for _, r in want]
    ok, orow = oracle.topk(keys, n + 3, oracle.ASC)
    want = sorted(rows)
    assert orow.tolist() == [r for _, r in want]
    # partial case against numpy's lexsort (a different library routine)
    for k in (1, 64, 777):
        _, orow = oracle.topk(keys, k, oracle.ASC)
        assert orow.tolist() == np.lexsort((np.arange(n), keys))[:k].tolist()


def test_empty_and_zero_k():
    e = np.zeros(0, dtype=np.int64)
    assert oracle.topk(e, 5)[1].shape == (0,)
    assert oracle.topk(np.arange(5, dtype=np.int64), 0)[1].shape == (0,)


def test_golden_regression():
    """tests/golden/topk_*.txt were written by tests/golden/make_golden.py from
    the oracle; they freeze the small reference outputs the GPU tests reuse."""
    from tests.golden import make_golden
    for case in make_golden.TOPK_CASES:
        want = make_golden.read_topk(case["name"])
        keys = make_golden.topk_input(case)
        ok, orow = oracle.topk(keys, case["k"], case["order"])
        assert orow.tolist() == want["rowids"]
        assert ok.view(np.uint64 if ok.dtype == np.int64 else np.uint32).tolist() == want["key_bits"]
