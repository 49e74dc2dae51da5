"""Pins of the two-column Top-K oracle (ORDER BY c0, c1 LIMIT K: the ORDER BY
of Sec. V-B with a second key column): brute-force selection from the
lexicographic definition on every small input over tiny alphabets, the
reduction to the one-column oracle when either column is constant, and
numpy's lexsort (a different sort) on larger mixed-type inputs, with float32
columns in IEEE totalOrder."""
import itertools

import numpy as np
import pytest

import oracle
from tests.test_oracle_topk import f32_specials

ORDERS = [(o0, o1) for o0 in (oracle.ASC, oracle.DESC) for o1 in (oracle.ASC, oracle.DESC)]


def _total_order_i64(bits_u32):
    """An int64 per float32 bit pattern, in IEEE totalOrder (negative patterns
    have their 31 magnitude bits flipped)."""
    x = bits_u32.astype(np.uint32).view(np.int32).astype(np.int64)
    return np.where(x < 0, x ^ 0x7FFFFFFF, x)


def _ordinal(col):
    """An int64 per key that orders like the key type's order."""
    if col.dtype == np.float32:
        return _total_order_i64(col.view(np.uint32))
    return col.astype(np.int64)


def _brute(c0, o0, c1, o1, rowids, k):
    """Repeated best pick, from the definition: row a goes before row b when
    its c0 is better, or c0 ties and its c1 is better, or both tie and its
    row-id is smaller; 'better' is smaller for ASC, larger for DESC."""
    v0, v1 = [int(x) for x in _ordinal(c0)], [int(x) for x in _ordinal(c1)]

    def before(a, b):
        if v0[a] != v0[b]:
            return (v0[a] < v0[b]) if o0 == oracle.ASC else (v0[a] > v0[b])
        if v1[a] != v1[b]:
            return (v1[a] < v1[b]) if o1 == oracle.ASC else (v1[a] > v1[b])
        return rowids[a] < rowids[b]

    rem = list(range(len(v0)))
    out = []
    for _ in range(min(k, len(v0))):
        best = rem[0]
        for i in rem[1:]:
            if before(i, best):
                best = i
        out.append(best)
        rem.remove(best)
    return out


def _check_brute(c0, c1, rowids, k, o0, o1):
    g0, g1, gr = oracle.topk_pair(c0, o0, c1, o1, k, rowids)
    rid = np.arange(c0.shape[0], dtype=np.uint32) if rowids is None else rowids
    want = _brute(c0, o0, c1, o1, [int(x) for x in rid], k)
    assert gr.tolist() == [int(rid[i]) for i in want]
    assert g0.view(np.uint8).tobytes() == c0[want].view(np.uint8).tobytes()
    assert g1.view(np.uint8).tobytes() == c1[want].view(np.uint8).tobytes()


@pytest.mark.parametrize("o0,o1", ORDERS)
def test_exhaustive_small_int_alphabets(o0, o1):
    a0 = np.array([-1, 0, 1], dtype=np.int32)
    a1 = np.array([0, 7], dtype=np.uint32)
    for n in range(0, 5):
        for s0 in itertools.product(range(3), repeat=n):
            for s1 in itertools.product(range(2), repeat=n):
                c0, c1 = a0[list(s0)], a1[list(s1)]
                for k in range(0, n + 2):
                    _check_brute(c0, c1, None, k, o0, o1)
                if n:
                    _check_brute(c0, c1, np.arange(n, dtype=np.uint32)[::-1].copy(), n, o0, o1)


@pytest.mark.parametrize("o0,o1", ORDERS)
def test_float_specials_both_columns(o0, o1):
    bits, _ = f32_specials()
    rng = np.random.default_rng(5)
    for n in (7, 40):
        for _ in range(20):
            c0 = bits[rng.integers(0, len(bits), n)].view(np.float32)
            c1 = bits[rng.integers(0, len(bits), n)].view(np.float32)
            for k in (1, n // 2, n):
                _check_brute(c0, c1, None, k, o0, o1)


@pytest.mark.parametrize("o0,o1", ORDERS)
def test_constant_column_reduces_to_one_column(o0, o1):
    rng = np.random.default_rng(6)
    n = 5000
    x = rng.integers(-50, 50, n).astype(np.int32)
    const = np.full(n, 3, dtype=np.int32)
    rowids = rng.permutation(n).astype(np.uint32)
    for k in (1, 100, n):
        # c1 constant: the order of c0 alone
        g0, _, gr = oracle.topk_pair(x, o0, const, o1, k, rowids)
        w0, wr = oracle.topk(x, k, o0, rowids)
        np.testing.assert_array_equal(gr, wr)
        np.testing.assert_array_equal(g0, w0)
        # c0 constant: the order of c1 alone
        _, g1, gr = oracle.topk_pair(const, o0, x, o1, k, rowids)
        w1, wr = oracle.topk(x, k, o1, rowids)
        np.testing.assert_array_equal(gr, wr)
        np.testing.assert_array_equal(g1, w1)


@pytest.mark.parametrize("t0,t1", [(np.int32, np.int32), (np.float32, np.int32), (np.uint32, np.float32)])
@pytest.mark.parametrize("o0,o1", ORDERS)
def test_larger_inputs_against_lexsort(t0, t1, o0, o1):
    rng = np.random.default_rng(7)
    n = 60_000

    def col(t):
        if t == np.float32:
            return rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32).view(np.float32)
        if t == np.uint32:
            return rng.integers(0, 40, n).astype(np.uint32)
        return rng.integers(-30, 30, n).astype(np.int32)

    c0, c1 = col(t0), col(t1)
    rowids = rng.integers(0, 1 << 20, n).astype(np.uint32)       # repeats allowed
    v0, v1 = _ordinal(c0), _ordinal(c1)
    if o0 == oracle.DESC:
        v0 = -v0
    if o1 == oracle.DESC:
        v1 = -v1
    idx = np.lexsort((np.arange(n), rowids, v1, v0))           # last key is the primary one
    for k in (1, 1000, n):
        g0, g1, gr = oracle.topk_pair(c0, o0, c1, o1, k, rowids)
        np.testing.assert_array_equal(gr, rowids[idx[:k]])
        np.testing.assert_array_equal(g0.view(np.uint32), c0[idx[:k]].view(np.uint32))
        np.testing.assert_array_equal(g1.view(np.uint32), c1[idx[:k]].view(np.uint32))
