"""Pins for the join oracle (Sec. III-B: key-based join probe returning the
set of matched pointers).  Checked against a pure-Python nested loop, the
pair-count identity, key equality of every pair and the generator's own
record of which probes were drawn as hits."""
import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import datagen

I64_MIN = -(1 << 63)
I64_MAX = (1 << 63) - 1


def py_nested(bk, br, pk, pr):
    out = []
    for p in range(len(pk)):
        for b in range(len(bk)):
            if int(pk[p]) == int(bk[b]):
                out.append((int(pr[p]) << 32) | int(br[b]))
    return sorted(out)


@pytest.mark.parametrize("seed", range(6))
def test_against_python_nested_loop(seed):
    rng = np.random.default_rng(seed)
    alphabet = np.array([I64_MIN, I64_MAX, 0, -1, 1, 42, -7], dtype=np.int64)
    nb, npr = int(rng.integers(0, 60)), int(rng.integers(0, 80))
    bk = alphabet[rng.integers(0, len(alphabet), nb)]
    pk = alphabet[rng.integers(0, len(alphabet), npr)]
    br = rng.integers(0, 1 << 32, nb, dtype=np.uint64).astype(np.uint32)
    pr = rng.integers(0, 1 << 32, npr, dtype=np.uint64).astype(np.uint32)
    want = py_nested(bk, br, pk, pr)
    assert oracle.join(bk, pk, br, pr).tolist() == want
    assert oracle.join_nested(bk, pk, br, pr).tolist() == want
    # implicit row-ids (row-id = index)
    assert oracle.join(bk, pk).tolist() == py_nested(bk, np.arange(nb), pk, np.arange(npr))


@pytest.mark.parametrize("mult,dist,hit", [("unique", "uniform", 0.1), ("unique", "zipf", 0.9),
                                           ("mult14", "uniform", 0.9), ("mult14", "zipf", 0.1)])
def test_invariants_generated(mult, dist, hit):
    b = datagen.join_build(4000, mult, seed=5)
    p = datagen.join_probe(20000, b, hit, dist, seed=5)
    pairs = oracle.join(b.keys, p.keys, b.rowids, p.rowids)
    # count identity: sum over probes of the build multiplicity of the probe key
    vals, counts = np.unique(b.keys, return_counts=True)
    pos = np.searchsorted(vals, p.keys)
    pos = np.minimum(pos, len(vals) - 1)
    mult_of_probe = np.where(vals[pos] == p.keys, counts[pos], 0)
    assert pairs.shape[0] == int(mult_of_probe.sum())
    # every pair joins equal keys; sorted; misses emit nothing
    pr = (pairs >> np.uint64(32)).astype(np.int64)
    br = (pairs & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.array_equal(p.keys[pr], b.keys[br])
    assert np.all(pairs[1:] >= pairs[:-1])
    assert not np.any(~p.hit[pr])
    # closed form: with a unique build, one pair per generated hit
    if mult == "unique":
        assert pairs.shape[0] == int(p.hit.sum())
    # multiplicities of the generator are 1..4
    if mult == "mult14":
        assert counts.min() >= 1 and counts.max() <= 4


def test_empty_sides():
    e = np.zeros(0, dtype=np.int64)
    x = np.array([1, 2, 3], dtype=np.int64)
    assert oracle.join(e, x).shape == (0,)
    assert oracle.join(x, e).shape == (0,)


def test_golden_regression():
    from tests.golden import make_golden
    for case in make_golden.JOIN_CASES:
        b, p = make_golden.join_input(case)
        got = oracle.join(b.keys, p.keys, b.rowids, p.rowids)
        assert got.tolist() == make_golden.read_join(case["name"])
        assert got.tolist() == py_nested(b.keys, b.rowids, p.keys, p.rowids)
