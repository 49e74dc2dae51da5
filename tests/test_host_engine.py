"""The serving harness's host engine (the CPU engine the gate keeps requests
on) returns exactly what the oracle does: Top-K bit-exact, probe pairs as a
multiset.  Host code only: runs without a GPU."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import build, datagen, olap


@pytest.fixture(scope="module")
def eng():
    build.build()
    e = olap.HostEngine(threads=4)
    yield e
    e.close()


@pytest.mark.parametrize("kt,dist", [("i64", "uniform"), ("f32", "uniform"), ("i64", "dup1024"),
                                     ("f32", "ascending"), ("f64", "uniform"), ("f64", "ascending"),
                                     ("u64", "uniform"), ("i32", "dup1024"), ("u32", "uniform")])
@pytest.mark.parametrize("n", [1, 1000, 200_003])
def test_topk_matches_oracle(eng, kt, dist, n):
    keys = datagen.topk_keys(n, dist, kt, seed=n)
    for k, order in ((1, olap.DESC), (100, olap.ASC), (5000, olap.DESC)):
        cnt = min(k, n)
        ok = np.empty(max(1, cnt), dtype=keys.dtype)
        orow = np.empty(max(1, cnt), dtype=np.uint32)
        r = olap.olap_serve_request(olap.OP_TOPK, olap.key_type_of(keys), order, 0, keys.ctypes.data, None, n, k,
                                    None, 0.0, 0.0, ok.ctypes.data, orow.ctypes.data, None, 0)
        assert eng.run(r) == olap.OK and r.out_count == cnt
        wk, wr = oracle.topk(keys, k, order)
        np.testing.assert_array_equal(orow[:cnt], wr)
        np.testing.assert_array_equal(ok[:cnt].view(np.uint8), wk.view(np.uint8))


@pytest.mark.parametrize("mult,hit", [("unique", 0.9), ("mult14", 0.3)])
def test_probe_matches_oracle(eng, mult, hit):
    b = datagen.join_build(50_000, mult, seed=4)
    tid = eng.add_table(b.keys)
    p = datagen.join_probe(300_000, b, hit, "zipf", seed=4)
    need = p.expected_pairs(b)
    out = np.empty((need, 2), dtype=np.uint32)
    r = olap.olap_serve_request(olap.OP_PROBE, olap.KEY_I64, 0, tid, p.keys.ctypes.data, None, p.keys.shape[0], 0,
                                None, float(need), 0.0, None, None, out.ctypes.data, need)
    assert eng.run(r) == olap.OK and r.out_count == need
    got = np.sort((out[:, 0].astype(np.uint64) << np.uint64(32)) | out[:, 1])
    np.testing.assert_array_equal(got, oracle.join(b.keys, p.keys))


@pytest.mark.parametrize("row_bytes,off,dtype", [(108, 0, np.float64), (13, 5, np.uint32), (64, 56, np.int64)])
def test_extract_key_column(eng, row_bytes, off, dtype):
    rng = np.random.default_rng(row_bytes)
    rows = rng.integers(0, 256, (300_001, row_bytes), dtype=np.uint8)
    got = eng.extract(rows, row_bytes, off, dtype)
    w = np.dtype(dtype).itemsize
    np.testing.assert_array_equal(got.view(np.uint8).reshape(-1, w), rows[:, off:off + w])
