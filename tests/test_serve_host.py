"""The serving loop's host side (Sec. II-B, Sec. IV), run with every request
kept on the host engine: that policy creates no device context, so the
dispatcher, the arrival schedule, the worker queue and the latency
statistics are checked here without a GPU.  Results are compared with the
oracle; the reported percentiles are recomputed from the per-request
timestamps by the nearest-rank rule."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import build, datagen, olap

KINDS = ["i64", "f32", "f64", "u64", "i32", "u32"]


@pytest.fixture(scope="module")
def eng():
    build.build()
    e = olap.HostEngine(threads=4)
    yield e
    e.close()


def _requests(eng, count, seed, rate_per_ms, closed=False):
    rng = np.random.default_rng(seed)
    arrivals = np.zeros(count) if closed else datagen.poisson_arrivals(count, rate_per_ms * 1e3, seed=seed) * 1e3
    b = datagen.join_build(40_000, "mult14", seed=seed)
    tid = eng.add_table(b.keys)
    reqs, keep = [], []
    for i in range(count):
        if i % 3 != 2:
            kt = KINDS[i % len(KINDS)]
            n = int(rng.integers(1, 60_000))
            k = int(rng.integers(1, 400))
            keys = datagen.topk_keys(n, "dup1024" if i % 2 else "uniform", kt, seed=seed * 100 + i)
            rid = (datagen.splitmix64(seed * 100 + i, n) >> np.uint64(40)).astype(np.uint32) if i % 4 == 0 else None
            order = olap.DESC if i % 5 else olap.ASC
            ok = np.empty(max(1, k), dtype=keys.dtype)
            orow = np.empty(max(1, k), dtype=np.uint32)
            keep.append(("topk", keys, rid, k, order, ok, orow))
            reqs.append(olap.olap_serve_request(olap.OP_TOPK, olap.key_type_of(keys), order, 0, keys.ctypes.data,
                                                None if rid is None else rid.ctypes.data, n, k, None, 0.0,
                                                float(arrivals[i]), ok.ctypes.data, orow.ctypes.data, None, 0))
        else:
            n = int(rng.integers(0, 80_000))
            p = datagen.join_probe(n, b, 0.6, "uniform", seed=seed * 100 + i)
            need = p.expected_pairs(b)
            out = np.empty((max(1, need), 2), dtype=np.uint32)
            keep.append(("probe", p.keys, b, need, out))
            reqs.append(olap.olap_serve_request(olap.OP_PROBE, olap.KEY_I64, 0, tid, p.keys.ctypes.data, None, n, 0,
                                                None, float(need), float(arrivals[i]), None, None,
                                                out.ctypes.data, need))
    return (olap.olap_serve_request * count)(*reqs), keep


def _nearest_rank(sorted_lat, p):
    idx = math.ceil(p / 100.0 * len(sorted_lat))
    return sorted_lat[min(max(idx - 1, 0), len(sorted_lat) - 1)]


def _check_results(arr, keep):
    for r, kp in zip(arr, keep):
        assert r.status == olap.OK and r.on_gpu == 0
        if kp[0] == "topk":
            _, keys, rid, k, order, ok, orow = kp
            cnt = min(k, keys.shape[0])
            assert r.out_count == cnt
            wk, wr = oracle.topk(keys, k, order, rid)
            np.testing.assert_array_equal(orow[:cnt], wr)
            np.testing.assert_array_equal(ok[:cnt].view(np.uint8), wk.view(np.uint8))
        else:
            _, keys, b, need, out = kp
            assert r.out_count == need
            got = np.sort((out[:need, 0].astype(np.uint64) << np.uint64(32)) | out[:need, 1])
            np.testing.assert_array_equal(got, oracle.join(b.keys, keys))


def test_open_loop_results_schedule_and_statistics(eng):
    arr, keep = _requests(eng, 60, seed=31, rate_per_ms=0.5)
    st = olap.serve(arr, olap.SERVE_ALWAYS_HOST, host=eng, cpu_workers=3)
    _check_results(arr, keep)
    assert st.n_host == len(arr) and st.n_gpu == 0 and st.n_failed == 0
    assert st.offload_fraction == 0.0 and st.peak_reserved_bytes == 0
    for r in arr:                      # nothing starts before it arrives
        assert r.start_ms >= r.arrival_ms - 1e-6 and r.done_ms >= r.start_ms
    lat = sorted(r.done_ms - r.arrival_ms for r in arr)
    for p, got in ((50, st.p50_ms), (95, st.p95_ms), (99, st.p99_ms)):
        assert got == _nearest_rank(lat, p)
    assert st.max_ms == lat[-1]
    assert math.isclose(st.mean_ms, sum(r.done_ms - r.arrival_ms for r in arr) / len(arr), rel_tol=1e-12)
    assert st.wall_ms == max(r.done_ms for r in arr)
    assert math.isclose(st.throughput_rps, len(arr) / (st.wall_ms / 1e3), rel_tol=1e-12)
    # the arrival schedule spans the trace: the run cannot end before the last arrival
    assert st.wall_ms >= max(r.arrival_ms for r in arr) - 1e-6


def test_closed_loop_latency_is_completion_time(eng):
    arr, keep = _requests(eng, 30, seed=32, rate_per_ms=1.0, closed=True)
    st = olap.serve(arr, olap.SERVE_ALWAYS_HOST, host=eng, cpu_workers=2, closed_loop=True)
    _check_results(arr, keep)
    lat = sorted(r.done_ms for r in arr)
    assert st.p99_ms == _nearest_rank(lat, 99) and st.max_ms == lat[-1]


def test_request_failures_are_reported_per_request(eng):
    b = datagen.join_build(1000, "unique", seed=33)
    tid = eng.add_table(b.keys)
    p = datagen.join_probe(5000, b, 0.9, "uniform", seed=33)
    need = p.expected_pairs(b)
    out = np.empty((need, 2), dtype=np.uint32)
    mk = lambda table_id, cap: olap.olap_serve_request(olap.OP_PROBE, olap.KEY_I64, 0, table_id, p.keys.ctypes.data,
                                                      None, 5000, 0, None, float(need), 0.0, None, None,
                                                      out.ctypes.data, cap)
    arr = (olap.olap_serve_request * 3)(mk(tid, need), mk(tid + 100, need), mk(tid, need - 1))
    st = olap.serve(arr, olap.SERVE_ALWAYS_HOST, host=eng, cpu_workers=1)
    assert [r.status for r in arr] == [olap.OK, olap.E_INVALID, olap.E_OVERFLOW]
    assert arr[0].out_count == need and arr[2].out_count == need     # overflow reports the size needed
    assert st.n_failed == 2 and st.n_host == 3


def test_serve_rejects_bad_options(eng):
    arr, _ = _requests(eng, 3, seed=34, rate_per_ms=1.0)
    with pytest.raises(olap.OlapError) as ei:
        olap.serve(arr, olap.SERVE_ALWAYS_HOST)                      # no host engine to run them
    assert ei.value.status == olap.E_INVALID
    with pytest.raises(olap.OlapError):
        olap.serve(arr, olap.SERVE_GATED, host=eng)                  # the gate needs both models
    with pytest.raises(olap.OlapError):
        olap.serve(arr, 7, host=eng)                                 # no such policy
    st = olap.serve((olap.olap_serve_request * 0)(), olap.SERVE_ALWAYS_HOST, host=eng)
    assert st.n_host == 0 and st.p99_ms == 0.0 and st.throughput_rps == 0.0


def test_engine_on_a_core_set_gives_the_same_results_and_pins_its_callers():
    """An engine created on a core set computes the same results as one that
    is not, and pins the threads that call it to that set (run in a thread of
    its own, so the test process keeps its cores)."""
    import os
    import threading
    build.build()
    cpus = sorted(os.sched_getaffinity(0))
    mine = cpus[-2:] if len(cpus) > 2 else cpus
    e = olap.HostEngine(threads=2, cpus=mine)
    seen = {}

    def work():
        arr, keep = _requests(e, 24, seed=31, rate_per_ms=1.0, closed=True)
        for r in arr:
            r.status = e.run(r)
        _check_results(arr, keep)
        seen["affinity"] = sorted(os.sched_getaffinity(0))

    t = threading.Thread(target=work)
    t.start()
    t.join()
    e.close()
    assert seen["affinity"] == mine
    assert sorted(os.sched_getaffinity(0)) == cpus          # the test's own thread is untouched
