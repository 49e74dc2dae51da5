"""The serving loop (Sec. II-B gate, Sec. IV gated vs always-on): requests of
mixed kind and size arrive while others run; GPU requests are admitted into
slots under a device-memory budget and overlap on the device.  Every result
in the mix is identical to the same request run alone (through the blocking
library call) and to the oracle; the gate sends some requests to the host
engine and their results are identical too."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import datagen, olap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = olap.Context(0)
    host = olap.HostEngine(threads=8)
    builds, tables = [], []
    for t, (nb, mult) in enumerate([(200_000, "unique"), (300_000, "mult14")]):
        b = datagen.join_build(nb, mult, seed=20 + t)
        builds.append(b)
        tables.append(ctx.join_build(b.keys))
        assert host.add_table(b.keys) == t
    yield ctx, host, builds, tables
    for t in tables:
        t.free()
    host.close()
    ctx.close()


def _requests(builds, tables, count=80, seed=9, rate_per_ms=2.0):
    rng = np.random.default_rng(seed)
    arrivals = datagen.poisson_arrivals(count, rate_per_ms * 1e3, seed=seed) * 1e3
    arena = datagen.topk_keys(3_000_000, "uniform", "i64", seed=seed)
    farena = datagen.topk_keys(3_000_000, "dup1024", "f32", seed=seed)
    reqs, keep = [], []
    for i in range(count):
        if i % 2 == 0:
            n = int(np.floor(1e3 * (2e6 / 1e3) ** rng.random()))
            k = int(min(n, np.floor(10 ** (4 * rng.random()))))
            f32 = rng.random() < 0.3
            off = int(rng.integers(0, 3_000_000 - n + 1))
            keys = (farena if f32 else arena)[off:off + n]
            order = olap.DESC if rng.random() < 0.7 else olap.ASC
            ok = np.empty(max(1, k), dtype=keys.dtype)
            orow = np.empty(max(1, k), dtype=np.uint32)
            keep.append(("topk", keys, k, order, ok, orow))
            reqs.append(olap.olap_serve_request(olap.OP_TOPK, olap.key_type_of(keys), order, 0, keys.ctypes.data,
                                                None, n, k, None, 0.0, float(arrivals[i]), ok.ctypes.data,
                                                orow.ctypes.data, None, 0))
        else:
            t = int(rng.integers(0, 2))
            n = int(np.floor(1e3 * (1e6 / 1e3) ** rng.random()))
            p = datagen.join_probe(n, builds[t], float(rng.choice([0.1, 0.9])), "uniform", seed=seed * 1000 + i)
            need = p.expected_pairs(builds[t])
            out = np.empty((max(1, need), 2), dtype=np.uint32)
            keep.append(("probe", p.keys, t, need, out))
            reqs.append(olap.olap_serve_request(olap.OP_PROBE, olap.KEY_I64, 0, t, p.keys.ctypes.data, None, n, 0,
                                                tables[t].h.value, float(need), float(arrivals[i]), None, None,
                                                out.ctypes.data, need))
    return (olap.olap_serve_request * count)(*reqs), keep


def _check_results(ctx, arr, keep, builds, tables):
    for r, kp in zip(arr, keep):
        assert r.status == olap.OK
        if kp[0] == "topk":
            _, keys, k, order, ok, orow = kp
            cnt = min(k, keys.shape[0])
            wk, wr = oracle.topk(keys, k, order)
            np.testing.assert_array_equal(orow[:cnt], wr)
            np.testing.assert_array_equal(ok[:cnt].view(np.uint8), wk.view(np.uint8))
            ak, ar = ctx.topk(keys, k, order)                          # alone
            np.testing.assert_array_equal(ar, orow[:cnt])
        else:
            _, keys, t, need, out = kp
            assert r.out_count == need
            got = np.sort((out[:need, 0].astype(np.uint64) << np.uint64(32)) | out[:need, 1])
            np.testing.assert_array_equal(got, oracle.join(builds[t].keys, keys))
            alone = ctx.join_probe(tables[t], keys)
            np.testing.assert_array_equal(
                np.sort((alone[:, 0].astype(np.uint64) << np.uint64(32)) | alone[:, 1]), got)


def test_always_gpu_mix_equals_alone_and_oracle(setup):
    ctx, host, builds, tables = setup
    arr, keep = _requests(builds, tables)
    st = olap.serve(arr, olap.SERVE_ALWAYS_GPU, gpu_slots=4, mem_budget_bytes=256 << 20)
    assert st.n_failed == 0 and st.n_gpu == len(arr) and st.offload_fraction == 1.0
    assert st.peak_reserved_bytes > 0
    assert st.p50_ms <= st.p95_ms <= st.p99_ms <= st.max_ms
    assert any(r.on_gpu for r in arr)
    _check_results(ctx, arr, keep, builds, tables)


def test_gated_mix_uses_both_engines(setup):
    ctx, host, builds, tables = setup
    arr, keep = _requests(builds, tables, seed=10)
    # a gate whose break-even sits inside the request sizes: small requests
    # stay on the host engine, large ones go to the GPU
    topk_model = olap.olap_gate_model(olap.OP_TOPK, olap.CPU_NLOGN, 2e-6, 0.0, 5e-9, 0.2, 1e-7, 0.05, 0.0, 0.01,
                                      0.0, 0.0, 0.0)
    probe_model = olap.olap_gate_model(olap.OP_PROBE, olap.CPU_NM, 1e-5, 0.0, 5e-9, 0.2, 1e-7, 0.05, 1e-8, 0.01,
                                       0.0, 0.0, 0.0)
    st = olap.serve(arr, olap.SERVE_GATED, topk_model, probe_model, host, gpu_slots=3, cpu_workers=4)
    assert st.n_failed == 0
    assert 0 < st.n_gpu < len(arr) and st.n_host == len(arr) - st.n_gpu
    for r in arr:                              # the gate's choice follows the model
        w = 4.0 if (r.op == olap.OP_TOPK and r.key_type == olap.KEY_F32) else 8.0
        d = olap.gate_estimate(topk_model if r.op == olap.OP_TOPK else probe_model, r.op, r.n,
                               r.k if r.op == olap.OP_TOPK else 1.0 + r.expected_pairs / r.n,
                               w * r.n, min(r.k, r.n) if r.op == olap.OP_TOPK else r.expected_pairs,
                               w, 0.0 if r.op == olap.OP_TOPK else r.expected_pairs / r.n)
        assert bool(r.on_gpu) == bool(d.offload)
    _check_results(ctx, arr, keep, builds, tables)


def test_budget_forces_one_at_a_time(setup):
    ctx, host, builds, tables = setup
    arr, keep = _requests(builds, tables, count=16, seed=11, rate_per_ms=1000.0)
    st = olap.serve(arr, olap.SERVE_ALWAYS_GPU, gpu_slots=4, mem_budget_bytes=1, closed_loop=True)
    assert st.n_failed == 0
    spans = sorted((r.start_ms, r.done_ms) for r in arr)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-3                 # never two in flight
    _check_results(ctx, arr, keep, builds, tables)
