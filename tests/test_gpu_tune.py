"""Tunable kernel parameters and the autotuner: every digit width and filter
block size gives the oracle's Top-K bit for bit (sampled path, direct path,
merge path for K > 4096, sample fallback), batches created on a tuned context
stay exact, and olap_autotune returns a configuration from its candidate set
and leaves the context producing exact results."""
import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import datagen, olap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


CASES = [
    (3_000_001, "uniform", "i64", 1000),     # sampled path
    (2_500_000, "dup1024", "f32", 77),       # sampled path, heavy ties
    ((1 << 21) + 3, "uniform", "f32", 5000),  # sampled path, K above one CTA's sort (merge path)
    (1 << 20, "uniform", "i64", 9000),       # direct path, merge path
    (2_200_000, "ascending", "i64", 10),     # sampled path, adversarial order
]


@pytest.mark.parametrize("digit", [8, 10, 11, 12])
@pytest.mark.parametrize("block", [256, 1024])
def test_digit_width_and_block_size(digit, block):
    _need_gpu()
    ctx = olap.Context(0, topk_digit_bits=digit, block_threads=block)
    try:
        for n, dist, kt, k in CASES:
            keys = datagen.topk_keys(n, dist, kt, seed=n % 97)
            for order in (olap.DESC, olap.ASC):
                gk, gr = ctx.topk(torch.from_numpy(keys).cuda(), k, order)
                wk, wr = oracle.topk(keys, k, order)
                np.testing.assert_array_equal(gr, wr)
                np.testing.assert_array_equal(gk.view(np.uint8), wk.view(np.uint8))
        # all keys equal: the sample cannot separate anything
        keys = np.full(3_000_000, 5, dtype=np.int64)
        gk, gr = ctx.topk(torch.from_numpy(keys).cuda(), 100, olap.DESC)
        np.testing.assert_array_equal(gr, np.arange(100))
    finally:
        ctx.close()


@pytest.mark.parametrize("digit", [8, 11])
def test_batch_digit_width(digit):
    _need_gpu()
    ctx = olap.Context(0, topk_digit_bits=digit)
    try:
        ns = [1, 4096, 4097, 70_000, 1_000_003]
        items, keep = [], []
        for i, n in enumerate(ns):
            keys = datagen.topk_keys(n, "uniform" if i % 2 else "dup1024", "i64", seed=i)
            dk = torch.from_numpy(keys).cuda()
            k = min(1000, n)
            ok = torch.empty(k, dtype=torch.int64, device="cuda")
            orow = torch.empty(k, dtype=torch.int32, device="cuda")
            c = torch.zeros(1, dtype=torch.int64, device="cuda")
            items.append(olap.topk_item(dk, k, olap.DESC, ok, orow, c))
            keep.append((keys, k, ok, orow, dk))
        b = ctx.batch(items)
        b.run()
        ctx.sync()
        assert b.errors() == 0
        for keys, k, ok, orow, _ in keep:
            wk, wr = oracle.topk(keys, k, olap.DESC)
            np.testing.assert_array_equal(orow.cpu().numpy().view(np.uint32), wr)
        b.free()
    finally:
        ctx.close()


def test_autotune_picks_from_candidates_and_stays_exact():
    _need_gpu()
    ctx = olap.Context(0)
    try:
        r = ctx.autotune(topk_n=1 << 22, topk_k=100, join_build_n=1 << 18, join_probe_n=1 << 21,
                         join_hit_rate=0.5, reps=3)
        assert r["block_threads"] in (256, 512, 1024)
        assert r["topk_digit_bits"] in (8, 10, 11, 12)
        assert r["load_factor"] in (0.25, 0.35, 0.5, 0.7)
        assert r["join_partitions"] in (0, 1)
        assert r["join_bucket_loads"] in (olap.LOADS_L1, olap.LOADS_L2_ONLY)
        assert 0 < r["topk_ms"] <= r["topk_default_ms"]
        assert 0 < r["join_probe_ms"] <= r["join_probe_default_ms"]
        assert r["candidates"] == 6 + 4 + 16           # Top-K; join builds; join probes
        # the tuned context still returns the oracle's results
        keys = datagen.topk_keys(3_000_000, "uniform", "i64", seed=41)
        gk, gr = ctx.topk(torch.from_numpy(keys).cuda(), 100, olap.DESC)
        np.testing.assert_array_equal(gr, oracle.topk(keys, 100, olap.DESC)[1])
        b = datagen.join_build(200_000, "mult14", seed=41)
        p = datagen.join_probe(600_000, b, 0.5, "uniform", seed=41)
        t = ctx.join_build(b.keys)                  # built at the tuned load factor
        got = ctx.join_probe(t, p.keys).astype(np.uint64)
        got = np.sort((got[:, 0] << np.uint64(32)) | got[:, 1])
        np.testing.assert_array_equal(got, oracle.join(b.keys, p.keys))
        t.free()
    finally:
        ctx.close()


def test_autotune_rejects_bad_requests():
    _need_gpu()
    ctx = olap.Context(0)
    try:
        for kw in ({"join_probe_n": 10}, {"topk_n": 1 << 32}, {"join_build_n": 10, "join_hit_rate": 1.5}):
            with pytest.raises(olap.OlapError) as ei:
                ctx.autotune(**kw)
            assert ei.value.status == olap.E_INVALID
    finally:
        ctx.close()
