"""GPU parity of Top-K (ORDER BY key LIMIT K, Sec. III-A) against the CPU
oracle, bit-exact: the same K row-ids and key bits in the same order.

Small and medium sizes compare element by element with the oracle; they span
several 4096-entry tiles, ragged tails, the direct path (N <= 2^21), the
sampled single-pass path and its fallback.  Full-size cases (N = 2^28) check
properties that fix the answer uniquely: K real input rows, distinct row-ids,
sorted, and exactly K-1 input rows strictly ahead of the last one.
"""
import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import datagen, olap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0)
    yield c
    c.close()


def _bits(a):
    a = np.asarray(a)
    return a.view(np.uint64 if a.dtype == np.int64 else np.uint32)


def _gpu_topk(ctx, keys, k, order, rowids=None, where="device"):
    if where == "device":
        dk = torch.from_numpy(keys).cuda()
        dr = None if rowids is None else torch.from_numpy(rowids.view(np.int32)).cuda()
        cnt = min(k, keys.shape[0])
        ok = torch.empty(max(cnt, 1), dtype=dk.dtype, device="cuda")
        orow = torch.empty(max(cnt, 1), dtype=torch.int32, device="cuda")
        got_k, got_r = ctx.topk(dk, k, order, rowids=dr, out_keys=ok, out_rowids=orow)
        return got_k.cpu().numpy(), got_r.cpu().numpy().view(np.uint32)
    if where == "pinned":
        pk = torch.from_numpy(keys).pin_memory()
        pr = None if rowids is None else torch.from_numpy(rowids.view(np.int32)).pin_memory()
        cnt = min(k, keys.shape[0])
        ok = torch.empty(max(cnt, 1), dtype=pk.dtype).pin_memory()
        orow = torch.empty(max(cnt, 1), dtype=torch.int32).pin_memory()
        got_k, got_r = ctx.topk(pk, k, order, rowids=pr, out_keys=ok, out_rowids=orow)
        return got_k.numpy(), got_r.numpy().view(np.uint32)
    got_k, got_r = ctx.topk(keys, k, order, rowids=rowids)
    return got_k, got_r


def _check(ctx, keys, k, order, rowids=None, where="device"):
    gk, gr = _gpu_topk(ctx, keys, k, order, rowids, where)
    ok, orow = oracle.topk(keys, k, order, rowids)
    assert gr.shape == orow.shape
    np.testing.assert_array_equal(gr, orow)
    np.testing.assert_array_equal(_bits(gk), _bits(ok))


SIZES = [1, 2, 31, 32, 33, 1000, 4095, 4096, 4097, 65537, 1 << 20]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kt", ["i64", "f32"])
def test_small_sizes_all_k(ctx, n, kt):
    keys = datagen.topk_keys(n, "uniform", kt, seed=n)
    for k in sorted({1, 10, 100, 1000, 4096, 4097, n - 1, n, n + 1}):
        if k < 1:
            continue
        for order in (olap.DESC, olap.ASC):
            _check(ctx, keys, k, order)


@pytest.mark.parametrize("dist", ["uniform", "ascending", "dup1024"])
@pytest.mark.parametrize("kt", ["i64", "f32"])
@pytest.mark.parametrize("n", [100_000, (1 << 21) + 3, 3_000_001])
def test_distributions(ctx, dist, kt, n):
    keys = datagen.topk_keys(n, dist, kt, seed=7)
    for k in (1, 10, 1000, 5000):
        _check(ctx, keys, k, olap.DESC)
    _check(ctx, keys, 100, olap.ASC)


@pytest.mark.parametrize("n", [4097, (1 << 21) + 17, 5_000_000])
def test_explicit_rowids_with_duplicates(ctx, n):
    keys = datagen.topk_keys(n, "dup1024", "i64", seed=3)
    rowids = (datagen.splitmix64(77, n) >> np.uint64(40)).astype(np.uint32)   # many repeats
    for k in (1, 100, 4096, 20000):
        _check(ctx, keys, k, olap.DESC, rowids)
        _check(ctx, keys, k, olap.ASC, rowids)


def test_large_k_merge_path(ctx):
    n = 3_000_000
    keys = datagen.topk_keys(n, "uniform", "i64", seed=11)
    for k in (4097, 100_000, 262_144):
        _check(ctx, keys, k, olap.DESC)
    f = datagen.topk_keys(n, "dup1024", "f32", seed=11)
    _check(ctx, f, 100_000, olap.ASC)


def test_all_equal_keys_fallback(ctx):
    # every key equal: the sampled threshold admits all N rows, more than the
    # candidate buffer holds, so the selection falls back to the full input.
    n = 4_000_000
    keys = np.full(n, -5, dtype=np.int64)
    _check(ctx, keys, 100, olap.DESC)
    _check(ctx, keys, 5000, olap.ASC)


def test_float_specials(ctx):
    from tests.test_oracle_topk import f32_specials
    bits, _ = f32_specials()
    rng = np.random.default_rng(1)
    for n in (7, 1000, 70_000):
        keys = bits[rng.integers(0, len(bits), n)].view(np.float32)
        for k in (1, 5, n // 2, n):
            _check(ctx, keys, k, olap.DESC)
            _check(ctx, keys, k, olap.ASC)


def test_int64_extremes(ctx):
    ext = np.array([-(1 << 63), (1 << 63) - 1, 0, -1, 1], dtype=np.int64)
    rng = np.random.default_rng(2)
    keys = ext[rng.integers(0, len(ext), 50_000)]
    for k in (1, 3, 10_000, 50_000):
        _check(ctx, keys, k, olap.DESC)
        _check(ctx, keys, k, olap.ASC)


@pytest.mark.parametrize("where", ["pinned", "pageable"])
def test_host_memory_kinds(ctx, where):
    n = 3_000_000
    keys = datagen.topk_keys(n, "uniform", "i64", seed=5)
    rowids = datagen.identity_rowids(n)[::-1].copy()
    _check(ctx, keys, 100, olap.DESC, rowids, where=where)
    f = datagen.topk_keys(n, "uniform", "f32", seed=5)
    _check(ctx, f, 1000, olap.ASC, None, where=where)


def test_empty_and_zero_k(ctx):
    e = np.zeros(0, dtype=np.int64)
    gk, gr = ctx.topk(e, 10)
    assert gr.shape == (0,)
    gk, gr = ctx.topk(np.arange(10, dtype=np.int64), 0)
    assert gr.shape == (0,)


def test_unaligned_device_pointer(ctx):
    # keys starting 8 bytes past a 16-byte boundary: scalar head, vector body
    n = (1 << 21) + 1001
    keys = datagen.topk_keys(n + 1, "uniform", "i64", seed=9)
    dk = torch.from_numpy(keys).cuda()[1:]
    ok = torch.empty(100, dtype=torch.int64, device="cuda")
    orow = torch.empty(100, dtype=torch.int32, device="cuda")
    ctx.topk(dk, 100, olap.DESC, out_keys=ok, out_rowids=orow)
    wk, wr = oracle.topk(keys[1:], 100, olap.DESC)
    np.testing.assert_array_equal(orow.cpu().numpy().view(np.uint32), wr)
    np.testing.assert_array_equal(ok.cpu().numpy(), wk)


@pytest.mark.parametrize("kt", ["i64", "f32"])
def test_filter_flavours_agree(ctx, kt):
    """The register-load (default) and bulk-copy streaming passes give the same bits."""
    regs = olap.Context(0, topk_filter=olap.FILTER_BULK)
    try:
        for n, dist, k in (((1 << 21) + 5, "uniform", 100), (6_000_011, "dup1024", 3000),
                           (4_194_304, "ascending", 10)):
            keys = datagen.topk_keys(n, dist, kt, seed=n)
            wk, wr = oracle.topk(keys, k, olap.DESC)
            for c in (ctx, regs):
                gk, gr = _gpu_topk(c, keys, k, olap.DESC)
                np.testing.assert_array_equal(gr, wr)
                np.testing.assert_array_equal(_bits(gk), _bits(wk))
                info = c.topk_info()
                assert info["path"] in (1, 2) and info["candidates"] >= k
    finally:
        regs.close()


def test_golden_fixtures(ctx):
    from tests.golden import make_golden
    for case in make_golden.TOPK_CASES:
        keys = make_golden.topk_input(case)
        want = make_golden.read_topk(case["name"])
        gk, gr = _gpu_topk(ctx, keys, case["k"], case["order"])
        assert gr.tolist() == want["rowids"]
        assert _bits(gk).tolist() == want["key_bits"]


def test_async_matches_blocking_and_status(ctx):
    n = 5_000_000
    keys = datagen.topk_keys(n, "uniform", "f32", seed=21)
    dk = torch.from_numpy(keys).cuda()
    ok = torch.empty(1000, dtype=torch.float32, device="cuda")
    orow = torch.empty(1000, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ctx.topk_async(dk, 1000, olap.DESC, ok, orow, dev_status=status)
    ctx.sync()
    assert int(status.item()) == olap.OK
    wk, wr = oracle.topk(keys, 1000, olap.DESC)
    np.testing.assert_array_equal(orow.cpu().numpy().view(np.uint32), wr)
    np.testing.assert_array_equal(_bits(ok.cpu().numpy()), _bits(wk))


# ---------------------------------------------------------------------------
# Full size: N = 2^28, the configuration the benchmark times.
# ---------------------------------------------------------------------------

def _total_order_i32(bits_u32):
    """A signed int32 key that sorts float32 bit patterns by IEEE totalOrder
    (negative patterns have their 31 magnitude bits flipped)."""
    x = bits_u32.view(np.int32)
    return x ^ ((x >> 31) & np.int32(0x7FFFFFFF))


def test_kernel_timing_events(ctx):
    # per-kernel CUDA events: each kernel of the sampled path is timed, the
    # results are unchanged, and the direct path reports no filter kernel
    keys = datagen.topk_keys(1 << 24, "uniform", "i64", seed=31)
    dk = torch.from_numpy(keys).cuda()
    ok = torch.empty(100, dtype=dk.dtype, device="cuda")
    orow = torch.empty(100, dtype=torch.int32, device="cuda")
    ctx.time_kernels(True)
    try:
        ctx.topk_async(dk, 100, olap.DESC, ok, orow)
        t = ctx.kernel_ms()
        assert t["topk_prepare_ms"] > 0 and t["topk_filter_ms"] > 0 and t["topk_select_ms"] > 0
        assert t["join_probe_ms"] == -1.0
        wk, wr = oracle.topk(keys, 100, olap.DESC)
        np.testing.assert_array_equal(orow.cpu().numpy().view(np.uint32), wr)
        small = dk[:100_000]
        ctx.topk_async(small, 100, olap.DESC, ok, orow)
        t = ctx.kernel_ms()
        assert t["topk_filter_ms"] == -1.0 and t["topk_select_ms"] > 0
    finally:
        ctx.time_kernels(False)


def test_total_order_key_matches_fixture():
    from tests.test_oracle_topk import f32_specials
    bits, _ = f32_specials()
    k = _total_order_i32(bits)
    assert np.all(k[1:] > k[:-1])


def _rank_dev(t):
    """A signed integer per key, in the keys' total order, on the device:
    int64 as is; float32 bits mapped like ``_total_order_i32``."""
    if t.dtype == torch.int64:
        return t
    x = t.view(torch.int32)
    return (x ^ ((x >> 31) & 0x7FFFFFFF)).to(torch.int64)


def _full_size_properties(dk, k, order, ok, orow, reversed_rowids=False):
    """Properties that fix the Top-K of a full-size column uniquely (checked
    on the device): K distinct real input rows with their own key bits, in
    (key, row-id) order, and exactly K-1 rows of the whole column strictly
    ahead of the last one.  Row-ids are the index, or n-1-index when the
    caller passed reversed row-ids."""
    n = dk.numel()
    rid = orow.to(torch.int64) & 0xFFFFFFFF
    assert rid.numel() == k and bool((rid < n).all())
    idx = (n - 1 - rid) if reversed_rowids else rid
    assert torch.unique(idx).numel() == k                                   # distinct rows
    ibits = torch.int64 if dk.dtype == torch.int64 else torch.int32
    assert torch.equal(dk[idx].view(ibits), ok.view(ibits))                 # real input rows
    ko = _rank_dev(ok)
    pk, nk, pr, nr = ko[:-1], ko[1:], rid[:-1], rid[1:]
    better = (pk > nk) if order == olap.DESC else (pk < nk)
    assert bool((better | ((pk == nk) & (pr < nr))).all())                  # sorted, ties by row-id
    lk, lr = ko[-1], rid[-1]
    ahead = 0
    step = 1 << 26
    for s0 in range(0, n, step):
        blk = _rank_dev(dk[s0:s0 + step])
        rows = torch.arange(s0, min(n, s0 + step), dtype=torch.int64, device=dk.device)
        if reversed_rowids:
            rows = n - 1 - rows
        b = (blk > lk) if order == olap.DESC else (blk < lk)
        ahead += int((b | ((blk == lk) & (rows < lr))).sum().item())
    assert ahead == k - 1


FULL_CELLS = [(kt, dist) for kt in ("i64", "f32") for dist in ("uniform", "ascending", "dup1024")]


@pytest.mark.parametrize("kt,dist", FULL_CELLS)
def test_full_size_2p28(ctx, kt, dist):
    """Every Top-K-at-scale cell: N = 2^28 keys of {int64, float32} x
    {uniform, ascending, 1024 distinct} x K in {10, 1000, 100000}, DESC (and
    ASC at K = 1000), device resident, the call the benchmark times."""
    n = 1 << 28
    dk = torch.from_numpy(datagen.topk_keys(n, dist, kt, seed=1)).cuda()
    for k in (10, 1000, 100_000):
        ok = torch.empty(k, dtype=dk.dtype, device="cuda")
        orow = torch.empty(k, dtype=torch.int32, device="cuda")
        for order in (olap.DESC, olap.ASC) if k == 1000 else (olap.DESC,):
            ctx.topk(dk, k, order, out_keys=ok, out_rowids=orow)
            _full_size_properties(dk, k, order, ok, orow)
            if dist == "ascending":                                        # closed form
                want = np.arange(n - 1, n - 1 - k, -1) if order == olap.DESC else np.arange(k)
                np.testing.assert_array_equal(orow.cpu().numpy().view(np.uint32).astype(np.int64), want)
    del dk
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kt", ["i64", "f32"])
def test_full_size_explicit_rowids(ctx, kt):
    """2^28 keys with 1024 distinct values and explicit u32 row-ids n-1..0, so
    the row-id tie-break runs against the index order inside every tie group."""
    n = 1 << 28
    dk = torch.from_numpy(datagen.topk_keys(n, "dup1024", kt, seed=1)).cuda()
    dr = torch.arange(n - 1, -1, -1, dtype=torch.int64, device="cuda").to(torch.int32)
    for k, order in ((1000, olap.DESC), (1000, olap.ASC), (100_000, olap.DESC)):
        ok = torch.empty(k, dtype=dk.dtype, device="cuda")
        orow = torch.empty(k, dtype=torch.int32, device="cuda")
        ctx.topk(dk, k, order, rowids=dr, out_keys=ok, out_rowids=orow)
        _full_size_properties(dk, k, order, ok, orow, reversed_rowids=True)
    del dk, dr
    torch.cuda.empty_cache()
