"""GPU parity of the hash join (Sec. III-B: key-based join probe returning the
set of matched (probe, build) row pointers) against the CPU oracle: the pair
multiset, compared sorted, bit-exact.

Small and medium sizes compare every pair.  The full-size workload (2^24
build rows, 2^28 probes, all eight cells) checks the exact pair count the
generator fixes (sum of build multiplicities over the hits), key equality and
distinctness of every pair, and the exact pairs of a sample of probe rows
against the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import datagen, olap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I64_MIN, I64_MAX = -(1 << 63), (1 << 63) - 1


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0)
    yield c
    c.close()


def packed(pairs):
    p = np.asarray(pairs, dtype=np.uint32).reshape(-1, 2).astype(np.uint64)
    return np.sort((p[:, 0] << np.uint64(32)) | p[:, 1])


def _check(ctx, bk, pk, br=None, pr=None, load=0.0, device=True):
    if device:
        t = ctx.join_build(torch.from_numpy(bk).cuda(),
                           None if br is None else torch.from_numpy(br.view(np.int32)).cuda(), load)
        dk = torch.from_numpy(pk).cuda()
        dr = None if pr is None else torch.from_numpy(pr.view(np.int32)).cuda()
        want = oracle.join(bk, pk, br, pr)
        out = torch.empty((max(1, want.shape[0]), 2), dtype=torch.int32, device="cuda")
        got = ctx.join_probe(t, dk, dr, out=out)
        got = got.cpu().numpy().view(np.uint32)
    else:
        t = ctx.join_build(bk, br, load)
        got = ctx.join_probe(t, pk, pr)
        want = oracle.join(bk, pk, br, pr)
    np.testing.assert_array_equal(packed(got), want)
    t.free()
    return want.shape[0]


@pytest.mark.parametrize("mult", ["unique", "mult14"])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
@pytest.mark.parametrize("hit", [0.1, 0.9])
def test_generated_medium(ctx, mult, dist, hit):
    b = datagen.join_build(200_003, mult, seed=11)
    p = datagen.join_probe(1_000_003, b, hit, dist, seed=11)
    cnt = _check(ctx, b.keys, p.keys)
    assert cnt == p.expected_pairs(b)


@pytest.mark.parametrize("load", [0.25, 0.5, 0.7, 0.9])
def test_load_factors(ctx, load):
    b = datagen.join_build(50_000, "mult14", seed=3)
    p = datagen.join_probe(300_000, b, 0.5, "uniform", seed=3)
    _check(ctx, b.keys, p.keys, load=load)


def test_small_and_empty(ctx):
    for nb, npr in [(0, 10), (10, 0), (1, 1), (31, 33), (1000, 4097)]:
        rng = np.random.default_rng(nb + npr)
        bk = rng.integers(-50, 50, nb).astype(np.int64)
        pk = rng.integers(-50, 50, npr).astype(np.int64)
        _check(ctx, bk, pk)


def test_extreme_keys_and_empty_marker(ctx):
    # -1 is the table's empty marker: such build rows live in the side list.
    rng = np.random.default_rng(4)
    alphabet = np.array([I64_MIN, I64_MAX, 0, -1, 1, -2], dtype=np.int64)
    bk = alphabet[rng.integers(0, len(alphabet), 3000)]
    pk = alphabet[rng.integers(0, len(alphabet), 5000)]
    _check(ctx, bk, pk)
    # all build keys -1
    _check(ctx, np.full(100, -1, dtype=np.int64), np.array([-1, 0, -1], dtype=np.int64))


def test_explicit_rowids(ctx):
    b = datagen.join_build(100_000, "mult14", seed=6)
    p = datagen.join_probe(400_000, b, 0.7, "zipf", seed=6)
    br = (datagen.splitmix64(1, b.keys.shape[0]) >> np.uint64(33)).astype(np.uint32)
    pr = (datagen.splitmix64(2, p.keys.shape[0]) >> np.uint64(33)).astype(np.uint32)
    _check(ctx, b.keys, p.keys, br, pr)


def test_heavy_build_duplicates(ctx):
    # long chains: 5000 copies of a few keys
    bk = np.repeat(np.array([7, -7, 123456789], dtype=np.int64), 5000)
    pk = np.array([7, 8, -7, 123456789, 7], dtype=np.int64)
    _check(ctx, bk, pk)


@pytest.mark.parametrize("where", ["pinned", "pageable"])
def test_host_memory(ctx, where):
    b = datagen.join_build(100_000, "unique", seed=9)
    p = datagen.join_probe(300_000, b, 0.5, "uniform", seed=9)
    if where == "pinned":
        t = ctx.join_build(torch.from_numpy(b.keys).pin_memory())
        out = torch.empty((200_000, 2), dtype=torch.int32).pin_memory()
        got = ctx.join_probe(t, torch.from_numpy(p.keys).pin_memory(), out=out).numpy().view(np.uint32)
        t.free()
        np.testing.assert_array_equal(packed(got), oracle.join(b.keys, p.keys))
    else:
        _check(ctx, b.keys, p.keys, device=False)


def test_overflow_reports_required_count(ctx):
    b = datagen.join_build(10_000, "mult14", seed=12)
    p = datagen.join_probe(50_000, b, 0.9, "uniform", seed=12)
    need = p.expected_pairs(b)
    t = ctx.join_build(b.keys)
    out = np.empty((need // 2, 2), dtype=np.uint32)
    with pytest.raises(olap.OlapError) as ei:
        ctx.join_probe(t, p.keys, out=out)
    assert ei.value.status == olap.E_OVERFLOW and str(need) in str(ei.value)
    got = ctx.join_probe(t, p.keys)            # own buffer: retried at the exact size
    assert got.shape[0] == need
    t.free()


def test_golden_fixtures(ctx):
    from tests.golden import make_golden
    for case in make_golden.JOIN_CASES:
        b, p = make_golden.join_input(case)
        t = ctx.join_build(b.keys)
        got = packed(ctx.join_probe(t, p.keys))
        assert got.tolist() == make_golden.read_join(case["name"])
        t.free()


@pytest.fixture(scope="module")
def part_ctxs():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    cs = {p: olap.Context(0, join_partitions=p) for p in (2, 8, 64, 256)}
    yield cs
    for c in cs.values():
        c.close()


@pytest.mark.parametrize("parts", [2, 8, 64, 256])
@pytest.mark.parametrize("mult,dist,hit", [("unique", "uniform", 0.9), ("mult14", "zipf", 0.5)])
def test_partitioned_probe_matches_oracle(part_ctxs, parts, mult, dist, hit):
    """The radix-partitioned probe, forced on: same pair multiset as the oracle
    for every partition count (a table of 2^17 buckets, chains that cross
    partition boundaries, a ragged last tile)."""
    c = part_ctxs[parts]
    b = datagen.join_build(100_003, mult, seed=21)
    p = datagen.join_probe(700_001, b, hit, dist, seed=21)
    cnt = _check(c, b.keys, p.keys)
    assert cnt == p.expected_pairs(b)


def test_partitioned_probe_edges(part_ctxs):
    c = part_ctxs[64]
    # fewer probe rows than partitions, one row, none; explicit row-ids; the
    # empty-marker key on both sides; a build smaller than the partition count
    rng = np.random.default_rng(22)
    alphabet = np.array([I64_MIN, I64_MAX, 0, -1, 1, -2], dtype=np.int64)
    bk = alphabet[rng.integers(0, len(alphabet), 3000)]
    for npr in (0, 1, 5, 63, 64, 65, 2049, 50_000):
        pk = alphabet[rng.integers(0, len(alphabet), npr)]
        _check(c, bk, pk)
    _check(c, np.array([5, -1, 5], dtype=np.int64), np.array([5, -1, 7, 5], dtype=np.int64))
    b = datagen.join_build(40_000, "mult14", seed=23)
    p = datagen.join_probe(300_000, b, 0.7, "zipf", seed=23)
    br = (datagen.splitmix64(3, b.keys.shape[0]) >> np.uint64(33)).astype(np.uint32)
    pr = (datagen.splitmix64(4, p.keys.shape[0]) >> np.uint64(33)).astype(np.uint32)
    _check(c, b.keys, p.keys, br, pr)
    _check(c, b.keys, p.keys, br, pr, device=False)       # host memory in and out


@pytest.mark.parametrize("loads", [olap.LOADS_L1, olap.LOADS_L2_ONLY])
@pytest.mark.parametrize("parts", [1, 16])
def test_bucket_load_paths(loads, parts):
    """Both cache paths of the 256-bit bucket reads, direct and partitioned."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0, join_partitions=parts, join_bucket_loads=loads)
    try:
        b = datagen.join_build(150_000, "mult14", seed=24)
        p = datagen.join_probe(500_000, b, 0.8, "zipf", seed=24)
        assert _check(c, b.keys, p.keys) == p.expected_pairs(b)
        _check(c, np.array([-1, 3, -1], dtype=np.int64), np.array([-1, 3, 4, -1], dtype=np.int64))
    finally:
        c.close()


@pytest.mark.parametrize("parts", [1, 8])
def test_prefilter_forced_matches_oracle(parts):
    """The Bloom pre-probe (Sec. III-B, "bloom-filter/partitioned hash")
    forced on, before a direct and a partitioned probe: the same pair
    multiset as the oracle; it drops rows (hit rate 0.1) but never a match,
    and keeps probe rows with the empty-marker key for the side list."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0, join_partitions=parts, join_prefilter=olap.PREFILTER_ON)
    try:
        for mult, dist, hit, n in (("unique", "uniform", 0.1, 600_001), ("mult14", "zipf", 0.5, 300_007),
                                   ("unique", "uniform", 1.0, 100_000)):
            b = datagen.join_build(120_011, mult, seed=31)
            p = datagen.join_probe(n, b, hit, dist, seed=31)
            assert _check(c, b.keys, p.keys) == p.expected_pairs(b)
            info = c.join_probe_info()
            assert info["prefiltered"] and info["parts"] == parts
            hits = int(p.hit.sum())
            assert hits <= info["rows_probed"] <= hits + n // 50       # few false positives
        b = datagen.join_build(50_000, "mult14", seed=32)
        p = datagen.join_probe(200_000, b, 0.3, "zipf", seed=32)
        br = (datagen.splitmix64(5, b.keys.shape[0]) >> np.uint64(33)).astype(np.uint32)
        pr = (datagen.splitmix64(6, p.keys.shape[0]) >> np.uint64(33)).astype(np.uint32)
        _check(c, b.keys, p.keys, br, pr)
        _check(c, b.keys, p.keys, br, pr, device=False)
        rng = np.random.default_rng(33)
        alphabet = np.array([I64_MIN, I64_MAX, 0, -1, 1, -2], dtype=np.int64)
        bk = alphabet[rng.integers(0, len(alphabet), 3000)]
        for npr in (1, 5, 63, 4097, 20_000):
            _check(c, bk, alphabet[rng.integers(0, len(alphabet), npr)])
        _check(c, np.array([5, -1, 5], dtype=np.int64), np.array([-1, 7, -1, 5], dtype=np.int64))
    finally:
        c.close()


def test_prefilter_auto_decides_on_the_device():
    """Automatic mode: a table above L2 carries a filter; the pre-probe's
    sample drops rows at hit rate 0.1 and leaves them at 0.9, and the pairs
    match the oracle either way."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0)
    try:
        b = datagen.join_build(1 << 22, "unique", seed=34)
        t = c.join_build(torch.from_numpy(b.keys).cuda())
        for hit, want in ((0.1, True), (0.9, False)):
            p = datagen.join_probe((1 << 21) + 7, b, hit, "uniform", seed=34)
            need = p.expected_pairs(b)
            out = torch.empty((need, 2), dtype=torch.int32, device="cuda")
            got = c.join_probe(t, torch.from_numpy(p.keys).cuda(), out=out)
            info = c.join_probe_info()
            assert info["prefiltered"] == want
            np.testing.assert_array_equal(packed(got.cpu().numpy().view(np.uint32)), oracle.join(b.keys, p.keys))
        t.free()
    finally:
        c.close()
    off = olap.Context(0, join_prefilter=olap.PREFILTER_OFF)
    try:
        t = off.join_build(b.keys)
        p = datagen.join_probe(1 << 21, b, 0.1, "uniform", seed=35)
        off.join_probe(t, p.keys)
        assert not off.join_probe_info()["prefiltered"]
        t.free()
    finally:
        off.close()


@pytest.mark.parametrize("loads", [olap.LOADS_AUTO, olap.LOADS_L2_ONLY])
@pytest.mark.parametrize("prefilter", [olap.PREFILTER_AUTO, olap.PREFILTER_OFF])
def test_skewed_probe_goes_direct(prefilter, loads):
    """A table above L2 with a probe side large enough to partition: the
    device-side sample sends a Zipf-distributed probe stream (its sampled keys
    repeat) straight to the direct probe, skipping the partition passes, and
    leaves a uniform stream partitioned; the pairs match the oracle either
    way, with the pre-probe on its own choice or off, through either bucket
    load path."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0, join_prefilter=prefilter, join_bucket_loads=loads)
    try:
        b = datagen.join_build(1 << 22, "mult14", seed=36)
        t = c.join_build(torch.from_numpy(b.keys).cuda())
        n = (1 << 21) + 13
        planned = c.join_probe_partitions(t, n)
        assert planned > 1
        for dist, hit, direct in (("zipf", 0.9, True), ("uniform", 0.9, False), ("zipf", 0.1, None)):
            p = datagen.join_probe(n, b, hit, dist, seed=36)
            need = p.expected_pairs(b)
            out = torch.empty((need, 2), dtype=torch.int32, device="cuda")
            got = c.join_probe(t, torch.from_numpy(p.keys).cuda(), out=out)
            info = c.join_probe_info()
            if direct is not None:
                assert info["parts"] == (1 if direct else planned)
            elif prefilter == olap.PREFILTER_AUTO:
                # hit rate 0.1: the kept rows are mostly the Zipf hits, which repeat
                assert info["prefiltered"] and info["parts"] == 1
            assert got.shape[0] == need
            np.testing.assert_array_equal(packed(got.cpu().numpy().view(np.uint32)), oracle.join(b.keys, p.keys))
        t.free()
    finally:
        c.close()


_BUILDS = {}


def _full_build(mult):
    """The 2^24-row build side of a full-size cell, generated once per
    multiplicity for the whole module."""
    if mult not in _BUILDS:
        _BUILDS.clear()
        _BUILDS[mult] = datagen.join_build(1 << 24, mult, seed=2)
    return _BUILDS[mult]


@pytest.mark.parametrize("hit", [0.1, 0.9])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
@pytest.mark.parametrize("mult", ["unique", "mult14"])
def test_full_size(ctx, mult, dist, hit):
    """Every join cell at full size: 2^24 build rows, 2^28 probe keys, device
    resident, the benchmark's call (the table is 8x L2, so the automatic mode
    takes the partitioned probe).  The pair set is fixed by four checks:
    the exact count the generator implies (the sum of build multiplicities
    over the hits), every pair joining equal keys, every pair distinct
    (sorted on the device, strictly increasing), and the exact pairs of 4096
    sampled probe rows against the oracle.  Distinct valid pairs as many as
    the join has are the join."""
    b = _full_build(mult)
    p = datagen.join_probe(1 << 28, b, hit, dist, seed=2)
    need = p.expected_pairs(b)
    t = ctx.join_build(torch.from_numpy(b.keys).cuda())
    dk = torch.from_numpy(p.keys).cuda()
    out = torch.empty((need, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx.join_probe_async(t, dk, out, need, cnt)
    ctx.sync()
    t.free()
    assert int(cnt.item()) == need
    info = ctx.join_probe_info()
    assert info["prefiltered"] == (hit < 0.5)                 # the automatic pre-probe's choice
    assert (info["parts"] == 1) == (dist == "zipf")           # the sample's skew check: Zipf probes go direct
    pr = out[:, 0].to(torch.int64) & 0xFFFFFFFF
    br = out[:, 1].to(torch.int64) & 0xFFFFFFFF
    assert bool((pr < (1 << 28)).all()) and bool((br < (1 << 24)).all())
    bkd = torch.from_numpy(b.keys).cuda()
    assert torch.equal(dk[pr], bkd[br])                       # every pair joins equal keys
    del bkd
    packed_d = torch.sort((pr << 32) | br).values
    del br
    assert bool((packed_d[1:] > packed_d[:-1]).all())          # no pair twice
    del packed_d
    # exact pairs of a sample of probe rows against the oracle
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(1 << 28, 4096, replace=False))
    sel = torch.isin(pr, torch.from_numpy(rows).cuda())
    got = packed(out[sel].cpu().numpy().view(np.uint32))
    want = oracle.join(b.keys, p.keys[rows], None, rows.astype(np.uint32))
    np.testing.assert_array_equal(got, want)
    del dk, out, pr, sel
    torch.cuda.empty_cache()


def test_probe_partitions_query():
    """olap_join_probe_partitions reports the probe's mode: direct for a small
    probe, a power of two above 1 for a table well above L2 with a large
    probe side, the forced count when the option sets one."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    b = datagen.join_build(1 << 22, "unique", seed=61)          # 2^22 buckets x 32 B = 128 MiB, above L2
    c = olap.Context(0)
    try:
        t = c.join_build(torch.from_numpy(b.keys).cuda())
        assert c.join_probe_partitions(t, 1000) == 1           # too few rows to pay for partitioning
        parts = c.join_probe_partitions(t, 1 << 24)
        assert parts > 1 and parts & (parts - 1) == 0
        small = c.join_build(b.keys[:1000])
        assert c.join_probe_partitions(small, 1 << 24) == 1     # the table fits in L2
        small.free()
        with pytest.raises(olap.OlapError) as ei:
            c.join_probe_partitions(small, 10)                  # freed
        assert ei.value.status == olap.E_INVALID
        t.free()
    finally:
        c.close()
    for opt, want in ((1, 1), (16, 16)):
        c = olap.Context(0, join_partitions=opt)
        try:
            t = c.join_build(b.keys[:100_000])
            assert c.join_probe_partitions(t, 5000) == want
            t.free()
        finally:
            c.close()
