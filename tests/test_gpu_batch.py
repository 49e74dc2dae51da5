"""The batched persistent executor: every item of a mixed batch (Top-K of
uneven sizes, K and key types, and probe batches against one resident table)
equals the oracle bit-exact, through the captured graph and through one call
per query; corrupted descriptors are rejected on the device."""
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


def _packed(p):
    p = np.asarray(p, dtype=np.uint32).reshape(-1, 2).astype(np.uint64)
    return np.sort((p[:, 0] << np.uint64(32)) | p[:, 1])


def _make(ctx, n_topk=300, n_probe=40, seed=5):
    rng = np.random.default_rng(seed)
    ns = datagen.log_uniform(1e3, 2e6, datagen.stream_seed(seed, 8), n_topk)
    ns[:6] = [1, 31, 4096, 4097, 70_000, 5]                      # edge sizes
    ks = (rng.integers(1, 1001, n_topk)).astype(np.int64)
    ks[:6] = [1, 40, 4096, 1000, 4096, 9]
    kinds = rng.integers(0, 4, n_topk)
    q = []
    items = []
    big = datagen.topk_keys(int(ns.sum()), "uniform", "i64", seed=seed)
    bigf = datagen.topk_keys(int(ns.sum()), "dup1024", "f32", seed=seed)
    off = 0
    for i in range(n_topk):
        n, k = int(ns[i]), int(ks[i])
        f32 = kinds[i] >= 2
        keys = (bigf if f32 else big)[off:off + n].copy()
        off += n
        order = olap.DESC if kinds[i] % 2 == 0 else olap.ASC
        dk = torch.from_numpy(keys).cuda()
        cnt = min(k, n)
        ok = torch.empty(max(1, cnt), dtype=dk.dtype, device="cuda")
        orow = torch.empty(max(1, cnt), dtype=torch.int32, device="cuda")
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        items.append(olap.topk_item(dk, k, order, ok, orow, c, d_status=st))
        q.append(("topk", keys, k, order, dk, ok, orow, c, st))
    b = datagen.join_build(1 << 18, "mult14", seed=seed)
    table = ctx.join_build(torch.from_numpy(b.keys).cuda())
    pns = datagen.log_uniform(1e3, 2e5, datagen.stream_seed(seed, 10), n_probe)
    pns[:5] = [0, 1, 32768, 32769, 700_000]       # empty, one chunk exactly, one row over, 22 chunks
    for i in range(n_probe):
        p = datagen.join_probe(int(pns[i]), b, 0.5, "uniform", seed=seed * 100 + i)
        need = p.expected_pairs(b)
        dk = torch.from_numpy(p.keys).cuda()
        out = torch.empty((max(1, need), 2), dtype=torch.int32, device="cuda")
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        items.append(olap.probe_item(table, dk, out, need, c, d_status=st))
        q.append(("probe", p.keys, need, None, dk, out, None, c, st))
    return items, q, b, table


def _verify(q, b):
    for kind, keys, k, order, dk, o1, o2, c, st in q:
        assert int(st.item()) == olap.OK
        if kind == "topk":
            wk, wr = oracle.topk(keys, k, order)
            assert int(c.item()) == len(wr)
            got_r = o2.cpu().numpy().view(np.uint32)[:len(wr)]
            got_k = o1.cpu().numpy()[:len(wr)]
            np.testing.assert_array_equal(got_r, wr)
            np.testing.assert_array_equal(got_k.view(np.uint8), wk.view(np.uint8))
        else:
            assert int(c.item()) == k
            got = _packed(o1.cpu().numpy().view(np.uint32)[:k])
            np.testing.assert_array_equal(got, oracle.join(b.keys, keys))


def test_batch_graph_and_per_query_match_oracle(ctx):
    items, q, b, table = _make(ctx)
    batch = ctx.batch(items)
    for _ in range(2):                      # replayed graph, results each time
        for e in q:
            e[7].zero_()
            e[8].fill_(-1)
        batch.run()
        ctx.sync()
        assert batch.errors() == 0
        _verify(q, b)
    for e in q:
        e[7].zero_()
        e[5].zero_()
    batch.run_per_query()
    ctx.sync()
    for kind, keys, k, order, dk, o1, o2, c, st in q:       # per-query path writes counts for probes
        if kind == "topk":
            wk, wr = oracle.topk(keys, k, order)
            np.testing.assert_array_equal(o2.cpu().numpy().view(np.uint32)[:len(wr)], wr)
        else:
            assert int(c.item()) == k
    batch.free()
    table.free()


def test_corrupted_descriptor_is_rejected_on_device(ctx):
    keys = torch.from_numpy(datagen.topk_keys(10_000, "uniform", "i64", seed=1)).cuda()
    ok = torch.empty(10, dtype=torch.int64, device="cuda")
    orow = torch.empty(10, dtype=torch.int32, device="cuda")
    c = torch.zeros(3, dtype=torch.int64, device="cuda")
    st = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    good = olap.topk_item(keys, 10, olap.DESC, ok, orow, c[0:1], d_status=st[0:1])
    bad_keys = olap.topk_item(keys, 10, olap.DESC, ok, orow, c[1:2], d_status=st[1:2])
    bad_keys.keys = None                    # n > 0 with no keys
    bad_out = olap.topk_item(keys, 10, olap.DESC, ok, orow, c[2:3], d_status=st[2:3])
    bad_out.out_rowids = None
    batch = ctx.batch([good, bad_keys, bad_out])
    batch.run()
    ctx.sync()
    assert batch.errors() == 2
    assert st.cpu().tolist() == [olap.OK, olap.E_DEVICE, olap.E_DEVICE]
    wk, wr = oracle.topk(keys.cpu().numpy(), 10, olap.DESC)
    np.testing.assert_array_equal(orow.cpu().numpy().view(np.uint32), wr)
    batch.free()


def test_corrupted_probe_descriptor_skips_only_its_chunks(ctx):
    b = datagen.join_build(50_000, "mult14", seed=8)
    table = ctx.join_build(torch.from_numpy(b.keys).cuda())
    p = datagen.join_probe(200_000, b, 0.7, "uniform", seed=8)      # 7 chunks
    need = p.expected_pairs(b)
    dk = torch.from_numpy(p.keys).cuda()
    out = torch.empty((need, 2), dtype=torch.int32, device="cuda")
    c = torch.full((2,), 77, dtype=torch.int64, device="cuda")
    st = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    good = olap.probe_item(table, dk, out, need, c[0:1], d_status=st[0:1])
    bad = olap.probe_item(table, dk, out, need, c[1:2], d_status=st[1:2])
    bad.keys = None                         # n > 0 with no keys
    batch = ctx.batch([bad, good])
    batch.run()
    ctx.sync()
    assert batch.errors() == 1
    assert st.cpu().tolist() == [olap.OK, olap.E_DEVICE]
    assert c.cpu().tolist() == [need, 77]   # the rejected item's count is left alone
    np.testing.assert_array_equal(_packed(out.cpu().numpy().view(np.uint32)), oracle.join(b.keys, p.keys))
    batch.free()
    table.free()


def test_host_rejects_k_above_limit(ctx):
    keys = torch.zeros(5000, dtype=torch.int64, device="cuda")
    out = torch.empty(5000, dtype=torch.int64, device="cuda")
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(olap.OlapError) as ei:
        ctx.batch([olap.topk_item(keys, 4097, olap.DESC, out, out, c)])
    assert ei.value.status == olap.E_INVALID


def test_side_by_side_branches_match_oracle():
    """The graph with the Top-K and probe kernels on two branches gives the
    same results as the serial graph."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0, batch_overlap=1)
    try:
        items, q, b, table = _make(c, n_topk=60, n_probe=12, seed=21)
        batch = c.batch(items)
        batch.run()
        c.sync()
        assert batch.errors() == 0
        _verify(q, b)
        batch.free()
        table.free()
    finally:
        c.close()


@pytest.mark.slow
def test_full_size_batch_sampled():
    """The batched workload at full size, in the configuration the benchmark
    times: 4096 Top-K queries (N ~ logU[1e3, 4e6), K ~ U{1..1000}, int64
    uniform keys drawn on the device, DESC) and 1024 probe batches
    (n ~ logU[1e3, 1e6), hit rate 0.5) against one 2^22-key unique table, on
    an autotuned context, one graph launch.  Every item: status OK and the
    exact count; every Top-K output: sorted, ties by row-id, and each key the
    key of its row; a sample of items (the largest and a random draw) against
    the oracle bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0)
    try:
        c.autotune(topk_n=1 << 20, topk_k=500, join_build_n=1 << 22, join_probe_n=1 << 20,
                   join_hit_rate=0.5, reps=3)
        n_topk, n_probe = 4096, 1024
        ns, ks = datagen.batched_topk_queries(n_topk, 1e3, 4e6, 1000, seed=3)
        offs = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        kseed = datagen.stream_seed(3, 0)
        keys = datagen.splitmix64_torch(kseed, int(offs[-1]), device="cuda")
        cnt = np.minimum(ks, ns)
        koffs = np.concatenate([[0], np.cumsum(ks)]).astype(np.int64)
        out_k = torch.empty(int(koffs[-1]), dtype=torch.int64, device="cuda")
        out_r = torch.empty(int(koffs[-1]), dtype=torch.int32, device="cuda")
        counts = torch.zeros(n_topk + n_probe, dtype=torch.int64, device="cuda")
        status = torch.full((n_topk + n_probe,), -1, dtype=torch.int32, device="cuda")
        items = []
        for i in range(n_topk):
            a, e = int(koffs[i]), int(koffs[i + 1])
            items.append(olap.topk_item(keys[int(offs[i]):int(offs[i + 1])], int(ks[i]), olap.DESC,
                                        out_k[a:e], out_r[a:e], counts[i:i + 1], d_status=status[i:i + 1]))
        b = datagen.join_build(1 << 22, "unique", seed=3)
        table = c.join_build(torch.from_numpy(b.keys).cuda())
        pns = datagen.batched_probe_sizes(n_probe, 1e3, 1e6, seed=3)
        poffs = np.concatenate([[0], np.cumsum(pns)]).astype(np.int64)
        p = datagen.join_probe(int(poffs[-1]), b, 0.5, "uniform", seed=3)
        hits = np.concatenate([[0], np.cumsum(p.hit)]).astype(np.int64)
        pk = torch.from_numpy(p.keys).cuda()
        pairs = torch.empty((int(hits[-1]) + 1, 2), dtype=torch.int32, device="cuda")
        for j in range(n_probe):
            a, e = int(poffs[j]), int(poffs[j + 1])
            h0, h1 = int(hits[a]), int(hits[e])
            items.append(olap.probe_item(table, pk[a:e], pairs[h0:h1 + 1], h1 - h0,
                                         counts[n_topk + j:n_topk + j + 1],
                                         d_status=status[n_topk + j:n_topk + j + 1]))
        batch = c.batch(items)
        batch.run()
        c.sync()
        assert batch.errors() == 0
        assert int((status != olap.OK).sum().item()) == 0
        got_counts = counts.cpu().numpy()
        np.testing.assert_array_equal(got_counts[:n_topk], cnt)
        np.testing.assert_array_equal(got_counts[n_topk:], np.diff(hits[poffs]))

        # every Top-K output: a real row, in order (rank DESC, row-id ASC on ties)
        valid = torch.from_numpy(np.concatenate([np.arange(koffs[i], koffs[i] + cnt[i]) for i in range(n_topk)])).cuda()
        seg = torch.from_numpy(np.repeat(np.arange(n_topk), cnt)).cuda()
        ok_k, ok_r = out_k[valid], out_r[valid].to(torch.int64)
        assert int(((ok_r < 0) | (ok_r >= torch.from_numpy(ns).cuda()[seg])).sum().item()) == 0
        src = torch.from_numpy(offs[:-1]).cuda()[seg] + ok_r
        assert torch.equal(keys[src], ok_k)
        same = seg[1:] == seg[:-1]
        desc = (ok_k[:-1] > ok_k[1:]) | ((ok_k[:-1] == ok_k[1:]) & (ok_r[:-1] < ok_r[1:]))
        assert int((same & ~desc).sum().item()) == 0

        # a sample against the oracle: the largest items and a seeded draw
        rng = np.random.default_rng(7)
        t_pick = np.unique(np.concatenate([np.argsort(ns)[-6:], rng.choice(n_topk, 20, replace=False)]))
        hk, hr = out_k.cpu().numpy(), out_r.cpu().numpy().view(np.uint32)
        for i in t_pick:
            host = datagen.splitmix64(kseed, int(ns[i]), start=int(offs[i])).view(np.int64)
            wk, wr = oracle.topk(host, int(ks[i]), olap.DESC)
            a = int(koffs[i])
            np.testing.assert_array_equal(hr[a:a + len(wr)], wr)
            np.testing.assert_array_equal(hk[a:a + len(wr)], wk)
        p_pick = np.unique(np.concatenate([np.argsort(pns)[-3:], rng.choice(n_probe, 9, replace=False)]))
        hp = pairs.cpu().numpy().view(np.uint32)
        for j in p_pick:
            a, e = int(poffs[j]), int(poffs[j + 1])
            h0, h1 = int(hits[a]), int(hits[e])
            np.testing.assert_array_equal(_packed(hp[h0:h1]), oracle.join(b.keys, p.keys[a:e]))
        batch.free()
        table.free()
    finally:
        c.close()


def test_launch_counter_counts_every_kernel():
    """olap_ctx_launches: the direct Top-K is two kernels (prepare, select),
    the sampled one three (prepare, filter, select); a build without key -1
    two (insert, chain counts); a direct probe one, a partitioned probe three; a batch replay the
    kernels of its graph (probe reset, probe, Top-K, and the merge of split
    Top-K items: the 2^20-key item here is split); the per-query run the sum
    of its calls.  A staged context launches no copy kernels."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0, host_access=olap.HOST_STAGED)
    try:
        def delta(fn):
            c0 = c.launches()
            fn()
            c.sync()
            return c.launches() - c0
        small = torch.from_numpy(datagen.topk_keys(1 << 20, "uniform", "i64", seed=70)).cuda()
        big = torch.from_numpy(datagen.topk_keys(1 << 22, "uniform", "i64", seed=71)).cuda()
        ok = torch.empty(100, dtype=torch.int64, device="cuda")
        orow = torch.empty(100, dtype=torch.int32, device="cuda")
        assert delta(lambda: c.topk_async(small, 100, olap.DESC, ok, orow)) == 2
        assert delta(lambda: c.topk_async(big, 100, olap.DESC, ok, orow)) == 3
        assert delta(lambda: c.topk(small.cpu().numpy(), 100, olap.DESC)) == 2      # staged copies are not kernels
        b = datagen.join_build(50_000, "unique", seed=72)
        holder = []
        assert delta(lambda: holder.append(c.join_build(torch.from_numpy(b.keys).cuda()))) == 2
        t = holder[0]
        p = datagen.join_probe(40_000, b, 0.5, "uniform", seed=72)
        pk = torch.from_numpy(p.keys).cuda()
        need = p.expected_pairs(b)
        out = torch.empty((need, 2), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert c.join_probe_partitions(t, 40_000) == 1
        assert delta(lambda: c.join_probe_async(t, pk, out, need, cnt)) == 1
        cnt2 = torch.zeros(2, dtype=torch.int64, device="cuda")
        items = [olap.topk_item(small, 100, olap.DESC, ok, orow, cnt2[0:1]),
                 olap.probe_item(t, pk, out, need, cnt2[1:2])]
        bt = c.batch(items)
        assert delta(bt.run) == 4
        assert delta(bt.run_per_query) == 3
        bt.free()
        t.free()
    finally:
        c.close()
    cp = olap.Context(0, join_partitions=4, host_access=olap.HOST_STAGED)
    try:
        t = cp.join_build(b.keys)
        c0 = cp.launches()
        got = cp.join_probe(t, p.keys)
        assert cp.launches() - c0 == 3                          # count, scatter, probe
        assert got.shape[0] == need
        t.free()
    finally:
        cp.close()


def test_split_items_match_oracle(ctx):
    """Top-K items of 2^19 keys and more run as parts of about 2^18 keys and a
    merge launch: every split item equals the oracle bit for bit, at the split
    threshold and above it, for both key widths and orders, the largest k,
    and explicit row-ids (reversed, so the merge's row-id tie-break is not
    the index order)."""
    cases = [(1 << 19, 1, olap.DESC, "i64", False), ((1 << 19) + 1, 4096, olap.ASC, "i64", False),
             (3 * (1 << 18) + 5, 1000, olap.DESC, "f32", False), (1_500_007, 777, olap.ASC, "f32", True),
             (2_000_003, 4096, olap.DESC, "i64", True), ((1 << 19) - 1, 100, olap.DESC, "i64", False)]
    items, q = [], []
    for j, (n, k, order, kt, explicit) in enumerate(cases):
        keys = datagen.topk_keys(n, "dup1024" if kt == "f32" else "uniform", kt, seed=40 + j)
        rid = np.arange(n, dtype=np.uint32)[::-1].copy() if explicit else None
        dk = torch.from_numpy(keys).cuda()
        dr = None if rid is None else torch.from_numpy(rid.view(np.int32)).cuda()
        ok = torch.empty(k, dtype=dk.dtype, device="cuda")
        orow = torch.empty(k, dtype=torch.int32, device="cuda")
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        items.append(olap.topk_item(dk, k, order, ok, orow, c, d_rowids=dr, d_status=st))
        q.append((keys, rid, k, order, dk, dr, ok, orow, c, st))
    bt = ctx.batch(items)
    try:
        bt.run()
        ctx.sync()
        assert bt.errors() == 0
        for keys, rid, k, order, _dk, _dr, ok, orow, c, st in q:
            assert int(st.item()) == olap.OK and int(c.item()) == k
            wk, wr = oracle.topk(keys, k, order, rid)
            np.testing.assert_array_equal(orow.cpu().numpy().view(np.uint32), wr)
            np.testing.assert_array_equal(ok.cpu().numpy().view(np.uint8), wk.view(np.uint8))
    finally:
        bt.free()
