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
