"""GPU parity of the two-column Top-K (ORDER BY c0, c1 LIMIT K: Sec. III-A's
Top-K with a second key column) against the CPU oracle, bit-exact: the same
row-ids and both columns' key bits, in the same order.

Medium sizes compare with the oracle element by element (direct path below
2^21 rows, sampled single pass above, tiles and ragged tails, every pair of
orders, mixed 4-byte types, IEEE totalOrder for float32, explicit row-ids
with repeats, host memory, columns of unequal alignment).  At full size
(2^28 rows) the properties that fix the answer are checked on the device."""
import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import datagen, olap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDERS = [(o0, o1) for o0 in (olap.ASC, olap.DESC) for o1 in (olap.ASC, olap.DESC)]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0)
    yield c
    c.close()


def _cols(n, t0, t1, seed):
    """c0 with heavy ties (1024 distinct values), c1 uniform bit patterns."""
    c0 = datagen.topk_keys(n, "dup1024", t0, seed=seed)
    c1 = datagen.topk_keys(n, "uniform", t1, seed=seed + 1)
    return c0, c1


def _check(ctx, c0, o0, c1, o1, k, rowids=None, where="device"):
    if where == "device" and np.uint32 in (c0.dtype.type, c1.dtype.type):
        where = "pageable"                      # torch has no full uint32 support: host columns
    if where == "device":
        d0, d1 = torch.from_numpy(c0).cuda(), torch.from_numpy(c1).cuda()
        dr = None if rowids is None else torch.from_numpy(rowids.view(np.int32)).cuda()
        cnt = max(1, min(k, c0.shape[0]))
        g0 = torch.empty(cnt, dtype=d0.dtype, device="cuda")
        g1 = torch.empty(cnt, dtype=d1.dtype, device="cuda")
        gr = torch.empty(cnt, dtype=torch.int32, device="cuda")
        g0, g1, gr = ctx.topk_pair(d0, o0, d1, o1, k, rowids=dr, out_keys0=g0, out_keys1=g1, out_rowids=gr)
        g0, g1, gr = g0.cpu().numpy(), g1.cpu().numpy(), gr.cpu().numpy().view(np.uint32)
    elif where == "pinned":
        p0, p1 = torch.from_numpy(c0).pin_memory(), torch.from_numpy(c1).pin_memory()
        pr = None if rowids is None else torch.from_numpy(rowids.view(np.int32)).pin_memory()
        cnt = max(1, min(k, c0.shape[0]))
        o_0 = torch.empty(cnt, dtype=p0.dtype).pin_memory()
        o_1 = torch.empty(cnt, dtype=p1.dtype).pin_memory()
        o_r = torch.empty(cnt, dtype=torch.int32).pin_memory()
        g0, g1, gr = ctx.topk_pair(p0, o0, p1, o1, k, rowids=pr, out_keys0=o_0, out_keys1=o_1, out_rowids=o_r)
        g0, g1, gr = g0.numpy(), g1.numpy(), gr.numpy().view(np.uint32)
    else:
        g0, g1, gr = ctx.topk_pair(c0, o0, c1, o1, k, rowids=rowids)
    w0, w1, wr = oracle.topk_pair(c0, o0, c1, o1, k, rowids)
    np.testing.assert_array_equal(gr, wr)
    np.testing.assert_array_equal(g0.view(np.uint32), w0.view(np.uint32))
    np.testing.assert_array_equal(g1.view(np.uint32), w1.view(np.uint32))


@pytest.mark.parametrize("t0,t1", [("i32", "i32"), ("f32", "i32"), ("u32", "f32")])
@pytest.mark.parametrize("n", [1, 33, 4097, 100_003, (1 << 21) + 3, 3_000_001])
def test_sizes_types_orders(ctx, t0, t1, n):
    c0, c1 = _cols(n, t0, t1, seed=n % 97)
    for o0, o1 in ORDERS:
        for k in (1, 10, 1000, 5000):
            _check(ctx, c0, o0, c1, o1, k)


def test_large_k_and_explicit_rowids(ctx):
    c0, c1 = _cols(2_500_000, "i32", "u32", seed=5)
    rowids = (datagen.splitmix64(9, c0.shape[0]) >> np.uint64(41)).astype(np.uint32)   # many repeats
    for o0, o1 in ORDERS[:2]:
        _check(ctx, c0, o0, c1, o1, 100_000, rowids)
        _check(ctx, c0, o0, c1, o1, 10, rowids)


def test_all_ties_on_both_columns_fall_back(ctx):
    # every row equal on both columns: the sampled threshold admits them all,
    # more than the candidate buffer, so the selection runs on the input
    n = 4_000_000
    c0 = np.full(n, 7, dtype=np.int32)
    c1 = np.full(n, -3, dtype=np.int32)
    _check(ctx, c0, olap.DESC, c1, olap.ASC, 100)


@pytest.mark.parametrize("where", ["pinned", "pageable"])
def test_host_memory(ctx, where):
    c0, c1 = _cols(3_000_000, "f32", "i32", seed=11)
    rowids = datagen.identity_rowids(c0.shape[0])[::-1].copy()
    _check(ctx, c0, olap.DESC, c1, olap.DESC, 1000, rowids, where=where)
    # pinned row-ids on the sampled path are read in place, pageable ones copied
    assert ctx.topk_info()["rowids_in_place"] == (where == "pinned")


def test_pinned_rowids_in_place_on_the_fallback_path(ctx):
    # all rows tie on both columns: the selection runs on the input and
    # reads every row-id in pinned host memory
    n = 3_000_000
    c0 = np.full(n, 7, dtype=np.int32)
    c1 = np.full(n, -3, dtype=np.int32)
    rowids = datagen.identity_rowids(n)[::-1].copy()
    _check(ctx, c0, olap.DESC, c1, olap.ASC, 100, rowids, where="pinned")
    info = ctx.topk_info()
    assert info["rowids_in_place"] and info["path"] == 2


def test_unequal_alignment_uses_row_loads(ctx):
    # c1 starts 4 bytes past c0's alignment: the row-by-row flavour
    n = (1 << 21) + 1001
    c0, c1 = _cols(n + 1, "i32", "i32", seed=13)
    d0 = torch.from_numpy(c0).cuda()[:n]
    d1 = torch.from_numpy(c1).cuda()[1:]
    g0 = torch.empty(500, dtype=torch.int32, device="cuda")
    g1 = torch.empty(500, dtype=torch.int32, device="cuda")
    gr = torch.empty(500, dtype=torch.int32, device="cuda")
    ctx.topk_pair(d0, olap.DESC, d1, olap.ASC, 500, out_keys0=g0, out_keys1=g1, out_rowids=gr)
    w0, w1, wr = oracle.topk_pair(c0[:n], olap.DESC, c1[1:], olap.ASC, 500)
    np.testing.assert_array_equal(gr.cpu().numpy().view(np.uint32), wr)
    np.testing.assert_array_equal(g0.cpu().numpy(), w0)
    np.testing.assert_array_equal(g1.cpu().numpy(), w1)


def test_eight_byte_columns_are_not_supported(ctx):
    a = np.arange(10, dtype=np.int64)
    b = np.arange(10, dtype=np.int32)
    with pytest.raises(olap.OlapError) as ei:
        ctx.topk_pair(a, olap.DESC, b, olap.ASC, 3)
    assert ei.value.status == olap.E_UNIMPLEMENTED


def _ordinal_dev(t):
    """int64 per key in its type's order, on the device."""
    if t.dtype == torch.float32:
        x = t.view(torch.int32)
        return (x ^ ((x >> 31) & 0x7FFFFFFF)).to(torch.int64)
    if t.dtype == torch.int32:
        return t.to(torch.int64)
    return t.view(torch.int32).to(torch.int64) & 0xFFFFFFFF       # uint32 held as int32 bits


@pytest.mark.parametrize("t0,t1", [("i32", "i32"), ("f32", "i32")])
def test_full_size_2p28(ctx, t0, t1):
    """2^28 rows: K distinct real rows with their own key bits, in
    (c0, c1, row-id) order, and exactly K-1 rows of the whole input ahead of
    the last one -- checked on the device."""
    n = 1 << 28
    c0, c1 = _cols(n, t0, t1, seed=1)
    d0, d1 = torch.from_numpy(c0).cuda(), torch.from_numpy(c1).cuda()
    del c0, c1
    dt = {"i32": torch.int32, "f32": torch.float32}
    for k, o0, o1 in ((1000, olap.DESC, olap.ASC), (1000, olap.ASC, olap.DESC), (100_000, olap.DESC, olap.DESC)):
        g0 = torch.empty(k, dtype=dt[t0], device="cuda")
        g1 = torch.empty(k, dtype=dt[t1], device="cuda")
        gr = torch.empty(k, dtype=torch.int32, device="cuda")
        ctx.topk_pair(d0, o0, d1, o1, k, out_keys0=g0, out_keys1=g1, out_rowids=gr)
        idx = gr.to(torch.int64) & 0xFFFFFFFF
        assert bool((idx < n).all()) and torch.unique(idx).numel() == k
        assert torch.equal(d0[idx].view(torch.int32), g0.view(torch.int32))
        assert torch.equal(d1[idx].view(torch.int32), g1.view(torch.int32))
        s0 = 1 if o0 == olap.ASC else -1
        s1 = 1 if o1 == olap.ASC else -1
        v0, v1 = _ordinal_dev(g0) * s0, _ordinal_dev(g1) * s1
        ok = (v0[:-1] < v0[1:]) | ((v0[:-1] == v0[1:]) & ((v1[:-1] < v1[1:]) |
                                                          ((v1[:-1] == v1[1:]) & (idx[:-1] < idx[1:]))))
        assert bool(ok.all())
        l0, l1, lr = v0[-1], v1[-1], idx[-1]
        ahead = 0
        step = 1 << 26
        for s in range(0, n, step):
            a0 = _ordinal_dev(d0[s:s + step]) * s0
            a1 = _ordinal_dev(d1[s:s + step]) * s1
            rows = torch.arange(s, min(n, s + step), dtype=torch.int64, device="cuda")
            ahead += int(((a0 < l0) | ((a0 == l0) & ((a1 < l1) | ((a1 == l1) & (rows < lr))))).sum().item())
        assert ahead == k - 1
    del d0, d1
    torch.cuda.empty_cache()
