"""GPU parity of Top-K over every key type (olap_key_type) against the CPU
oracle, bit-exact: float64 (the paper's key column is a double, Sec. V-A)
by IEEE 754-2019 totalOrder, uint64, int32 and uint32 by value.  Sizes cover
the direct path (N <= 2^21), the sampled single pass, K above one CTA's sort
(merge path), ragged and unaligned inputs, the batched executor, pageable
host memory, and a full-size float64 column of 2^28 keys checked by the
properties that fix the answer."""
import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import datagen, olap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NEW = ["f64", "u64", "i32", "u32"]
TORCH_OK = {"f64": True, "u64": False, "i32": True, "u32": False}   # torch lacks full uint support


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0)
    yield c
    c.close()


def _to_dev(a):
    """Device copy of a numpy key column (unsigned types through a same-width view)."""
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda(), True
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda(), True
    return torch.from_numpy(a).cuda(), False


def _gpu_topk(ctx, keys, k, order, rowids=None):
    """Through the blocking call, device keys when torch has the type, else
    host keys (pageable)."""
    if TORCH_OK.get({np.float64: "f64", np.int32: "i32"}.get(keys.dtype.type, ""), False):
        dk, _ = _to_dev(keys)
        dr = None if rowids is None else torch.from_numpy(rowids.view(np.int32)).cuda()
        return ctx.topk(dk, k, order, rowids=dr)
    return ctx.topk(keys, k, order, rowids=rowids)


def _same(gk, gr, wk, wr):
    np.testing.assert_array_equal(np.asarray(gr).view(np.uint32), wr)
    np.testing.assert_array_equal(np.asarray(gk).view(np.uint8), wk.view(np.uint8))


@pytest.mark.parametrize("kt", NEW)
@pytest.mark.parametrize("dist", ["uniform", "ascending", "dup1024"])
@pytest.mark.parametrize("n", [1, 31, 4097, 100_003, 3_000_001])
def test_sizes_and_distributions(ctx, kt, dist, n):
    keys = datagen.topk_keys(n, dist, kt, seed=n % 101)
    for k, order in ((1, olap.DESC), (100, olap.ASC), (1000, olap.DESC)):
        gk, gr = _gpu_topk(ctx, keys, k, order)
        _same(gk, gr, *oracle.topk(keys, k, order))


@pytest.mark.parametrize("kt", NEW)
def test_merge_path_and_rowids(ctx, kt):
    keys = datagen.topk_keys((1 << 21) + 5, "dup1024", kt, seed=9)
    rid = (datagen.splitmix64(10, keys.shape[0]) >> np.uint64(40)).astype(np.uint32)
    gk, gr = _gpu_topk(ctx, keys, 9000, olap.DESC, rid)
    _same(gk, gr, *oracle.topk(keys, 9000, olap.DESC, rid))


@pytest.mark.parametrize("off", [1, 3])
@pytest.mark.parametrize("kt", NEW)
def test_unaligned_host_slices(ctx, kt, off):
    base = datagen.topk_keys(2_500_011, "uniform", kt, seed=11 + off)
    keys = base[off:]
    gk, gr = ctx.topk(keys, 777, olap.ASC)
    _same(gk, gr, *oracle.topk(keys, 777, olap.ASC))


def test_f64_specials(ctx):
    from tests.test_oracle_keytypes import f64_specials
    bits, _ = f64_specials()
    rng = np.random.default_rng(12)
    for n in (26, 5000, 3_000_000):
        keys = bits[rng.integers(0, len(bits), n)].view(np.float64)
        for order in (olap.ASC, olap.DESC):
            for k in (1, 25, 2000):
                gk, gr = _gpu_topk(ctx, keys, k, order)
                _same(gk, gr, *oracle.topk(keys, k, order))


def test_extremes_of_integer_types(ctx):
    for dt in (np.uint64, np.int32, np.uint32):
        info = np.iinfo(dt)
        alphabet = np.array([info.min, info.min + 1, 0 if info.min < 0 else 1, info.max - 1, info.max], dtype=dt)
        rng = np.random.default_rng(13)
        for n in (5, 4099, 2_200_000):
            keys = alphabet[rng.integers(0, len(alphabet), n)]
            for order in (olap.ASC, olap.DESC):
                gk, gr = ctx.topk(keys, 300, order)
                _same(gk, gr, *oracle.topk(keys, 300, order))


@pytest.mark.parametrize("kt", NEW)
def test_batched_items(ctx, kt):
    items, keep = [], []
    for i, n in enumerate([1, 4096, 70_000, 1_000_003]):
        keys = datagen.topk_keys(n, "uniform" if i % 2 else "dup1024", kt, seed=i)
        dk, _ = _to_dev(keys)
        k = min(500, n)
        ok = torch.empty(k, dtype=dk.dtype, device="cuda")
        orow = torch.empty(k, dtype=torch.int32, device="cuda")
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        it = olap.topk_item(dk, k, olap.DESC, ok, orow, c)
        it.key_type = olap.key_type_of(keys)                 # the unsigned kinds travel as signed views
        items.append(it)
        keep.append((keys, k, ok, orow, dk))
    b = ctx.batch(items)
    b.run()
    ctx.sync()
    assert b.errors() == 0
    for keys, k, ok, orow, _ in keep:
        wk, wr = oracle.topk(keys, k, olap.DESC)
        np.testing.assert_array_equal(orow.cpu().numpy().view(np.uint32), wr)
        np.testing.assert_array_equal(ok.cpu().numpy().view(np.uint8), wk.view(np.uint8))
    b.free()


def _f64_order(bits):
    """IEEE totalOrder image of float64 bit patterns as signed int64."""
    b = bits.view(np.int64)
    return b ^ ((b >> 63) & np.int64(0x7FFFFFFFFFFFFFFF))


@pytest.mark.slow
def test_full_size_f64_2p28(ctx):
    n, k = 1 << 28, 1000
    keys = datagen.topk_keys(n, "uniform", "f64", seed=1)
    dk = torch.from_numpy(keys).cuda()
    ok = torch.empty(k, dtype=torch.float64, device="cuda")
    orow = torch.empty(k, dtype=torch.int32, device="cuda")
    ctx.topk_async(dk, k, olap.DESC, ok, orow)
    ctx.sync()
    gk, gr = ok.cpu().numpy(), orow.cpu().numpy().view(np.uint32)
    idx = gr.astype(np.int64)
    assert np.unique(idx).shape[0] == k
    np.testing.assert_array_equal(keys[idx].view(np.uint64), gk.view(np.uint64))       # real rows
    img = _f64_order(gk.view(np.uint64))
    assert np.all((img[:-1] > img[1:]) | ((img[:-1] == img[1:]) & (idx[:-1] < idx[1:])))   # sorted
    # exactly k - 1 rows strictly ahead of the last one (count on the device)
    full = torch.from_numpy(_f64_order(keys.view(np.uint64))).cuda()
    last, lr = int(img[-1]), int(idx[-1])
    ahead = int((full > last).sum().item())
    ties = torch.nonzero(full == last).flatten()
    ahead += int((ties < lr).sum().item())
    assert ahead == k - 1
