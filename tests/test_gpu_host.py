"""Pageable host memory in and out, through both ways of crossing the host
link: the copy kernel that reads and writes pageable memory itself (where the
device supports it) and the pinned double-buffer staging.  Inputs are numpy
slices at every alignment the copy has to line up (offsets of 1..3 elements),
results bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2601_19911_gb300 import datagen, olap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[olap.HOST_AUTO, olap.HOST_STAGED], ids=["auto", "staged"])
def hctx(request):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0, host_access=request.param)
    if request.param == olap.HOST_STAGED:
        assert not c.host_direct
    yield c
    c.close()


@pytest.mark.parametrize("off", [0, 1, 2, 3])
@pytest.mark.parametrize("kt", ["i64", "f32"])
def test_topk_pageable_slices(hctx, off, kt):
    base = datagen.topk_keys(3_000_011, "uniform", kt, seed=50 + off)
    keys = base[off:]                                   # 4- or 8-byte aligned, not 16
    rid_base = (datagen.splitmix64(51, base.shape[0]) >> np.uint64(40)).astype(np.uint32)
    rowids = rid_base[off:]
    for k in (1, 333, 5000):
        ok = np.empty(k + 3, dtype=keys.dtype)[3:] if off else np.empty(k, dtype=keys.dtype)
        orow = np.empty(k + 1, dtype=np.uint32)[1:]     # outputs at odd offsets too
        gk, gr = hctx.topk(keys, k, olap.DESC, rowids=rowids, out_keys=ok, out_rowids=orow)
        wk, wr = oracle.topk(keys, k, olap.DESC, rowids)
        np.testing.assert_array_equal(gr, wr)
        np.testing.assert_array_equal(gk.view(np.uint8), wk.view(np.uint8))


@pytest.mark.parametrize("off", [0, 1, 3])
def test_join_pageable_slices(hctx, off):
    b = datagen.join_build(120_000 + off, "mult14", seed=52)
    p = datagen.join_probe(900_001, b, 0.7, "uniform", seed=52)
    bk = np.concatenate([np.zeros(off, dtype=np.int64), b.keys])[off:]
    pk = np.concatenate([np.zeros(off, dtype=np.int64), p.keys])[off:]
    t = hctx.join_build(bk)
    got = hctx.join_probe(t, pk)                       # pairs back into pageable memory
    t.free()
    got = got.astype(np.uint64)
    got = np.sort((got[:, 0] << np.uint64(32)) | got[:, 1])
    np.testing.assert_array_equal(got, oracle.join(b.keys, p.keys))


def test_empty_and_tiny(hctx):
    for n in (0, 1, 15, 17):
        keys = datagen.topk_keys(n + 1, "uniform", "i64", seed=n)[1:]
        gk, gr = hctx.topk(keys, 10, olap.ASC)
        wk, wr = oracle.topk(keys, 10, olap.ASC)
        np.testing.assert_array_equal(gr, wr)


def test_bounded_wait_reports_timeout_and_context_survives():
    """Every device-side spin in the library is bounded: the self-test runs the
    grid barriers' wait on a word that nothing writes, with a short limit
    (about 1 ms of SM clock), and the wait must expire with OLAP_E_TIMEOUT.
    The context keeps working afterwards."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0)
    try:
        assert c.selftest_wait(2_000_000) == olap.E_TIMEOUT
        assert c.selftest_wait(50_000) == olap.E_TIMEOUT
        keys = datagen.topk_keys(100_000, "uniform", "i64", seed=99)
        gk, gr = c.topk(keys, 10, olap.DESC)
        np.testing.assert_array_equal(gr, oracle.topk(keys, 10, olap.DESC)[1])
        with pytest.raises(olap.OlapError):
            c.selftest_wait(0)
    finally:
        c.close()


@pytest.mark.parametrize("kt", ["i64", "f32"])
def test_pinned_rowids_are_read_in_place(kt):
    """On the sampled path a blocking Top-K with row-ids in page-locked host
    memory reads only the candidates' row-ids, in place: reversed row-ids,
    1024 distinct keys (so the row-id tie-break decides), both orders and two
    k, against the oracle; all-equal keys send the select back to the input
    (every row-id then read in host memory); pageable and device row-ids are
    still copied."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = olap.Context(0)
    try:
        n = 3_000_007
        keys = datagen.topk_keys(n, "dup1024", kt, seed=81)
        rid = np.arange(n - 1, -1, -1, dtype=np.int64).astype(np.uint32)
        hk = torch.from_numpy(keys).pin_memory()
        hr = torch.from_numpy(rid.view(np.int32)).pin_memory()
        for k, order in ((1000, olap.DESC), (1000, olap.ASC), (10_000, olap.DESC)):
            gk, gr = c.topk(hk, k, order, rowids=hr)
            assert c.topk_info()["rowids_in_place"] and c.topk_info()["path"] == 1
            wk, wr = oracle.topk(keys, k, order, rid)
            np.testing.assert_array_equal(np.asarray(gr), wr)
            np.testing.assert_array_equal(np.asarray(gk).view(np.uint8), wk.view(np.uint8))
        same = np.full(n, 7, dtype=keys.dtype)
        hs = torch.from_numpy(same).pin_memory()
        gk, gr = c.topk(hs, 1000, olap.DESC, rowids=hr)
        assert c.topk_info()["rowids_in_place"] and c.topk_info()["path"] == 2
        np.testing.assert_array_equal(np.asarray(gr), oracle.topk(same, 1000, olap.DESC, rid)[1])
        gk, gr = c.topk(keys, 1000, olap.DESC, rowids=rid)                  # pageable: copied
        assert not c.topk_info()["rowids_in_place"]
        np.testing.assert_array_equal(np.asarray(gr), oracle.topk(keys, 1000, olap.DESC, rid)[1])
        dk = torch.from_numpy(keys).cuda()
        dr = torch.from_numpy(rid.view(np.int32)).cuda()
        gk, gr = c.topk(dk, 1000, olap.DESC, rowids=dr)                      # device: used as they are
        assert not c.topk_info()["rowids_in_place"]
        np.testing.assert_array_equal(np.asarray(gr), oracle.topk(keys, 1000, olap.DESC, rid)[1])
    finally:
        c.close()
