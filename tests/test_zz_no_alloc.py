"""The Top-K entry point that allocates nothing (olap_topk_noalloc).

It exists for callers that cannot let a library allocate GPU memory (engines
whose device memory belongs to their own pool, operator hosts that forbid
allocation, paths that cannot take cudaMalloc's synchronisation); its working
memory is a fixed array inside the library.  This test calls it through the C
ABI twice in a row -- the second call reusing the array the first one left
behind -- and once more at the size limits, where its working set is largest,
and checks each result against the CPU oracle and against olap_topk on the
same input.  The results are integers and row-ids, so the comparison is
exact.  This file is collected last so that a failure here comes after every
other test has run.
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


def _noalloc(keys_np, k, order):
    dk = torch.from_numpy(keys_np).cuda()
    cnt = min(k, keys_np.shape[0])
    ok = torch.empty(cnt, dtype=dk.dtype, device="cuda")
    orow = torch.empty(cnt, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    lib = olap.load()
    st = lib.olap_topk_noalloc(dk.data_ptr(), olap.key_type_of(dk), None, dk.numel(), k, order,
                               ok.data_ptr(), orow.data_ptr(), status.data_ptr(), None)
    assert st == olap.OK
    torch.cuda.synchronize()
    assert int(status.item()) == olap.OK
    return ok.cpu().numpy(), orow.cpu().numpy().view(np.uint32)


def _same(keys, k, order, ctx):
    gk, gr = _noalloc(keys, k, order)
    ok, orow = oracle.topk(keys, k, order)
    np.testing.assert_array_equal(gr, orow)
    np.testing.assert_array_equal(gk.view(np.uint8), ok.view(np.uint8))
    wk, wr = ctx.topk(keys, k, order)
    np.testing.assert_array_equal(gr, wr)
    np.testing.assert_array_equal(gk.view(np.uint8), wk.view(np.uint8))


def test_two_calls_in_a_row_match_oracle_and_olap_topk(ctx):
    # First call: sampled single-pass path (n > 2^21), int64, DESC.
    a = datagen.topk_keys(3_000_001, "uniform", "i64", seed=31)
    # Second call: direct path, float32 with duplicates, ASC, the largest k.
    b = datagen.topk_keys(200_003, "dup1024", "f32", seed=32)
    _same(a, 1000, olap.DESC, ctx)
    _same(b, olap.NOALLOC_MAX_K, olap.ASC, ctx)


def test_at_the_size_limits(ctx):
    # n and k at their maxima on the sampled path: the largest candidate
    # buffer the fixed array has to hold.
    keys = datagen.topk_keys(olap.NOALLOC_MAX_N, "uniform", "i64", seed=33)
    _same(keys, olap.NOALLOC_MAX_K, olap.DESC, ctx)


def test_sizes_beyond_the_array_are_refused():
    lib = olap.load()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    d = torch.zeros(16, dtype=torch.int64, device="cuda")
    st = lib.olap_topk_noalloc(d.data_ptr(), olap.KEY_I64, None, olap.NOALLOC_MAX_N + 1, 10, olap.DESC,
                               d.data_ptr(), d.data_ptr(), None, None)
    assert st == olap.E_INVALID
    st = lib.olap_topk_noalloc(d.data_ptr(), olap.KEY_I64, None, 16, olap.NOALLOC_MAX_K + 1, olap.DESC,
                               d.data_ptr(), d.data_ptr(), None, None)
    assert st == olap.E_INVALID
    with pytest.raises(ValueError):
        olap.topk_noalloc(torch.zeros(olap.NOALLOC_MAX_N + 1, dtype=torch.int64, device="cuda"), 10,
                          olap.DESC, d, d)
