"""Full-row offload (olap_topk_rows), the foil of key-only transfer with late
materialization (Sec. II-C, Sec. V-E): the returned rows are exactly the rows
the oracle's Top-K of the key field selects, in order, for aligned and
unaligned key fields, every key width, host and device tables; and they equal
the key-only result materialized on the host by row-id."""
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


def _table(n, row_bytes, key_offset, keys, seed):
    payload = np.frombuffer(datagen.splitmix64(seed, (n * row_bytes + 7) // 8).tobytes(), dtype=np.uint8)
    t = payload[: n * row_bytes].copy().reshape(n, row_bytes)
    kb = keys.view(np.uint8).reshape(n, keys.dtype.itemsize)
    t[:, key_offset:key_offset + keys.dtype.itemsize] = kb
    return t


@pytest.mark.parametrize("kt,row_bytes,key_offset", [("f64", 108, 0), ("f64", 103, 3), ("i64", 64, 56),
                                                      ("i32", 100, 96), ("f32", 13, 5), ("u64", 8, 0)])
@pytest.mark.parametrize("where", ["host", "device"])
def test_rows_match_oracle(ctx, kt, row_bytes, key_offset, where):
    for n, k in ((1, 5), (4097, 100), (3_000_017, 1000)):
        keys = datagen.topk_keys(n, "uniform" if n % 2 else "dup1024", kt, seed=n % 89)
        t = _table(n, row_bytes, key_offset, keys, seed=n)
        src = t if where == "host" else torch.from_numpy(t).cuda()
        for order in (olap.DESC, olap.ASC):
            got_rows, got_rid = ctx.topk_rows(src, row_bytes, key_offset, olap.key_type_of(keys), k, order)
            wk, wr = oracle.topk(keys, k, order)
            np.testing.assert_array_equal(got_rid, wr)
            np.testing.assert_array_equal(got_rows[: len(wr) * row_bytes].reshape(-1, row_bytes), t[wr])
            # key-only + late materialization gives the same rows
            ko, kr = ctx.topk(keys, k, order)
            np.testing.assert_array_equal(t[kr], t[wr])


def test_bad_key_field(ctx):
    t = np.zeros((10, 16), dtype=np.uint8)
    with pytest.raises(olap.OlapError) as ei:
        ctx.topk_rows(t, 16, 12, olap.KEY_I64, 3)
    assert ei.value.status == olap.E_INVALID
