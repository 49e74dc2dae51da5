"""The seeded generators: determinism, chunk independence and the shapes the
workloads ask for."""
import numpy as np

from paper_2601_19911_gb300 import datagen


def test_splitmix_chunk_independent():
    a = datagen.splitmix64(11, (1 << 22) + 1000)
    b = np.concatenate([datagen.splitmix64(11, 1000), datagen.splitmix64(11, (1 << 22), start=1000)])
    assert np.array_equal(a, b)
    assert np.array_equal(datagen.splitmix64(11, 10), datagen.splitmix64(11, 10))
    assert not np.array_equal(datagen.splitmix64(11, 10), datagen.splitmix64(12, 10))


def test_splitmix_first_value():
    # seed 0: the first output is mix(0x9E3779B97F4A7C15), computed with Python ints
    z = 0x9E3779B97F4A7C15
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & (2**64 - 1)
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & (2**64 - 1)
    z ^= z >> 31
    assert int(datagen.splitmix64(0, 1)[0]) == z


def test_topk_shapes():
    for kt in ("i64", "f32"):
        a = datagen.topk_keys(10000, "ascending", kt)
        if kt == "i64":
            assert np.all(np.diff(a) > 0)
        else:
            assert np.all(np.isfinite(a)) and np.all(a[1:] > a[:-1])
        d = datagen.topk_keys(50000, "dup1024", kt, seed=1)
        assert np.unique(d.view(np.uint64 if kt == "i64" else np.uint32)).shape[0] == 1024
    u = datagen.topk_keys(1 << 16, "uniform", "f32")
    assert np.isnan(u).sum() > 0          # full 32-bit patterns include NaNs


def test_join_shapes():
    b = datagen.join_build(10000, "mult14", seed=3)
    assert b.keys.shape[0] == 10000
    _, c = np.unique(b.keys, return_counts=True)
    assert c.min() >= 1 and c.max() <= 4 and abs(c.mean() - 2.5) < 0.1
    u = datagen.join_build(10000, "unique", seed=3)
    assert np.unique(u.keys).shape[0] == 10000
    p = datagen.join_probe(50000, u, 0.1, "uniform", seed=3)
    assert abs(p.hit.mean() - 0.1) < 0.01
    assert np.all(np.isin(p.keys[p.hit], u.keys)) and not np.any(np.isin(p.keys[~p.hit], u.keys))


def test_log_uniform_range():
    ns, ks = datagen.batched_topk_queries(4096)
    assert ns.min() >= 1000 and ns.max() < 4e6 and ks.min() >= 1 and ks.max() <= 1000


def test_torch_stream_equals_numpy_stream():
    torch = __import__("pytest").importorskip("torch")
    a = datagen.splitmix64(stream_seed := datagen.stream_seed(3, 0), 5000, start=17)
    b = datagen.splitmix64_torch(stream_seed, 5000, start=17, device="cpu", chunk=777).numpy().view(np.uint64)
    assert np.array_equal(a, b)
