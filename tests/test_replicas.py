"""The N-GPU path is N replicas (no collective on the data path): two gloo
ranks on the CPU check the bookkeeping the benchmark uses -- rank/world from
the launcher's environment, the barrier, the maximum of the per-rank times
on every rank, and the whole-job throughput (all ranks' units over the
slowest rank's time)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    from paper_2601_19911_gb300 import replicas
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = replicas.env()
        replicas.barrier(w)
        my_time = 0.5 + rank                    # rank 1 is the slower one
        t = replicas.max_over_ranks(my_time, w, device="cpu")
        rate = replicas.whole_job_rate(1000.0, w, t)
        replicas.barrier(w)
        q.put((r, w, lr, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for r, w, lr, t, rate in got:
        assert w == 2 and lr == r
        assert t == 1.5                          # every rank sees the slowest time
        assert rate == pytest.approx(2 * 1000.0 / 1.5)


def test_single_process_defaults(monkeypatch):
    from paper_2601_19911_gb300 import replicas
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.env() == (1, 0, 0)
    assert replicas.max_over_ranks(3.25, 1) == 3.25
    replicas.barrier(1)
    assert replicas.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_prints_only_on_rank_zero(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = bench.build_parser().parse_args(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
