"""The N-rank path of bench.py on CPU: world-size-2 gloo ranks.

The bench runs one independent replica per GPU (gathers are independent: no
collective on the data path) and reports the whole job: the slowest rank's
time, and every rank's units over it.  This checks that aggregation with two
gloo ranks that report different times, and that the reference arm runs on
rank 0 only.
"""
import contextlib
import io
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    t, value = bench.whole_job_rate(0.5 + rank, 10.0, world, dist, "cpu")
    out.put((rank, t, value))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, value in res:
        assert t == pytest.approx(1.5)
        assert value == pytest.approx(2 * 10.0 / 1.5)


def test_single_rank_rate():
    import bench
    t, value = bench.whole_job_rate(2.0, 8.0, 1)
    assert (t, value) == (2.0, 4.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), dict(warmup=0, steps=1, gpus=2))()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
