"""The multi-rank path of the benchmark on CPU (gloo, world size 2): every
rank runs its own replica, the timed region is the slowest rank's, and the
whole-job throughput counts all ranks' flops over that time; the reference
arm runs on rank 0 only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        t = bench.slowest_rank_ms(10.0 + 5.0 * rank, dist, torch.device("cpu"))
        out.put((r, ws, local, t, bench.whole_job_tflops(ws, 2.0e12, 4, t)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 and r[2] == r[0] for r in res)
    assert all(r[3] == 15.0 for r in res)                       # the slowest rank's time, on every rank
    assert all(abs(r[4] - 2 * 2.0e12 * 4 / 15e-3 / 1e12) < 1e-9 for r in res)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        n, steps, warmup = 64, 1, 0
    bench.reference_arm(Args())            # rank 1: returns at once, prints nothing
    assert capsys.readouterr().out == ""
