"""The multi-GPU path of the bench is replicas only (one independent grid
per rank, no data-path collective): its host logic -- the slowest rank's
time taken by every rank, whole-job throughput, only rank 0 reporting -- run
as two gloo ranks on the CPU."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        value = bench.job_throughput(world, 1000, 4, t)
        buf = io.StringIO()
        with redirect_stdout(buf):
            args = type("A", (), {"steps": 1, "warmup": 0, "n": 4})()
            rc = bench.run_reference(args, rank, world) if rank != 0 else 0
        q.put((rank, t, value, rc, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value, rc, out in res:
        assert t == 2.5                       # the slower rank's time, on every rank
        assert value == pytest.approx(2 * 1000 * 4 / 2.5)
        assert rc == 0
    # the reference arm: ranks other than 0 exit without work or output
    assert res[1][4] == ""


def test_single_process_passthrough():
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.job_throughput(1, 10, 2, 4.0) == 5.0
