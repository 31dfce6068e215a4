"""The replicas-only multi-GPU path of bench.py on the host: two gloo ranks on CPU.

The all-pairs path does not shard here (one GPU per process, every rank runs the whole problem
on its own copy), so the only collective is the maximum over the ranks of each measured time,
and the whole-job rate counts every rank's pairs against the slowest rank's time. The reference
arm runs on rank 0 alone; other ranks return without work.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (world, rank, rank)
        # rank r measured (1 + r) ms, (3 - r) ms and 5 ms: every rank sees the slowest of each
        got = bench.max_over_ranks([1.0 + rank, 3.0 - rank, 5.0], "cpu", world)
        rate = bench.whole_job_rate(1000, got[0], world)
        # the reference arm: rank 0 alone prints (here with a tiny sample), the others return
        args = bench.parse(["--impl", "reference", "--N", "40", "--L", "20", "--steps", "1",
                                          "--warmup", "0", "--ref-models", "12"])
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.run_reference(args)
        q.put((rank, got, rate, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict()
    for _ in range(2):
        rank, got, rate, printed = q.get(timeout=240)
        res[rank] = (got, rate, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        got, rate, _ = res[rank]
        assert got == [2.0, 3.0, 5.0]
        assert rate == pytest.approx(2 * 1000 / 2e-3)
    assert '"impl": "reference"' in res[0][2] and res[1][2] == ""
