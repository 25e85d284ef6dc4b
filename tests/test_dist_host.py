"""Host side of the multi-GPU path on CPU: two gloo ranks.

The workload shards as independent replicas (cells are independent, so
every rank builds its own copy and no collective touches the data); what
the ranks share is the barrier and the max-over-ranks time from which the
whole-job value is computed.  The reference arm runs on rank 0 only.
"""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    ws, r, _ = bench.dist_init(None)
    assert dist.get_backend() == "gloo"
    bench.barrier(ws)
    slowest = bench.max_over_ranks(ws, 1.0 + r)          # rank 1 is the slow one
    value = bench.aggregate(ws, 1000.0, 0.5 + 0.25 * r)
    out.put((r, ws, slowest, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_barrier_and_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, ws, slowest, value in got:
        assert ws == 2
        assert slowest == 2.0
        assert value == pytest.approx(2 * 1000.0 / 0.75)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
