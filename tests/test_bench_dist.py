"""The multi-rank path of bench.py on CPU (gloo, world size 2): ranks run
independent replicas, the job time is the slowest rank's, the throughput
aggregates all ranks' bytes (weak scaling), and no collective touches the
data path."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    ms = [4.0, 10.0][rank]                      # rank 1 is the slow one
    slowest = bench.max_over_ranks(ms, world)
    gbs = bench.job_throughput(5e9, ms, world)  # 5 GB per rank
    bench.barrier(world)
    q.put((rank, slowest, gbs))
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, gbs in out:
        assert slowest == 10.0
        assert gbs == pytest.approx(2 * 5e9 / 10e-3 / 1e9)
