"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
read-set figures, must agree on the whole-job totals (sums of (k+1)-mers and
SdBG entries, maximum of the timed durations).  No GPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    res = bench.job_totals(dist, "cpu", kmers=1000 * (rank + 1), edges=10 * (rank + 1), ms=5.0 + rank,
                           e2e_s=0.5 * (world - rank))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, res))


@pytest.mark.parametrize("world", [2, 3])
def test_job_totals_over_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = {"kmers": 1000 * world * (world + 1) // 2, "edges": 10 * world * (world + 1) // 2,
            "ms": 5.0 + world - 1, "e2e_s": 0.5 * world}
    for r in range(world):
        assert out[r] == want


def test_job_totals_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(None, "cpu", 7, 3, 2.0, 1.0) == {"kmers": 7, "edges": 3, "ms": 2.0, "e2e_s": 1.0}
