"""The multi-GPU path of bench.py on CPU with gloo (world size 2): each rank
aligns its own batch (distinct seeds), and the whole-job throughput is the
units of all ranks over the slowest rank's time.  No collective touches the
data path; pairs never cross ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    pairs = synth.config2(seed=bench.rank_seed(2, rank), n=3)
    units, secs = bench.job_totals(100.0 * (rank + 1), 1.0 + rank, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, units, secs, pairs[0].prot))


def test_two_ranks_weak_scaling_totals():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, units, secs, _ in res:
        assert units == 300.0 and secs == 2.0          # sum of units, max of times
    assert res[0][3] != res[1][3]                      # each rank aligns its own pairs


def test_single_process_totals():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_totals(5.0, 2.0) == (5.0, 2.0)
    assert bench.rank_seed(2, 0) == 2 and bench.rank_seed(2, 3) == 3002
