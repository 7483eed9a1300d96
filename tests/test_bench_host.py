"""Host-side logic of the multi-rank benchmark: each rank advances its own
replica; the job's value is the units of all ranks over the slowest rank's
time.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.allmax(world, 1.0 + rank)          # slowest rank: 2 s
    u = bench.allsum(world, 100.0 * (rank + 1))  # 100 + 200 units
    bench.barrier(world)
    out.put((rank, u / t))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {0: 150.0, 1: 150.0}


def test_step_units_follow_the_paper_rate():
    import bench
    import kg_inputs as KI
    m = KI.make(1)
    units, att = bench.step_units(m)
    assert units == m.M * 50
    assert att == pytest.approx(1e-3 * m.M * 50 * 0.01)     # R_MC = 1e-3 per monomer per tau
