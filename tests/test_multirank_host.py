"""The N > 1 bench path on CPU: world_size-2 gloo ranks (no GPU).  Each rank
advances its own replica -- the BSSN path does not shard -- so the only
collective is the max over ranks of the timed region, and the whole-job rate
is the units all ranks processed over that max."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 100.0 + 50.0 * rank          # the slower rank decides
    rate, ms = bench.whole_job_rate(1000, 10, ms_local, world)
    out[rank] = (rate, ms, bench.max_over_ranks(float(rank), world))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_uses_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        rate, ms, mx = out[r]
        assert ms == pytest.approx(150.0)
        assert rate == pytest.approx(1000 * 10 * 2 / 0.150 / 1e6)
        assert mx == 1.0
