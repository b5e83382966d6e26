"""Multi-process host logic of bench.py on CPU (gloo, world size 2):
every ensemble lattice goes to exactly one rank, and the timing reduction
takes the maximum over ranks."""
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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import mhd_inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    draws = mhd_inputs.ensemble(512)
    mine = bench.partition(draws, rank, world)
    out[rank] = ([d["seed"] for d in mine], bench.reduce_max(10.0 * (rank + 1), dist),
                 bench.reduce_max(sum(d["n"] ** 2 for d in mine), dist))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_and_max_reduction_over_two_gloo_ranks():
    import mhd_inputs
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    seeds = res[0][0] + res[1][0]
    all_seeds = [d["seed"] for d in mhd_inputs.ensemble(512)]
    assert sorted(seeds) == sorted(all_seeds) and len(set(res[0][0]) & set(res[1][0])) == 0
    assert res[0][1] == res[1][1] == 20.0
    assert res[0][2] == res[1][2] == max(sum(d["n"] ** 2 for d in mhd_inputs.ensemble(512)[r::2])
                                         for r in range(2))
