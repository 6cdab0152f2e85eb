"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas), the
timed region's duration is the maximum over ranks, throughput counts the units
of all ranks, and every rank draws its own seeded particles."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    wl, X0, _ = bench.initial_state(rank)
    out[rank] = (ms, bench.job_throughput(wl.N * wl.p, 4, world, ms), float(X0[0, :8].sum()))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    import bench
    bench.WL.update(N=2000, p=4)  # small replicas: the rank logic, not the workload
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_entry, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0                     # max over ranks
    assert res[0][1] == pytest.approx(2000 * 4 * 4 * 2 / 0.02)  # all ranks' units
    assert res[0][2] != res[1][2]                              # each replica its own seed


def _rank_entry(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    bench.WL.update(N=2000, p=4)
    _rank(rank, world, port, out)
