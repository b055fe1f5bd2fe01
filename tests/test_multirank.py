"""The N > 1 path of bench.py on the CPU: two gloo ranks (127.0.0.1), each an
independent replica with a seed of its own.  Checks the host logic that the
GPU run uses -- rank/world from the environment, barrier, whole-job
aggregation (units summed, time of the slowest rank) -- and that replicas
differ and step independently (the oracle stands in for the device step, so
nothing here needs a GPU).  The reference arm's non-zero ranks exit without
work."""
import argparse
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r = bench._dist()
        assert (ws, r) == (world, rank)
        w = bench.headline_workload("heat_bath", rank, n_cells=3, per_cell=200)
        o = oracle.from_workload(w)
        n0 = o.count(0)
        o.step(2)
        bench._barrier()
        units, secs = bench.aggregate(float(n0 * 2), 1.0 + rank)
        v, q, s, c = o.read_particles(0)
        # the reference arm: ranks other than 0 return at once, printing nothing
        rc = bench.run_reference(argparse.Namespace(steps=1, warmup=0, workload="exchange")) if rank != 0 else 0
        out.put((rank, n0, units, secs, float(np.sum(v * v)), rc))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_replicas_and_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, u0, s0, e0, rc0), (r1, n1, u1, s1, e1, rc1) = res
    assert u0 == u1 == 2.0 * (n0 + n1)      # units summed over ranks
    assert s0 == s1 == 2.0                  # the slowest rank's time
    assert e0 != e1                         # replicas have seeds of their own
    assert rc1 == 0
