"""The N > 1 path of bench.py on the CPU: two gloo ranks (127.0.0.1), each
stepping a contiguous range of one workload's cells.  Checks the host logic
that the GPU run uses -- rank/world from the environment, barrier, whole-job
aggregation (units summed, time of the slowest rank) -- and that the split
does not change the result: the two ranges, stepped as separate contexts on
separate ranks, reproduce the unsplit run of all cells bit for bit (the
oracle stands in for the device step, so nothing here needs a GPU).  The
reference arm's non-zero ranks exit without work."""
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
        w = bench.headline_workload("heat_bath", rank, world, cells_per_rank=3, per_cell=200)
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
    assert e0 != e1                         # the ranks hold different cells
    assert rc1 == 0


def _split_rank(rank, world, port, out, kind, total, per_cell, steps):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_2606_31548_b300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c0, c1 = rank * total // world, (rank + 1) * total // world
        w = W.cell_range(kind, c0, c1, total, per_cell=per_cell)
        o = oracle.from_workload(w)
        o.step(steps)
        v, q, s, c = o.read_particles(0)
        parts = [None] * world
        dist.all_gather_object(parts, (v, q, s, c + c0, o.read_counters(0), o.read_cell_sgmax(0, w.n_cells)))
        out.put((rank, parts if rank == 0 else None))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
@pytest.mark.parametrize("kind,total,per_cell,steps", [("exchange", 6, 300, 3), ("heat_bath", 5, 200, 4)])
def test_two_gloo_ranks_split_equals_unsplit(kind, total, per_cell, steps):
    """One workload split into two contiguous cell ranges, one per gloo rank,
    each stepped as a separate oracle context keyed by its global cell
    indices: the gathered particles, counters and (sigma g)_max equal the
    unsplit run of all cells bit for bit (the heat bath with dissociation
    creates particles in both ranges)."""
    import oracle
    from paper_2606_31548_b300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank, args=(r, 2, port, q, kind, total, per_cell, steps)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=240) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = got[0]
    whole = W.cell_range(kind, 0, total, total, per_cell=per_cell)
    o = oracle.from_workload(whole)
    o.step(steps)
    v, qn, s, c = o.read_particles(0)
    assert np.array_equal(np.concatenate([p[3] for p in parts]), c)
    assert np.array_equal(np.concatenate([p[2] for p in parts]), s)
    assert np.array_equal(np.concatenate([p[1] for p in parts]), qn)
    assert np.array_equal(np.concatenate([p[0] for p in parts]), v)
    cnt = o.read_counters(0)
    assert np.array_equal(parts[0][4] + parts[1][4] - np.array([0] * 7 + [steps] + [0] * (len(cnt) - 8), np.uint64),
                          cnt)  # the step counter is per context
    assert np.array_equal(np.concatenate([p[5] for p in parts]), o.read_cell_sgmax(0, total))
    # keyed by the local index instead, the upper range would draw other numbers
    w1 = W.cell_range(kind, total // 2, total, total, per_cell=per_cell)
    w1.cell_base = 0
    o1 = oracle.from_workload(w1)
    o1.step(steps)
    assert not np.array_equal(o1.read_particles(0)[0], parts[1][0])
