"""Batched reservoirs: many independent 0D reservoirs advanced by one launch
sequence (CUDA graph) give, reservoir by reservoir, exactly what each gives
alone, in both precisions; FP64 matches the oracle bit for bit; the launch-shape
autotuner does not change any result."""
import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _small_batch(n_res=6, steps=10):
    return W.batched_reservoirs(n_res=n_res, n_min=1500, n_max=20000, T_min=5000.0, T_max=30000.0,
                                steps=steps, seed=0x5EED)


def _state(ctx, res):
    v, q, s, c = ctx.read_particles(res)
    return v, q, s, c


@pytest.mark.parametrize("precision", [hcao.FP64, hcao.FP32])
def test_batched_equals_each_alone(precision):
    bw = _small_batch()
    g = hcao.from_batched(bw, precision=precision)
    g.step(bw.steps)  # CUDA-graph path
    g.sync()
    for i, w in enumerate(bw.reservoirs):
        a = hcao.from_workload(w, precision=precision)
        for _ in range(bw.steps):
            a.step(1)  # one launch sequence per step
        va, qa, sa, ca = _state(a, 0)
        vb, qb, sb, cb = _state(g, i)
        assert np.array_equal(qa, qb) and np.array_equal(sa, sb) and np.array_equal(ca, cb)
        assert np.array_equal(va, vb)
        a.close()


def test_batched_fp64_matches_oracle():
    bw = _small_batch(n_res=4, steps=6)
    g = hcao.from_batched(bw, precision=hcao.FP64)
    g.step(bw.steps)
    g.sync()
    o = oracle.from_batched(bw)
    o.step(bw.steps)
    for i in range(len(bw.reservoirs)):
        vg, qg, sg, cg = _state(g, i)
        vo, qo, so, co = o.read_particles(i)
        assert np.array_equal(qg, qo) and np.array_equal(sg, so)
        assert np.array_equal(vg, vo)


def test_autotune_does_not_change_results():
    bw = _small_batch(n_res=5, steps=9)
    a = hcao.from_batched(bw, precision=hcao.FP32)
    chosen = a.autotune(1)  # 7 steps while timing grids, 2 more for the work-class placement
    done = int(a.read_counters(0)[7])
    assert done == 9  # triatomic and CH4-like reservoirs: two work classes
    a.step(11 - done)
    b = hcao.from_batched(bw, precision=hcao.FP32)
    b.step(11)
    for i in range(len(bw.reservoirs)):
        va, qa, _, _ = _state(a, i)
        vb, qb, _, _ = _state(b, i)
        assert np.array_equal(qa, qb) and np.array_equal(va, vb)
    assert chosen[0] > 0 and chosen[1] > 0 and chosen[2] in (0, 1)


def test_autotune_single_work_class():
    """One species: a single work class, so the queue goes straight to its
    place (no placement kernel) and the autotuner times only the grids."""
    w = W.relaxation_triatomic(n_particles=20000, n_cells=8)
    g = hcao.from_workload(w, precision=hcao.FP32)
    n0 = g.kernel_launches()
    g.step(1)
    assert g.kernel_launches() - n0 == 2 + 2 * 2 + 2  # set-up, (select, relax) x 2 rounds, finish
    chosen = g.autotune(1)
    assert int(g.read_counters(0)[7]) == 8 and chosen[2] == 0


def test_remove_all_then_add_again():
    """Reservoirs come and go (the serving pattern): removing the last one and
    adding another keeps the context usable and the results unchanged."""
    bw = _small_batch(n_res=3, steps=4)
    p = hcao.Context(precision=hcao.FP32)
    p.set_species(bw.species)
    results = []
    for w in bw.reservoirs:
        rid = p.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
        p.load_particles(rid, w.v, w.qn0(), w.species_idx, w.cell)
        p.init_vibration(rid, w.T_vib0)
        p.step(bw.steps)
        results.append(p.read_particles(rid))
        p.remove_reservoir(rid)
    g = hcao.from_batched(bw, precision=hcao.FP32)
    g.step(bw.steps)
    for i, (v, q, s, c) in enumerate(results):
        v2, q2, s2, c2 = g.read_particles(i)
        assert np.array_equal(q, q2) and np.array_equal(v, v2)
