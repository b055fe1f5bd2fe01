"""The multi-GPU split on one GPU: a workload cut into contiguous cell ranges,
each loaded as a reservoir keyed by its global cell indices
(hcao_set_cell_base), steps exactly as the whole workload: the ranges'
particles, in order, equal the unsplit run bit for bit in both precisions,
and equal the oracle's in FP64 mode.  This is what each rank of bench.py
--gpus N does with its range (no data-path collective)."""
import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _ranges(kind, total, per_cell, cuts, precision):
    g = hcao.Context(precision=precision)
    whole = W.cell_range(kind, 0, total, total, per_cell=per_cell)
    g.set_species(whole.species)
    g.set_reactions(whole.reactions)
    bounds = [0] + list(cuts) + [total]
    for a, b in zip(bounds[:-1], bounds[1:]):
        w = W.cell_range(kind, a, b, total, per_cell=per_cell)
        rid = g.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
        g.set_cell_base(rid, w.cell_base)
        g.load_particles(rid, w.v, w.qn0(), w.species_idx, w.cell)
        g.init_vibration(rid, w.T_vib0)
    return g, bounds


@pytest.mark.parametrize("precision", [hcao.FP64, hcao.FP32])
@pytest.mark.parametrize("kind,total,per_cell", [("exchange", 40, 600), ("heat_bath", 30, 400)])
def test_split_ranges_equal_whole(kind, total, per_cell, precision):
    steps = 4
    g, bounds = _ranges(kind, total, per_cell, [13, 27] if total == 40 else [11], precision)
    whole = W.cell_range(kind, 0, total, total, per_cell=per_cell)
    u = hcao.from_workload(whole, precision=precision)
    g.step(steps)
    u.step(steps)
    vu, qu, su, cu = u.read_particles(0)
    parts = [g.read_particles(r) for r in range(len(bounds) - 1)]
    assert np.array_equal(np.concatenate([p[3] + b for p, b in zip(parts, bounds)]), cu)
    assert np.array_equal(np.concatenate([p[2] for p in parts]), su)
    assert np.array_equal(np.concatenate([p[1] for p in parts]), qu)
    assert np.array_equal(np.concatenate([p[0] for p in parts]), vu)
    if precision == hcao.FP64:
        o = oracle.from_workload(whole)
        o.step(steps)
        vo, qo, so, co = o.read_particles(0)
        assert np.array_equal(vo, vu) and np.array_equal(qo, qu) and np.array_equal(so, su)


def test_cell_base_only_before_load():
    w = W.cell_range("exchange", 2, 4, 8, per_cell=50)
    g = hcao.from_workload(w, precision=hcao.FP64)
    with pytest.raises(hcao.HcaoError):
        g.set_cell_base(0, 5)
