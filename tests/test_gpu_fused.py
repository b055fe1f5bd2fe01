"""The fused per-cell collision kernel (one CTA per cell, records staged in
shared memory) against the per-round queue kernels, FP32 mode.

Both paths draw every random number from the same (step, cell, round, pair)
keyed streams and evaluate every floating-point expression with explicit
roundings, so after any number of steps they must agree bit for bit: every
particle's velocity, quantum numbers and species, every counter, every
cell's (sigma_T g)_max and the K5 work counts.  The full-size exchange
mixture (16384 cells x 1200, the benchmark's configuration) is checked for
conservation and, on sampled cells, against the fused kernel on those cells
alone (cells are independent and keyed by their index).
"""
import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _ragged():
    base = W.relaxation_triatomic(n_particles=10, n_cells=1)
    counts = np.array([0, 1, 2, 3, 5, 64, 127, 300, 0, 2, 1000, 2047])
    rng = np.random.default_rng(19)
    n = int(counts.sum())
    cell = np.repeat(np.arange(len(counts), dtype=np.int32), counts)
    base.cell = cell[rng.permutation(n)]
    base.n_cells = len(counts)
    base.species_idx = np.zeros(n, np.int32)
    base.v = W.maxwellian(rng, n, np.full(n, base.species[0].mass), 20000.0)
    base.weight = 1e23 * base.cell_volume / counts.max()
    return base


def _ragged_multitile():
    """1000 cells (four set-up tiles of 256) of 0..299 particles, a fifth of
    them empty: tile offsets and the block-cell table across tiles."""
    base = W.relaxation_triatomic(n_particles=10, n_cells=1)
    rng = np.random.default_rng(23)
    counts = rng.integers(0, 300, 1000)
    counts[rng.random(1000) < 0.2] = 0
    n = int(counts.sum())
    cell = np.repeat(np.arange(len(counts), dtype=np.int32), counts)
    base.cell = cell[rng.permutation(n)]
    base.n_cells = len(counts)
    base.species_idx = np.zeros(n, np.int32)
    base.v = W.maxwellian(rng, n, np.full(n, base.species[0].mass), 20000.0)
    base.weight = 1e23 * base.cell_volume / counts.max()
    return base


def _many_species():
    """Nine species of 0, 1, 3, 4, 6 and 9 modes: 31 distinct work keys
    (the mode counts of the molecules a pair relaxes, in order), more than the
    queue path's 16 work classes, so the lightest keys share the last class."""
    names = ["H2O", "OH", "N2", "HCN", "CH4", "CH3", "H2", "H", "N"]
    species = [W.paper_species(n) for n in names]
    return W._build("many_species", species, [], 40, np.full(40, 300), [1.0] * len(names), 4.64e-6, 1e23,
                    2.0e-9, 8000.0, 8000.0, 0x4D535053, 10)


def _two_rounds():
    w = W.relaxation_triatomic(n_particles=4000, n_cells=4)
    w.dt *= 3.0  # N_sel > N/2: two pairing rounds per step
    return w


CASES = {
    "exchange_4000K": (lambda: W.ch4_h_exchange(n_cells=48, per_cell=1200, T0=4000.0), {}),
    "exchange_2000K": (lambda: W.ch4_h_exchange(n_cells=24, per_cell=1200, T0=2000.0), {}),
    "ch4_bath_no_dissociation": (lambda: W.ch4_heat_bath(n_cells=40, per_cell=500, dissociation=False), {}),
    "triatomic_multicell": (lambda: W.relaxation_triatomic(n_particles=12000, n_cells=6), {}),
    "ragged_cells": (_ragged, {}),
    "ragged_multitile": (_ragged_multitile, {}),
    "many_species": (_many_species, {}),
    "two_rounds": (_two_rounds, {"max_rounds": 4}),
}


def _state(g, w):
    v, q, s, c = g.read_particles(0)
    return v, q, s, c, g.read_counters(0), g.read_cell_sgmax(0, w.n_cells), g.read_work()


@pytest.mark.parametrize("name", sorted(CASES))
def test_fused_equals_queue_path(name):
    make, kw = CASES[name]
    w = make()
    f = hcao.from_workload(w, precision=hcao.FP32, **kw)
    q = hcao.from_workload(w, precision=hcao.FP32, **kw)
    assert q.step_path() == hcao.PATH_QUEUE  # the default
    f.set_step_path(hcao.PATH_FUSED)
    assert f.step_path() == hcao.PATH_FUSED
    assert q.step_path() == hcao.PATH_QUEUE
    for s in (1, 1, 3, 5):
        f.step(s)
        q.step(s)
        a, b = _state(f, w), _state(q, w)
        for x, y, what in zip(a, b, ("v", "qn", "species", "cell", "counters", "sgmax", "work")):
            assert np.array_equal(x, y), (name, what)
    # one more step each with profiling on: the K5 work is counted then
    f.set_profiling(True)
    q.set_profiling(True)
    f.step(1)
    q.step(1)
    a, b = _state(f, w), _state(q, w)
    for x, y, what in zip(a, b, ("v", "qn", "species", "cell", "counters", "sgmax", "work")):
        assert np.array_equal(x, y), (name, what)
    assert a[6][3] > 0  # relaxed pairs counted
    c = f.read_counters(0)
    assert c[1] > 0 and c[7] == 11  # collisions happened; eleven steps
    if name.startswith("exchange"):
        assert c[8] > 0  # exchange events
    if name == "two_rounds":
        f.set_log(True)  # a per-pair log needs the queue path
        assert f.step_path() == hcao.PATH_QUEUE
        with pytest.raises(hcao.HcaoError):
            f.step(1)


def test_fused_path_eligibility():
    # dissociation creates particles: queue path, and the fused path is refused
    w = W.ch4_heat_bath(n_cells=8, per_cell=200)
    g = hcao.from_workload(w, precision=hcao.FP32)
    assert g.step_path() == hcao.PATH_QUEUE
    g.set_step_path(hcao.PATH_FUSED)
    with pytest.raises(hcao.HcaoError) as e:
        g.step(1)
    assert e.value.code == -1
    g.set_step_path(hcao.PATH_AUTO)
    g.step(1)
    # FP64 mode: queue path (the bit-exact oracle parity mode)
    w2 = W.ch4_h_exchange(n_cells=4, per_cell=300)
    assert hcao.from_workload(w2, precision=hcao.FP64).step_path() == hcao.PATH_QUEUE
    # a cell beyond the shared-memory limit (4096 slots): queue path
    w3 = W.relaxation_triatomic(n_particles=5000, n_cells=1)
    g3 = hcao.from_workload(w3, precision=hcao.FP32)
    g3.set_step_path(hcao.PATH_FUSED)
    assert g3.step_path() == hcao.PATH_QUEUE
    # no chemistry, small cells: fused on request; one fused launch per step
    w4 = W.relaxation_triatomic(n_particles=4000, n_cells=4)
    g4 = hcao.from_workload(w4, precision=hcao.FP32)
    assert g4.step_path() == hcao.PATH_QUEUE
    g4.set_step_path(hcao.PATH_FUSED)
    assert g4.step_path() == hcao.PATH_FUSED
    n0 = g4.kernel_launches()
    g4.step(7)
    assert g4.kernel_launches() - n0 == 7


def test_queue_path_launch_count():
    """The launches a step's CUDA graph replays are counted from its capture:
    the same count as the profiled step, which launches kernel by kernel.
    Exchange mixture, two rounds: set-up 2, per round select, work-class
    placement, relax and react, then the finish count and the cell update."""
    w = W.ch4_h_exchange(n_cells=16, per_cell=600)
    g = hcao.from_workload(w, precision=hcao.FP32)
    p = hcao.from_workload(w, precision=hcao.FP32)
    p.set_profiling(True)
    n0, m0 = g.kernel_launches(), p.kernel_launches()
    g.step(3)
    p.step(3)
    assert g.kernel_launches() - n0 == p.kernel_launches() - m0 == 3 * 12
    a, b = _state(g, w), _state(p, w)
    for x, y in zip(a[:6], b[:6]):
        assert np.array_equal(x, y)
    # the K5 work is counted on profiled steps only
    assert int(a[6].sum()) == 0 and b[6][3] > 0


def test_fused_profiling_class():
    w = W.ch4_h_exchange(n_cells=16, per_cell=1200)
    g = hcao.from_workload(w, precision=hcao.FP32)
    g.set_step_path(hcao.PATH_FUSED)
    g.set_profiling(True)
    g.step(3)
    ms, n = g.read_profile()
    assert int(n[5]) == 3 and ms[5] > 0.0
    assert int(n[:5].sum()) == 0


def test_full_size_exchange_sampled_cells_and_conservation():
    """16384 cells x 1200 (19.7M particles) in the benchmark's configuration
    (FP32, the default queue path), two steps: the totals (particles, energy
    with formation energies, momentum) are conserved, and 5 sampled cells
    equal the fused kernel's run of those cells alone (cells are independent
    and keyed by their index)."""
    w = W.ch4_h_exchange()
    g = hcao.from_workload(w, precision=hcao.FP32)
    assert g.step_path() == hcao.PATH_QUEUE

    def totals():
        m = g.read_moments(0)
        mass = sum(m.n[i] * w.species[i].mass for i in range(len(w.species)))
        E = m.E_tr + sum(m.E_vib[i] for i in range(16)) + m.E_form
        return E, np.array(m.momentum[:]), sum(m.n[i] for i in range(16)), float(np.sqrt(2.0 * mass * m.E_tr))

    E0, p0, n0, ps = totals()
    g.step(2)
    E1, p1, n1, _ = totals()
    assert n1 == n0 == w.n
    assert abs(E1 - E0) <= 1e-6 * abs(E0)
    assert np.all(np.abs(p1 - p0) <= 1e-6 * ps)
    assert g.read_counters(0)[8] > 100000  # exchange events
    vg, qg, sg, cg = g.read_particles(0)
    g.close()
    pick = [0, 1, 4097, 9999, 16383]
    sel = np.isin(w.cell, pick)
    q = hcao.Context(precision=hcao.FP32)
    q.set_species(w.species)
    q.set_reactions(w.reactions)
    q.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
    q.load_particles(0, w.v[sel], w.qn0()[sel], w.species_idx[sel], w.cell[sel])
    q.init_vibration(0, w.T_vib0)
    q.set_step_path(hcao.PATH_FUSED)
    q.step(2)
    vq, qq, sq, cq = q.read_particles(0)
    out = np.isin(cg, pick)
    assert np.array_equal(cg[out], cq)
    assert np.array_equal(sg[out], sq)
    assert np.array_equal(qg[out], qq)
    assert np.array_equal(vg[out], vq)


def test_full_size_exchange_fp64_sampled_cells_match_oracle():
    """The same workload in FP64 mode (queue path), one step: sampled cells
    equal the oracle's run of those cells bit for bit."""
    w = W.ch4_h_exchange()
    g = hcao.from_workload(w, precision=hcao.FP64)
    g.step(1)
    vg, qg, sg, cg = g.read_particles(0)
    g.close()
    pick = [0, 777, 8191, 16383]
    sel = np.isin(w.cell, pick)
    o = oracle.Oracle()
    for s in w.species:
        o.add_species(s)
    for r in w.reactions:
        o.add_reaction(r)
    o.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
    o.load(0, w.v[sel], w.qn0()[sel], w.species_idx[sel], w.cell[sel])
    o.init_vibration(0, w.T_vib0)
    o.step(1)
    vo, qo, so, co = o.read_particles(0)
    out = np.isin(cg, pick)
    assert np.array_equal(cg[out], co)
    assert np.array_equal(sg[out], so)
    assert np.array_equal(qg[out], qo)
    assert np.array_equal(vg[out], vo)
