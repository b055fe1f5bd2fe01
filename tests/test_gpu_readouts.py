"""Readouts of the collision phase's bookkeeping (Sec. "Implementation of the
polyatomic HCAO model": level populations, vibrational energy and the
zero-point search for T_vib) against the oracle's particles.

FP64 mode steps bit for bit like the oracle, so the GPU's level populations
must equal counts taken from the oracle's particles exactly, and its moments
must equal sums over the oracle's particles up to the summation order of the
device reduction.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _stepped(w, steps, precision=hcao.FP64):
    g = hcao.from_workload(w, precision=precision)
    o = oracle.from_workload(w)
    g.step(steps)
    g.sync()
    o.step(steps)
    return g, o


WORKLOADS = {
    "triatomic": lambda: W.relaxation_triatomic(n_particles=6000, n_cells=3),
    "ch4_dissociation": lambda: W.ch4_heat_bath(n_cells=12, per_cell=400),
    "ch4_h_exchange": lambda: W.ch4_h_exchange(n_cells=6, per_cell=800, T0=6000.0),
}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_level_populations_equal_oracle_counts(name):
    w = WORKLOADS[name]()
    g, o = _stepped(w, 6)
    _, qo, so, _ = o.read_particles(0)
    checked = 0
    for sp, s in enumerate(w.species):
        for mode in range(s.n_modes):
            got = g.read_level_populations(0, sp, mode, 256)
            exp = np.bincount(qo[so == sp, mode].astype(np.int64), minlength=256).astype(np.uint64)
            assert np.array_equal(got, exp), (s.name, mode)
            checked += int(exp.sum())
    assert checked > 0
    # fewer slots than levels: the first max_levels counts
    got = g.read_level_populations(0, 0, 0, 3)
    assert np.array_equal(got, np.bincount(qo[so == 0, 0], minlength=256)[:3].astype(np.uint64))


def test_level_populations_fp32_equal_own_particles():
    w = W.ch4_heat_bath(n_cells=16, per_cell=300)
    g = hcao.from_workload(w, precision=hcao.FP32)
    g.step(4)
    _, q, s, _ = g.read_particles(0)
    for sp in (0, 1):
        for mode in range(w.species[sp].n_modes):
            got = g.read_level_populations(0, sp, mode, 256)
            exp = np.bincount(q[s == sp, mode].astype(np.int64), minlength=256).astype(np.uint64)
            assert np.array_equal(got, exp)


def test_level_populations_reject_bad_arguments():
    w = W.relaxation_triatomic(n_particles=100)
    g = hcao.from_workload(w)
    for sp, mode in ((1, 0), (0, 3), (-1, 0), (0, -1)):
        with pytest.raises(hcao.HcaoError):
            g.read_level_populations(0, sp, mode, 16)
    with pytest.raises(hcao.HcaoError):
        g.read_level_populations(7, 0, 0, 16)  # no such reservoir


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_moments_fp64_equal_oracle_sums(name):
    w = WORKLOADS[name]()
    g, o = _stepped(w, 6)
    m = g.read_moments(0)
    vo, qo, so, _ = o.read_particles(0)
    mass = np.array([s.mass for s in w.species])[so]
    n_sp = np.bincount(so, minlength=16)
    assert list(m.n) == [int(x) for x in n_sp]
    # momentum: sums near zero, compared against the scale of sum |m v|
    for d in range(3):
        exp = math.fsum(mass * vo[:, d])
        scale = math.fsum(np.abs(mass * vo[:, d]))
        assert abs(m.momentum[d] - exp) <= 1e-13 * scale, (d, m.momentum[d], exp)
    e_tr = math.fsum(0.5 * mass * np.sum(vo * vo, axis=1))
    assert abs(m.E_tr - e_tr) <= 1e-12 * e_tr
    e_form = math.fsum(np.array([s.E_form for s in w.species])[so])
    assert abs(m.E_form - e_form) <= 1e-12 * max(abs(e_form), 1e-30)
    for sp, s in enumerate(w.species):
        sel = so == sp
        if s.n_modes == 0 or not sel.any():
            assert m.E_vib[sp] == 0.0
            continue
        lev = [o.levels(sp, j) for j in range(s.n_modes)]
        ev = np.zeros(int(sel.sum()))
        for j in range(s.n_modes):
            ev += lev[j][qo[sel, j]]
        exp = math.fsum(ev)
        assert abs(m.E_vib[sp] - exp) <= 1e-12 * exp, (s.name, m.E_vib[sp], exp)
        # T_vib: the zero-point search on both sides (root of the mean
        # vibrational energy above the ZPE), bisection to the same tolerance
        tv_o = o.tvib(0, sp)
        assert abs(m.T_vib[sp] - tv_o) <= 1e-9 * tv_o, (s.name, m.T_vib[sp], tv_o)
    # translational temperature from the peculiar kinetic energy
    M = float(mass.sum())
    p2 = sum(math.fsum(mass * vo[:, d]) ** 2 for d in range(3))
    T_tr = 2.0 / 3.0 * (e_tr - 0.5 * p2 / M) / (len(so) * W.KB)
    assert abs(m.T_tr - T_tr) <= 1e-11 * T_tr


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_moments_fp32_against_exact_sums(name):
    """FP32 mode sums momentum and translational energy in int64 fixed point
    from float products of each particle's velocity and its mass (held as a
    float pair, so the mass is not rounded): per particle at most a few float
    roundings (<= 3e-7 relative), unbiased, so the totals sit far closer to
    the exact sums of the same particles."""
    w = WORKLOADS[name]()
    g = hcao.from_workload(w, precision=hcao.FP32)
    g.step(6)
    m = g.read_moments(0)
    v, q, sp, _ = g.read_particles(0)
    mass = np.array([s.mass for s in w.species])[sp]
    assert list(m.n) == [int(x) for x in np.bincount(sp, minlength=16)]
    e_tr = math.fsum(0.5 * mass * np.sum(v * v, axis=1))
    assert abs(m.E_tr - e_tr) <= 3e-7 * e_tr
    assert abs(m.E_tr - e_tr) <= 5e-9 * e_tr, (m.E_tr, e_tr)
    for d in range(3):
        exp = math.fsum(mass * v[:, d])
        scale = math.fsum(np.abs(mass * v[:, d]))
        assert abs(m.momentum[d] - exp) <= 1e-9 * scale, (d, m.momentum[d], exp)
    e_form = math.fsum(np.array([s.E_form for s in w.species])[sp])
    assert abs(m.E_form - e_form) <= 1e-12 * max(abs(e_form), 1e-30)
    counts = g.read_counters(0)  # summed over the cells on the device
    assert counts[7] == 6 and counts[0] >= counts[1] > 0


def test_tvib_equals_translational_temperature_at_equilibrium():
    """Equilibrated triatomic reservoir (FP64, GPU alone): T_vib from the
    zero-point search meets T_tr (Sec. implementation: T_vib is the
    temperature whose Boltzmann mean vibrational energy equals the measured
    one)."""
    w = W.relaxation_triatomic(n_particles=20000, n_cells=1)
    w.T_vib0 = w.T_tr0 = 8000.0
    g = hcao.from_workload(w, precision=hcao.FP64)
    g.step(200)
    m = g.read_moments(0)
    assert abs(m.T_vib[0] - m.T_tr) / m.T_tr < 0.03, (m.T_vib[0], m.T_tr)


@pytest.mark.parametrize("precision", [hcao.FP32, hcao.FP64])
def test_load_with_fp32_velocities(precision):
    """hcao_load_particles_f32 (12 bytes of velocity per particle over the
    link) gives the records of hcao_load_particles with the same values, and
    the same run after three steps."""
    w = W.ch4_heat_bath(n_cells=37, per_cell=123)
    vf = w.v.astype(np.float32)
    ctxs = []
    for v in (vf.astype(np.float64), vf):
        g = hcao.Context(precision=precision)
        g.set_species(w.species)
        g.set_reactions(w.reactions)
        rid = g.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
        g.load_particles(rid, v, w.qn0(), w.species_idx, w.cell)
        g.init_vibration(rid, w.T_vib0)
        ctxs.append(g)
    for steps in (0, 3):
        if steps:
            for g in ctxs:
                g.step(steps)
        a, b = ctxs[0].read_particles(0), ctxs[1].read_particles(0)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_rejection_cap_reports_and_keeps_state_fp64():
    """A rejection loop that hits its cap (reject_cap = 1: a K5 trial that
    would restart fails the draw instead) keeps the molecule's state and
    reports HCAO_EREJECT_LIMIT from the next synchronising call, without any
    device fault; after hcao_clear_error the context reads out and steps on.
    The particles equal the oracle's run with the same cap, which also
    reports the cap."""
    # ground-state molecules (the initialiser's own rejection loop would hit
    # the cap of 1 too)
    w = W.ch4_heat_bath(n_cells=8, per_cell=400, dissociation=False)
    g = hcao.from_workload(w, precision=hcao.FP64, reject_cap=1, init_vib=False)
    o = oracle.Oracle(reject_cap=1)
    for s in w.species:
        o.add_species(s)
    res = o.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
    o.load(res, w.v, w.qn0(), w.species_idx, w.cell)
    o_failed = False
    for _ in range(3):
        g.step(1)
        try:
            o.step(1)
        except RuntimeError:
            o_failed = True
    with pytest.raises(hcao.HcaoError) as e:
        g.sync()
    assert e.value.code == -4 and o_failed
    g.clear_error()
    g.sync()
    vg, qg, sg, cg = g.read_particles(0)
    vo, qo, so, co = o.read_particles(0)
    assert np.array_equal(cg, co) and np.array_equal(sg, so) and np.array_equal(qg, qo)
    assert np.array_equal(vg, vo)
    g.step(1)
    g.clear_error()
    g.sync()
