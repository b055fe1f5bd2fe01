"""Recombination B + C + M -> A + M on the GPU (reading A14) against the oracle.

FP64 mode: every decision -- accepted pairs, recombination and dissociation
events, the third body, the removed particle and the compacted order of each
cell -- and every FP64 velocity equals the oracle's bit for bit.  The rate
tables are built independently on both sides (the library groups identical
modes, the oracle enumerates every level combination) and agree to 1e-11.
FP32 mode: exact-to-rounding conservation and the oracle's statistics.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W

pytestmark = pytest.mark.gpu

KB = 1.380649e-23


def _assert_same(g, o):
    lg, lo = g.read_log(), o.read_log()
    assert len(lg) == len(lo)
    for f in ("step", "cell", "round_k", "p", "q", "event", "aux"):
        assert np.array_equal(lg[f], lo[f]), f
    vg, qg, sg, cg = g.read_particles(0)
    vo, qo, so, co = o.read_particles(0)
    assert np.array_equal(cg, co) and np.array_equal(sg, so) and np.array_equal(qg, qo)
    assert np.array_equal(vg, vo), np.max(np.abs(vg - vo))


def test_rate_tables_match_oracle():
    w = W.ch4_recombination(n_cells=1, per_cell=10)
    g = hcao.from_workload(w, precision=hcao.FP64)
    o = oracle.from_workload(w)
    for T in (2000.0, 2031.7, 4000.0, 4100.5):
        for m in range(3):
            kg, ko = g.recomb_rate(1, m, T), o.rec_rate(1, m, T)
            assert abs(kg - ko) <= 1e-11 * ko, (T, m, kg, ko)
    # clamped at the ends of the table
    assert g.recomb_rate(1, 2, 100.0) == g.recomb_rate(1, 2, 500.0)
    with pytest.raises(hcao.HcaoError):
        g.recomb_rate(0, 0, 3000.0)  # reaction 0 is the dissociation


def _wr(w):
    for r in w.reactions:
        if r.type == "recomb":
            r.recomb_prob = "wr"
    return w


def test_wr_rate_tables_match_oracle():
    """The recombination rate tables built from the WR form of P (the sampled
    sum with the Whitten-Rabinovitch density, Sec. "Recombination
    reactions"): library against oracle at nodes and between them, and below
    the exact-sum tables as the WR form runs low for CH4."""
    w = _wr(W.ch4_recombination(n_cells=1, per_cell=10))
    g = hcao.from_workload(w, precision=hcao.FP64)
    o = oracle.from_workload(w)
    ge = hcao.from_workload(W.ch4_recombination(n_cells=1, per_cell=10), precision=hcao.FP64)
    for T in (2000.0, 2031.7, 4000.0, 9000.0):
        for m in range(3):
            kg, ko = g.recomb_rate(1, m, T), o.rec_rate(1, m, T)
            assert abs(kg - ko) <= 1e-10 * ko, (T, m, kg, ko)
        ratio = g.recomb_rate(1, 2, T) / ge.recomb_rate(1, 2, T)
        assert 0.4 < ratio < 0.95, (T, ratio)


def test_parity_recombination_wr_fp64():
    """A recombination run with the WR rate tables: bit-exact with the
    oracle's run with its own WR tables (FP64 mode)."""
    w = _wr(W.ch4_recombination(n_cells=6, per_cell=800, T0=3000.0, n_density=1e26))
    g = hcao.from_workload(w, precision=hcao.FP64, log=True)
    o = oracle.from_workload(w, log=True)
    for _ in range(4):
        g.step(1)
        o.step(1)
        _assert_same(g, o)
    assert g.read_reaction_counts(0, 2)[1] > 20  # recombinations happened


@pytest.mark.parametrize("case", ["one_round", "four_rounds"])
def test_parity_recombination_fp64(case):
    w = W.ch4_recombination(n_cells=6, per_cell=800, T0=2000.0, n_density=1e26)
    kw = {}
    if case == "four_rounds":
        w.dt *= 3.0  # N_sel > N/2: later rounds meet particles removed earlier in the step
        kw = {"max_rounds": 4}
    g = hcao.from_workload(w, precision=hcao.FP64, log=True, **kw)
    o = oracle.from_workload(w, log=True)
    for _ in range(5):
        g.step(1)
        o.step(1)
        _assert_same(g, o)
    cg, co = g.read_counters(0), o.read_counters(0)
    assert np.array_equal(cg, co[: len(cg)]), (cg, co)
    assert cg[9] > 10  # recombinations happened
    if case == "four_rounds":
        lg = g.read_log()
        assert np.any((lg["round_k"] >> 24) >= 1)


def test_parity_recombination_single_large_cell_fp64():
    """One cell of 12,000 particles (its event slots span several 1024-slot
    chunks, so the removed positions are gathered by several warps in no
    fixed order before the compaction sorts them): bit-exact with the
    oracle."""
    w = W.ch4_recombination(n_cells=1, per_cell=12000, T0=2500.0, n_density=1e26)
    g = hcao.from_workload(w, precision=hcao.FP64, log=True)
    o = oracle.from_workload(w, log=True)
    for _ in range(3):
        g.step(1)
        o.step(1)
        _assert_same(g, o)
    assert g.read_counters(0)[9] > 50  # recombinations happened


def _totals(g, species):
    m = g.read_moments(0)
    E = m.E_tr + sum(m.E_vib[i] for i in range(16)) + m.E_form
    return E, np.array(m.momentum[:]), [m.n[i] for i in range(len(species))]


def test_fp32_recombination_conserves_and_counts():
    w = W.ch4_recombination(n_cells=16, per_cell=2000, T0=2000.0, n_density=1e26)
    g = hcao.from_workload(w, precision=hcao.FP32)
    E0, p0, n0 = _totals(g, w.species)
    prev = E0
    for _ in range(8):
        g.step(1)
        E, p, n = _totals(g, w.species)
        assert abs(E - prev) < 1e-6 * abs(prev)
        prev = E
    c = g.read_counters(0)
    diss, rec = int(c[8]), int(c[9])
    assert rec > 50
    # CH4 + diss - rec, CH3 - diss + rec ...
    assert n[0] == n0[0] - diss + rec
    assert n[1] == n0[1] + diss - rec
    assert n[2] == n0[2] + diss - rec
    assert g.count(0) == w.n + diss - rec


def test_fp32_recombination_matches_oracle_statistics():
    """Recombination counts over 6 steps: FP32 GPU vs the FP64 oracle on the
    same workload, within 3.5 sigma of Poisson counts."""
    w = W.ch4_recombination(n_cells=8, per_cell=1000, T0=2000.0, n_density=1e26)
    g = hcao.from_workload(w, precision=hcao.FP32)
    g.step(6)
    o = oracle.from_workload(w)
    o.step(6)
    ng, no = int(g.read_counters(0)[9]), int(o.read_counters(0)[9])
    assert abs(ng - no) < 3.5 * math.sqrt(2 * max(no, 1)) + 3, (ng, no)


def test_fp32_recombination_rate_law():
    """Recombinations per step vs k_r(T) n_B n_C n V dt / w with the library's
    own tabulated k_r (third bodies in proportion to the composition), FP32
    mode, within 3.5 sigma of the Poisson spread plus 2%."""
    w = W.ch4_recombination(n_cells=1, per_cell=100000, T0=2500.0, n_density=3e25,
                            fractions=(0.0, 1.0, 1.0))
    g = hcao.from_workload(w, precision=hcao.FP32)
    expected, counted = 0.0, 0
    for _ in range(20):
        m = g.read_moments(0)
        N = sum(m.n[i] for i in range(3))
        nd = [m.n[i] * w.weight / w.cell_volume for i in range(3)]
        n3 = (N - 2) * w.weight / w.cell_volume
        kr = sum(m.n[k] / N * g.recomb_rate(1, k, m.T_tr) for k in range(3))
        expected += kr * nd[1] * nd[2] * n3 * w.cell_volume * w.dt / w.weight
        before = int(g.read_counters(0)[9])
        g.step(1)
        counted += int(g.read_counters(0)[9]) - before
    assert expected > 1000
    assert abs(counted - expected) < 3.5 * math.sqrt(expected) + 0.02 * expected, (counted, expected)


def test_steady_state_balance():
    """A closed CH4 / CH3 / H reservoir reaches a steady state in which
    dissociations and recombinations per step balance.  The composition
    settles at n_B n_C / n_A = 1-3 K_eq(T), not K_eq itself: recombined CH4
    carries the released energy as vibration (the LB product redistribution
    of all reactions) and dissociates again faster than thermal CH4, for
    which k_f = k_r K_eq holds."""
    w = W.ch4_recombination(n_cells=1, per_cell=200000, T0=4000.0, n_density=1e26)
    g = hcao.from_workload(w, precision=hcao.FP32)
    o = oracle.from_workload(W.ch4_recombination(n_cells=1, per_cell=10))
    g.step(1500)
    c0 = g.read_counters(0)
    ratios, temps = [], []
    for _ in range(20):
        g.step(25)
        m = g.read_moments(0)
        n = [m.n[i] * w.weight / w.cell_volume for i in range(3)]
        ratios.append(n[1] * n[2] / n[0])
        temps.append(m.T_tr)
    c1 = g.read_counters(0)
    diss, rec = int(c1[8] - c0[8]), int(c1[9] - c0[9])
    assert rec > 10000
    assert abs(diss - rec) < 4.0 * math.sqrt(diss + rec), (diss, rec)
    r = float(np.mean(ratios)) / o.keq(1, float(np.mean(temps)))
    assert 1.0 < r < 3.0, r
