"""The collision-temperature product split (HCAO_SPLIT_TCOLL, Sec.
"Polyatomic QK reaction modeling": the energy left after a reaction shared
by equipartition at a collision temperature) on the GPU against the oracle.

FP64 mode: dissociation, exchange and recombination runs equal the oracle's
bit for bit (T_c by bisection with the same exponential on both sides; the
products' levels through the exponent-1/2 tables where the exponent falls
below 3/2 - omega).  FP32 mode (b1 interpolated from a per-reaction table):
the exchange products' mean vibrational energies against the oracle's on
independent seeds, a clear difference from the relaxation-table reading,
and exact-to-rounding conservation through dissociation and recombination.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W

pytestmark = pytest.mark.gpu
TC = "collision_temperature"


def _split(w, split=TC):
    w.reactions = [dataclasses.replace(r, product_split=split) for r in w.reactions]
    return w


def _assert_same(g, o):
    lg, lo = g.read_log(), o.read_log()
    assert len(lg) == len(lo)
    for f in ("step", "cell", "round_k", "p", "q", "event", "aux"):
        assert np.array_equal(lg[f], lo[f]), f
    vg, qg, sg, cg = g.read_particles(0)
    vo, qo, so, co = o.read_particles(0)
    assert np.array_equal(cg, co) and np.array_equal(sg, so) and np.array_equal(qg, qo)
    assert np.array_equal(vg, vo), np.max(np.abs(vg - vo))


CASES = {
    "dissociation": (lambda: W.ch4_heat_bath(n_cells=6, per_cell=400), 8),
    "exchange": (lambda: W.ch4_h_exchange(n_cells=6, per_cell=800, T0=6000.0), 8),
    "recombination": (lambda: W.ch4_recombination(n_cells=6, per_cell=800, T0=3000.0, n_density=1e26), 9),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_parity_tcoll_fp64(name):
    make, counter = CASES[name]
    w = _split(make())
    g = hcao.from_workload(w, precision=hcao.FP64, log=True)
    o = oracle.from_workload(w, log=True)
    for _ in range(4):
        g.step(1)
        o.step(1)
        _assert_same(g, o)
    cg, co = g.read_counters(0), o.read_counters(0)
    assert np.array_equal(cg, co[: len(cg)]), (cg, co)
    assert cg[counter] > 10, cg  # the reaction happened


def _product_means(run, w, levels):
    v, q, sp, c = run.read_particles(0)
    out = {}
    for s in (2, 3):
        idx = np.where(sp == s)[0]
        ev = np.zeros(len(idx))
        for j, L in enumerate(levels[s]):
            ev += L[q[idx, j]] - L[0]
        out[s] = (ev.mean(), ev.var(ddof=1) / len(ev), len(ev))
    return out


def test_fp32_tcoll_exchange_products_match_oracle():
    """CH4 + H -> CH3 + H2 at 6000 K, one step from no products: every CH3
    and H2 is an exchange product.  Their mean vibrational energies in FP32
    mode agree with the oracle's (independent seeds, 4 sigma) and differ from
    the relaxation-table reading's by more than 8 sigma."""
    def make(seed_off, split):
        return _split(W.ch4_h_exchange(n_cells=200, per_cell=1200, T0=6000.0, seed=0x5EED0 + seed_off), split)

    wg, wo, wr = make(1, TC), make(2, TC), make(1, "relaxation")
    o = oracle.from_workload(wo)
    levels = {s: [np.array(o.levels(s, j)) for j in range(wo.species[s].n_modes)] for s in (2, 3)}
    o.step(1)
    mo = _product_means(o, wo, levels)
    g = hcao.from_workload(wg, precision=hcao.FP32)
    g.step(1)
    mg = _product_means(g, wg, levels)
    r = hcao.from_workload(wr, precision=hcao.FP32)
    r.step(1)
    mr = _product_means(r, wr, levels)
    for s in (2, 3):
        assert mg[s][2] > 3000 and mo[s][2] > 3000
        se = math.sqrt(mg[s][1] + mo[s][1])
        assert abs(mg[s][0] - mo[s][0]) < 4 * se, (s, mg[s], mo[s])
        se_r = math.sqrt(mg[s][1] + mr[s][1])
        assert abs(mg[s][0] - mr[s][0]) > 8 * se_r, (s, mg[s], mr[s])


def _mean_evib_of(run, sp_id, levels):
    v, q, sp, c = run.read_particles(0)
    idx = np.where(sp == sp_id)[0]
    ev = np.zeros(len(idx))
    for j, L in enumerate(levels):
        ev += L[q[idx, j]] - L[0]
    return ev.mean(), ev.var(ddof=1) / len(ev), len(ev)


@pytest.mark.parametrize("name", ["dissociation", "recombination"])
def test_fp32_tcoll_products_match_oracle(name):
    """One step from a state without the product species: the products' mean
    vibrational energy in FP32 mode against the oracle's (independent seeds,
    4 sigma).  Dissociation CH4 + M -> CH3 + H + M at 15000 K (CH3 exponent
    2: H has no modes); recombination CH3 + H + M -> CH4 + M at 3000 K
    (exponent 1/2, through the exponent-1/2 tables).  For the dissociation the
    relaxation-table reading is also run and must differ by > 8 sigma."""
    def make(seed_off, split):
        if name == "dissociation":
            w = W.ch4_heat_bath(n_cells=200, per_cell=500, seed=0x7C0D0 + seed_off)
        else:
            w = W.ch4_recombination(n_cells=4, per_cell=50000, T0=3000.0, n_density=1e26,
                                    fractions=(0.0, 1.0, 1.0), seed=0x7C0E0 + seed_off)
        return _split(w, split)

    prod = 1 if name == "dissociation" else 0
    wg, wo = make(1, TC), make(2, TC)
    o = oracle.from_workload(wo)
    levels = [np.array(o.levels(prod, j)) for j in range(wo.species[prod].n_modes)]
    o.step(1)
    mo = _mean_evib_of(o, prod, levels)
    g = hcao.from_workload(wg, precision=hcao.FP32)
    g.step(1)
    mg = _mean_evib_of(g, prod, levels)
    assert mg[2] > 1000 and mo[2] > 1000
    se = math.sqrt(mg[1] + mo[1])
    assert abs(mg[0] - mo[0]) < 4 * se, (mg, mo)
    if name == "dissociation":
        r = hcao.from_workload(make(1, "relaxation"), precision=hcao.FP32)
        r.step(1)
        mr = _mean_evib_of(r, prod, levels)
        assert abs(mg[0] - mr[0]) > 8 * math.sqrt(mg[1] + mr[1]), (mg, mr)


@pytest.mark.parametrize("name", ["dissociation", "recombination"])
def test_fp32_tcoll_conserves(name):
    if name == "dissociation":
        w = _split(W.ch4_heat_bath(n_cells=32, per_cell=500))
    else:
        w = _split(W.ch4_recombination(n_cells=16, per_cell=2000, T0=3000.0, n_density=1e26))
    g = hcao.from_workload(w, precision=hcao.FP32)

    def totals():
        m = g.read_moments(0)
        return m.E_tr + sum(m.E_vib[i] for i in range(16)) + m.E_form, np.array(m.momentum[:])

    E0, p0 = totals()
    for _ in range(6):
        g.step(1)
        E, p = totals()
        assert abs(E - E0) < 1e-6 * abs(E0)
        E0 = E
    c = g.read_counters(0)
    assert c[8] > 10 or c[9] > 10


@pytest.mark.parametrize("split", ["relaxation", TC])
def test_steady_state_both_readings(split):
    """The closed CH4 / CH3 / H reservoir under each product reading: a
    steady state with balanced dissociation and recombination, composition
    n_B n_C / n_A between 1 and 3 K_eq(T) (printed: the two readings'
    ratios)."""
    w = _split(W.ch4_recombination(n_cells=1, per_cell=200000, T0=4000.0, n_density=1e26), split)
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
    print(f"steady state, {split}: n_B n_C / n_A = {r:.3f} K_eq at T = {np.mean(temps):.0f} K")
    assert 1.0 < r < 3.0, r
