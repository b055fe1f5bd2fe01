"""FP32 mode (the production path) against the FP64 oracle.

FP32 mode stores velocities in FP32 and keeps every energy in int64 fixed
point, so it cannot match the oracle bit for bit; it must match the oracle's
statistics.  Each comparison runs the two sides on independent seeds (so the
difference is a genuine two-sample statistic, not two views of one random
stream) and allows 3 standard errors of the difference (3.5 where several
correlated checkpoints of one curve are tested together).

* Exchange (Eq. Ecoll-exch, CH4 + H -> CH3 + H2, one stretch coupled):
  the single-step exchange probability per CH4-H collision and the accepted
  collisions per particle-step at 2000, 4000 and 6000 K.
* Relaxation (Sec. "Implementation of the polyatomic HCAO model"): the
  triatomic's T_vib(t) curve over 16 seeds.
* Conservation: every accepted non-reacting or exchange collision conserves
  its pair's energy to 1e-6 relative and its momentum, and leaves every other
  particle untouched.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _two_sample(kg, ng, ko, no):
    """Difference of two binomial proportions and its standard error."""
    pg, po = kg / ng, ko / no
    p = (kg + ko) / (ng + no)
    se = math.sqrt(p * (1 - p) * (1.0 / ng + 1.0 / no))
    return pg - po, se


def _mixed_exchange(ctx_log, v0_sp, cell0, n_cells):
    """(exchange events, accepted CH4-H collisions) of the last step's log."""
    lg = ctx_log.read_log()
    acc = lg[lg["event"] >= 0]
    start = np.concatenate([[0], np.cumsum(np.bincount(cell0, minlength=n_cells))[:-1]])
    ip = start[acc["cell"]] + acc["p"]
    iq = start[acc["cell"]] + acc["q"]
    mixed = v0_sp[ip] != v0_sp[iq]
    return int(np.sum(acc["event"][mixed] == 1)), int(np.sum(mixed)), len(acc)


@pytest.mark.parametrize("T", [2000.0, 4000.0, 6000.0])
def test_fp32_exchange_probability_matches_oracle(T):
    """One step from the Boltzmann state at T: the exchange probability per
    CH4-H collision (Eq. Ecoll-exch) of FP32 mode against the oracle's, on
    independent seeds (binomial two-sample, 3 sigma), and the accepted
    collisions per particle-step."""
    wo = W.ch4_h_exchange(n_cells=400, per_cell=1200, T0=T)
    wg = W.ch4_h_exchange(n_cells=400, per_cell=1200, T0=T, seed=wo.seed + 101)
    o = oracle.from_workload(wo, log=True)
    _, _, so, co = o.read_particles(0)
    o.step(1)
    ex_o, mix_o, acc_o = _mixed_exchange(o, so, co, wo.n_cells)
    g = hcao.from_workload(wg, precision=hcao.FP32, log=True)
    _, _, sg, cg = g.read_particles(0)
    g.step(1)
    ex_g, mix_g, acc_g = _mixed_exchange(g, sg, cg, wg.n_cells)
    assert ex_o > 500 and ex_g > 500
    d, se = _two_sample(ex_g, mix_g, ex_o, mix_o)
    assert abs(d) < 3 * se, (T, ex_g / mix_g, ex_o / mix_o, se)
    # collision rate: accepted collisions per particle-step (Poisson counts)
    rg, ro = acc_g / wg.n, acc_o / wo.n
    assert abs(rg - ro) < 3 * math.sqrt(acc_g + acc_o) / wo.n, (rg, ro)


def test_fp32_relaxation_curve_matches_oracle():
    seeds, n = 16, 4000
    marks = [1, 2, 4, 8, 16, 32, 64, 120]  # steps at which T_vib is read
    curves = {"gpu": [], "oracle": []}
    for i in range(seeds):
        for side in ("gpu", "oracle"):
            # independent seeds per side
            w = W.relaxation_triatomic(n_particles=n, seed=0x7E1A0000 + 2 * i + (side == "gpu"))
            c = []
            done = 0
            if side == "gpu":
                g = hcao.from_workload(w, precision=hcao.FP32)
                c.append(g.read_moments(0).T_vib[0])
                for m in marks:
                    g.step(m - done)
                    done = m
                    c.append(g.read_moments(0).T_vib[0])
                g.close()
            else:
                o = oracle.from_workload(w)
                c.append(o.tvib(0, 0))
                for m in marks:
                    o.step(m - done)
                    done = m
                    c.append(o.tvib(0, 0))
                o.close()
            curves[side].append(c)
    cg, co = np.array(curves["gpu"]), np.array(curves["oracle"])
    mg, mo = cg.mean(0), co.mean(0)
    se = np.sqrt(cg.var(0, ddof=1) / seeds + co.var(0, ddof=1) / seeds)
    assert np.all(np.abs(mg - mo) < 3.5 * se), (mg, mo, se)
    # the curve relaxes: T_vib rises from 300 K by thousands of kelvin
    assert mo[0] < 400.0 and mo[-1] > mo[0] + 3000.0 and mg[-1] > mg[0] + 3000.0


def _pair_energy(v, q, sp, idx, species, levels):
    """Total energy (kinetic + vibrational + formation) and momentum of the
    particles idx, and the energy scale kinetic + vibrational (the formation
    energies of reactants and products nearly cancel, so the total alone can
    be small)."""
    e, scale = 0.0, 0.0
    p = np.zeros(3)
    for i in idx:
        s = species[sp[i]]
        ke = 0.5 * s.mass * float(v[i] @ v[i])
        ev = sum(levels[sp[i]][j][q[i, j]] for j in range(s.n_modes))
        e += ke + ev + s.E_form
        scale += ke + ev
        p += s.mass * v[i]
    return e, p, scale


@pytest.mark.parametrize("name", ["triatomic", "exchange"])
def test_fp32_per_collision_conservation(name):
    if name == "triatomic":
        w = W.relaxation_triatomic(n_particles=6000, n_cells=4)
    else:
        w = W.ch4_h_exchange(n_cells=8, per_cell=1200, T0=6000.0)
    g = hcao.from_workload(w, precision=hcao.FP32, log=True)
    levels = [[np.array([g.level_energy(s, j, i) for i in range(g.n_levels(s, j))])
               for j in range(sp.n_modes)] for s, sp in enumerate(w.species)]
    g.step(2)  # (sigma g)_max settles
    v0, q0, s0, c0 = g.read_particles(0)
    g.step(1)
    v1, q1, s1, c1 = g.read_particles(0)
    assert np.array_equal(c0, c1)  # no particle created or removed
    log = g.read_log()
    start = np.searchsorted(c0, np.arange(w.n_cells))
    acc = log[log["event"] >= 0]
    touched = np.zeros(len(c0), bool)
    members = np.concatenate([start[acc["cell"]] + acc["p"], start[acc["cell"]] + acc["q"]])
    uniq, cnt = np.unique(members, return_counts=True)
    once = set(uniq[cnt == 1].tolist())
    touched[members] = True
    n_checked, worst = 0, 0.0
    for rec in acc:
        ip, iq = start[rec["cell"]] + rec["p"], start[rec["cell"]] + rec["q"]
        if ip not in once or iq not in once:
            continue  # in two pairs of this step (a second pairing round)
        e0, p0, scale = _pair_energy(v0, q0, s0, (ip, iq), w.species, levels)
        e1, p1, _ = _pair_energy(v1, q1, s1, (ip, iq), w.species, levels)
        ke = 0.5 * (w.species[s0[ip]].mass * float(v0[ip] @ v0[ip]) +
                    w.species[s0[iq]].mass * float(v0[iq] @ v0[iq]))
        rel = abs(e1 - e0) / scale
        worst = max(worst, rel)
        assert rel <= 1e-6, (rec, e0, e1)
        pscale = math.sqrt(2.0 * (w.species[s0[ip]].mass + w.species[s0[iq]].mass) * ke)
        assert np.all(np.abs(p1 - p0) <= 1e-6 * pscale), (rec, p0, p1)
        n_checked += 1
    assert n_checked > 200
    if name == "exchange":
        assert np.any(acc["event"] == 1)  # exchange events among the checked pairs
    # particles in no accepted pair are untouched, bit for bit
    idle = ~touched
    assert np.array_equal(v0[idle], v1[idle]) and np.array_equal(q0[idle], q1[idle])
    assert np.array_equal(s0[idle], s1[idle])
