"""Pins of the oracle's rotation (Sec. "Rotation coupling"): a classical
rotational energy per molecule, relaxed by the classical LB draw, coupled to
the QK collision energies by gamma.

* ora_ln, the logarithm the rotation draws use, against math.log;
* the LB rotational fraction against scipy's Beta(rot_dof/2, (5-2 omega)/2);
* the initial rotational energy against scipy's Gamma(rot_dof/2) kT;
* an adiabatic reservoir reaches equipartition: <E_rot> = rot_dof/2 k T_tr and
  the rotational energies follow Gamma(rot_dof/2) k T_tr; energy is conserved;
* with gamma = 1 the single-step dissociation probability of CH4 colliding
  with H is sum_E p(E_vib = E) Q(5/2 - omega + rot_dof/2, (X - E)/kT) (the
  rotational energy adds to the collision-weighted translational energy);
  with gamma = 0 it is the same sum with Q(5/2 - omega, .).
"""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2606_31548_b300 import workloads as W
from test_oracle_pins import KB, EV, _energy_momentum, _evib_distribution

rng = np.random.default_rng(5)


def test_ln_matches_math_log():
    xs = np.concatenate([rng.uniform(1e-300, 1e-290, 50), rng.uniform(0.0, 1.0, 2000) + 1e-17,
                         rng.uniform(0.99, 1.01, 500), np.exp(rng.uniform(-700, 700, 1000)),
                         [1.0, 2.0, 0.5, 1.0 - 2 ** -53, 1.0 + 2 ** -52]])
    worst = 0.0
    for x in xs:
        a, b = oracle.ln(float(x)), math.log(float(x))
        worst = max(worst, abs(a - b) / max(abs(b), 1e-300) if abs(b) > 1e-12 else abs(a - b))
    assert worst < 1e-15, worst  # a few ulp
    assert oracle.ln(1.0) == 0.0


def _rot_species(dof, omega=0.75):
    s = W.triatomic()
    s.rot_dof = dof
    s.omega = omega
    return s


@pytest.mark.parametrize("dof,omega", [(2, 0.75), (3, 0.75), (3, 0.5), (2, 1.0)])
def test_rot_fraction_is_beta(dof, omega):
    o = oracle.Oracle()
    o.add_species(_rot_species(dof, omega))
    x = o.sample_rot_fraction(0, 99 + dof, 40000)
    assert stats.kstest(x, stats.beta(dof / 2, 2.5 - omega).cdf).pvalue > 1e-4
    # a plausible mistake (the vibrational exponent on the wrong side) is rejected
    assert stats.kstest(x, stats.beta(2.5 - omega, dof / 2).cdf).pvalue < 1e-6


def _rot_reservoir(dof, T_rot0, n=6000, T=10000.0, steps=0):
    w = W.relaxation_triatomic(n_particles=n, n_cells=2)
    w.species = [_rot_species(dof)]
    w.T_tr0 = T
    w.T_rot0 = T_rot0
    return w


@pytest.mark.parametrize("dof", [2, 3])
def test_initial_rotation_is_gamma(dof):
    T = 3000.0
    w = _rot_reservoir(dof, T)
    o = oracle.from_workload(w)
    e = o.read_erot(0) / (KB * T)
    assert stats.kstest(e, stats.gamma(dof / 2).cdf).pvalue > 1e-4
    assert stats.kstest(e, stats.gamma((dof + 1) / 2).cdf).pvalue < 1e-6


@pytest.mark.parametrize("dof", [2, 3])
def test_rotation_equipartition_and_conservation(dof):
    w = _rot_reservoir(dof, 300.0, n=4000)
    o = oracle.from_workload(w)

    def total():
        E, p, ps = _energy_momentum(o, 0, w.species)
        return E + o.read_erot(0).sum(), p, ps

    E0, p0, ps = total()
    assert o.read_erot(0).mean() / KB < 1000.0  # starts cold
    o.step(150)
    E1, p1, _ = total()
    assert abs(E1 - E0) <= 1e-12 * abs(E0)
    assert np.all(np.abs(p1 - p0) <= 1e-12 * ps)
    v, _, sp, _ = o.read_particles(0)
    m = w.species[0].mass
    N = len(v)
    pc = m * v.sum(0)
    T_tr = 2.0 / 3.0 * (0.5 * m * (v * v).sum() - 0.5 * (pc @ pc) / (m * N)) / (N * KB)
    er = o.read_erot(0)
    T_rot = er.mean() / (dof / 2 * KB)
    assert abs(T_rot / T_tr - 1.0) < 0.03, (T_rot, T_tr)
    assert stats.kstest(er / (KB * T_tr), stats.gamma(dof / 2).cdf).pvalue > 1e-4


@pytest.mark.parametrize("gamma", [0.0, 1.0])
def test_rotation_coupling_dissociation_probability(gamma):
    T = 7000.0
    w = W.ch4_h_exchange(n_cells=200, per_cell=1000, T0=T)
    w.species[0].rot_dof = 3  # CH4 rotates; H does not
    w.reactions = [W.Reaction("diss", [0], [2, 1], diss_mode_mask=0xF, gamma=gamma)]
    o = oracle.from_workload(w, log=True)
    _, _, s0, c0 = o.read_particles(0)
    o.step(1)
    lg = o.read_log()
    acc = lg[lg["event"] >= 0]
    start = np.concatenate([[0], np.cumsum(np.bincount(c0, minlength=w.n_cells))[:-1]])
    ip, iq = start[acc["cell"]] + acc["p"], start[acc["cell"]] + acc["q"]
    mixed = s0[ip] != s0[iq]
    n_coll = int(mixed.sum())
    n_ev = int(np.sum(acc["event"][mixed] == 1))
    lev = [o.levels(0, j) for j in range(9)]
    X = 4.5 * EV + o.zpe(0) + o.zpe(2) + o.zpe(1) - lev[0][0]
    e, p = _evib_distribution(lev, T)
    a = 1.75 + (1.5 if gamma == 1.0 else 0.0)
    P = float(np.sum(p * special.gammaincc(a, np.maximum(0.0, (X - e) / (KB * T)))))
    P_other = float(np.sum(p * special.gammaincc(3.25 if gamma == 0.0 else 1.75,
                                                 np.maximum(0.0, (X - e) / (KB * T)))))
    sd = math.sqrt(P * (1 - P) / n_coll)
    assert n_ev > 100
    assert abs(n_ev / n_coll - P) < 3.5 * sd, (n_ev / n_coll, P, n_coll)
    assert abs(P_other - P) > 10 * sd
