"""Pins of the oracle's recombination (Sec. "Recombination reactions", reading
A14) against what the mathematics fixes independently of its code path:

* Q(a, x) against scipy's incomplete gamma (another implementation);
* the thermal dissociation probability P of Eq. recomb-correct against a
  binned convolution of the per-mode Boltzmann distributions (another
  algorithm) and, for one mode, against the level sum written with scipy;
* K_eq's vibrational factor against the geometric-series closed form of a
  harmonic oscillator;
* the cell temperature against numpy's centre-of-mass kinetic energy;
* the DSMC-level probability k_r n / (sigma_T g) against the macroscopic rate
  law R = k_r n_B n_C n_M (counted events over many steps);
* exact conservation of energy (kinetic + vibrational + formation) and
  momentum through recombination, and the removal bookkeeping.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from paper_2606_31548_b300 import workloads as W

KB = 1.380649e-23
H = 6.62607015e-34
HC = H * 299792458.0
EV = 1.602176634e-19
AMU = 1.66053906660e-27


def _boltzmann(E, T):
    w = np.exp(-(E - E[0]) / (KB * T))
    return w / w.sum()


def _evib_hist(levels, T, cap, de=1e-4 * EV):
    """Boltzmann distribution of a molecule's total vibrational energy on a
    grid of width de (convolution of the per-mode distributions); all the
    probability at or above cap is kept in the last bin."""
    nb = int(cap / de) + 2
    dist = np.zeros(nb)
    dist[0] = 1.0
    for E in levels:
        p = _boltzmann(E, T)
        nd = np.zeros(nb)
        for e, pe in zip(E, p):
            if pe < 1e-16:
                continue
            k = int(round(e / de))
            if k >= nb:
                nd[-1] += dist.sum() * pe
                continue
            nd[k:] += dist[: nb - k] * pe
            if k:
                nd[-1] += dist[nb - k:].sum() * pe
        dist = nd
    e = np.arange(nb) * de
    e[-1] = max(e[-1], cap)
    return e, dist


def _ch4_system():
    o = oracle.Oracle()
    for s in (W.ch4_like(), W.ch3_like(), W.h_atom()):
        o.add_species(s)
    o.add_reaction(W.Reaction("diss", [0], [1, 2], diss_mode_mask=0xF))
    o.add_reaction(W.Reaction("recomb", [1, 2], [0, -1], diss_mode_mask=0xF))
    return o


@pytest.mark.parametrize("a", [1.5, 1.75, 2.0])
def test_gamma_q_matches_scipy(a):
    for x in [0.0, 1e-8, 0.01, 0.3, 1.0, a + 0.999, a + 1.0, 3.7, 10.0, 35.0, 120.0, 500.0]:
        q, ref = oracle.gamma_q(a, x), special.gammaincc(a, x)
        assert abs(q - ref) <= 1e-13 * ref + 1e-300, (a, x, q, ref)


def _threshold(o, A, B, C, De, mode=0):
    E0 = o.levels(A, mode)[0]
    return De + o.zpe(A) + o.zpe(B) + o.zpe(C) - E0


@pytest.mark.parametrize("T", [3000.0, 4000.0, 9000.0])
def test_diss_prob_ch4_matches_binned_convolution(T):
    """P(T) for the 9-mode CH4-like molecule: the oracle's exact level sum vs
    E[Q(5/2 - omega, max(0, (D - E_vib)/kT))] over a binned E_vib
    distribution; D from the QK threshold of the reverse dissociation."""
    o = _ch4_system()
    D = _threshold(o, 0, 1, 2, 4.5 * EV)
    lev = [o.levels(0, j) for j in range(9)]
    e, p = _evib_hist(lev, T, cap=D + 0.01 * EV)
    ref = float(np.sum(p * special.gammaincc(1.75, np.maximum(0.0, (D - e) / (KB * T)))))
    P = o.diss_prob(1, T)
    assert abs(P - ref) < 3e-3 * ref, (P, ref)
    assert 1e-8 < P < 1.0


def test_diss_prob_single_mode_level_sum():
    """One Morse stretch: P = sum_i p_i Q(a, max(0, (D - E_i)/kT)) exactly."""
    ab = W.Species("AB", 14.0 * AMU, 3.5e-10, we=[2000 * 100.0], wexe=[15 * 100.0], De=[3.0 * EV])
    a, b = W.Species("A", 7.0 * AMU, 3e-10, E_form=1.5 * EV), W.Species("B", 7.0 * AMU, 3e-10, E_form=1.5 * EV)
    o = oracle.Oracle()
    for s in (ab, a, b):
        o.add_species(s)
    o.add_reaction(W.Reaction("recomb", [1, 2], [0, -1], diss_mode_mask=1))
    D = _threshold(o, 0, 1, 2, 3.0 * EV)
    for T in (2500.0, 6000.0, 15000.0):
        E = o.levels(0, 0)
        p = _boltzmann(E, T)
        ref = float(np.sum(p * special.gammaincc(1.75, np.maximum(0.0, (D - E) / (KB * T)))))
        P = o.diss_prob(0, T)
        assert abs(P - ref) <= 1e-12 * ref, (T, P, ref)


def test_keq_harmonic_closed_form():
    """A nearly untruncated harmonic stretch (wexe = 0, large De): the
    vibrational factor of K_eq is 1 - exp(-theta/T) (geometric series), the
    translational one (2 pi mu k T / h^2)^(3/2), mu = m_B m_C / m_A."""
    we = 1000 * 100.0
    theta = HC * we / KB
    ab = W.Species("AB", 20.0 * AMU, 3.5e-10, we=[we], wexe=[0.0], De=[60.0 * EV])
    a = W.Species("A", 12.0 * AMU, 3e-10, E_form=3.0 * EV)
    b = W.Species("B", 8.0 * AMU, 3e-10, E_form=1.0 * EV)
    o = oracle.Oracle()
    for s in (ab, a, b):
        o.add_species(s)
    o.add_reaction(W.Reaction("recomb", [1, 2], [0, -1], diss_mode_mask=1))
    for T in (800.0, 3000.0, 7000.0):
        mu = (12.0 * 8.0 / 20.0) * AMU
        qtr = (2 * math.pi * mu * KB * T / H ** 2) ** 1.5
        zpe = 0.5 * HC * we
        dE0 = 4.0 * EV - zpe
        ref = qtr * (1.0 - math.exp(-theta / T)) * math.exp(-dE0 / (KB * T))
        assert abs(o.keq(0, T) - ref) < 1e-9 * ref, (T, o.keq(0, T), ref)


def test_rate_table_interpolation_and_nodes():
    o = _ch4_system()
    assert oracle.rec_node_T(0) == 500.0 and oracle.rec_node_T(32) == 1000.0
    assert oracle.rec_node_T(oracle.REC_NODES - 1) == 64000.0
    i = 112  # 500 * 2^3.5
    T0, T1 = oracle.rec_node_T(i), oracle.rec_node_T(i + 1)
    k0, k1 = o.rec_rate_node(1, 2, i), o.rec_rate_node(1, 2, i + 1)
    assert o.rec_rate(1, 2, T0) == k0
    Tm = 0.5 * (T0 + T1)
    assert abs(o.rec_rate(1, 2, Tm) - 0.5 * (k0 + k1)) <= 1e-15 * k0
    # k_r = P <sigma g>_{A,M} / K_eq at a node
    kf = o.diss_prob(1, T0) * o.mean_sigma_g(0, 2, T0)
    assert abs(k0 - kf / o.keq(1, T0)) <= 1e-14 * k0


def test_cell_temperature_matches_numpy():
    w = W.ch4_heat_bath(n_cells=3, per_cell=700, T0=8000.0)
    o = oracle.from_workload(w)
    v, qn, sp, cell = o.read_particles(0)
    m = np.array([s.mass for s in w.species])[sp]
    for c in range(3):
        s = cell == c
        V = np.sum(m[s, None] * v[s], axis=0) / np.sum(m[s])
        T = np.sum(m[s] * np.sum((v[s] - V) ** 2, axis=1)) / (3 * KB * np.sum(s))
        assert abs(o.cell_temperature(0, c) - T) < 1e-9 * T


def _mix(n_cells, per_cell, T, n_density, fractions, seed, steps=50):
    sp = [W.ch4_like(), W.ch3_like(), W.h_atom()]
    rx = [W.Reaction("recomb", [1, 2], [0, -1], diss_mode_mask=0xF)]
    dt = 0.2 / W.vhs_collision_frequency(sp[1], n_density, T)
    return W._build("recomb_mix", sp, rx, n_cells, np.full(n_cells, per_cell), fractions, 4.64e-6,
                    n_density, dt, T, T, seed, steps)


def _energy_momentum(o, species):
    v, qn, sp, cell = o.read_particles(0)
    m = np.array([s.mass for s in species])[sp]
    E = 0.5 * np.sum(m * np.sum(v * v, axis=1)) + np.sum(np.array([s.E_form for s in species])[sp])
    for k, s in enumerate(species):
        sel = sp == k
        for j in range(s.n_modes):
            lev = np.array([o.L.ora_level_energy(o.ctx, k, j, i) for i in range(o.n_levels(k, j))])
            E += lev[qn[sel, j]].sum()
    return E, np.sum(m[:, None] * v, axis=0), np.sum(m * np.linalg.norm(v, axis=1)), sp


def test_recombination_conserves_and_removes():
    w = _mix(4, 500, 2000.0, 1e26, [0.0, 0.5, 0.5], seed=11)
    o = oracle.from_workload(w)
    E0, p0, ps, sp0 = _energy_momentum(o, w.species)
    n0 = o.count(0)
    for _ in range(4):
        o.step(1)
    E1, p1, _, sp1 = _energy_momentum(o, w.species)
    nrec = int(o.read_counters(0)[8])
    assert nrec > 20
    assert o.count(0) == n0 - nrec
    assert np.bincount(sp1, minlength=3)[0] == nrec
    assert np.bincount(sp1, minlength=3)[1] == np.bincount(sp0, minlength=3)[1] - nrec
    assert np.all(sp1 >= 0)
    assert abs(E1 - E0) <= 1e-12 * abs(E0)
    assert np.all(np.abs(p1 - p0) <= 1e-12 * ps)


def test_recombination_rate_law():
    """Counted recombinations per step vs k_r(T_cell) n_B n_C n V dt / w
    summed over steps and cells (n the third-body density), within 3.5 sigma
    of the Poisson spread."""
    w = _mix(6, 600, 2500.0, 3e25, [0.0, 0.5, 0.5], seed=12)
    o = oracle.from_workload(w)
    expected = 0.0
    counted = 0
    for _ in range(20):
        v, qn, sp, cell = o.read_particles(0)
        for c in range(w.n_cells):
            s = cell == c
            N = int(np.sum(s))
            nB = np.sum(sp[s] == 1) * w.weight / w.cell_volume
            nC = np.sum(sp[s] == 2) * w.weight / w.cell_volume
            n3 = (N - 2) * w.weight / w.cell_volume
            T = o.cell_temperature(0, c)
            # third bodies of each species in proportion to the cell's composition
            kr = sum(np.sum(sp[s] == k) / N * o.rec_rate(0, k, T) for k in range(3))
            expected += kr * nB * nC * n3 * w.cell_volume * w.dt / w.weight
        before = int(o.read_counters(0)[8])
        o.step(1)
        counted += int(o.read_counters(0)[8]) - before
    assert expected > 120
    assert abs(counted - expected) < 3.5 * math.sqrt(expected) + 0.02 * expected, (counted, expected)
