"""Pins of the oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code path: published
known-answer vectors, closed forms of a different shape than the oracle's
formula (level spacings, fundamentals), brute-force enumeration of small
state spaces, conservation laws and kinetic-theory closed forms.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2606_31548_b300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
KB = 1.380649e-23
HC = 6.62607015e-34 * 299792458.0
EV = 1.602176634e-19


# ---------------------------------------------------------------- RNG
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox(v[0:4], v[4:6]) == v[6:10]


@pytest.mark.parametrize("N", [2, 3, 5, 16, 17, 100, 1000, 1200, 4096, 4097, 20000, 65535])
def test_pair_perm_is_bijection(N):
    """The pairing permutation is a bijection of [0,N) (exhaustive)."""
    key = [0x12345678, 0x9ABCDEF0, 0x0F1E2D3C, 0x4B5A6978 ^ N]
    img = [oracle.pair_perm(x, N, key) for x in range(N)]
    assert sorted(img) == list(range(N))
    if N >= 100:  # not the identity
        assert sum(i == x for x, i in enumerate(img)) < N // 10


def test_pair_perm_pairs_are_uniform():
    """Over random keys, pair 0's members are uniform over the cell, their
    offset is uniform over the other particles, and within one key the pairs'
    members do not follow their index (reading A9: every pair of particles
    equally likely)."""
    N = 1200
    rng = np.random.default_rng(77)
    keys = rng.integers(0, 2 ** 32, size=(20000, 4))
    a = np.array([oracle.pair_perm(0, N, list(map(int, k))) for k in keys])
    b = np.array([oracle.pair_perm(1, N, list(map(int, k))) for k in keys])
    assert stats.chisquare(np.bincount(a * 40 // N, minlength=40)).pvalue > 1e-4
    off = (b - a) % N
    assert off.min() >= 1
    assert stats.chisquare(np.bincount((off - 1) * 40 // (N - 1), minlength=40)).pvalue > 1e-4
    key = list(map(int, keys[0]))
    img = np.array([oracle.pair_perm(x, N, key) for x in range(N)])
    assert abs(np.corrcoef(np.arange(N // 2), img[0::2])[0, 1]) < 0.15
    assert abs(np.corrcoef(img[0::2], img[1::2])[0, 1]) < 0.15


# ---------------------------------------------------------------- levels
def _oracle_with(*species, M=2048, span=64 * EV):
    o = oracle.Oracle(M, span)
    for s in species:
        o.add_species(s)
    return o


def test_morse_levels_spacing_and_truncation():
    """Eq. energy-AHO: consecutive spacing hc(we - 2 wexe (i+1)), ground level
    hc(we/2 - wexe/4); the list stops at the last level below De (reading A2)."""
    s = W.triatomic()
    o = _oracle_with(s)
    E = o.levels(0, 0)
    we, wexe, De = s.we[0], s.wexe[0], s.De[0]
    assert E[0] == pytest.approx(HC * (we / 2 - wexe / 4), rel=1e-14)
    dE = np.diff(E)
    i = np.arange(1, len(E))
    assert np.allclose(dE, HC * (we - 2 * wexe * i), rtol=1e-12, atol=0)
    # fundamental transition of the synthetic triatomic: 3800 - 2*80 = 3640 cm^-1
    assert dE[0] / (HC * 100) == pytest.approx(3640.0, rel=1e-12)
    # truncation by brute force: next level would reach De (or stop rising)
    assert E[-1] < De
    nxt = E[-1] + HC * (we - 2 * wexe * len(E))
    assert nxt >= De or nxt <= E[-1]
    assert len(E) == 17
    # C2 stretches: 18 levels; total ZPE of the CH4-like preset
    o2 = _oracle_with(W.ch4_like())
    assert o2.n_levels(0, 0) == 18
    zpe = 4 * HC * (3100e2 / 2 - 60e2 / 4) + 0.5 * HC * (3 * 1300e2 + 2 * 1550e2)
    assert o2.zpe(0) == pytest.approx(zpe, rel=1e-9)


def test_harmonic_levels():
    """Bends: equal spacing k Theta, ground level k Theta / 2."""
    s = W.triatomic()
    o = _oracle_with(s)
    E = o.levels(0, 2)
    kth = KB * s.theta[0]
    assert E[0] == pytest.approx(0.5 * kth, rel=1e-14)
    assert np.allclose(np.diff(E), kth, rtol=1e-9)
    assert len(E) == 256


# ---------------------------------------------------------------- LB sampler
def _enumerate_states(levels, Ec):
    """All states with sum E < Ec, by recursion over modes (brute force)."""
    out = []

    def rec(j, rem, cur):
        if j == len(levels):
            out.append((tuple(cur), rem))
            return
        for i, e in enumerate(levels[j]):
            if e >= rem:
                break
            cur.append(i)
            rec(j + 1, rem - e, cur)
            cur.pop()

    rec(0, Ec, [])
    return out


def _lb_target(levels, Ec, a):
    st = _enumerate_states(levels, Ec)
    keys = [s for s, _ in st]
    w = np.array([r ** a for _, r in st])
    return keys, w / w.sum()


def _chi2(keys, p, samples, n_modes):
    idx = {k: i for i, k in enumerate(keys)}
    cnt = np.zeros(len(keys))
    for row in samples[:, :n_modes]:
        cnt[idx[tuple(int(x) for x in row)]] += 1
    exp = p * len(samples)
    big = exp >= 5
    obs = np.append(cnt[big], cnt[~big].sum())
    ex = np.append(exp[big], exp[~big].sum())
    if ex[-1] == 0:
        obs, ex = obs[:-1], ex[:-1]
    return stats.chisquare(obs, ex).pvalue


@pytest.mark.parametrize("method", ["table", "literal"])
@pytest.mark.parametrize("Ec_eV", [0.9, 2.0, 3.5])
def test_lb_sampler_triatomic_matches_enumerated_target(method, Ec_eV):
    """Relaxation step: p(i) ~ (Ec - sum E)^(xi_rel/2-1), xi_rel = 5 - 2 omega."""
    s = W.triatomic()
    o = _oracle_with(s)
    levels = [o.levels(0, j) for j in range(3)]
    Ec = Ec_eV * EV
    keys, p = _lb_target(levels, Ec, 0.75)
    smp, tr = o.sample_lb(0, Ec, seed=1234 + int(Ec_eV * 10), n=60000, method=method)
    assert _chi2(keys, p, smp, 3) > 1e-4
    # a plausible mistake (linear weight instead of ^0.75) is rejected
    keys1, p1 = _lb_target(levels, Ec, 1.0)
    if Ec_eV > 1.0:
        assert _chi2(keys1, p1, smp, 3) < 1e-6


def test_lb_sampler_pentatomic_matches_enumerated_target():
    """Nine-mode CH4-like molecule at a collision energy small enough to enumerate."""
    s = W.ch4_like()
    o = _oracle_with(s)
    levels = [o.levels(0, j) for j in range(9)]
    Ec = o.zpe(0) + 0.9 * EV
    keys, p = _lb_target(levels, Ec, 0.75)
    assert len(keys) > 200
    smp, tr = o.sample_lb(0, Ec, seed=99, n=80000)
    assert _chi2(keys, p, smp, 9) > 1e-4
    assert 80000 / tr > 0.3  # the table sampler needs few trials


@pytest.mark.parametrize("omega,a", [(0.5, 1.0), (1.0, 0.5)])
def test_lb_sampler_other_vhs_exponents(omega, a):
    s = W.triatomic()
    s.omega = omega
    o = _oracle_with(s)
    levels = [o.levels(0, j) for j in range(3)]
    Ec = 2.5 * EV
    keys, p = _lb_target(levels, Ec, a)
    smp, _ = o.sample_lb(0, Ec, seed=7, n=50000)
    assert _chi2(keys, p, smp, 3) > 1e-4


def test_k5_tables_bound_the_exact_sums():
    """H_k(g) >= sum over the states of modes k..n-1 of (g - sum E)^a (brute force)."""
    s = W.triatomic()
    o = _oracle_with(s, M=512, span=8 * EV)
    levels = [o.levels(0, j) for j in range(3)]
    cq = 8 * EV / 512 ** 2  # quadratic grid g_m = base + cq m^2
    for k in range(3):
        H = o.table(0, k)
        base = sum(l[0] for l in levels[k:])
        for m in [1, 5, 40, 120, 300, 500]:
            g = base + cq * m * m
            exact = sum(r ** 0.75 for _, r in _enumerate_states(levels[k:], g))
            assert H[m] >= exact * (1 - 1e-12)
            if g - base > 0.25 * EV:  # above the ground-state-only range the bound is tight
                assert H[m] <= exact * 1.25 + 1e-30


# ---------------------------------------------------------------- init
def test_initial_populations_are_boltzmann():
    """Initial bend (P6) and stretch (P7, reading A7) levels follow the
    Boltzmann distribution over each mode's levels at T_vib."""
    s = W.triatomic()
    o = _oracle_with(s)
    T = 6000.0
    smp = o.sample_init(0, T, seed=5, n=60000)
    for j in range(3):
        E = o.levels(0, j)
        w = np.exp(-(E - E[0]) / (KB * T))
        p = w / w.sum()
        cnt = np.bincount(smp[:, j], minlength=len(E))[: len(E)]
        ex = p * len(smp)
        big = ex >= 5
        pv = stats.chisquare(np.append(cnt[big], cnt[~big].sum()),
                             np.append(ex[big], ex[~big].sum())).pvalue
        assert pv > 1e-4, (j, pv)


# ---------------------------------------------------------------- DSMC
def _energy_momentum(o, res, species):
    v, qn, sp, cell = o.read_particles(res)
    m = np.array([s.mass for s in species])[sp]
    ke = 0.5 * np.sum(m * np.sum(v * v, axis=1))
    ev = 0.0
    for k, s in enumerate(species):
        sel = sp == k
        for j in range(s.n_modes):
            E = o.levels(k, j)
            ev += E[qn[sel, j]].sum()
    ef = np.sum(np.array([s.E_form for s in species])[sp])
    p = np.sum(m[:, None] * v, axis=0)
    pscale = np.sum(m * np.linalg.norm(v, axis=1))
    return ke + ev + ef, p, pscale


@pytest.mark.parametrize("wl", ["tri", "ch4diss", "exch"])
def test_conservation(wl):
    """Per-collision momentum and energy conservation (summed over a step)."""
    if wl == "tri":
        w = W.relaxation_triatomic(n_particles=3000, n_cells=3)
    elif wl == "ch4diss":
        w = W.ch4_heat_bath(n_cells=4, per_cell=400)
    else:
        w = W.ch4_h_exchange(n_cells=4, per_cell=600, T0=6000.0)
    o = oracle.from_workload(w)
    E0, p0, ps = _energy_momentum(o, 0, w.species)
    for _ in range(6):
        o.step(1)
        E1, p1, _ = _energy_momentum(o, 0, w.species)
        assert abs(E1 - E0) <= 1e-12 * abs(E0) + 1e-30
        assert np.all(np.abs(p1 - p0) <= 1e-12 * ps)
    cnt = o.read_counters(0)
    if wl != "tri":
        assert cnt[8] > 0  # reactions happened


def test_collision_frequency_vhs_closed_form():
    """NTC/VHS: accepted collisions per molecule per second equal the VHS
    closed form nu = 4 d^2 n sqrt(pi k T_ref / m) (T/T_ref)^(1-omega) (the
    paper's recombination rate expression with P = 1, delta_sym = 2)."""
    sp = W.h_atom()
    sp.mass = 40 * W.AMU
    sp.d_ref = 4.0e-10
    T = 3000.0
    N, cells = 40000, 8
    rng = np.random.default_rng(3)
    v = W.maxwellian(rng, N, np.full(N, sp.mass), T)
    cell = np.repeat(np.arange(cells, dtype=np.int32), N // cells)
    n_dens = 1e23
    V = 4.64e-6
    w = n_dens * V / N
    nu = 4 * sp.d_ref ** 2 * n_dens * math.sqrt(math.pi * KB * 273.0 / sp.mass) * (T / 273.0) ** 0.25
    dt = 0.2 / nu
    o = oracle.Oracle()
    o.add_species(sp)
    o.add_reservoir(cells, V / cells, w, dt, 77, T)
    o.load(0, v, np.zeros((N, 16), np.uint8), np.zeros(N, np.int32), cell)
    steps = 10
    o.step(steps)
    acc = int(o.read_counters(0)[1])
    expected = 0.5 * nu * N * dt * steps
    assert abs(acc - expected) < 3.5 * math.sqrt(expected), (acc, expected)


def _boltzmann_mode(E, T):
    w = np.exp(-(E - E[0]) / (KB * T))
    return w / w.sum()


def test_relaxation_reaches_boltzmann_equilibrium_and_detailed_balance():
    """Adiabatic triatomic reservoir: the final level populations equal the
    Boltzmann distribution at the temperature fixed by energy conservation
    (E/N = 3/2 kT + <E_vib>(T), brute-force level sums), T_vib (zero-point
    search) equals that T, and transitions obey detailed balance."""
    w = W.relaxation_triatomic(n_particles=4000, n_cells=4)
    w.T_vib0 = 2000.0
    o = oracle.from_workload(w)
    s = w.species[0]
    lev = [o.levels(0, j) for j in range(3)]
    o.step(250)
    v, qn, sp, _ = o.read_particles(0)
    E_tot, _, _ = _energy_momentum(o, 0, w.species)
    N = len(v)
    m = s.mass
    ptot = np.sum(m * v, axis=0)
    e_int = (E_tot - 0.5 * np.dot(ptot, ptot) / (m * N)) / N

    def e_of_T(T):
        ev = sum(np.sum(_boltzmann_mode(E, T) * E) for E in lev)
        return 1.5 * KB * T + ev

    lo, hi = 100.0, 50000.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if e_of_T(mid) < e_int else (lo, mid)
    Teq = 0.5 * (lo + hi)
    counts = [np.zeros(len(E)) for E in lev]
    trans = np.zeros((16, 16))
    o.set_log(True)
    for _ in range(150):
        q_before = o.read_particles(0)[1][:, 2].copy()
        o.step(1)
        q_after = o.read_particles(0)[1]
        for j in range(3):
            counts[j] += np.bincount(q_after[:, j], minlength=len(lev[j]))[: len(lev[j])]
        a, b = q_before, q_after[:, 2]
        ok = (a < 16) & (b < 16)
        np.add.at(trans, (a[ok], b[ok]), 1)
    # populations vs Boltzmann at Teq (stretch 0 and the bend)
    for j in (0, 2):
        p = _boltzmann_mode(lev[j], Teq)
        tot = counts[j].sum()
        # samples are correlated across steps: compare the fractions with a
        # tolerance of a few standard errors of N independent molecules
        for i in range(4):
            se = math.sqrt(p[i] * (1 - p[i]) / N)
            assert abs(counts[j][i] / tot - p[i]) < 5 * se + 2e-3, (j, i, counts[j][i] / tot, p[i])
    assert abs(o.tvib(0, 0) - Teq) / Teq < 0.05
    # detailed balance in equilibrium: n(i->j) = n(j->i)
    for i in range(4):
        for j in range(i + 1, 5):
            a, b = trans[i, j], trans[j, i]
            if a + b > 50:
                assert abs(a - b) < 4 * math.sqrt(a + b), (i, j, a, b)


def _evib_distribution(levels, T, de=2e-4 * EV):
    """Boltzmann distribution of the total vibrational energy of one molecule
    (energies from the well bottom) on a grid of width de, by convolving the
    per-mode Boltzmann distributions (brute force)."""
    top = sum(E[-1] for E in levels)
    nb = int(top / de) + 2
    dist = np.zeros(nb)
    dist[0] = 1.0
    for E in levels:
        p = _boltzmann_mode(E, T)
        nd = np.zeros(nb)
        for e, pe in zip(E, p):
            if pe < 1e-15:
                continue
            k = int(round(e / de))
            nd[k:] += dist[: nb - k] * pe
        dist = nd
    return np.arange(nb) * de, dist


def test_dissociation_probability_single_step():
    """Eq. Ecoll-diss with the competing-reaction rule: in a Boltzmann state
    at T, P(reaction | collision) = sum over both partners' vibrational
    energies of Q(5/2 - omega, (X - max(Ev_P, Ev_Q))/kT), X = De + ZPE_A +
    ZPE_B + ZPE_C - E_j(0), because every C-H stretch is identical."""
    T = 7000.0
    w = W.ch4_heat_bath(n_cells=200, per_cell=500, T0=T)
    o = oracle.from_workload(w, log=True)
    o.step(1)
    lg = o.read_log()
    acc = lg[lg["event"] >= 0]
    n_coll = len(acc)
    n_react = int(np.sum(acc["event"] == 1))
    lev = [o.levels(0, j) for j in range(9)]
    X = 4.5 * EV + o.zpe(0) + o.zpe(1) + o.zpe(2) - lev[0][0]
    e, p = _evib_distribution(lev, T)
    kT = KB * T
    F = np.cumsum(p)
    pmax = np.diff(np.concatenate([[0.0], F * F]))  # distribution of max(Ev_P, Ev_Q)
    P = float(np.sum(pmax * special.gammaincc(1.75, np.maximum(0.0, (X - e) / kT))))
    sd = math.sqrt(P * (1 - P) / n_coll)
    assert abs(n_react / n_coll - P) < 3.5 * sd + 0.004, (n_react / n_coll, P, n_coll)
    assert 0.05 < P < 0.95


def test_exchange_probability_single_step():
    """Eq. Ecoll-exch with alpha = 1 on one stretch (reading A18) and the ZPE
    included (reading A12): P(exchange | CH4-H collision) =
    sum_i p_i Q(5/2 - omega, max(0, (Ea - E_i)/kT))."""
    T = 4000.0
    w = W.ch4_h_exchange(n_cells=100, per_cell=1200, T0=T)
    o = oracle.from_workload(w, log=True)
    v0, q0, sp0, cell0 = o.read_particles(0)
    o.step(1)
    lg = o.read_log()
    acc = lg[lg["event"] >= 0]
    # the log gives positions within a cell; particles are read cell by cell
    start = np.concatenate([[0], np.cumsum(np.bincount(cell0, minlength=w.n_cells))[:-1]])
    ip = start[acc["cell"]] + acc["p"]
    iq = start[acc["cell"]] + acc["q"]
    mixed = sp0[ip] != sp0[iq]
    n_coll = int(np.sum(mixed))
    n_react = int(np.sum(acc["event"][mixed] == 1))
    E = o.levels(0, 0)
    p = _boltzmann_mode(E, T)
    P = float(np.sum(p * special.gammaincc(1.75, np.maximum(0.0, (1.03e-19 - E) / (KB * T)))))
    sd = math.sqrt(P * (1 - P) / n_coll)
    assert abs(n_react / n_coll - P) < 3.5 * sd, (n_react / n_coll, P, n_coll)
    # reading A12 matters: without the ZPE the probability differs by far
    P_noz = float(np.sum(p * special.gammaincc(1.75, np.maximum(0.0, (1.03e-19 - (E - E[0])) / (KB * T)))))
    assert abs(P_noz - P) > 10 * sd
