"""More pins of the oracle: the competing-reaction choice, the exchange
energy with per-mode coupling and a steric factor, the relaxation sampler at
the collision energies of the hot benchmarks, and the recombination rate
table's interpolation.

Each expected value is computed here from the paper's definitions with
numpy/scipy (level energies are the only thing read from the oracle), so a
plausible mistake in the oracle -- a uniform instead of an E_excess-weighted
channel choice, the coupling applied to the wrong energy, a steric factor
ignored, a sampler that is right only at low energy -- fails one of them.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2606_31548_b300 import workloads as W
from test_oracle_pins import KB, EV, _boltzmann_mode, _chi2, _evib_distribution, _lb_target

U = W.AMU


def _chisq_p(ob, ex, min_expected=5.0):
    """chi^2 p-value of counts ob against expected counts ex; bins expected
    below min_expected are pooled into one (dropped if empty)."""
    ob, ex = np.asarray(ob, float), np.asarray(ex, float)
    big = ex >= min_expected
    o2, e2 = ob[big], ex[big]
    if ex[~big].sum() > 0:
        o2, e2 = np.append(o2, ob[~big].sum()), np.append(e2, ex[~big].sum())
    e2 = e2 * (o2.sum() / e2.sum())
    return stats.chisquare(o2, e2).pvalue


# ---------------------------------------------------------------- P21
def _two_particle_cells(o_factory, species, q_p, q_q, Etr, n_cells, seed):
    """n_cells cells of two CH4 molecules each, in fixed vibrational states
    q_p and q_q with relative translational energy Etr; the time step makes
    one candidate pair per cell with probability 0.8, always accepted."""
    m = species[0].mass
    g = math.sqrt(2.0 * Etr / (0.5 * m))  # Etr = 1/2 (m/2) g^2
    n = 2 * n_cells
    v = np.zeros((n, 3))
    v[0::2, 0] = 0.5 * g
    v[1::2, 0] = -0.5 * g
    qn = np.zeros((n, 16), np.uint8)
    qn[0::2, : len(q_p)] = q_p
    qn[1::2, : len(q_q)] = q_q
    sp = np.zeros(n, np.int32)
    cell = np.repeat(np.arange(n_cells, dtype=np.int32), 2)
    Vc, w = 1e-12, 1.0
    probe = o_factory()
    probe.add_reservoir(n_cells, Vc, w, 1e-9, seed, 300.0)
    probe.load(0, v, qn, sp, cell)
    sgmax = probe.read_cell_sgmax(0, n_cells)[0]
    probe.close()
    # N_sel = 1/2 N (N-1) w sgmax dt / V_c = 0.8 for N = 2; (sigma g)_max of
    # 300 K is far below the pair's sigma g, so every candidate is accepted
    dt = 0.8 * Vc / (w * sgmax)
    o = o_factory()
    o.add_reservoir(n_cells, Vc, w, dt, seed, 300.0)
    o.load(0, v, qn, sp, cell)
    return o


def test_competing_reactions_weighted_by_excess_energy():
    """Sec. "Competing reactions": when several channels have E_excess > 0,
    one is chosen with probability E_excess_i / sum E_excess.  Two CH4
    molecules collide with both above every C-H threshold (Eq. Ecoll-diss:
    E_excess,j = E_tr + E_vib,A - ZPE_A - ZPE_B - ZPE_C + E_A,j,0 - D_e,j; all
    four stretches of a molecule share it).  The fraction of dissociations of
    the less excited partner must be 4 X_Q / (4 X_P + 4 X_Q), not 1/2."""
    species = [W.ch4_like(), W.ch3_like(), W.h_atom()]
    rx = W.Reaction("diss", [0], [1, 2], diss_mode_mask=0xF)

    def fac():
        o = oracle.Oracle()
        for s in species:
            o.add_species(s)
        o.add_reaction(rx)
        return o

    q_p = [6, 5, 0, 0, 1, 0, 0, 0, 0]
    q_q = [2, 2, 0, 0, 0, 0, 0, 0, 0]
    Etr = 4.5 * EV
    lev = oracle.Oracle()
    for s in species:
        lev.add_species(s)
    L = [lev.levels(0, j) for j in range(9)]
    zpe_sum = lev.zpe(0) + lev.zpe(1) + lev.zpe(2)
    ev = lambda q: sum(L[j][q[j]] for j in range(9))
    X = [Etr + ev(q) - zpe_sum + L[0][0] - 4.5 * EV for q in (q_p, q_q)]
    assert X[0] > X[1] > 0.0
    o = _two_particle_cells(fac, species, q_p, q_q, Etr, 6000, 0x21C0)
    o.set_log(True)
    o.step(1)
    lg = o.read_log()
    acc = lg[lg["event"] >= 0]
    assert len(acc) > 4000 and np.all(acc["event"] == 1)  # every accepted pair reacts
    # the member at slot p is the more excited one (even index) or not,
    # depending on the pairing permutation
    p_is_first = (acc["p"] % 2) == 0
    side_q = acc["aux"] >= 16
    broke_less_excited = np.where(p_is_first, side_q, ~side_q)
    frac = float(np.mean(broke_less_excited))
    expect = X[1] / (X[0] + X[1])
    sd = math.sqrt(expect * (1 - expect) / len(acc))
    assert abs(frac - expect) < 3 * sd, (frac, expect, sd)
    assert abs(0.5 - expect) > 10 * sd  # a uniform choice is rejected
    # within a molecule the four stretches are equally likely
    stretch = (acc["aux"] % 16).astype(int)
    cnt = np.bincount(stretch, minlength=4)
    assert len(cnt) == 4
    assert stats.chisquare(cnt).pvalue > 1e-4


# ---------------------------------------------------------------- Eq. Ecoll-exch
def test_exchange_per_mode_coupling_and_steric_factor():
    """Eq. Ecoll-exch with the paper's CH4 + H preset form: alpha_j = 0.21 on
    every mode of CH4 (vibrational energies with their ZPE, reading A12) and a
    steric factor 0.5.  From a Boltzmann state at T the single-step exchange
    probability of a CH4-H collision is
    sigma sum_E p(E_vib = E) Q(5/2 - omega, max(0, (E_a - 0.21 E)/kT)),
    with p(E_vib) the brute-force convolution of the per-mode Boltzmann
    distributions."""
    T = 3000.0
    w = W.ch4_h_exchange(n_cells=120, per_cell=1200, T0=T)
    w.reactions = [W.Reaction("exch", [0, 1], [2, 3], Ea=1.03e-19, steric=0.5,
                              alpha_mode="per_mode", alpha=[0.21] * 9)]
    o = oracle.from_workload(w, log=True)
    v0, q0, sp0, cell0 = o.read_particles(0)
    o.step(1)
    lg = o.read_log()
    acc = lg[lg["event"] >= 0]
    start = np.concatenate([[0], np.cumsum(np.bincount(cell0, minlength=w.n_cells))[:-1]])
    ip = start[acc["cell"]] + acc["p"]
    iq = start[acc["cell"]] + acc["q"]
    mixed = sp0[ip] != sp0[iq]
    n_coll = int(np.sum(mixed))
    n_react = int(np.sum(acc["event"][mixed] == 1))
    lev = [o.levels(0, j) for j in range(9)]
    e, p = _evib_distribution(lev, T)
    kT = KB * T

    def prob(alpha, steric, shift=0.0):
        x = (1.03e-19 - alpha * (e - shift)) / kT
        return steric * float(np.sum(p * special.gammaincc(1.75, np.maximum(0.0, x))))

    P = prob(0.21, 0.5)
    sd = math.sqrt(P * (1 - P) / n_coll)
    assert abs(n_react / n_coll - P) < 3 * sd, (n_react / n_coll, P, n_coll)
    # the steric factor and the coupling both matter at this sample size
    assert abs(prob(0.21, 1.0) - P) > 10 * sd
    assert abs(prob(0.0, 0.5) - P) > 10 * sd
    assert abs(prob(1.0, 0.5) - P) > 10 * sd
    assert abs(prob(0.21, 0.5, shift=o.zpe(0)) - P) > 10 * sd  # coupling without the ZPE


# ---------------------------------------------------------------- sampler at high energy
@pytest.mark.parametrize("dE_eV", [5.0, 10.0, 20.0])
def test_lb_samplers_triatomic_at_high_energy(dE_eV):
    """The K5 table sampler and the literal sampler (uniform proposals per
    mode, joint acceptance: Sec. "Implementation of the polyatomic HCAO
    model") against the enumerated LB target at collision energies far above
    the ZPE (the hot benchmarks run at several eV), and against each other on
    the joint (stretch, stretch) table."""
    s = W.triatomic()
    o = oracle.Oracle()
    o.add_species(s)
    levels = [o.levels(0, j) for j in range(3)]
    Ec = o.zpe(0) + dE_eV * EV
    keys, p = _lb_target(levels, Ec, 0.75)
    assert len(keys) > 500
    n = 60000
    k5, _ = o.sample_lb(0, Ec, seed=4000 + int(dE_eV), n=n)
    lit, tr = o.sample_lb(0, Ec, seed=5000 + int(dE_eV), n=n, method="literal")
    # too many states for a cell-wise chi^2: test the two stretches' joint
    # table and the bend's marginal against the target's
    ks = np.array(keys)
    for smp in (k5, lit):
        joint_t = np.zeros((17, 17))
        np.add.at(joint_t, (ks[:, 0], ks[:, 1]), p)
        joint_s = np.zeros((17, 17))
        np.add.at(joint_s, (smp[:, 0].astype(int), smp[:, 1].astype(int)), 1)
        assert _chisq_p(joint_s.ravel(), joint_t.ravel() * n) > 1e-4
        nb = int(ks[:, 2].max()) + 1
        bend_t = np.bincount(ks[:, 2], weights=p, minlength=nb) * n
        bend_s = np.bincount(smp[:, 2].astype(int), minlength=nb)[:nb]
        assert _chisq_p(bend_s, bend_t) > 1e-4
    # two-sample: K5 against the literal sampler on the joint stretch table
    t = np.zeros((2, 17 * 17))
    for r, smp in enumerate((k5, lit)):
        np.add.at(t[r], smp[:, 0].astype(int) * 17 + smp[:, 1].astype(int), 1)
    keep = t.sum(0) >= 10
    t2 = t[:, keep]
    if t[:, ~keep].sum() > 0:
        t2 = np.concatenate([t2, t[:, ~keep].sum(1, keepdims=True)], axis=1)
    assert stats.chi2_contingency(t2)[1] > 1e-4


def _marginals_by_convolution(levels, Ec, a, de):
    """Exact-to-binning marginals of the LB target p(i) ~ (Ec - sum E)^a:
    for mode k, sum over the other modes' states of (Ec - E_k(i) - sum)^a,
    with the other modes' energy sums binned on a grid of width de (brute
    force convolution of their level lists)."""
    out = []
    nb = int(Ec / de) + 2
    for k in range(len(levels)):
        dens = np.zeros(nb)
        dens[0] = 1.0
        for j, E in enumerate(levels):
            if j == k:
                continue
            nd = np.zeros(nb)
            for e in E:
                b = int(round(e / de))
                if b >= nb:
                    break
                nd[b:] += dens[: nb - b]
            dens = nd
        grid = np.arange(nb) * de
        m = []
        for e in levels[k]:
            r = Ec - e - grid
            m.append(float(np.sum(dens[r > 0] * r[r > 0] ** a)) if e < Ec else 0.0)
        m = np.array(m)
        out.append(m / m.sum())
    return out


@pytest.mark.parametrize("dE_eV", [3.0, 6.0, 10.0])
def test_k5_sampler_ch4_marginals_at_high_energy(dE_eV):
    """Nine-mode CH4-like molecule at collision energies of the heat bath
    (too many states to enumerate): every mode's marginal of the K5 sampler
    against the target's marginal from a binned convolution (chi^2)."""
    s = W.ch4_like()
    o = oracle.Oracle()
    o.add_species(s)
    levels = [o.levels(0, j) for j in range(9)]
    Ec = o.zpe(0) + dE_eV * EV
    marg = _marginals_by_convolution(levels, Ec, 0.75, 2e-4 * EV)
    n = 100000
    smp, _ = o.sample_lb(0, Ec, seed=6000 + int(dE_eV), n=n)
    for k in range(9):
        ex = marg[k] * n
        ob = np.bincount(smp[:, k].astype(int), minlength=len(ex))[: len(ex)]
        pv = _chisq_p(ob, ex)
        assert pv > 1e-4, (k, pv)
    # a linear weight (the exponent of a wrong xi_rel) is rejected on some mode
    lin = _marginals_by_convolution(levels, Ec, 1.0, 2e-4 * EV)
    pvs = []
    for k in range(9):
        ex = lin[k] * n
        ob = np.bincount(smp[:, k].astype(int), minlength=len(ex))[: len(ex)]
        pvs.append(_chisq_p(ob, ex))
    assert min(pvs) < 1e-6


# ---------------------------------------------------------------- recombination table
def test_recombination_rate_table_interpolation_bound():
    """The recombination rate k_r(T) = P(T) <sigma_T g>_{A,M}(T) / K_eq(T)
    (Sec. "Recombination reactions", reading A14) is evaluated in the DSMC
    step from a table at T_i = 500 K 2^(i/32), linearly interpolated (the
    device and the oracle use the same table so that their decisions agree
    bit for bit).  Half-way between nodes, from 1400 K up, the table stays
    within 0.2% of k_r computed at T itself (the interpolation error grows
    towards the coldest nodes: ~1% at 700 K); at a node it is exact."""
    w = W.ch4_recombination()
    o = oracle.Oracle()
    for s in w.species:
        o.add_species(s)
    for r in w.reactions:
        o.add_reaction(r)
    rx, spM = 1, 2

    def exact(T):
        return o.diss_prob(rx, T) * o.mean_sigma_g(0, spM, T) / o.keq(rx, T)

    for i in (48, 96, 128):  # 1430, 4044, 8087 K
        T = 500.0 * 2 ** ((i + 0.5) / 32)
        assert abs(o.rec_rate(rx, spM, T) / exact(T) - 1.0) < 2e-3, T
    T = oracle.rec_node_T(96)
    assert abs(o.rec_rate(rx, spM, T) / exact(T) - 1.0) < 1e-12
