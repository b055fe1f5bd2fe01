"""Pins of the oracle's second reading of the product redistribution
(Sec. "Polyatomic QK reaction modeling": the energy left after a reaction is
shared by LB over the products' degrees of freedom by equipartition, the
vibrational ones found by root-finding at a collision temperature T_c).

The reading, restated independently of the oracle's code:

* T_c solves xi_tr/2 k T_c + sum_p <E_vib,p>(T_c) = E_x, E_x the available
  energy above the products' ground states, xi_tr = 3 per relative motion of
  the products (6 after a dissociation, 3 after an exchange or a
  recombination), <E_vib> the Boltzmann mean above the ground level (a
  stretch over its level list, a bend the harmonic kTheta/(e^(Theta/T) - 1));
* the first product's levels follow (E - E_state)^b1 at the available energy
  minus the partner's ZPE, b1 = (xi_tr + xi_vib,2(T_c))/2 - 1 with
  xi_vib = 2 <E_vib>(T_c) / (k T_c); the second product's follow
  (E - E_state)^(xi_tr/2 - 1) at what the first left; a recombination's
  product (E - E_state)^(1/2) at the whole available energy.

Each test enumerates the target by brute force and checks the draws of
ora_sample_products against it (chi^2 or a randomised probability-integral
transform), rejects the relaxation-table reading (exponent 3/2 - omega), and
checks exact conservation in every event.
"""
import math

import numpy as np
from scipy import optimize, stats

import oracle
from paper_2606_31548_b300 import workloads as W
from test_oracle_products import (EV, _budget_velocity, _chi2_p, _evib, _levels, _lb_pmf, _totals)

KB = 1.380649e-23
N = 20000
TC = "collision_temperature"


def _mean_evib(levels, species, T):
    """Boltzmann mean vibrational energy above the ground level."""
    e = 0.0
    ns = len(species.we)
    for j, L in enumerate(levels):
        if j >= ns:
            th = species.theta[j - ns]
            e += KB * th / math.expm1(th / T) if th / T < 700.0 else 0.0
        else:
            de = L - L[0]
            w = np.exp(-de / (KB * T))
            e += float((de * w).sum() / w.sum())
    return e


def _t_coll(xi_tr, prods, Ex):
    def f(T):
        return 0.5 * xi_tr * KB * T + sum(_mean_evib(L, s, T) for L, s in prods) - Ex
    return optimize.brentq(f, 1.0, 1e7, xtol=1e-9, rtol=1e-14)


def _system():
    sp = [W.ch4_like(), W.h_atom(), W.ch3_like(), W.h2()]
    o = oracle.Oracle()
    for s in sp:
        o.add_species(s)
    o.add_reaction(W.Reaction("diss", [0], [2, 1], diss_mode_mask=0xF, product_split=TC))
    o.add_reaction(W.Reaction("exch", [0, 1], [2, 3], Ea=1.03e-19, steric=1.0, alpha_mode="one_random_stretch",
                              product_split=TC))
    return o, sp


def test_own_exponential():
    """The oracle's own exponential (T_c and the acceptance powers use it, so
    that the device can reproduce them bit for bit) against the C library's
    over its range: within 2 ulp, exact at 0, 0 below -708."""
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(-708.0, 709.0, 20000), rng.uniform(-1.0, 1.0, 20000),
                         rng.uniform(-1e-9, 1e-9, 200), [-708.0, 709.0, 1.0, -1.0, 0.5 * math.log(2.0)]])
    rel = max(abs(oracle.exp(float(x)) - math.exp(float(x))) / math.exp(float(x)) for x in xs)
    assert rel < 4.5e-16, rel
    assert oracle.exp(0.0) == 1.0
    assert oracle.exp(-709.5) == 0.0
    # x^y = e^(y ln x) through the two own series
    for x, y in [(0.3, 0.25), (0.9, 1.5), (1e-6, 0.5), (0.5, 2.0)]:
        assert abs(oracle.exp(y * oracle.ln(x)) - x ** y) < 1e-15 * x ** y


def test_tcoll_dissociation_products():
    """CH4 + M -> CH3 + H + M: H has no modes, so T_c drops out and CH3's
    levels follow exponent b1 = 6/2 - 1 = 2 at the whole available energy."""
    o, sp = _system()
    vA, vM, Eav = _budget_velocity(o, sp, 0, 1, [2, 1], 1.0 * EV)
    qA = np.zeros(16, np.uint8)
    v, q = o.sample_products(0, [(0, vA, qA), (1, vM, np.zeros(16, np.uint8))], seed=17, n=N)
    assert len(v) == N
    mA, mB, mC, mM = sp[0].mass, sp[2].mass, sp[1].mass, sp[1].mass
    LB = _levels(o, 2, sp[2])
    P0, E0 = _totals([mA, mM], [sp[0].E_form, sp[1].E_form], [vA, vM], o.zpe(0))
    scale = mA * float(np.linalg.norm(vM)) + mM * float(np.linalg.norm(vM))
    for i in range(0, N, 97):
        EvB = _evib(LB, q[i, 0])
        P1, E1 = _totals([mB, mC, mM], [sp[2].E_form, sp[1].E_form, sp[1].E_form], list(v[i]), EvB)
        assert np.all(np.abs(P1 - P0) <= 1e-12 * scale)
        assert abs(E1 - E0) <= 1e-12 * abs(E0)
    keys, p = _lb_pmf(LB, Eav, 2.0)
    assert _chi2_p(keys, p, q[:, 0], sp[2].n_modes) > 1e-3
    keys, p = _lb_pmf(LB, Eav, 0.75)  # the relaxation tables' exponent
    assert _chi2_p(keys, p, q[:, 0], sp[2].n_modes) < 1e-6


def test_tcoll_exchange_products():
    """CH4 + H -> CH3 + H2 at 2 eV above the products' ground states: CH3's
    levels follow b1 = (3 + xi_vib,H2(T_c))/2 - 1, H2's exponent 1/2 at what
    CH3 left."""
    o, sp = _system()
    vA, vB, Eav = _budget_velocity(o, sp, 0, 1, [2, 3], 2.0 * EV)
    v, q = o.sample_products(1, [(0, vA, np.zeros(16, np.uint8)), (1, vB, np.zeros(16, np.uint8))], seed=19, n=N)
    assert len(v) == N
    mA, mB, mC, mD = sp[0].mass, sp[1].mass, sp[2].mass, sp[3].mass
    LC, LD = _levels(o, 2, sp[2]), _levels(o, 3, sp[3])
    P0, E0 = _totals([mA, mB], [sp[0].E_form, sp[1].E_form], [vA, vB], o.zpe(0))
    scale = mB * float(np.linalg.norm(vB))
    EvC = np.array([_evib(LC, q[i, 0]) for i in range(N)])
    EvD = np.array([_evib(LD, q[i, 1]) for i in range(N)])
    for i in range(0, N, 97):
        P1, E1 = _totals([mC, mD], [sp[2].E_form, sp[3].E_form], [v[i, 0], v[i, 1]], EvC[i] + EvD[i])
        assert np.all(np.abs(P1 - P0) <= 1e-12 * scale)
        assert abs(E1 - E0) <= 1e-12 * abs(E0)
    Ex = Eav - o.zpe(2) - o.zpe(3)
    Tc = _t_coll(3.0, [(LC, sp[2]), (LD, sp[3])], Ex)
    xiD = 2.0 * _mean_evib(LD, sp[3], Tc) / (KB * Tc)
    b1 = (3.0 + xiD) / 2.0 - 1.0
    assert 3000.0 < Tc < 20000.0 and 0.3 < xiD < 2.0
    keys, p = _lb_pmf(LC, Eav - o.zpe(3), b1)
    assert _chi2_p(keys, p, q[:, 0], sp[2].n_modes) > 1e-3
    keys, p = _lb_pmf(LC, Eav - o.zpe(3), 0.75)
    assert _chi2_p(keys, p, q[:, 0], sp[2].n_modes) < 1e-6
    # H2 given CH3: randomised PIT at exponent 1/2 and the budget CH3 left
    rng = np.random.default_rng(23)
    E = LD[0]

    def pit_p(b):
        pit = np.empty(N)
        for i in range(N):
            Ec = Eav - EvC[i]
            w = np.where(E < Ec, np.maximum(Ec - E, 0.0) ** b, 0.0)
            w /= w.sum()
            k = int(q[i, 1, 0])
            pit[i] = w[:k].sum() + rng.random() * w[k]
        return stats.kstest(pit, stats.uniform().cdf).pvalue

    assert pit_p(0.5) > 1e-3
    mu = mC * mD / (mC + mD)
    Erel = 0.5 * mu * np.sum((v[:, 0] - v[:, 1]) ** 2, axis=1)
    assert np.allclose(Erel, Eav - EvC - EvD, rtol=1e-9, atol=0)


def test_tcoll_recombination_triatomic():
    """OH + H + M -> H2O + M: H2O's three modes follow exponent 1/2 at the
    whole available energy (drawn through the exponent-1/2 tables, since 1/2
    is below the relaxation tables' 3/4)."""
    sp = [W.paper_species("H2O"), W.paper_species("OH"), W.paper_species("H")]
    o = oracle.Oracle()
    for x in sp:
        o.add_species(x)
    o.add_reaction(W.Reaction("recomb", [1, 2], [0, -1], diss_mode_mask=1, product_split=TC))
    mW, mOH, mH = sp[0].mass, sp[1].mass, sp[2].mass
    z = np.zeros(16, np.uint8)
    u = 3000.0
    vB, vC, vM = np.array([0.2 * u, 0.0, 0.0]), np.array([-u, 0.1 * u, 0.0]), np.array([0.0, 0.0, u])
    v, q = o.sample_products(0, [(1, vB, z), (2, vC, z), (2, vM, z)], seed=29, n=N)
    assert len(v) == N
    P0 = mOH * vB + mH * vC + mH * vM
    KE0 = 0.5 * (mOH * float(vB @ vB) + mH * float(vC @ vC) + mH * float(vM @ vM))
    mt = mW + mH
    V = P0 / mt
    LW = _levels(o, 0, sp[0])
    Eav = KE0 - 0.5 * mt * float(V @ V) + o.zpe(1) - (sp[0].E_form - sp[1].E_form - sp[2].E_form)
    Ein = KE0 + o.zpe(1) + sp[1].E_form
    EvA = np.array([_evib(LW, q[i, 0]) for i in range(N)])
    for i in range(0, N, 97):
        P1 = mW * v[i, 0] + mH * v[i, 2]
        E1 = 0.5 * mW * float(v[i, 0] @ v[i, 0]) + 0.5 * mH * float(v[i, 2] @ v[i, 2]) + sp[0].E_form + EvA[i]
        assert np.all(np.abs(P1 - P0) <= 1e-12 * mH * u * 3)
        assert abs(E1 - Ein) <= 1e-12 * abs(Eav)
    keys, p = _lb_pmf(LW, Eav, 0.5)
    assert _chi2_p(keys, p, q[:, 0], 3) > 1e-3
    keys, p = _lb_pmf(LW, Eav, 0.75)
    assert _chi2_p(keys, p, q[:, 0], 3) < 1e-6
