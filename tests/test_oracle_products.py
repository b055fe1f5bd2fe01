"""Pins of the oracle's reaction products (Sec. "Polyatomic QK reaction
modeling": the remaining energy is redistributed over the products with the
Larsen-Borgnakke model; reading A13), from what the reading and the
mathematics fix independently of the oracle's code:

* exact conservation of momentum and of energy (kinetic + vibrational +
  formation) in every event;
* the first product's levels follow the enumerated LB target at the
  available energy minus its partner's ZPE, the second product's levels the
  target at what the first left (a randomised probability-integral transform
  of every event is uniform); the target without the ZPE reservation is
  rejected, so the test tells the readings apart;
* dissociation: the three-body translational energy splits as Beta(3/2, 3/2)
  between the B-C and (BC)-M relative motions, both directions isotropic and
  independent; exchange and recombination (B + C + M -> A + M, reading A14):
  the relative direction is isotropic and the relative kinetic energy is what
  the levels left.

All draws come from the oracle's own diagnostic ora_sample_products: n
independent executions of the reaction on one fixed pair of reactants.
"""
import math

import numpy as np
from scipy import stats

import oracle
from paper_2606_31548_b300 import workloads as W

EV = 1.602176634e-19
N = 20000


def _system():
    sp = [W.ch4_like(), W.h_atom(), W.ch3_like(), W.h2()]
    o = oracle.Oracle()
    for s in sp:
        o.add_species(s)
    o.add_reaction(W.Reaction("diss", [0], [2, 1], diss_mode_mask=0xF))
    o.add_reaction(W.Reaction("exch", [0, 1], [2, 3], Ea=1.03e-19, steric=1.0, alpha_mode="one_random_stretch"))
    return o, sp


def _a(sp):
    """LB exponent xi_rel/2 - 1, xi_rel = 5 - 2 omega."""
    return (5.0 - 2.0 * sp[0].omega) / 2.0 - 1.0


def _levels(o, k, s):
    return [np.array(o.levels(k, j)) for j in range(s.n_modes)]


def _evib(levels, q):
    return sum(levels[j][q[j]] for j in range(len(levels)))


def _budget_velocity(o, sp, iA, iM, products, E_extra):
    mA, mM = sp[iA].mass, sp[iM].mass
    mu = mA * mM / (mA + mM)
    dEf = sum(sp[p].E_form for p in products) - sp[iA].E_form - sp[iM].E_form
    EvA = o.zpe(iA)
    EvM = o.zpe(iM) if sp[iM].n_modes else 0.0
    Eav = sum(o.zpe(p) if sp[p].n_modes else 0.0 for p in products) + E_extra
    Erel = Eav + dEf - EvA - EvM
    g = math.sqrt(2.0 * Erel / mu)
    return np.zeros(3), np.array([0.3 * g, -0.4 * g, math.sqrt(0.75) * g]), Eav


def _lb_pmf(levels, Ec, a):
    """The LB target p(q) ~ (Ec - sum_j E_j(q_j))^a over the states with
    sum E < Ec, enumerated by brute force."""
    keys, w = [], []

    def rec(j, rem, cur):
        if j == len(levels):
            keys.append(tuple(cur))
            w.append(rem ** a)
            return
        for i, e in enumerate(levels[j]):
            if e >= rem:
                break
            cur.append(i)
            rec(j + 1, rem - e, cur)
            cur.pop()

    rec(0, Ec, [])
    w = np.array(w)
    return keys, w / w.sum()


def _chi2_p(keys, p, q, n_modes):
    idx = {k: i for i, k in enumerate(keys)}
    cnt = np.zeros(len(keys))
    for row in q[:, :n_modes]:
        cnt[idx[tuple(int(x) for x in row)]] += 1
    exp = p * len(q)
    big = exp >= 5
    obs = np.append(cnt[big], cnt[~big].sum())
    ex = np.append(exp[big], exp[~big].sum())
    if ex[-1] == 0:
        obs, ex = obs[:-1], ex[:-1]
    return stats.chisquare(obs, ex).pvalue


def _isotropic_p(u):
    """Two KS p-values: cos(theta) ~ U(-1, 1), phi ~ U(0, 2 pi)."""
    u = u / np.linalg.norm(u, axis=1)[:, None]
    p1 = stats.kstest(u[:, 2], stats.uniform(-1, 2).cdf).pvalue
    p2 = stats.kstest(np.arctan2(u[:, 1], u[:, 0]) % (2 * np.pi), stats.uniform(0, 2 * np.pi).cdf).pvalue
    return min(p1, p2), u


def _totals(masses, E_form, v, evib):
    P = sum(m * vi for m, vi in zip(masses, v))
    E = sum(0.5 * m * float(vi @ vi) for m, vi in zip(masses, v)) + sum(E_form) + evib
    return P, E


def test_dissociation_products():
    o, sp = _system()
    a = _a(sp)
    vA, vM, Eav = _budget_velocity(o, sp, 0, 1, [2, 1], 1.0 * EV)
    qA = np.zeros(16, np.uint8)
    v, q = o.sample_products(0, [(0, vA, qA), (1, vM, np.zeros(16, np.uint8))], seed=7, n=N)
    assert len(v) == N
    mA, mB, mC, mM = sp[0].mass, sp[2].mass, sp[1].mass, sp[1].mass
    LB = _levels(o, 2, sp[2])
    P0, E0 = _totals([mA, mM], [sp[0].E_form, sp[1].E_form], [vA, vM], o.zpe(0))
    scale = mA * float(np.linalg.norm(vM)) + mM * float(np.linalg.norm(vM))
    EvB = np.array([_evib(LB, q[i, 0]) for i in range(N)])
    for i in range(0, N, 97):
        P1, E1 = _totals([mB, mC, mM], [sp[2].E_form, sp[1].E_form, sp[1].E_form], list(v[i]), EvB[i])
        assert np.all(np.abs(P1 - P0) <= 1e-12 * scale)
        assert abs(E1 - E0) <= 1e-12 * abs(E0)
    assert np.all(q[:, 1] == 0)  # H has no modes
    # first product: LB target at Eav - ZPE(H) = Eav
    keys, p = _lb_pmf(LB, Eav, a)
    assert _chi2_p(keys, p, q[:, 0], sp[2].n_modes) > 1e-3
    # Beta(3/2, 3/2) split of the translational energy left
    vB, vC, vM1 = v[:, 0], v[:, 1], v[:, 2]
    mBC, mt = mB + mC, mB + mC + mM
    VBC = (mB * vB + mC * vC) / mBC
    E1 = 0.5 * (mB * mC / mBC) * np.sum((vB - vC) ** 2, axis=1)
    E2 = 0.5 * (mBC * mM / mt) * np.sum((VBC - vM1) ** 2, axis=1)
    assert np.allclose(E1 + E2, Eav - EvB, rtol=1e-9, atol=0)
    x = E1 / (E1 + E2)
    assert stats.kstest(x, stats.beta(1.5, 1.5).cdf).pvalue > 1e-3
    assert stats.kstest(x, stats.uniform().cdf).pvalue < 1e-6  # a wrong split is seen
    # both Jacobi directions isotropic, and independent of each other
    pa, u1 = _isotropic_p(vB - vC)
    pb, u2 = _isotropic_p(VBC - vM1)
    assert pa > 1e-3 and pb > 1e-3
    assert stats.kstest(np.sum(u1 * u2, axis=1), stats.uniform(-1, 2).cdf).pvalue > 1e-3


def test_exchange_products():
    o, sp = _system()
    a = _a(sp)
    vA, vB, Eav = _budget_velocity(o, sp, 0, 1, [2, 3], 1.0 * EV)
    v, q = o.sample_products(1, [(0, vA, np.zeros(16, np.uint8)), (1, vB, np.zeros(16, np.uint8))], seed=11, n=N)
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
    # first product CH3: LB target at Eav - ZPE(H2); without the reservation: rejected
    keys, p = _lb_pmf(LC, Eav - o.zpe(3), a)
    assert _chi2_p(keys, p, q[:, 0], sp[2].n_modes) > 1e-3
    keys_w, p_w = _lb_pmf(LC, Eav, a)
    assert _chi2_p(keys_w, p_w, q[:, 0], sp[2].n_modes) < 1e-6
    # second product H2 given the first: randomised PIT of its level is
    # uniform at the budget the first left, and not at the full budget
    rng = np.random.default_rng(5)
    E = LD[0]

    def pit_p(budget):
        pit = np.empty(N)
        for i in range(N):
            Ec = budget(i)
            w = np.where(E < Ec, np.maximum(Ec - E, 0.0) ** a, 0.0)
            w /= w.sum()
            k = int(q[i, 1, 0])
            pit[i] = w[:k].sum() + rng.random() * w[k]
        return stats.kstest(pit, stats.uniform().cdf).pvalue

    assert pit_p(lambda i: Eav - EvC[i]) > 1e-3
    assert pit_p(lambda i: Eav) < 1e-6
    # relative motion: the energy the levels left, isotropic direction
    mu = mC * mD / (mC + mD)
    Erel = 0.5 * mu * np.sum((v[:, 0] - v[:, 1]) ** 2, axis=1)
    assert np.allclose(Erel, Eav - EvC - EvD, rtol=1e-9, atol=0)
    pd, _ = _isotropic_p(v[:, 0] - v[:, 1])
    assert pd > 1e-3


def test_recombination_products():
    """H + H + M -> H2 + M: H2's level takes the LB target at the whole
    available energy (the released binding energy included), the A-M motion
    the rest in an isotropic direction."""
    sp = [W.h_atom(), W.h2()]
    o = oracle.Oracle()
    for x in sp:
        o.add_species(x)
    o.add_reaction(W.Reaction("recomb", [0, 0], [1, -1], diss_mode_mask=1))
    a = _a(sp)
    mH, mA = sp[0].mass, sp[1].mass
    u = math.sqrt(0.75 * 0.5 * EV / mH)  # 0.5 eV in the three bodies' centre-of-mass frame
    vB, vC, vM = np.array([u, 0.0, 0.0]), np.array([-u, 0.0, 0.0]), np.array([0.0, u, 0.0])
    z = np.zeros(16, np.uint8)
    v, q = o.sample_products(0, [(0, vB, z), (0, vC, z), (0, vM, z)], seed=13, n=N)
    assert len(v) == N
    P0 = mH * (vB + vC + vM)
    KE0 = 0.5 * mH * float(vB @ vB + vC @ vC + vM @ vM)
    mt = mA + mH
    V = P0 / mt
    Eav = KE0 - 0.5 * mt * float(V @ V) - sp[1].E_form  # E_form(H) = 0; no vibration in
    LA = _levels(o, 1, sp[1])
    EvA = np.array([LA[0][q[i, 0, 0]] for i in range(N)])
    vA, vM1 = v[:, 0], v[:, 2]
    for i in range(0, N, 97):
        P1 = mA * vA[i] + mH * vM1[i]
        E1 = 0.5 * mA * float(vA[i] @ vA[i]) + 0.5 * mH * float(vM1[i] @ vM1[i]) + sp[1].E_form + EvA[i]
        assert np.all(np.abs(P1 - P0) <= 1e-12 * mH * u)
        assert abs(E1 - KE0) <= 1e-12 * abs(sp[1].E_form)
    assert np.all(v[:, 1] == 0.0)
    # H2's level: LB target at Eav over its levels below Eav
    keys, p = _lb_pmf(LA, Eav, a)
    assert _chi2_p(keys, p, q[:, 0], 1) > 1e-3
    # the A-M motion: what the level left, isotropic
    mu = mA * mH / mt
    Erel = 0.5 * mu * np.sum((vA - vM1) ** 2, axis=1)
    assert np.allclose(Erel, Eav - EvA, rtol=1e-9, atol=0)
    pd, _ = _isotropic_p(vA - vM1)
    assert pd > 1e-3
