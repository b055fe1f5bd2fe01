"""Pins of the oracle's Whitten-Rabinovitch approximation of the recombination
probability P (the sampled form the paper gives beside Eq. recomb-correct),
from what the mathematics fixes independently of the oracle's code:

* the WR density of states approximates the exact density of harmonic
  oscillators: state counts over energy windows against the Beyer-Swinehart
  count of the same oscillators (integer wavenumbers).  With the decadic
  logarithm in the Omega correlation (the reading taken) CH4- and CH3-like
  sets agree within 6% from the zero-point energy up; the natural logarithm
  would be 15-50% off, so the count decides the reading;
* one oscillator has a constant density, so the WR sum is the midpoint rule
  of a Boltzmann average of Q over the energies below the threshold, which
  scipy's quadrature gives independently;
* the sum converges in the number of sample energies.

It also compares the WR form with the exact level sum for the CH4 molecule
(the exact sum is pinned in tests/test_oracle_recomb.py).
"""
import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_2606_31548_b300 import workloads as W

HC = 6.62607015e-34 * 299792458.0  # J m
CM = 100.0                          # 1 cm^-1 in m^-1
KB = 1.380649e-23


def _bs_counts(freqs_cm, emax):
    """Beyer-Swinehart: number of harmonic states at each integer wavenumber
    (exact for integer frequencies)."""
    rho = np.zeros(emax + 1)
    rho[0] = 1.0
    for f in freqs_cm:
        for e in range(f, emax + 1):
            rho[e] += rho[e - f]
    return rho


@pytest.mark.parametrize("freqs", [[2980] * 4 + [1300] * 3 + [1550] * 2,  # CH4-like
                                   [2980] * 3 + [606, 1401, 1401]])       # CH3-like
@pytest.mark.parametrize("x", [1.0, 2.0, 4.0])
def test_wr_density_counts_harmonic_states(freqs, x):
    hnu = [f * CM * HC for f in freqs]
    ez = 0.5 * sum(freqs)
    rho = _bs_counts(freqs, int(1.3 * x * ez) + 10)
    lo, hi = int(0.75 * x * ez), int(1.25 * x * ez)
    exact = rho[lo:hi].sum()
    wr = integrate.quad(lambda e: oracle.wr_density(hnu, e * CM * HC) * CM * HC, lo, hi, limit=200)[0]
    assert exact > 100
    assert abs(wr / exact - 1.0) < 0.06, (x, wr, exact)


def _h2_recombination():
    sp = [W.h_atom(), W.h2()]
    o = oracle.Oracle()
    for s in sp:
        o.add_species(s)
    o.add_reaction(W.Reaction("recomb", [0, 0], [1, -1], diss_mode_mask=1))
    return o, sp


@pytest.mark.parametrize("T", [3000.0, 8000.0, 20000.0])
def test_wr_probability_one_oscillator_is_the_boltzmann_average(T):
    """l = 1: rho is constant, so P = int_0^D Q(a, (D-E)/kT) e^(-E/kT) dE /
    int_0^D e^(-E/kT) dE, D the threshold above the ground level (for H2:
    its De less its ground level)."""
    o, sp = _h2_recombination()
    a = 2.5 - sp[1].omega
    D = sp[1].De[0] - o.levels(1, 0)[0]
    kT = KB * T
    num = integrate.quad(lambda e: special.gammaincc(a, (D - e) / kT) * np.exp(-e / kT), 0.0, D, limit=400)[0]
    den = integrate.quad(lambda e: np.exp(-e / kT), 0.0, D, limit=400)[0]
    P = o.diss_prob_wr(0, T, 4000)
    assert abs(P - num / den) <= 1e-6 * (num / den), (P, num / den)


def _ch4():
    o = oracle.Oracle()
    for s in (W.ch4_like(), W.ch3_like(), W.h_atom()):
        o.add_species(s)
    o.add_reaction(W.Reaction("diss", [0], [1, 2], diss_mode_mask=0xF))
    o.add_reaction(W.Reaction("recomb", [1, 2], [0, -1], diss_mode_mask=0xF))
    return o


@pytest.mark.parametrize("T", [2000.0, 6000.0, 15000.0])
def test_wr_probability_converges_and_stays_near_the_exact_sum(T):
    o = _ch4()
    p1, p8 = o.diss_prob_wr(1, T, 1000), o.diss_prob_wr(1, T, 8000)
    assert abs(p1 - p8) <= 1e-4 * p8
    # the WR form omits the states above the threshold and counts harmonic
    # levels; measured 0.56-0.84 of the exact sum for CH4 over 2000-15000 K
    r = p8 / o.diss_prob(1, T)
    assert 0.4 < r < 1.0, r
