"""The paper's species tables and verification cases as presets (Sec.
"Verification": tab:h2o, tab:hcn, tab:ch4, tab:ch3, the diatomics beside
them and the Arrhenius tables), run by the oracle on a small sample:

* the Morse levels follow Eq. energy-AHO with the tables' omega_e and chi_e
  and stop below D_e = h c omega_e / (4 chi_e);
* every case conserves energy (kinetic + vibrational + formation) and
  momentum per step with its QK and its TCE reactions, and reacts;
* hydrogen cyanide at 5000 K forms CN but no HC (the triple bond's channel is
  out of reach, the paper's qualitative result).
"""
import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import workloads as W
from test_oracle_pins import _energy_momentum

HC = 6.62607015e-34 * 299792458.0


def test_paper_morse_levels():
    s = W.paper_species("CH4")
    o = oracle.Oracle()
    o.add_species(s)
    E = o.levels(0, 0)
    we, chi = 312350.0, 0.0190
    i = np.arange(len(E))
    assert np.allclose(E, HC * we * (i + 0.5) - HC * we * chi * (i + 0.5) ** 2, rtol=1e-12)
    De = HC * we / (4 * chi)
    # kept while below D_e and still rising: E(i+1) - E(i) = h c omega_e (1 - 2 chi (i+1)) > 0
    assert E[-1] < De and len(E) == int(np.floor(1 / (2 * chi))) + 1
    assert np.all(np.diff(E) > 0)
    assert np.allclose(o.levels(0, 4)[:3], np.array([0.5, 1.5, 2.5]) * 1.380649e-23 * 1565.2, rtol=1e-12)


CASES = {
    "water": lambda m: W.paper_water(m, n_per_species=3000),
    "hcn_12000K": lambda m: W.paper_hcn(12000.0, m, n_per_species=3000),
    "methane_exchange": lambda m: W.paper_methane_exchange(m, n_per_species=1500),
    "methane_dissociation": lambda m: _wr(W.paper_methane_dissociation(m, n_per_species=2000)),
}


def _wr(w):
    # the recombination's rate tables from the WR form of P (the exact level
    # sum over this CH4's 27-level stretches takes minutes on one core)
    for r in w.reactions:
        if r.type == "recomb":
            r.recomb_prob = "wr"
    return w


@pytest.mark.parametrize("model", ["qk", "tce"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_paper_case_conserves_and_reacts(case, model):
    w = CASES[case](model)
    o = oracle.from_workload(w)
    E0, p0, ps = _energy_momentum(o, 0, w.species)
    for _ in range(8):
        o.step(1)
        E1, p1, _ = _energy_momentum(o, 0, w.species)
        assert abs(E1 - E0) <= 1e-11 * abs(E0)
        assert np.all(np.abs(p1 - p0) <= 1e-11 * ps)
    assert int(o.read_counters(0)[8]) > 0, (case, model)


def test_paper_hcn_5000K_forms_no_hc():
    w = W.paper_hcn(5000.0, "qk", n_per_species=4000)
    o = oracle.from_workload(w)
    o.step(40)
    c = o.read_counters(0)
    assert c[8] > 0 and c[9] == 0  # H + CN forms, HC + N does not
    _, _, sp, _ = o.read_particles(0)
    assert np.sum(sp == 4) == 0 and np.sum(sp == 3) > 0
