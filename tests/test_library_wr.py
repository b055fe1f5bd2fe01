"""The library's host computation of the Whitten-Rabinovitch density and of
the WR form of the dissociation probability against the oracle's (written
independently; the oracle's is pinned in tests/test_oracle_wr.py).  Both are
plain host code, so this runs on the CPU: the library loads without a GPU."""
import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W


def _ch4():
    o = oracle.Oracle()
    sp = [W.ch4_like(), W.ch3_like(), W.h_atom()]
    for s in sp:
        o.add_species(s)
    o.add_reaction(W.Reaction("diss", [0], [1, 2], diss_mode_mask=0xF))
    o.add_reaction(W.Reaction("recomb", [1, 2], [0, -1], diss_mode_mask=0xF))
    return o, sp


def _quanta(o, k, s):
    return np.array([o.levels(k, j)[1] - o.levels(k, j)[0] for j in range(s.n_modes)])


def test_wr_density_matches_oracle():
    o, sp = _ch4()
    for k in (0, 1):
        hnu = _quanta(o, k, sp[k])
        ez = 0.5 * hnu.sum()
        for x in (0.05, 0.3, 0.99, 1.0, 1.7, 4.0, 20.0):
            a, b = hcao.wr_density(hnu, x * ez), oracle.wr_density(hnu, x * ez)
            assert abs(a - b) <= 1e-12 * b, (k, x, a, b)


@pytest.mark.parametrize("T", [2000.0, 4000.0, 9000.0, 15000.0])
def test_wr_probability_matches_oracle(T):
    """Recombination 1 (CH3 + H -> CH4): the threshold above CH4's ground state
    is min over the breaking stretches of De_j + ZPE(CH4) + ZPE(CH3) + ZPE(H)
    - E_j(0), less ZPE(CH4)."""
    o, sp = _ch4()
    hnu = _quanta(o, 0, sp[0])
    zpe = o.zpe(0) + o.zpe(1)
    D = min(sp[0].De[j] + zpe - o.levels(0, j)[0] for j in range(4)) - o.zpe(0)
    a = hcao.wr_diss_prob(hnu, D, sp[0].omega, T, 1000)
    b = o.diss_prob_wr(1, T, 1000)
    assert abs(a - b) <= 1e-11 * b, (a, b)


def test_wr_rejects_bad_arguments():
    assert np.isnan(hcao.wr_density([1e-20, -1e-20], 1e-19))
    assert np.isnan(hcao.wr_density([], 1e-19))
    assert np.isnan(hcao.wr_diss_prob([1e-20], 1e-19, 0.75, 3000.0, 0))
    assert hcao.wr_diss_prob([1e-20], 0.0, 0.75, 3000.0, 10) == 1.0
