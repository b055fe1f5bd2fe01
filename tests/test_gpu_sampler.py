"""The relaxation step's sampler on the GPU (hcao_sample_lb, C ABI).

FP64: identical draws to the oracle's K5 sampler, bit for bit.  FP32 (the
flattened sampler of the fast collision kernel): the enumerated LB target
p(i) ~ (Ec - sum E)^(xi_rel/2 - 1), chi^2.
"""
import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W
from test_oracle_pins import _chi2, _lb_target

pytestmark = pytest.mark.gpu
EV = 1.602176634e-19


def _ctx(species, precision):
    c = hcao.Context(precision=precision)
    c.set_species(species)
    return c


@pytest.mark.parametrize("make,Ec_over_zpe_eV", [(W.triatomic, 0.9), (W.triatomic, 3.0),
                                                 (W.ch4_like, 0.5), (W.ch4_like, 9.0),
                                                 (W.ch4_like, 40.0)])
def test_fp64_sampler_equals_oracle(make, Ec_over_zpe_eV):
    s = make()
    g = _ctx([s], hcao.FP64)
    o = oracle.Oracle()
    o.add_species(s)
    Ec = o.zpe(0) + Ec_over_zpe_eV * EV
    qg, tg = g.sample_lb(0, Ec, 77, 20000)
    qo, to = o.sample_lb(0, Ec, 77, 20000)
    assert np.array_equal(qg, qo)
    assert tg == to


@pytest.mark.parametrize("make,Ec_over_zpe_eV,nm", [(W.triatomic, 0.9, 3), (W.triatomic, 2.5, 3),
                                                    (W.ch4_like, 0.9, 9), (W.ch4_like, 0.3, 9)])
def test_fp32_sampler_matches_enumerated_target(make, Ec_over_zpe_eV, nm):
    s = make()
    g = _ctx([s], hcao.FP32)
    levels = [np.array([g.level_energy(0, j, i) for i in range(g.n_levels(0, j))]) for j in range(nm)]
    zpe = sum(l[0] for l in levels)
    Ec = zpe + Ec_over_zpe_eV * EV
    keys, p = _lb_target(levels, Ec, 0.75)
    smp, tr = g.sample_lb(0, Ec, 1234, 200000)
    assert _chi2(keys, p, smp, nm) > 1e-4
    assert 200000 / tr > 0.5


def test_fp32_sampler_high_energy_mean():
    """At 12 eV above the ZPE (too many states to enumerate) the FP32 and FP64
    samplers agree on the mean of every mode's quantum number (5 sigma)."""
    s = W.ch4_like()
    g32 = _ctx([s], hcao.FP32)
    g64 = _ctx([s], hcao.FP64)
    o = oracle.Oracle()
    o.add_species(s)
    Ec = o.zpe(0) + 12 * EV
    a, _ = g32.sample_lb(0, Ec, 5, 200000)
    b, _ = g64.sample_lb(0, Ec, 6, 200000)
    for j in range(9):
        ma, mb = a[:, j].mean(), b[:, j].mean()
        se = np.sqrt(a[:, j].var() / len(a) + b[:, j].var() / len(b))
        assert abs(ma - mb) < 5 * se + 1e-9, (j, ma, mb)
