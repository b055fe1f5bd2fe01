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


# ------------------------------------------------------------- high energies
@pytest.mark.parametrize("dE_eV", [5.0, 10.0, 20.0])
def test_fp32_sampler_triatomic_high_energy(dE_eV):
    """The FP32 alias sampler against the enumerated LB target at collision
    energies far above the ZPE (the hot workloads reach several eV): the
    joint table of the two stretches and the bend's marginal (chi^2)."""
    from test_oracle_chemistry_pins import _chisq_p
    s = W.triatomic()
    g = _ctx([s], hcao.FP32)
    levels = [np.array([g.level_energy(0, j, i) for i in range(g.n_levels(0, j))]) for j in range(3)]
    Ec = sum(l[0] for l in levels) + dE_eV * EV
    keys, p = _lb_target(levels, Ec, 0.75)
    ks = np.array(keys)
    n = 400000
    smp, _ = g.sample_lb(0, Ec, 31 + int(dE_eV), n)
    joint_t = np.zeros((17, 17))
    np.add.at(joint_t, (ks[:, 0], ks[:, 1]), p)
    joint_s = np.zeros((17, 17))
    np.add.at(joint_s, (smp[:, 0].astype(int), smp[:, 1].astype(int)), 1)
    assert _chisq_p(joint_s.ravel(), joint_t.ravel() * n) > 1e-4
    nb = int(ks[:, 2].max()) + 1
    bend_t = np.bincount(ks[:, 2], weights=p, minlength=nb) * n
    bend_s = np.bincount(smp[:, 2].astype(int), minlength=nb)[:nb]
    assert _chisq_p(bend_s, bend_t) > 1e-4


@pytest.mark.parametrize("dE_eV", [3.0, 6.0, 10.0])
def test_fp32_sampler_ch4_marginals_high_energy(dE_eV):
    """Nine-mode CH4-like molecule at the heat bath's collision energies: every
    mode's marginal of the FP32 alias sampler against the target's marginal
    from a binned convolution (chi^2)."""
    from test_oracle_chemistry_pins import _chisq_p, _marginals_by_convolution
    s = W.ch4_like()
    g = _ctx([s], hcao.FP32)
    levels = [np.array([g.level_energy(0, j, i) for i in range(g.n_levels(0, j))]) for j in range(9)]
    Ec = sum(l[0] for l in levels) + dE_eV * EV
    marg = _marginals_by_convolution(levels, Ec, 0.75, 2e-4 * EV)
    n = 400000
    smp, _ = g.sample_lb(0, Ec, 71 + int(dE_eV), n)
    for k in range(9):
        ex = marg[k] * n
        ob = np.bincount(smp[:, k].astype(int), minlength=len(ex))[: len(ex)]
        assert _chisq_p(ob, ex) > 1e-4, k
