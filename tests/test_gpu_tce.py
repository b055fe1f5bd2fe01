"""The TCE reaction model (the paper's comparison model, Eq. arrhenius) on
the GPU against the oracle.

FP64 mode: bit-exact with the oracle -- TCE dissociation (created particles),
TCE exchange, and TCE beside QK channels (TCE reactions are tested first).
FP32 mode: the TCE dissociation probability per collision within 3 sigma of
the oracle's on independent seeds.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W
from test_gpu_recomb import _assert_same

pytestmark = pytest.mark.gpu
KB = 1.380649e-23


def _diss(A=2e-16, zeta=0.0):
    return W.Reaction("diss", [0], [1, 2], diss_mode_mask=0xF, model="tce", arrhenius=[A, 0.0, 51488.0 * KB],
                      tce_zeta=zeta)


@pytest.mark.parametrize("A,zeta", [(2e-16, 0.0), (5.26e-12, 0.0), (5.26e-14, 2.0)])
def test_parity_tce_dissociation_fp64(A, zeta):
    w = W.ch4_heat_bath(n_cells=12, per_cell=400, T0=15000.0)
    w.reactions = [_diss(A, zeta)]
    g = hcao.from_workload(w, precision=hcao.FP64, log=True)
    o = oracle.from_workload(w, log=True)
    for _ in range(5):
        g.step(1)
        o.step(1)
        _assert_same(g, o)
    assert g.read_reaction_counts(0, 1)[0] > 20
    assert np.array_equal(g.read_counters(0), o.read_counters(0)[: len(g.read_counters(0))])


def test_parity_tce_exchange_beside_qk_dissociation_fp64():
    """TCE exchange (the paper's CH4 + H parameters) with a QK dissociation
    in the same mixture: TCE is tested first, the QK channels after."""
    w = W.ch4_h_exchange(n_cells=10, per_cell=600, T0=6000.0)
    w.reactions = [W.Reaction("exch", [0, 1], [2, 3], model="tce", arrhenius=[1.03e-24, 2.5, 4825.0 * KB]),
                   W.Reaction("diss", [0], [2, 1], diss_mode_mask=0xF)]
    g = hcao.from_workload(w, precision=hcao.FP64, log=True)
    o = oracle.from_workload(w, log=True)
    for _ in range(5):
        g.step(1)
        o.step(1)
        _assert_same(g, o)
    c = g.read_reaction_counts(0, 2)
    assert c[0] > 50


def test_fp32_tce_dissociation_rate_matches_oracle():
    steps = 1
    wo = W.ch4_heat_bath(n_cells=300, per_cell=500, T0=20000.0)
    wg = W.ch4_heat_bath(n_cells=300, per_cell=500, T0=20000.0, seed=wo.seed + 7)
    wo.reactions = [_diss()]
    wg.reactions = [_diss()]
    o = oracle.from_workload(wo)
    o.step(steps)
    g = hcao.from_workload(wg, precision=hcao.FP32)
    g.step(steps)
    co, cg = o.read_counters(0), g.read_counters(0)
    ko, kg, no, ng = int(co[8]), int(cg[8]), int(co[1]), int(cg[1])
    assert ko > 100 and kg > 100
    p = (ko + kg) / (no + ng)
    se = math.sqrt(p * (1 - p) * (1 / no + 1 / ng))
    assert abs(kg / ng - ko / no) < 3 * se, (kg / ng, ko / no, se)


def test_tce_rejects_divergent_parameters():
    w = W.ch4_heat_bath(n_cells=2, per_cell=10)
    g = hcao.Context(precision=hcao.FP64)
    g.set_species(w.species)
    bad = W.Reaction("diss", [0], [1, 2], diss_mode_mask=0xF, model="tce", arrhenius=[1e-3, -2.6, 1e-19])
    with pytest.raises(hcao.HcaoError):
        g.set_reactions([bad])
