"""The paper's verification cases (Sec. "Verification") as presets on the GPU.

FP64 mode: each case with its QK and its TCE reactions equals the oracle bit
for bit over a few steps (small samples).  FP32 mode at the presets' sizes:
hydrogen cyanide at 5000 K forms CN and no HC (the paper's qualitative
result), and every case conserves energy to 1e-6 per step while it reacts.
"""
import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W
from test_gpu_recomb import _assert_same

pytestmark = pytest.mark.gpu


def _wr(w):
    for r in w.reactions:
        if r.type == "recomb":
            r.recomb_prob = "wr"
    return w


SMALL = {
    "water": lambda m: W.paper_water(m, n_per_species=3000, n_cells=4),
    "hcn_12000K": lambda m: W.paper_hcn(12000.0, m, n_per_species=3000, n_cells=4),
    "methane_exchange": lambda m: W.paper_methane_exchange(m, n_per_species=1500, n_cells=4),
    "methane_dissociation": lambda m: _wr(W.paper_methane_dissociation(m, n_per_species=2000, n_cells=4)),
}


@pytest.mark.parametrize("model", ["qk", "tce"])
@pytest.mark.parametrize("case", sorted(SMALL))
def test_paper_case_parity_fp64(case, model):
    w = SMALL[case](model)
    kw = {"max_rounds": 4} if case == "methane_dissociation" else {}
    g = hcao.from_workload(w, precision=hcao.FP64, log=True, **kw)
    o = oracle.from_workload(w, log=True)
    for _ in range(4):
        g.step(1)
        o.step(1)
        _assert_same(g, o)
    assert int(g.read_counters(0)[8]) > 0


def _energy(g, w):
    m = g.read_moments(0)
    return m.E_tr + sum(m.E_vib[i] for i in range(16)) + m.E_form, m


def test_paper_hcn_5000K_fp32_no_hc():
    w = W.paper_hcn(5000.0, "qk")
    g = hcao.from_workload(w, precision=hcao.FP32)
    E0, _ = _energy(g, w)
    g.step(300)
    E1, m = _energy(g, w)
    assert abs(E1 - E0) <= 1e-5 * abs(E0)
    c = g.read_counters(0)
    assert c[8] > 0 and c[9] == 0
    assert m.n[3] > 0 and m.n[4] == 0  # CN, no HC


@pytest.mark.parametrize("model", ["qk", "tce"])
@pytest.mark.parametrize("case", ["water", "methane_exchange"])
def test_paper_case_fp32_conserves(case, model):
    w = W.paper_water(model) if case == "water" else W.paper_methane_exchange(model)
    g = hcao.from_workload(w, precision=hcao.FP32)
    prev, _ = _energy(g, w)
    for _ in range(5):
        g.step(20)
        E, m = _energy(g, w)
        assert abs(E - prev) <= 2e-5 * abs(prev)  # 20 steps of at most 1e-6 each
        prev = E
    assert int(g.read_counters(0)[8]) > 0
