"""Rotation and rotation-vibration coupling (Sec. "Rotation coupling") on the
GPU against the oracle.

FP64 mode: bit-exact with the oracle -- the initial rotational energies, the
classical LB rotational relaxation after the vibrational draws, gamma E_rot
in the QK collision energies, rotation pooled by dissociation, exchange and
recombination (products start without rotation).  FP32 mode: energy with
rotation conserved per step, equipartition (T_rot -> T_tr), and the
relaxation of T_rot within 3.5 sigma of the oracle's on independent seeds.
"""
import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W
from test_gpu_recomb import _assert_same

pytestmark = pytest.mark.gpu
KB = 1.380649e-23


def _rotating(w, dof=3, T_rot=None):
    for s in w.species:
        if s.n_modes > 0:
            s.rot_dof = dof if s.n_modes > 1 else 2
    if T_rot is not None:
        w.T_rot0 = T_rot
    return w


def _same_rot(g, o):
    _assert_same(g, o)
    assert np.array_equal(g.read_erot(0), o.read_erot(0))


def test_init_rotation_matches_oracle():
    w = _rotating(W.relaxation_triatomic(n_particles=5000, n_cells=3), T_rot=4000.0)
    g = hcao.from_workload(w, precision=hcao.FP64)
    o = oracle.from_workload(w)
    eg, eo = g.read_erot(0), o.read_erot(0)
    assert np.array_equal(eg, eo)
    assert abs(eg.mean() / (1.5 * KB * 4000.0) - 1) < 0.05
    f = hcao.from_workload(w, precision=hcao.FP32)
    assert np.array_equal(f.read_erot(0), eo.astype(np.float32).astype(np.float64))
    # load / read round trip
    e = np.linspace(0.0, 1e-19, w.n)
    g.load_erot(0, e)
    back = g.read_erot(0)
    _, _, s, _ = g.read_particles(0)
    assert np.array_equal(back, e)


CASES = {
    "triatomic_relaxation": lambda: _rotating(W.relaxation_triatomic(n_particles=4000, n_cells=4), T_rot=300.0),
    "ch4_dissociation_gamma": lambda: _gamma(_rotating(W.ch4_heat_bath(n_cells=10, per_cell=300)), 0.5),
    "ch4_h_exchange_gamma": lambda: _gamma(_rotating(W.ch4_h_exchange(n_cells=8, per_cell=500, T0=5000.0)), 1.0),
    "ch4_recombination": lambda: _wr(_rotating(W.ch4_recombination(n_cells=5, per_cell=800, T0=3000.0,
                                                                     n_density=1e26))),
    # rotation pooled into the products' energy under the collision-temperature split
    "ch4_dissociation_gamma_tcoll": lambda: _tc(_gamma(_rotating(W.ch4_heat_bath(n_cells=10, per_cell=300)), 0.5)),
    "ch4_recombination_tcoll": lambda: _tc(_rotating(W.ch4_recombination(n_cells=5, per_cell=800, T0=3000.0,
                                                                         n_density=1e26))),
}


def _tc(w):
    for r in w.reactions:
        r.product_split = "collision_temperature"
    return w


def _gamma(w, g):
    for r in w.reactions:
        if r.type in ("diss", "exch"):
            r.gamma = g
    return w


def _wr(w):
    for r in w.reactions:
        if r.type == "recomb":
            r.recomb_prob = "wr"
    return w


@pytest.mark.parametrize("name", sorted(CASES))
def test_rotation_parity_fp64(name):
    w = CASES[name]()
    kw = {"max_rounds": 4} if name.startswith("ch4_recombination") else {}
    g = hcao.from_workload(w, precision=hcao.FP64, log=True, **kw)
    o = oracle.from_workload(w, log=True)
    for _ in range(5):
        g.step(1)
        o.step(1)
        _same_rot(g, o)
    m = g.read_moments(0)
    assert sum(m.E_rot[i] for i in range(16)) > 0.0
    if name != "triatomic_relaxation":
        assert int(sum(g.read_counters(0)[8:])) > 0


def _total(g, w):
    m = g.read_moments(0)
    return m.E_tr + sum(m.E_vib[i] for i in range(16)) + m.E_form + sum(m.E_rot[i] for i in range(16)), m


def test_rotation_fp32_conservation_and_equipartition():
    w = _rotating(W.relaxation_triatomic(n_particles=20000, n_cells=10), T_rot=300.0)
    g = hcao.from_workload(w, precision=hcao.FP32)
    E0, m0 = _total(g, w)
    assert m0.T_rot[0] < 400.0
    prev = E0
    for _ in range(10):
        g.step(20)
        E, m = _total(g, w)
        assert abs(E - prev) <= 2e-5 * abs(prev)
        prev = E
    assert abs(m.T_rot[0] / m.T_tr - 1.0) < 0.03, (m.T_rot[0], m.T_tr)


def test_rotation_fp32_relaxation_matches_oracle():
    seeds, marks = 10, [1, 2, 4, 8]
    cur = {"gpu": [], "oracle": []}
    for i in range(seeds):
        for side in ("gpu", "oracle"):
            w = _rotating(W.relaxation_triatomic(n_particles=3000, seed=0x7E2B0000 + 2 * i + (side == "gpu")),
                          T_rot=300.0)
            c, done = [], 0
            if side == "gpu":
                g = hcao.from_workload(w, precision=hcao.FP32)
                for m in marks:
                    g.step(m - done)
                    done = m
                    c.append(g.read_moments(0).T_rot[0])
                g.close()
            else:
                o = oracle.from_workload(w)
                for m in marks:
                    o.step(m - done)
                    done = m
                    c.append(o.read_erot(0).mean() / (1.5 * KB))
                o.close()
            cur[side].append(c)
    cg, co = np.array(cur["gpu"]), np.array(cur["oracle"])
    se = np.sqrt(cg.var(0, ddof=1) / seeds + co.var(0, ddof=1) / seeds)
    assert np.all(np.abs(cg.mean(0) - co.mean(0)) < 3.5 * se), (cg.mean(0), co.mean(0), se)
    assert co.mean(0)[-1] > 1000.0 and cg.mean(0)[-1] > 1000.0  # warming from 300 K
