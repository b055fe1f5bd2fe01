"""ctypes binding of the oracle (TEST INFRASTRUCTURE).

Only tests/, __graft_entry__.smoke() and bench.py's cpu-baseline leg may import
this package.  The CUDA library never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hcao_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAXM = 16


def build(force: bool = False) -> str:
    """Compile the oracle: -O2, no FMA contraction, IEEE doubles."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hcao_oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-Wall", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class _Species(C.Structure):
    _fields_ = [("mass", C.c_double), ("d_ref", C.c_double), ("T_ref", C.c_double),
                ("omega", C.c_double), ("E_form", C.c_double), ("n_stretch", C.c_int),
                ("we", C.c_double * MAXM), ("wexe", C.c_double * MAXM), ("De", C.c_double * MAXM),
                ("n_bend", C.c_int), ("theta", C.c_double * MAXM), ("rot_dof", C.c_int)]


class _Reaction(C.Structure):
    _fields_ = [("type", C.c_int), ("reactants", C.c_int * 2), ("products", C.c_int * 2),
                ("diss_mode_mask", C.c_uint32), ("Ea", C.c_double), ("steric", C.c_double),
                ("alpha_mode", C.c_int), ("alpha", C.c_double * MAXM), ("model", C.c_int),
                ("arrhenius", C.c_double * 3), ("tce_zeta", C.c_double), ("wr_samples", C.c_int),
                ("gamma", C.c_double), ("prod_split", C.c_int)]


def reaction_model_code(r) -> int:
    """The C model field of a workload reaction: TCE or QK; WR or exact P."""
    if r.type == "recomb":
        return 1 if getattr(r, "recomb_prob", "exact") == "wr" else 0
    return 1 if getattr(r, "model", "qk") == "tce" else 0


class LogRec(C.Structure):
    _fields_ = [("step", C.c_uint32), ("cell", C.c_uint32), ("round_k", C.c_uint32),
                ("p", C.c_uint32), ("q", C.c_uint32), ("event", C.c_int32), ("aux", C.c_uint32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.ora_create.restype = C.c_void_p
        L.ora_create.argtypes = [C.c_int, C.c_double, C.c_uint32]
        L.ora_destroy.argtypes = [C.c_void_p]
        L.ora_add_species.argtypes = [C.c_void_p, C.POINTER(_Species)]
        L.ora_add_reaction.argtypes = [C.c_void_p, C.POINTER(_Reaction)]
        L.ora_add_reservoir.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double,
                                        C.c_uint64, C.c_double]
        L.ora_load.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p]
        L.ora_init_vibration.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.ora_set_cell_base.argtypes = [C.c_void_p, C.c_int, C.c_uint32]
        L.ora_init_rotation.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.ora_load_erot.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.ora_read_erot.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.ora_ln.restype = C.c_double
        L.ora_ln.argtypes = [C.c_double]
        L.ora_exp.restype = C.c_double
        L.ora_exp.argtypes = [C.c_double]
        L.ora_sample_rot_fraction.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_int64, C.c_void_p]
        L.ora_step.argtypes = [C.c_void_p, C.c_int]
        L.ora_set_log.argtypes = [C.c_void_p, C.c_int]
        L.ora_log_count.restype = C.c_int64
        L.ora_log_count.argtypes = [C.c_void_p]
        L.ora_read_log.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        L.ora_count.restype = C.c_int64
        L.ora_count.argtypes = [C.c_void_p, C.c_int]
        L.ora_read_particles.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p]
        L.ora_read_cell_sgmax.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.ora_read_counters.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int]
        L.ora_n_levels.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.ora_level_energy.restype = C.c_double
        L.ora_level_energy.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
        L.ora_table_value.restype = C.c_double
        L.ora_table_value.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
        L.ora_table_entries.argtypes = [C.c_void_p, C.c_int]
        L.ora_zpe.restype = C.c_double
        L.ora_zpe.argtypes = [C.c_void_p, C.c_int]
        L.ora_sample_lb.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_int64, C.c_int,
                                    C.c_void_p, C.POINTER(C.c_uint64)]
        L.ora_sample_init.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_int64,
                                      C.c_void_p]
        L.ora_wr_density.restype = C.c_double
        L.ora_wr_density.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.ora_diss_prob_wr.restype = C.c_double
        L.ora_diss_prob_wr.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int]
        L.ora_sample_products.restype = C.c_int64
        L.ora_sample_products.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                          C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_uint64, C.c_int64, C.c_void_p, C.c_void_p]
        L.ora_pair_perm.restype = C.c_uint32
        L.ora_pair_perm.argtypes = [C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32)]
        L.ora_philox.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.ora_tvib.restype = C.c_double
        L.ora_tvib.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.ora_mean_sigma_g.restype = C.c_double
        L.ora_mean_sigma_g.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double]
        for name, args in (("ora_diss_prob", [C.c_void_p, C.c_int, C.c_double]),
                           ("ora_keq", [C.c_void_p, C.c_int, C.c_double]),
                           ("ora_rec_rate_node", [C.c_void_p, C.c_int, C.c_int, C.c_int]),
                           ("ora_rec_rate", [C.c_void_p, C.c_int, C.c_int, C.c_double]),
                           ("ora_cell_temperature", [C.c_void_p, C.c_int, C.c_int]),
                           ("ora_rec_node_T", [C.c_int]),
                           ("ora_gamma_q", [C.c_double, C.c_double]),
                           ("ora_tce_prob", [C.c_void_p, C.c_int, C.c_int, C.c_double])):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = args
        L.ora_last_error.restype = C.c_char_p
        L.ora_last_error.argtypes = [C.c_void_p]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox(ctr: Sequence[int], key: Sequence[int]) -> List[int]:
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().ora_philox(c, k, o)
    return list(o)


def pair_perm(x: int, N: int, key: Sequence[int]) -> int:
    """The keyed pairing permutation of [0, N)."""
    k = (C.c_uint32 * 4)(*key)
    return int(lib().ora_pair_perm(x, N, k))


class Oracle:
    """One oracle context: species, reactions, reservoirs."""

    def __init__(self, table_points: int = 2048, table_span_J: float = 64 * 1.602176634e-19,
                 reject_cap: int = 1 << 20):
        self.L = lib()
        self.ctx = self.L.ora_create(table_points, table_span_J, reject_cap)
        self.n_reactions = 0

    def close(self):
        if self.ctx:
            self.L.ora_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, r, what):
        if r < 0:
            raise RuntimeError(f"oracle {what} failed ({r}): {self.L.ora_last_error(self.ctx)}")
        return r

    def add_species(self, s) -> int:
        d = _Species()
        d.mass, d.d_ref, d.T_ref, d.omega, d.E_form = s.mass, s.d_ref, s.T_ref, s.omega, s.E_form
        d.n_stretch = len(s.we)
        for j in range(len(s.we)):
            d.we[j], d.wexe[j], d.De[j] = s.we[j], s.wexe[j], s.De[j]
        d.n_bend = len(s.theta)
        for j, t in enumerate(s.theta):
            d.theta[j] = t
        d.rot_dof = getattr(s, "rot_dof", 0)
        return self._chk(self.L.ora_add_species(self.ctx, C.byref(d)), "add_species")

    def add_reaction(self, r) -> int:
        d = _Reaction()
        d.type = {"diss": 1, "exch": 2, "recomb": 3}[r.type]
        rc = list(r.reactants) + [-1] * (2 - len(r.reactants))
        d.reactants[0], d.reactants[1] = rc[0], rc[1]
        d.products[0], d.products[1] = r.products[0], r.products[1]
        d.diss_mode_mask = r.diss_mode_mask
        d.Ea, d.steric = r.Ea, r.steric
        d.alpha_mode = 1 if r.alpha_mode == "one_random_stretch" else 0
        for j, a in enumerate(r.alpha):
            d.alpha[j] = a
        d.model = reaction_model_code(r)
        for j, a in enumerate(getattr(r, "arrhenius", None) or []):
            d.arrhenius[j] = a
        d.tce_zeta = getattr(r, "tce_zeta", 0.0)
        d.wr_samples = getattr(r, "wr_samples", 1000)
        d.gamma = getattr(r, "gamma", 0.0)
        d.prod_split = 1 if getattr(r, "product_split", "relaxation") == "collision_temperature" else 0
        self.n_reactions += 1
        return self._chk(self.L.ora_add_reaction(self.ctx, C.byref(d)), "add_reaction")

    def add_reservoir(self, n_cells, cell_volume, weight, dt, seed, T_sgmax) -> int:
        return self._chk(self.L.ora_add_reservoir(self.ctx, n_cells, cell_volume, weight, dt,
                                                  seed, T_sgmax), "add_reservoir")

    def load(self, res, v, qn, species, cell):
        v = np.ascontiguousarray(v, dtype=np.float64)
        qn = np.ascontiguousarray(qn, dtype=np.uint8)
        species = np.ascontiguousarray(species, dtype=np.int32)
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        self._chk(self.L.ora_load(self.ctx, res, v.shape[0], _p(v), _p(qn), _p(species), _p(cell)),
                  "load")

    def init_rotation(self, res, T_rot):
        self._chk(self.L.ora_init_rotation(self.ctx, res, T_rot), "init_rotation")

    def load_erot(self, res, erot):
        e = np.ascontiguousarray(erot, np.float64)
        self._chk(self.L.ora_load_erot(self.ctx, res, _p(e)), "load_erot")

    def read_erot(self, res) -> np.ndarray:
        out = np.zeros(self.count(res))
        self._chk(self.L.ora_read_erot(self.ctx, res, _p(out)), "read_erot")
        return out

    def sample_rot_fraction(self, sp, seed, n) -> np.ndarray:
        out = np.zeros(n)
        self._chk(self.L.ora_sample_rot_fraction(self.ctx, sp, seed, n, _p(out)), "sample_rot_fraction")
        return out

    def set_cell_base(self, res, base):
        self._chk(self.L.ora_set_cell_base(self.ctx, res, base), "set_cell_base")

    def init_vibration(self, res, T_vib):
        self._chk(self.L.ora_init_vibration(self.ctx, res, T_vib), "init_vibration")

    def step(self, n=1):
        self._chk(self.L.ora_step(self.ctx, n), "step")

    def set_log(self, on=True):
        self.L.ora_set_log(self.ctx, 1 if on else 0)

    def read_log(self) -> np.ndarray:
        n = self.L.ora_log_count(self.ctx)
        buf = (LogRec * max(n, 1))()
        self.L.ora_read_log(self.ctx, buf, n)
        a = np.frombuffer(buf, dtype=np.dtype([("step", "u4"), ("cell", "u4"), ("round_k", "u4"),
                                               ("p", "u4"), ("q", "u4"), ("event", "i4"),
                                               ("aux", "u4")]), count=n)
        return a.copy()

    def count(self, res) -> int:
        return int(self.L.ora_count(self.ctx, res))

    def read_particles(self, res):
        n = self.count(res)
        v = np.zeros((n, 3)); qn = np.zeros((n, 16), np.uint8)
        sp = np.zeros(n, np.int32); cell = np.zeros(n, np.int32)
        self.L.ora_read_particles(self.ctx, res, _p(v), _p(qn), _p(sp), _p(cell))
        return v, qn, sp, cell

    def read_cell_sgmax(self, res, n_cells) -> np.ndarray:
        out = np.zeros(n_cells)
        self.L.ora_read_cell_sgmax(self.ctx, res, _p(out))
        return out

    def read_counters(self, res) -> np.ndarray:
        out = np.zeros(8 + 32, np.uint64)
        n = self.L.ora_read_counters(self.ctx, res, _p(out), 40)
        return out[:n].copy()

    def n_levels(self, sp, mode) -> int:
        return int(self.L.ora_n_levels(self.ctx, sp, mode))

    def levels(self, sp, mode) -> np.ndarray:
        return np.array([self.L.ora_level_energy(self.ctx, sp, mode, i)
                         for i in range(self.n_levels(sp, mode))])

    def table(self, sp, k) -> np.ndarray:
        n = self.L.ora_table_entries(self.ctx, sp)
        return np.array([self.L.ora_table_value(self.ctx, sp, k, m) for m in range(n)])

    def zpe(self, sp) -> float:
        return float(self.L.ora_zpe(self.ctx, sp))

    def sample_lb(self, sp, Ec, seed, n, method="table"):
        out = np.zeros((n, 16), np.uint8)
        tr = C.c_uint64(0)
        self._chk(self.L.ora_sample_lb(self.ctx, sp, Ec, seed, n, 1 if method == "literal" else 0,
                                       _p(out), C.byref(tr)), "sample_lb")
        return out, int(tr.value)

    def diss_prob_wr(self, rx, T, n_samp=1000) -> float:
        return float(self.L.ora_diss_prob_wr(self.ctx, rx, T, n_samp))

    def sample_products(self, rx, reactants, seed, n):
        """n independent executions of reaction rx on one fixed set of
        reactants, a list of (species, velocity, levels): dissociation [A, M],
        exchange [A, B], recombination [B, C, M].  Returns (v, q) of the
        executed events: v (k, 3, 3) and q (k, 2, 16) as ora_sample_products
        lays them out."""
        args = []
        for j in range(3):
            if j < len(reactants):
                sp, vv, qq = reactants[j]
                vv = np.ascontiguousarray(vv, np.float64)
                qq = np.ascontiguousarray(np.resize(np.asarray(qq, np.uint8), 16))
            else:
                sp, vv, qq = -1, np.zeros(3), np.zeros(16, np.uint8)
            args += [sp, vv, qq]
        keep = args  # the arrays must outlive the call
        ov = np.zeros((n, 3, 3), np.float64)
        oq = np.zeros((n, 2, 16), np.uint8)
        k = int(self.L.ora_sample_products(self.ctx, rx, keep[0], _p(keep[1]), _p(keep[2]), keep[3], _p(keep[4]),
                                           _p(keep[5]), keep[6], _p(keep[7]), _p(keep[8]), seed, n,
                                           _p(ov), _p(oq)))
        self._chk(min(k, 0), "sample_products")
        return ov[:k], oq[:k]

    def sample_init(self, sp, T, seed, n):
        out = np.zeros((n, 16), np.uint8)
        self._chk(self.L.ora_sample_init(self.ctx, sp, T, seed, n, _p(out)), "sample_init")
        return out

    def tvib(self, res, sp) -> float:
        return float(self.L.ora_tvib(self.ctx, res, sp))

    def mean_sigma_g(self, a, b, T) -> float:
        return float(self.L.ora_mean_sigma_g(self.ctx, a, b, T))

    # -- recombination (reading A14)
    def diss_prob(self, rx, T) -> float:
        """Thermal dissociation probability per collision of recombination rx's molecule."""
        return float(self.L.ora_diss_prob(self.ctx, rx, T))

    def keq(self, rx, T) -> float:
        """Equilibrium constant n_B n_C / n_A (m^-3) of recombination rx."""
        return float(self.L.ora_keq(self.ctx, rx, T))

    def rec_rate(self, rx, spM, T) -> float:
        """Tabulated k_r (m^6/s), interpolated at T."""
        return float(self.L.ora_rec_rate(self.ctx, rx, spM, T))

    def rec_rate_node(self, rx, spM, i) -> float:
        return float(self.L.ora_rec_rate_node(self.ctx, rx, spM, i))

    def tce_prob(self, rx, m, Ec) -> float:
        """TCE reaction probability of reaction rx with a partner of species m at collision energy Ec."""
        return float(self.L.ora_tce_prob(self.ctx, rx, m, Ec))

    def cell_temperature(self, res, cell) -> float:
        return float(self.L.ora_cell_temperature(self.ctx, res, cell))


REC_NODES = 225


def rec_node_T(i: int) -> float:
    return float(lib().ora_rec_node_T(i))


def wr_density(hnu, E: float) -> float:
    """Whitten-Rabinovitch density of states (1/J) of oscillators with quanta
    hnu (J) at energy E (J) above the ground state."""
    h = np.ascontiguousarray(hnu, np.float64)
    return float(lib().ora_wr_density(_p(h), len(h), E))


def ln(x: float) -> float:
    """The oracle's own natural logarithm (rotation draws)."""
    return float(lib().ora_ln(x))


def exp(x: float) -> float:
    """The oracle's own exponential (used where the device must reproduce it)."""
    return float(lib().ora_exp(x))


def gamma_q(a: float, x: float) -> float:
    return float(lib().ora_gamma_q(a, x))


def from_workload(w, table_points=2048, table_span_J=64 * 1.602176634e-19, log=False,
                  init_vib=True) -> Oracle:
    """Oracle set up with a workload's species, reactions and initial state."""
    o = Oracle(table_points, table_span_J)
    for s in w.species:
        o.add_species(s)
    for r in w.reactions:
        o.add_reaction(r)
    res = o.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
    if getattr(w, "cell_base", 0):
        o.set_cell_base(res, w.cell_base)
    o.load(res, w.v, w.qn0(), w.species_idx, w.cell)
    if init_vib:
        o.init_vibration(res, w.T_vib0)
        if any(getattr(s, "rot_dof", 0) for s in w.species):
            o.init_rotation(res, getattr(w, "T_rot0", w.T_tr0))
    o.set_log(log)
    return o


def from_batched(bw, table_points=2048, table_span_J=64 * 1.602176634e-19, log=False,
                 only=None) -> Oracle:
    """Oracle holding the reservoirs of a batched workload (all, or the indices in `only`)."""
    o = Oracle(table_points, table_span_J)
    for s in bw.species:
        o.add_species(s)
    for r in bw.reactions:
        o.add_reaction(r)
    for i, w in enumerate(bw.reservoirs):
        if only is not None and i not in only:
            continue
        res = o.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
        o.load(res, w.v, w.qn0(), w.species_idx, w.cell)
        o.init_vibration(res, w.T_vib0)
    o.set_log(log)
    return o
