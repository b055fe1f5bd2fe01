"""Thin ctypes binding of libhcao (argument marshalling only).

Every step of the collision phase runs in the library's CUDA kernels; this
module only converts numpy arrays and workload presets into the C structs of
include/hcao.h.  It raises if the compiled library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhcao.so")

FP64, FP32 = 0, 1
PATH_AUTO, PATH_QUEUE, PATH_FUSED = 0, 1, 2
SPLIT_RELAX, SPLIT_TCOLL = 0, 1
DISS, EXCH, RECOMB = 1, 2, 3
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EREJECT_LIMIT",
          -5: "ELEVEL_OVERFLOW", -6: "EBUSY", -7: "ECAPACITY", -8: "EROUNDS", -9: "ENOTFOUND",
          -10: "ENONFINITE", -11: "ECANCELLED"}

EXPORTS = [
    "hcao_create", "hcao_destroy", "hcao_last_error", "hcao_default_config", "hcao_set_species",
    "hcao_set_reactions", "hcao_add_reservoir", "hcao_remove_reservoir", "hcao_load_particles",
    "hcao_init_vibration", "hcao_step", "hcao_sync", "hcao_count", "hcao_read_particles",
    "hcao_read_moments", "hcao_read_level_populations", "hcao_read_counters",
    "hcao_read_reaction_counts", "hcao_read_cell_sgmax", "hcao_set_log", "hcao_read_log",
    "hcao_cell_sort", "hcao_level_energy", "hcao_n_levels", "hcao_kernel_launches",
    "hcao_set_profiling", "hcao_read_profile", "hcao_sample_lb", "hcao_cell_sort_noalloc",
    "hcao_read_work", "hcao_autotune", "hcao_serve_start", "hcao_serve_submit", "hcao_serve_poll",
    "hcao_serve_stop", "hcao_serve_stats", "hcao_recomb_rate", "hcao_wr_density", "hcao_wr_diss_prob",
    "hcao_set_step_path", "hcao_get_step_path", "hcao_set_cell_base", "hcao_init_rotation",
    "hcao_load_erot", "hcao_read_erot", "hcao_load_particles_f32", "hcao_serve_timing",
    "hcao_serve_cancel", "hcao_debug_fail_allocs", "hcao_clear_error",
]
REC_NODES = 225
MAX_REMOVALS_PER_CELL = 4096
NOALLOC_SORT_MAX_KEYS = 1 << 19


class HcaoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("precision", C.c_int), ("device", C.c_int), ("cuda_stream", C.c_void_p),
                ("table_points", C.c_int), ("table_span_J", C.c_double), ("reject_cap", C.c_uint32),
                ("max_rounds", C.c_int), ("capacity_factor", C.c_double), ("capacity_extra", C.c_int)]


class _Species(C.Structure):
    _fields_ = [("mass", C.c_double), ("d_ref", C.c_double), ("T_ref", C.c_double),
                ("omega", C.c_double), ("E_form", C.c_double), ("n_stretch", C.c_int),
                ("we", C.POINTER(C.c_double)), ("wexe", C.POINTER(C.c_double)),
                ("De", C.POINTER(C.c_double)), ("n_bend", C.c_int), ("theta", C.POINTER(C.c_double)),
                ("rot_dof", C.c_int)]


class _Reaction(C.Structure):
    _fields_ = [("type", C.c_int), ("reactants", C.c_int * 2), ("products", C.c_int * 2),
                ("diss_mode_mask", C.c_uint32), ("Ea", C.c_double), ("steric", C.c_double),
                ("alpha_mode", C.c_int), ("alpha", C.POINTER(C.c_double)), ("model", C.c_int),
                ("arrhenius", C.c_double * 3), ("tce_zeta", C.c_double), ("wr_samples", C.c_int),
                ("gamma", C.c_double), ("prod_split", C.c_int)]


class LogRec(C.Structure):
    _fields_ = [("step", C.c_uint32), ("cell", C.c_uint32), ("round_k", C.c_uint32),
                ("p", C.c_uint32), ("q", C.c_uint32), ("event", C.c_int32), ("aux", C.c_uint32)]


LOG_DTYPE = np.dtype([("step", "u4"), ("cell", "u4"), ("round_k", "u4"), ("p", "u4"), ("q", "u4"),
                      ("event", "i4"), ("aux", "u4")])


class Moments(C.Structure):
    _fields_ = [("n", C.c_int64 * 16), ("momentum", C.c_double * 3), ("E_tr", C.c_double),
                ("E_vib", C.c_double * 16), ("E_form", C.c_double), ("T_tr", C.c_double),
                ("T_vib", C.c_double * 16), ("E_rot", C.c_double * 16), ("T_rot", C.c_double * 16)]


class Job(C.Structure):
    _fields_ = [("n_cells", C.c_int), ("cell_volume", C.c_double), ("weight", C.c_double),
                ("dt", C.c_double), ("seed", C.c_uint64), ("T_sgmax", C.c_double), ("n", C.c_int64),
                ("v", C.c_void_p), ("qn", C.c_void_p), ("species", C.c_void_p), ("cell", C.c_void_p),
                ("T_vib", C.c_double), ("n_steps", C.c_int)]


class JobResult(C.Structure):
    _fields_ = [("status", C.c_int), ("steps", C.c_int), ("n_particles", C.c_int64),
                ("moments", Moments), ("counters", C.c_uint64 * 16), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double)]


_lib = None


def lib() -> C.CDLL:
    """Load libhcao.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhcao.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl, u64 = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_uint64
        L.hcao_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
        L.hcao_destroy.argtypes = [vp]
        L.hcao_destroy.restype = None
        L.hcao_last_error.argtypes = [vp]
        L.hcao_last_error.restype = C.c_char_p
        L.hcao_default_config.argtypes = [C.POINTER(Config)]
        L.hcao_default_config.restype = None
        L.hcao_set_species.argtypes = [vp, C.POINTER(_Species), i32]
        L.hcao_set_reactions.argtypes = [vp, C.POINTER(_Reaction), i32]
        L.hcao_add_reservoir.argtypes = [vp, i32, dbl, dbl, dbl, u64, dbl, C.POINTER(i32)]
        L.hcao_remove_reservoir.argtypes = [vp, i32]
        L.hcao_load_particles.argtypes = [vp, i32, i64, vp, vp, vp, vp]
        L.hcao_load_particles_f32.argtypes = [vp, i32, i64, vp, vp, vp, vp]
        L.hcao_serve_timing.argtypes = [vp, vp]
        L.hcao_serve_cancel.argtypes = [vp, u64]
        L.hcao_debug_fail_allocs.argtypes = [vp, i32]
        L.hcao_clear_error.argtypes = [vp]
        L.hcao_init_vibration.argtypes = [vp, i32, dbl]
        L.hcao_step.argtypes = [vp, i32]
        L.hcao_sync.argtypes = [vp]
        L.hcao_count.argtypes = [vp, i32, C.POINTER(i64)]
        L.hcao_read_particles.argtypes = [vp, i32, vp, vp, vp, vp]
        L.hcao_read_moments.argtypes = [vp, i32, C.POINTER(Moments)]
        L.hcao_read_level_populations.argtypes = [vp, i32, i32, i32, vp, i32]
        L.hcao_read_counters.argtypes = [vp, i32, vp, i32, C.POINTER(i32)]
        L.hcao_read_reaction_counts.argtypes = [vp, i32, vp, i32]
        L.hcao_read_cell_sgmax.argtypes = [vp, i32, vp]
        L.hcao_set_log.argtypes = [vp, i32]
        L.hcao_wr_density.argtypes = [vp, i32, dbl]
        L.hcao_wr_density.restype = dbl
        L.hcao_wr_diss_prob.argtypes = [vp, i32, dbl, dbl, dbl, i32]
        L.hcao_wr_diss_prob.restype = dbl
        L.hcao_read_log.argtypes = [vp, vp, i64, C.POINTER(i64)]
        L.hcao_cell_sort.argtypes = [vp, vp, i64, C.c_uint32, vp, vp]
        L.hcao_level_energy.argtypes = [vp, i32, i32, i32, C.POINTER(dbl)]
        L.hcao_n_levels.argtypes = [vp, i32, i32, C.POINTER(i32)]
        L.hcao_sample_lb.argtypes = [vp, i32, dbl, u64, i64, vp, C.POINTER(u64)]
        L.hcao_cell_sort_noalloc.argtypes = [vp, i64, C.c_uint32, vp, vp, vp]
        L.hcao_read_work.argtypes = [vp, vp, i32, C.POINTER(i32)]
        L.hcao_autotune.argtypes = [vp, i32, vp]
        L.hcao_set_profiling.argtypes = [vp, i32]
        L.hcao_read_profile.argtypes = [vp, vp, vp, i32, C.POINTER(i32)]
        L.hcao_serve_start.argtypes = [vp, i64, i32, i32]
        L.hcao_serve_submit.argtypes = [vp, C.POINTER(Job), C.POINTER(u64)]
        L.hcao_serve_poll.argtypes = [vp, u64, C.POINTER(JobResult)]
        L.hcao_serve_stop.argtypes = [vp]
        L.hcao_serve_stats.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(u64)]
        L.hcao_recomb_rate.argtypes = [vp, i32, i32, dbl, C.POINTER(dbl)]
        L.hcao_set_step_path.argtypes = [vp, i32]
        L.hcao_set_cell_base.argtypes = [vp, i32, C.c_uint32]
        L.hcao_init_rotation.argtypes = [vp, i32, dbl]
        L.hcao_load_erot.argtypes = [vp, i32, vp]
        L.hcao_read_erot.argtypes = [vp, i32, vp]
        L.hcao_get_step_path.argtypes = [vp, C.POINTER(i32)]
        L.hcao_kernel_launches.argtypes = [vp]
        L.hcao_kernel_launches.restype = u64
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dptr(ptr) -> C.c_void_p:
    """Device pointer from an int or a torch tensor."""
    if hasattr(ptr, "data_ptr"):
        return C.c_void_p(ptr.data_ptr())
    return C.c_void_p(int(ptr))


def wr_density(hnu, E: float) -> float:
    """Whitten-Rabinovitch density of states (1/J) of oscillators with quanta
    hnu (J) at E (J) above the ground state (host computation, no GPU)."""
    h = np.ascontiguousarray(hnu, np.float64)
    return float(lib().hcao_wr_density(h.ctypes.data, len(h), E))


def wr_diss_prob(hnu, Dx: float, omega: float, T: float, n_samp: int = 1000) -> float:
    """The WR form of the dissociation probability (host computation)."""
    h = np.ascontiguousarray(hnu, np.float64)
    return float(lib().hcao_wr_diss_prob(h.ctypes.data, len(h), Dx, omega, T, n_samp))


class Context:
    """One libhcao context on one GPU."""

    def __init__(self, precision: int = FP64, device: int = 0, stream: Optional[int] = None,
                 table_points: int = 2048, table_span_J: float = 64 * 1.602176634e-19,
                 max_rounds: int = 2, capacity_factor: float = 2.0, capacity_extra: int = 64,
                 reject_cap: int = 1 << 20):
        self.L = lib()
        cfg = Config()
        self.L.hcao_default_config(C.byref(cfg))
        cfg.precision, cfg.device = precision, device
        cfg.cuda_stream = stream
        cfg.table_points, cfg.table_span_J = table_points, table_span_J
        cfg.max_rounds, cfg.capacity_factor, cfg.capacity_extra = max_rounds, capacity_factor, capacity_extra
        cfg.reject_cap = reject_cap
        h = C.c_void_p()
        r = self.L.hcao_create(C.byref(cfg), C.byref(h))
        if r != 0:
            raise HcaoError(r, "hcao_create failed")
        self.h = h
        self.precision = precision
        self._keep = []
        self.n_reactions = 0

    def close(self):
        if getattr(self, "h", None):
            self.L.hcao_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, r):
        if r != 0:
            raise HcaoError(r, self.L.hcao_last_error(self.h).decode())
        return r

    # -- setup
    def set_species(self, species: Sequence) -> None:
        arr = (_Species * len(species))()
        keep = []
        for i, s in enumerate(species):
            d = arr[i]
            d.mass, d.d_ref, d.T_ref, d.omega, d.E_form = s.mass, s.d_ref, s.T_ref, s.omega, s.E_form
            d.n_stretch, d.n_bend = len(s.we), len(s.theta)
            d.rot_dof = getattr(s, "rot_dof", 0)
            for name in ("we", "wexe", "De", "theta"):
                vals = list(getattr(s, name))
                buf = (C.c_double * max(1, len(vals)))(*vals)
                keep.append(buf)
                setattr(d, name, C.cast(buf, C.POINTER(C.c_double)))
        self._chk(self.L.hcao_set_species(self.h, arr, len(species)))

    def set_reactions(self, reactions: Sequence) -> None:
        if not reactions:
            return
        arr = (_Reaction * len(reactions))()
        keep = []
        for i, r in enumerate(reactions):
            d = arr[i]
            d.type = {"diss": DISS, "exch": EXCH, "recomb": RECOMB}[r.type]
            rc = list(r.reactants) + [-1] * (2 - len(r.reactants))
            d.reactants[0], d.reactants[1] = rc[0], rc[1]
            d.products[0], d.products[1] = r.products[0], r.products[1]
            d.diss_mode_mask = r.diss_mode_mask
            d.Ea, d.steric = r.Ea, r.steric
            d.alpha_mode = 1 if r.alpha_mode == "one_random_stretch" else 0
            if r.alpha:
                buf = (C.c_double * len(r.alpha))(*r.alpha)
                keep.append(buf)
                d.alpha = C.cast(buf, C.POINTER(C.c_double))
            if r.type == "recomb":
                d.model = 1 if getattr(r, "recomb_prob", "exact") == "wr" else 0
            else:
                d.model = 1 if getattr(r, "model", "qk") == "tce" else 0
            for j, a in enumerate(getattr(r, "arrhenius", None) or []):
                d.arrhenius[j] = a
            d.tce_zeta = getattr(r, "tce_zeta", 0.0)
            d.wr_samples = getattr(r, "wr_samples", 1000)
            d.gamma = getattr(r, "gamma", 0.0)
            split = getattr(r, "product_split", "relaxation")
            d.prod_split = {"relaxation": SPLIT_RELAX, "collision_temperature": SPLIT_TCOLL}[split]
        self._chk(self.L.hcao_set_reactions(self.h, arr, len(reactions)))
        self.n_reactions = len(reactions)

    def add_reservoir(self, n_cells, cell_volume, weight, dt, seed, T_sgmax) -> int:
        rid = C.c_int()
        self._chk(self.L.hcao_add_reservoir(self.h, n_cells, cell_volume, weight, dt, seed, T_sgmax,
                                            C.byref(rid)))
        return rid.value

    def set_cell_base(self, res: int, base: int) -> None:
        """Key reservoir res's cells as cells base, base + 1, ... of a larger workload."""
        self._chk(self.L.hcao_set_cell_base(self.h, res, base))

    def remove_reservoir(self, res: int) -> None:
        self._chk(self.L.hcao_remove_reservoir(self.h, res))

    def load_particles(self, res, v, qn, species, cell) -> None:
        """FP32 velocity arrays go through hcao_load_particles_f32 (half the
        bytes over the host-device link), anything else as FP64."""
        f32 = isinstance(v, np.ndarray) and v.dtype == np.float32
        v = np.ascontiguousarray(v, dtype=np.float32 if f32 else np.float64)
        qn = np.ascontiguousarray(qn, dtype=np.uint8)
        species = np.ascontiguousarray(species, dtype=np.int32)
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        fn = self.L.hcao_load_particles_f32 if f32 else self.L.hcao_load_particles
        self._chk(fn(self.h, res, v.shape[0], _p(v), _p(qn), _p(species), _p(cell)))

    def init_vibration(self, res, T_vib) -> None:
        self._chk(self.L.hcao_init_vibration(self.h, res, T_vib))

    def init_rotation(self, res, T_rot) -> None:
        self._chk(self.L.hcao_init_rotation(self.h, res, T_rot))

    def load_erot(self, res, erot) -> None:
        e = np.ascontiguousarray(erot, dtype=np.float64)
        self._chk(self.L.hcao_load_erot(self.h, res, _p(e)))

    def read_erot(self, res) -> np.ndarray:
        out = np.zeros(max(self.count(res), 1))
        self._chk(self.L.hcao_read_erot(self.h, res, _p(out)))
        return out[: self.count(res)]

    # -- run
    def step(self, n=1) -> None:
        self._chk(self.L.hcao_step(self.h, n))

    def sync(self) -> None:
        self._chk(self.L.hcao_sync(self.h))

    def set_log(self, on=True) -> None:
        self._chk(self.L.hcao_set_log(self.h, 1 if on else 0))

    # -- read
    def count(self, res) -> int:
        n = C.c_int64()
        self._chk(self.L.hcao_count(self.h, res, C.byref(n)))
        return n.value

    def read_particles(self, res):
        n = self.count(res)
        v = np.zeros((n, 3)); qn = np.zeros((n, 16), np.uint8)
        sp = np.zeros(n, np.int32); cell = np.zeros(n, np.int32)
        if n:
            self._chk(self.L.hcao_read_particles(self.h, res, _p(v), _p(qn), _p(sp), _p(cell)))
        return v, qn, sp, cell

    def read_moments(self, res) -> Moments:
        m = Moments()
        self._chk(self.L.hcao_read_moments(self.h, res, C.byref(m)))
        return m

    def read_level_populations(self, res, species, mode, max_levels=256) -> np.ndarray:
        out = np.zeros(max_levels, np.uint64)
        self._chk(self.L.hcao_read_level_populations(self.h, res, species, mode, _p(out), max_levels))
        return out

    def read_counters(self, res) -> np.ndarray:
        out = np.zeros(40, np.uint64)
        n = C.c_int()
        self._chk(self.L.hcao_read_counters(self.h, res, _p(out), 40, C.byref(n)))
        return out[: n.value].copy()

    def read_reaction_counts(self, res, n) -> np.ndarray:
        out = np.zeros(max(n, 1), np.uint64)
        self._chk(self.L.hcao_read_reaction_counts(self.h, res, _p(out), n))
        return out[:n]

    def read_cell_sgmax(self, res, n_cells) -> np.ndarray:
        out = np.zeros(n_cells)
        self._chk(self.L.hcao_read_cell_sgmax(self.h, res, _p(out)))
        return out

    def read_log(self) -> np.ndarray:
        n = C.c_int64()
        self._chk(self.L.hcao_read_log(self.h, None, 0, C.byref(n)))
        buf = np.zeros(max(n.value, 1), dtype=LOG_DTYPE)
        got = C.c_int64()
        self._chk(self.L.hcao_read_log(self.h, _p(buf), buf.shape[0], C.byref(got)))
        return buf[: got.value].copy()

    def cell_sort(self, keys_dev, n, n_cells, perm_dev, offsets_dev) -> None:
        self._chk(self.L.hcao_cell_sort(self.h, _dptr(keys_dev), n, n_cells, _dptr(perm_dev),
                                        _dptr(offsets_dev)))

    def level_energy(self, sp, mode, level) -> float:
        e = C.c_double()
        self._chk(self.L.hcao_level_energy(self.h, sp, mode, level, C.byref(e)))
        return e.value

    def n_levels(self, sp, mode) -> int:
        n = C.c_int()
        self._chk(self.L.hcao_n_levels(self.h, sp, mode, C.byref(n)))
        return n.value

    def sample_lb(self, sp, Ec, seed, n):
        """n post-collision states of species sp at collision energy Ec (device sampler)."""
        out = np.zeros((n, 16), np.uint8)
        tr = C.c_uint64(0)
        self._chk(self.L.hcao_sample_lb(self.h, sp, Ec, seed, n, _p(out), C.byref(tr)))
        return out, int(tr.value)

    def set_profiling(self, on=True) -> None:
        self._chk(self.L.hcao_set_profiling(self.h, 1 if on else 0))

    PROFILE_KERNELS = ("setup", "select", "relax", "react", "finish", "fused")

    def read_profile(self):
        """(ms, launches) per kernel class: setup, select, relax, react, finish
        (the queue path) and the fused per-cell kernel."""
        ms = np.zeros(6)
        n = np.zeros(6, np.uint64)
        got = C.c_int()
        self._chk(self.L.hcao_read_profile(self.h, _p(ms), _p(n), 6, C.byref(got)))
        return ms, n

    def set_step_path(self, path: int) -> None:
        """PATH_AUTO (default), PATH_QUEUE or PATH_FUSED."""
        self._chk(self.L.hcao_set_step_path(self.h, path))

    def step_path(self) -> int:
        """The collision-phase path the next step takes: PATH_QUEUE or PATH_FUSED."""
        p = C.c_int()
        self._chk(self.L.hcao_get_step_path(self.h, C.byref(p)))
        return p.value

    def autotune(self, steps_per_candidate=1):
        """Pick the launch schedule by timing candidates on live steps; returns
        (select grid, relax grid, queue placed by work class: 0 or 1)."""
        out = np.zeros(3, np.int32)
        self._chk(self.L.hcao_autotune(self.h, steps_per_candidate, _p(out)))
        return int(out[0]), int(out[1]), int(out[2])

    def read_work(self) -> np.ndarray:
        """[level evaluations, mode draws, molecule samples, relaxed pairs] (FP32 relax kernel)."""
        out = np.zeros(4, np.uint64)
        n = C.c_int()
        self._chk(self.L.hcao_read_work(self.h, _p(out), 4, C.byref(n)))
        return out

    def kernel_launches(self) -> int:
        return int(self.L.hcao_kernel_launches(self.h))

    def recomb_rate(self, reaction, spM, T) -> float:
        """The tabulated k_r (m^6/s) of a recombination with third-body species spM at T."""
        out = C.c_double()
        self._chk(self.L.hcao_recomb_rate(self.h, reaction, spM, T, C.byref(out)))
        return out.value

    # -- serving (continuous batching of reservoir jobs)
    def serve_start(self, hbm_budget_bytes=0, max_active=0, max_batch_steps=0) -> None:
        self._chk(self.L.hcao_serve_start(self.h, int(hbm_budget_bytes), max_active, max_batch_steps))

    def serve_submit(self, w, n_steps, T_vib=None) -> int:
        """Queue a reservoir job built from a workload; returns its id.  The
        host arrays are copied by the library before this returns."""
        v = np.ascontiguousarray(w.v, dtype=np.float64)
        qn = np.ascontiguousarray(w.qn0(), dtype=np.uint8)
        sp = np.ascontiguousarray(w.species_idx, dtype=np.int32)
        cell = np.ascontiguousarray(w.cell, dtype=np.int32)
        j = Job(n_cells=w.n_cells, cell_volume=w.cell_volume, weight=w.weight, dt=w.dt, seed=w.seed,
                T_sgmax=w.T_tr0, n=v.shape[0], v=_p(v), qn=_p(qn), species=_p(sp), cell=_p(cell),
                T_vib=w.T_vib0 if T_vib is None else T_vib, n_steps=n_steps)
        jid = C.c_uint64()
        self._chk(self.L.hcao_serve_submit(self.h, C.byref(j), C.byref(jid)))
        return jid.value

    def serve_poll(self, job_id):
        """None while the job is queued or running, else its JobResult
        (raises on a failed job)."""
        r = JobResult()
        st = self.L.hcao_serve_poll(self.h, job_id, C.byref(r))
        if st == -6:
            return None
        if st != 0:
            raise HcaoError(st, f"serving job {job_id} failed")
        return r

    def serve_stop(self) -> None:
        self._chk(self.L.hcao_serve_stop(self.h))

    def serve_stats(self):
        """(queued, resident, budgeted bytes in use, engine iterations)."""
        q, a, b, it = C.c_int64(), C.c_int64(), C.c_int64(), C.c_uint64()
        self._chk(self.L.hcao_serve_stats(self.h, C.byref(q), C.byref(a), C.byref(b), C.byref(it)))
        return q.value, a.value, b.value, it.value

    def serve_cancel(self, job_id) -> None:
        self._chk(self.L.hcao_serve_cancel(self.h, job_id))

    def clear_error(self) -> None:
        """Clear the sticky device error word (see hcao_clear_error)."""
        self._chk(self.L.hcao_clear_error(self.h))

    def debug_fail_allocs(self, n) -> None:
        """Test fault injection: the next n device allocations fail as out of memory."""
        self._chk(self.L.hcao_debug_fail_allocs(self.h, n))

    def serve_timing(self) -> dict:
        """The engine thread's seconds by activity since serve_start."""
        t = np.zeros(4)
        self._chk(self.L.hcao_serve_timing(self.h, _p(t)))
        return {"admit_s": float(t[0]), "step_s": float(t[1]), "retire_s": float(t[2]), "wait_s": float(t[3])}


def from_batched(bw, precision=FP64, init_vib=True, **kw) -> Context:
    """A context holding every reservoir of a batched workload (reservoir i = id i)."""
    c = Context(precision=precision, **kw)
    c.set_species(bw.species)
    c.set_reactions(bw.reactions)
    for w in bw.reservoirs:
        rid = c.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
        c.load_particles(rid, w.v, w.qn0(), w.species_idx, w.cell)
        if init_vib:
            c.init_vibration(rid, w.T_vib0)
    return c


def cell_sort_noalloc(keys_dev, n, n_cells, perm_dev, offsets_dev, stream=None) -> None:
    """hcao_cell_sort_noalloc: the stable cell sort without any device
    allocation (scratch in a fixed device array, n <= NOALLOC_SORT_MAX_KEYS)."""
    r = lib().hcao_cell_sort_noalloc(_dptr(keys_dev), n, n_cells, _dptr(perm_dev), _dptr(offsets_dev),
                                     None if stream is None else C.c_void_p(int(stream)))
    if r != 0:
        raise HcaoError(r, "hcao_cell_sort_noalloc failed")


def from_workload(w, precision=FP64, log=False, init_vib=True, **kw) -> Context:
    """A context loaded with a workload's species, reactions and initial state."""
    c = Context(precision=precision, **kw)
    c.set_species(w.species)
    c.set_reactions(w.reactions)
    rid = c.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
    if getattr(w, "cell_base", 0):
        c.set_cell_base(rid, w.cell_base)
    c.load_particles(rid, w.v, w.qn0(), w.species_idx, w.cell)
    if init_vib:
        c.init_vibration(rid, w.T_vib0)
        if any(getattr(s, "rot_dof", 0) for s in w.species):
            c.init_rotation(rid, getattr(w, "T_rot0", w.T_tr0))
    if log:
        c.set_log(True)
    return c
