"""Seeded synthetic workloads: species presets and initial particle arrays.

This module holds input data only -- species parameters, reservoir sizes and
seeded generators of initial velocities, species and cell assignments.  It does
none of the method's arithmetic (no level energies, no sampling of quantum
numbers, no collision physics) and serves both the CUDA library and the
oracle.  Unit conversions (cm^-1, eV, u) are the only computations.

Species presets follow the synthetic workloads built on the paper's
verification setups (Sec. "Verification": single reservoir cell of
V = 4.64e-6 m^3, n = 1e23 m^-3 for the water case, 1e22 m^-3 per species for
the CH4 + H exchange case), with the readings listed beside each preset.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

EV = 1.602176634e-19          # J
AMU = 1.66053906660e-27       # kg
CM1 = 100.0                   # cm^-1 -> m^-1
C2_RAD = 1.438776877e-2       # m K, second radiation constant hc/k (cm^-1 -> K)
KB = 1.380649e-23             # J/K (used only for Maxwellian input velocities)


@dataclasses.dataclass
class Species:
    name: str
    mass: float                     # kg
    d_ref: float                    # m
    T_ref: float = 273.0            # K
    omega: float = 0.75
    E_form: float = 0.0             # J, from the well bottom
    we: List[float] = dataclasses.field(default_factory=list)     # m^-1 per stretch
    wexe: List[float] = dataclasses.field(default_factory=list)   # m^-1 per stretch
    De: List[float] = dataclasses.field(default_factory=list)     # J per stretch
    theta: List[float] = dataclasses.field(default_factory=list)  # K per bend
    coupling_m1: float = 0.0        # stretch-bend coupling, stored, unused (reading A1)
    rot_dof: int = 0                # classical rotational degrees of freedom (0, 2 or 3)

    @property
    def n_modes(self) -> int:
        return len(self.we) + len(self.theta)


@dataclasses.dataclass
class Reaction:
    type: str                       # "diss", "exch" or "recomb"
    reactants: List[int]
    products: List[int]
    diss_mode_mask: int = 0
    Ea: float = 0.0
    steric: float = 1.0
    alpha_mode: str = "per_mode"    # or "one_random_stretch" (reading A18)
    alpha: List[float] = dataclasses.field(default_factory=list)
    model: str = "qk"               # diss / exch: "qk" or "tce" (Arrhenius via TCE)
    arrhenius: Optional[List[float]] = None   # TCE: A (m^3/s K^-b), b, E_a (J)
    tce_zeta: float = 0.0           # TCE: internal DOF (half the pair's sum) in the collision energy
    recomb_prob: str = "exact"      # recomb: "exact" level sum or "wr" (Whitten-Rabinovitch)
    wr_samples: int = 1000
    gamma: float = 0.0              # rotation-vibration coupling: gamma E_rot,A in the QK collision energy
    product_split: str = "relaxation"  # products' levels: "relaxation" (reading A13) or
                                       # "collision_temperature" (equipartition at T_c)


def triatomic() -> Species:
    """Synthetic triatomic: 2 Morse stretches (we 3800, wexe 80 cm^-1, De 5.1 eV),
    1 bend at 1600 cm^-1, coupling -50 cm^-1 (stored only), 18.015 u."""
    return Species("triatomic", 18.015 * AMU, 4.0e-10,
                   we=[3800 * CM1] * 2, wexe=[80 * CM1] * 2, De=[5.1 * EV] * 2,
                   theta=[1600 * CM1 * C2_RAD], coupling_m1=-50 * CM1)


def ch4_like() -> Species:
    """CH4-like: 4 Morse C-H stretches (we 3100, wexe 60 cm^-1, De 4.5 eV) and
    bends 3 x 1300 + 2 x 1550 cm^-1 (reading A3), 16.043 u."""
    return Species("CH4", 16.043 * AMU, 4.0e-10,
                   we=[3100 * CM1] * 4, wexe=[60 * CM1] * 4, De=[4.5 * EV] * 4,
                   theta=[1300 * CM1 * C2_RAD] * 3 + [1550 * CM1 * C2_RAD] * 2)


def ch3_like() -> Species:
    """CH3 product: the paper's CH3 bends (872.1 K x1, 2016.2 K x2) with the C-H
    stretch parameters of ch4_like; E_form = +4.5 eV so that breaking one C-H
    bond of CH4 costs exactly its De (reading A13)."""
    return Species("CH3", 15.035 * AMU, 4.0e-10, E_form=4.5 * EV,
                   we=[3100 * CM1] * 3, wexe=[60 * CM1] * 3, De=[4.5 * EV] * 3,
                   theta=[872.1, 2016.2, 2016.2])


def h_atom() -> Species:
    return Species("H", 1.008 * AMU, 2.5e-10)


def h2() -> Species:
    """H2 with the paper's Morse constants (we = 439524 m^-1, chi_e = 0.0287);
    De = 4.7469 eV and E_form = -De (two H atoms bind)."""
    we = 439524.0
    De = 4.746866797 * EV
    return Species("H2", 2.016 * AMU, 2.9e-10, E_form=-De, we=[we], wexe=[0.0287 * we], De=[De])


def maxwellian(rng: np.random.Generator, n: int, mass: np.ndarray, T: float) -> np.ndarray:
    """Velocities (n,3) from a Maxwellian at T: each component N(0, kT/m)."""
    sig = np.sqrt(KB * T / mass)
    return rng.standard_normal((n, 3)) * sig[:, None]


@dataclasses.dataclass
class Workload:
    name: str
    species: List[Species]
    reactions: List[Reaction]
    n_cells: int
    cell_volume: float
    weight: float
    dt: float
    T_tr0: float
    T_vib0: float
    seed: int
    v: np.ndarray
    species_idx: np.ndarray
    cell: np.ndarray
    steps: int
    cell_base: int = 0              # index of the first cell in the random-number keys

    @property
    def n(self) -> int:
        return int(self.v.shape[0])

    def qn0(self) -> np.ndarray:
        return np.zeros((self.n, 16), dtype=np.uint8)


def _build(name, species, reactions, n_cells, per_cell_counts, fractions, V_total, n_density,
           dt, T_tr0, T_vib0, seed, steps, shuffle=True) -> Workload:
    rng = np.random.default_rng(seed)
    n = int(np.sum(per_cell_counts))
    cell = np.repeat(np.arange(n_cells, dtype=np.int32), per_cell_counts)
    sp = rng.choice(len(fractions), size=n, p=np.asarray(fractions) / np.sum(fractions)).astype(np.int32) \
        if len(fractions) > 1 else np.zeros(n, dtype=np.int32)
    if shuffle:
        perm = rng.permutation(n)
        cell = cell[perm]
    mass = np.array([species[i].mass for i in range(len(species))])[sp]
    v = maxwellian(rng, n, mass, T_tr0)
    weight = n_density * V_total / n
    return Workload(name, species, reactions, n_cells, V_total / n_cells, weight, dt, T_tr0, T_vib0,
                    seed, np.ascontiguousarray(v, dtype=np.float64), sp.astype(np.int32),
                    cell.astype(np.int32), steps)


def relaxation_triatomic(n_particles: int = 20000, n_cells: int = 1, steps: int = 1000,
                         seed: int = 0x48434131) -> Workload:
    """0D adiabatic reservoir of the synthetic triatomic: T_tr0 = 10000 K,
    T_vib0 = 300 K, no chemistry; n = 1e23 m^-3 in V = 4.64e-6 m^3;
    dt = 2.0e-9 s (0.2 / nu(T_tr0) of the VHS closed form, reading A19)."""
    counts = np.full(n_cells, n_particles // n_cells)
    counts[: n_particles % n_cells] += 1
    return _build("relaxation_triatomic", [triatomic()], [], n_cells, counts, [1.0], 4.64e-6,
                  1e23, 2.0e-9, 10000.0, 300.0, seed, steps)


def ch4_heat_bath(n_cells: int = 4096, per_cell: int = 500, steps: int = 500,
                  seed: int = 0x48434132, T0: float = 15000.0, dissociation: bool = True) -> Workload:
    """0D CH4-like heat bath at 15000 K (T_tr0 = T_vib0, reading A20),
    dissociation CH4 + M -> CH3 + H + M on all four stretches; n = 1e23 m^-3 in
    V = 4.64e-6 m^3 split into n_cells cells; dt = 1.7e-9 s (0.2 / nu(T0))."""
    sp = [ch4_like(), ch3_like(), h_atom()]
    rx = [Reaction("diss", [0], [1, 2], diss_mode_mask=0xF)] if dissociation else []
    counts = np.full(n_cells, per_cell)
    return _build("ch4_heat_bath", sp, rx, n_cells, counts, [1.0], 4.64e-6, 1e23, 1.7e-9,
                  T0, T0, seed, steps)


def ch4_h_exchange(n_cells: int = 16384, per_cell: int = 1200, steps: int = 2000,
                   seed: int = 0x48434133, T0: float = 5000.0) -> Workload:
    """CH4 + H -> CH3 + H2, 50/50 CH4/H, Ea = 1.03e-19 J, steric factor 1,
    alpha = 1 on one stretch chosen per collision (reading A18); n = 1e22 m^-3
    per species (2e22 total) in V = 4.64e-6 m^3; dt = 0.2/nu(T0) of the
    mixture, tabulated for 2000..6000 K."""
    dts = {2000.0: 8.2e-9, 3000.0: 7.4e-9, 4000.0: 6.9e-9, 5000.0: 6.5e-9, 6000.0: 6.2e-9}
    dt = dts.get(float(T0), 6.5e-9)
    sp = [ch4_like(), h_atom(), ch3_like(), h2()]
    rx = [Reaction("exch", [0, 1], [2, 3], Ea=1.03e-19, steric=1.0, alpha_mode="one_random_stretch")]
    counts = np.full(n_cells, per_cell)
    return _build("ch4_h_exchange", sp, rx, n_cells, counts, [0.5, 0.5], 4.64e-6, 2e22, dt,
                  T0, T0, seed, steps)


def ch4_recombination(n_cells: int = 8, per_cell: int = 2000, steps: int = 500,
                      seed: int = 0x48434136, T0: float = 4000.0, n_density: float = 3e23,
                      fractions=(1.0, 1.0, 1.0), recombination: bool = True) -> Workload:
    """CH4 + M <-> CH3 + H + M (the paper's methane dissociation-recombination
    case, Sec. "Verification"): CH4 : CH3 : H in the given proportions at total
    number density n_density, T_tr0 = T_vib0 = T0, dissociation on all four
    C-H stretches and its recombination; dt = 0.2 / nu(T0) of CH4 at that
    density."""
    sp = [ch4_like(), ch3_like(), h_atom()]
    rx = [Reaction("diss", [0], [1, 2], diss_mode_mask=0xF)]
    if recombination:
        rx.append(Reaction("recomb", [1, 2], [0, -1], diss_mode_mask=0xF))
    dt = 0.2 / vhs_collision_frequency(sp[0], n_density, T0)
    return _build("ch4_recombination", sp, rx, n_cells, np.full(n_cells, per_cell), list(fractions),
                  4.64e-6, n_density, dt, T0, T0, seed, steps)


def cell_range(kind: str, c0: int, c1: int, total_cells: int, per_cell: Optional[int] = None,
               T0: Optional[float] = None, seed: Optional[int] = None) -> Workload:
    """Cells [c0, c1) of a workload of total_cells cells whose initial state
    is drawn cell by cell, from a generator seeded by (seed, cell), so that
    any split of the cells into contiguous ranges holds exactly the
    particles of the whole: the unit of the multi-GPU split (each rank one
    range; cell_base = c0 keys the range's cells by their global index).
    kind "exchange": the CH4 + H mixture of ch4_h_exchange (50/50, 1200 per
    cell, 4000 K); kind "heat_bath": the CH4 bath of ch4_heat_bath (500 per
    cell, 15000 K).  Weight and cell volume are those of the whole."""
    if kind == "exchange":
        T = 4000.0 if T0 is None else T0
        ref = ch4_h_exchange(n_cells=1, per_cell=2, T0=T)
        pc = 1200 if per_cell is None else per_cell
        fractions, n_density, sd = np.array([0.5, 0.5]), 2e22, 0x48434133
    elif kind == "heat_bath":
        T = 15000.0 if T0 is None else T0
        ref = ch4_heat_bath(n_cells=1, per_cell=2, T0=T)
        pc = 500 if per_cell is None else per_cell
        fractions, n_density, sd = np.array([1.0]), 1e23, 0x48434132
    else:
        raise ValueError(kind)
    sd = sd if seed is None else seed
    V_total = 4.64e-6
    n_loc = (c1 - c0) * pc
    sp = np.zeros(n_loc, np.int32)
    v = np.zeros((n_loc, 3))
    masses = np.array([s.mass for s in ref.species])
    for i, c in enumerate(range(c0, c1)):
        rng = np.random.default_rng((sd, c))
        s_c = rng.choice(len(fractions), size=pc, p=fractions / fractions.sum()).astype(np.int32) \
            if len(fractions) > 1 else np.zeros(pc, np.int32)
        sp[i * pc:(i + 1) * pc] = s_c
        v[i * pc:(i + 1) * pc] = maxwellian(rng, pc, masses[s_c], T)
    cell = np.repeat(np.arange(c1 - c0, dtype=np.int32), pc)
    weight = n_density * V_total / (total_cells * pc)
    return Workload(f"{ref.name}_cells_{c0}_{c1}_of_{total_cells}", ref.species, ref.reactions, c1 - c0,
                    V_total / total_cells, weight, ref.dt, T, T, sd, np.ascontiguousarray(v), sp, cell, ref.steps,
                    cell_base=c0)


def random_levels(rng: np.random.Generator, n: int, n_levels: List[int], n_modes: int) -> np.ndarray:
    """Uniformly random valid quantum numbers for load-path tests (no physics)."""
    q = np.zeros((n, 16), dtype=np.uint8)
    for j in range(n_modes):
        q[:, j] = rng.integers(0, n_levels[j], size=n)
    return q


def vhs_collision_frequency(sp: Species, n_density: float, T: float) -> float:
    """Mean collision frequency of a simple VHS gas, nu = 4 d^2 n sqrt(pi k T_ref / m)
    (T/T_ref)^(1-omega) (Bird's VHS closed form), used only to choose a time step
    dt = 0.2 / nu(T0) for a workload."""
    import math
    return 4.0 * sp.d_ref ** 2 * n_density * math.sqrt(math.pi * KB * sp.T_ref / sp.mass) * \
        (T / sp.T_ref) ** (1.0 - sp.omega)


@dataclasses.dataclass
class BatchedWorkload:
    """Many independent single-cell 0D reservoirs sharing one species table."""
    name: str
    species: List[Species]
    reactions: List[Reaction]
    reservoirs: List[Workload]
    steps: int

    @property
    def n(self) -> int:
        return int(sum(r.n for r in self.reservoirs))


def batched_reservoirs(n_res: int = 256, n_min: int = 10_000, n_max: int = 2_000_000,
                       T_min: float = 5000.0, T_max: float = 30000.0, steps: int = 1000,
                       seed: int = 0x48434134) -> BatchedWorkload:
    """Independent 0D reservoirs (one cell of V = 4.64e-6 m^3, n = 1e23 m^-3):
    particle counts log-uniform in [n_min, n_max], T uniform in [T_min, T_max]
    (T_tr0 = T_vib0), species the synthetic triatomic or the CH4-like
    pentatomic with probability 1/2 each, no chemistry, dt = 0.2 / nu(T0)."""
    rng = np.random.default_rng(seed)
    species = [triatomic(), ch4_like()]
    out = []
    for i in range(n_res):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        T = float(rng.uniform(T_min, T_max))
        s = int(rng.integers(0, 2))
        dt = 0.2 / vhs_collision_frequency(species[s], 1e23, T)
        r = _build(f"reservoir{i}", species, [], 1, np.array([n]), [1.0], 4.64e-6, 1e23, dt, T, T,
                   seed + 1 + i, steps, shuffle=False)
        r.species_idx[:] = s
        mass = np.full(n, species[s].mass)
        r.v = np.ascontiguousarray(maxwellian(np.random.default_rng(seed + 100000 + i), n, mass, T))
        out.append(r)
    return BatchedWorkload("batched_reservoirs", species, [], out, steps)


@dataclasses.dataclass
class ServedJob:
    arrival: float       # s after the first arrival
    kind: str
    workload: Workload
    steps: int


@dataclasses.dataclass
class ServedWorkload:
    """Poisson-arriving single-cell reservoir jobs sharing one species and
    reaction table (the serving engine's input)."""
    name: str
    species: List[Species]
    reactions: List[Reaction]
    jobs: List[ServedJob]

    @property
    def particle_steps(self) -> int:
        return int(sum(j.workload.n * j.steps for j in self.jobs))


def served_jobs(n_jobs: int = 48, rate: float = 50.0, n_min: int = 10_000, n_max: int = 4_000_000,
                steps_min: int = 200, steps_max: int = 2000, recombination: bool = False,
                seed: int = 0x48434135) -> ServedWorkload:
    """Reservoir jobs arriving as a Poisson process of the given rate (1/s):
    particle counts log-uniform in [n_min, n_max], step counts uniform in
    [steps_min, steps_max], one cell of V = 4.64e-6 m^3 each.  Species table
    [triatomic, CH4-like, CH3-like, H]; reactions CH4 + M -> CH3 + H + M
    (+ its recombination if asked).  Job kinds, 1/3 each:
      relax  -- triatomic, n = 1e23 m^-3, T_tr0 uniform 5000-30000 K, T_vib0 = 300 K;
      bath   -- CH4-like heat bath, n = 1e23 m^-3, T_tr0 = T_vib0 uniform 6000-10000 K;
      equil  -- CH4 : CH3 : H = 1 : 1 : 1 at n = 1e23 m^-3 each, T_tr0 = T_vib0 = 4000 K.
    dt = 0.2 / nu(T0) of the job's first species at the job's total density."""
    rng = np.random.default_rng(seed)
    species = [triatomic(), ch4_like(), ch3_like(), h_atom()]
    rx = [Reaction("diss", [1], [2, 3], diss_mode_mask=0xF)]
    if recombination:
        rx.append(Reaction("recomb", [2, 3], [1, -1], diss_mode_mask=0xF))
    t = 0.0
    jobs = []
    for i in range(n_jobs):
        if i:
            t += float(rng.exponential(1.0 / rate))
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        steps = int(rng.integers(steps_min, steps_max + 1))
        kind = ("relax", "bath", "equil")[int(rng.integers(0, 3))]
        js = seed + 1 + i
        if kind == "relax":
            T = float(rng.uniform(5000.0, 30000.0))
            dt = 0.2 / vhs_collision_frequency(species[0], 1e23, T)
            w = _build(f"job{i}", species, rx, 1, np.array([n]), [1.0], 4.64e-6, 1e23, dt, T, 300.0,
                       js, steps, shuffle=False)
        elif kind == "bath":
            T = float(rng.uniform(6000.0, 10000.0))
            dt = 0.2 / vhs_collision_frequency(species[1], 1e23, T)
            w = _build(f"job{i}", species, rx, 1, np.array([n]), [0.0, 1.0], 4.64e-6, 1e23, dt, T, T,
                       js, steps, shuffle=False)
        else:
            T = 4000.0
            dt = 0.2 / vhs_collision_frequency(species[1], 3e23, T)
            w = _build(f"job{i}", species, rx, 1, np.array([n]), [0.0, 1.0, 1.0, 1.0], 4.64e-6, 3e23,
                       dt, T, T, js, steps, shuffle=False)
        jobs.append(ServedJob(t, kind, w, steps))
    return ServedWorkload("served_jobs", species, rx, jobs)


# ----------------------------------------------------------------- paper presets
# The species and reaction tables of the paper's verification cases (Sec.
# "Verification": tab:h2o, tab:hcn, tab:ch4, tab:ch3 and the Arrhenius
# tables).  The tables give omega_e (m^-1) and chi_e of each Morse stretch and
# Theta (K) of each bend.  Readings (the tables leave these open):
#   - a stretch's dissociation energy is the Morse value
#     D_e = h c omega_e / (4 chi_e) (Eq. energy-AHO with chi_e = h c omega_e /
#     (4 D_e)); its levels are kept below it;
#   - masses are the molecular masses, VHS d_ref 4e-10 m for polyatomic
#     molecules, 3.5e-10 m for diatomics, 3.0e-10 m for N and 2.5e-10 m for
#     H, T_ref = 273 K and omega = 0.75 for all;
#   - formation energies from the well bottoms: the fragment that keeps a
#     bond's partner carries that bond's D_e, so that breaking it costs
#     exactly D_e (reading A13);
#   - the paper's particle weights and number densities would give 1e14 to
#     1e17 particles for its reservoir volume; the presets keep the number
#     densities and temperatures and choose the particle count, w = n V / N;
#   - Arrhenius E_a values are given in K and converted with k.
HC_JM = 6.62607015e-34 * 299792458.0   # h c, J m


def morse(we_m1: float, chi_e: float):
    """(omega_e, omega_e chi_e, D_e) of a Morse stretch from omega_e (m^-1)
    and chi_e (the paper's table form)."""
    return we_m1, we_m1 * chi_e, HC_JM * we_m1 / (4.0 * chi_e)


def _morse_species(name, mass_u, d_ref, stretches, thetas, E_form=0.0) -> Species:
    we, wexe, De = [], [], []
    for w_, c_ in stretches:
        a, b, d = morse(w_, c_)
        we.append(a); wexe.append(b); De.append(d)
    return Species(name, mass_u * AMU, d_ref, E_form=E_form, we=we, wexe=wexe, De=De, theta=list(thetas))


def paper_species(name: str) -> Species:
    """Species of the paper's verification tables (tab:h2o, tab:hcn, tab:ch4,
    tab:ch3 and the diatomics named beside them)."""
    oh = (387620.0, 0.021774)
    hc = (342040.0, 0.0146)
    cn_in_hcn = (211920.0, 0.00368)
    ch = (312350.0, 0.0190)
    h2 = (439524.0, 0.0287)
    if name == "H2O":
        return _morse_species("H2O", 18.015, 4.0e-10, [oh, oh], [2294.3])
    if name == "OH":  # the water molecule's O-H stretch parameters
        return _morse_species("OH", 17.007, 3.5e-10, [oh], [], E_form=morse(*oh)[2])
    if name == "N2":
        return _morse_species("N2", 28.014, 3.5e-10, [(234599.0, 0.007439)], [])
    if name == "HCN":  # modes: HC stretch, CN stretch, two bends
        return _morse_species("HCN", 27.025, 4.0e-10, [hc, cn_in_hcn], [1023.9, 1023.9])
    if name == "CN":  # the paper's CN constants (chi_e as printed beside the table)
        return _morse_species("CN", 26.017, 3.5e-10, [(211920.0, 0.0146)], [], E_form=morse(*hc)[2])
    if name == "HC":
        return _morse_species("HC", 13.019, 3.5e-10, [hc], [], E_form=morse(*cn_in_hcn)[2])
    if name == "CH4":
        return _morse_species("CH4", 16.043, 4.0e-10, [ch] * 4, [1565.2, 1565.2, 1360.3, 1360.3, 1360.3])
    if name == "CH3":
        return _morse_species("CH3", 15.035, 4.0e-10, [ch] * 3, [872.1, 2016.2, 2016.2], E_form=morse(*ch)[2])
    if name == "H2":
        return _morse_species("H2", 2.016, 2.9e-10, [h2], [], E_form=-morse(*h2)[2])
    if name == "H":
        return Species("H", 1.008 * AMU, 2.5e-10)
    if name == "N":
        return Species("N", 14.007 * AMU, 3.0e-10)
    raise ValueError(name)


# Arrhenius parameters of the paper's TCE reference runs: A (m^3/s K^-b), b,
# E_a (K), and the internal degrees of freedom (half the pair's sum) that the
# TCE collision energy counts (reading: 0, translation only, except for HCN,
# whose b = -2.6 needs zeta > 1.1 for the probability to stay finite at the
# threshold; zeta = 2, HCN's two bends and two stretches halved)
PAPER_ARRHENIUS = {
    "H2O+M->H+OH+M": ([8e-15, 0.0, 52920.0], 0.0),
    "HCN+M->H+CN+M": ([5.9283e-4, -2.6, 62845.0], 2.0),
    "CH4+H->CH3+H2": ([1.03e-24, 2.5, 4825.0], 0.0),
    "CH4+M->CH3+H+M": ([5.26e-12, 0.0, 51488.0], 0.0),
}


def _tce(key):
    (A, b, Ea_K), zeta = PAPER_ARRHENIUS[key]
    return dict(model="tce", arrhenius=[A, b, Ea_K * KB], tce_zeta=zeta)


def paper_water(model: str = "qk", n_per_species: int = 200_000, n_cells: int = 1,
                seed: int = 0x48434140) -> Workload:
    """H2O + N2 -> H + OH + N2 (Sec. "Verification", water case): T0 = 6000 K,
    n = 1e23 m^-3 of H2O and of N2, dt = 2e-9 s; QK (either O-H stretch may
    break) or TCE with the paper's Arrhenius parameters."""
    sp = [paper_species(s) for s in ("H2O", "N2", "H", "OH")]
    kw = _tce("H2O+M->H+OH+M") if model == "tce" else {}
    rx = [Reaction("diss", [0], [3, 2], diss_mode_mask=0b11, **kw)]
    counts = np.full(n_cells, 2 * n_per_species // n_cells)
    return _build(f"paper_water_{model}", sp, rx, n_cells, counts, [1.0, 1.0, 0.0, 0.0], 4.64e-6, 2e23,
                  2e-9, 6000.0, 6000.0, seed, 2000)


def paper_hcn(T0: float = 5000.0, model: str = "qk", n_per_species: int = 200_000, n_cells: int = 1,
              seed: int = 0x48434141) -> Workload:
    """HCN + N, the two dissociation channels H + CN and HC + N (Sec.
    "Verification", hydrogen cyanide case): n = 3e24 m^-3 of HCN and of N at
    T0 = 5000 or 12000 K; QK (both channels) or TCE (the H + CN channel
    only, the paper's Arrhenius parameters).  dt = 0.2 / nu(T0)."""
    sp = [paper_species(s) for s in ("HCN", "N", "H", "CN", "HC")]
    if model == "tce":
        rx = [Reaction("diss", [0], [3, 2], diss_mode_mask=0b01, **_tce("HCN+M->H+CN+M"))]
    else:
        rx = [Reaction("diss", [0], [3, 2], diss_mode_mask=0b01),
              Reaction("diss", [0], [4, 1], diss_mode_mask=0b10)]
    dt = 0.2 / vhs_collision_frequency(sp[0], 6e24, T0)
    counts = np.full(n_cells, 2 * n_per_species // n_cells)
    return _build(f"paper_hcn_{model}_{T0:.0f}K", sp, rx, n_cells, counts, [1.0, 1.0, 0.0, 0.0, 0.0], 4.64e-6,
                  6e24, dt, T0, T0, seed, 2000)


def paper_methane_exchange(model: str = "qk", n_per_species: int = 100_000, n_cells: int = 1,
                           seed: int = 0x48434142) -> Workload:
    """CH4 + H -> CH3 + H2 (Sec. "Verification", methane case): CH4, H, CH3
    and H2 at n = 1e22 m^-3 each, T0 = 5000 K, dt = 5e-9 s; QK with 21% of
    every mode's energy coupled (alpha_j = 0.21) and E_a = 1.03e-19 J, or TCE
    with the paper's Arrhenius parameters."""
    sp = [paper_species(s) for s in ("CH4", "H", "CH3", "H2")]
    if model == "tce":
        rx = [Reaction("exch", [0, 1], [2, 3], **_tce("CH4+H->CH3+H2"))]
    else:
        rx = [Reaction("exch", [0, 1], [2, 3], Ea=1.03e-19, steric=1.0, alpha_mode="per_mode", alpha=[0.21] * 9)]
    counts = np.full(n_cells, 4 * n_per_species // n_cells)
    return _build(f"paper_methane_exchange_{model}", sp, rx, n_cells, counts, [1.0, 1.0, 1.0, 1.0], 4.64e-6,
                  4e22, 5e-9, 5000.0, 5000.0, seed, 2000)


def paper_methane_dissociation(model: str = "qk", n_per_species: int = 100_000, n_cells: int = 1,
                               seed: int = 0x48434143) -> Workload:
    """CH4 + M <-> CH3 + H + M (Sec. "Verification", methane case): CH4, CH3
    and H at n = 1e23 m^-3 each, T0 = 9000 K; the forward dissociation by QK
    or TCE (the paper's Arrhenius parameters), the backward recombination
    from the equilibrium constant in both.  dt = 0.2 / nu(T0)."""
    sp = [paper_species(s) for s in ("CH4", "CH3", "H")]
    kw = _tce("CH4+M->CH3+H+M") if model == "tce" else {}
    rx = [Reaction("diss", [0], [1, 2], diss_mode_mask=0xF, **kw),
          Reaction("recomb", [1, 2], [0, -1], diss_mode_mask=0xF)]
    dt = 0.2 / vhs_collision_frequency(sp[0], 3e23, 9000.0)
    counts = np.full(n_cells, 3 * n_per_species // n_cells)
    return _build(f"paper_methane_dissociation_{model}", sp, rx, n_cells, counts, [1.0, 1.0, 1.0], 4.64e-6,
                  3e23, dt, 9000.0, 9000.0, seed, 2000)
