/*
 * hcao.h -- C ABI of libhcao: the DSMC collision phase with the HCAO
 * vibrational model and QK-type chemistry on one NVIDIA B300 (sm_103a).
 *
 * Paper: "A harmonically-coupled-anharmonic-oscillator approach for polyatomic
 * chemistry modeling in DSMC" (Lauterbach, Tuttas, Pfeiffer).
 *
 * Conventions (every entry point):
 *   - Returns hcao_status; HCAO_OK (0) on success, a negative code otherwise.
 *     hcao_last_error() gives a one-line description of the last failure.
 *     No C++ exception crosses this boundary.
 *   - SI units throughout: J, K, m, kg, s.
 *   - Pointers named host_* or documented as "host" are host memory owned by the
 *     caller; the library copies what it needs before returning (or, for reads,
 *     has filled them when the call returns).  Pointers documented as "device"
 *     are device memory owned by the caller.
 *   - The context owns all of its device memory (cudaMallocAsync on its
 *     stream) and frees it in hcao_destroy.
 *   - All work is issued on the context's stream (hcao_config.cuda_stream,
 *     borrowed, may be PyTorch's current stream; NULL = the legacy default
 *     stream).  Calls on one context are not thread-safe.
 *   - Device-side failures (rejection-loop cap, capacity, round limit) set a
 *     sticky error word on the device; hcao_sync() and every read call return
 *     it as a status.
 */
#ifndef HCAO_H
#define HCAO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HCAO_OK = 0,
    HCAO_EINVAL = -1,          /* bad argument or call order */
    HCAO_ENOMEM = -2,          /* device allocation failed */
    HCAO_ECUDA = -3,           /* a CUDA runtime call failed */
    HCAO_EREJECT_LIMIT = -4,   /* an LB/init rejection loop hit its cap */
    HCAO_ELEVEL_OVERFLOW = -5, /* a quantum number outside a mode's level list */
    HCAO_EBUSY = -6,           /* job still running (serving) */
    HCAO_ECAPACITY = -7,       /* a cell ran out of particle slots, or would pair over 2^24
                                  pairs in one NTC round (N/2, N/3 with recombination) */
    HCAO_EROUNDS = -8,         /* NTC needed more pairing rounds than configured */
    HCAO_ENOTFOUND = -9,
    HCAO_ENONFINITE = -10,     /* a non-finite velocity or (sigma_T g)_max was met */
    HCAO_ECANCELLED = -11      /* a served job cancelled before it finished */
} hcao_status;

enum { HCAO_FP64 = 0, HCAO_FP32 = 1 };
enum { HCAO_DISS = 1, HCAO_EXCH = 2, HCAO_RECOMB = 3 };
enum { HCAO_ALPHA_PER_MODE = 0, HCAO_ALPHA_ONE_RANDOM_STRETCH = 1 };

#define HCAO_MAX_MODES 16
#define HCAO_MAX_SPECIES 16
#define HCAO_MAX_REACTIONS 8

typedef struct {
    int precision;          /* HCAO_FP64 (bit-exact parity mode) or HCAO_FP32 */
    int device;             /* CUDA device ordinal */
    void* cuda_stream;      /* borrowed cudaStream_t; NULL = default stream */
    int table_points;       /* K5 grid, 16..4000 (default 2048): FP64 quadratic grid points M;
                               FP32 2M geometric buckets (8 mantissa bits) over M/128 octaves
                               below the span */
    double table_span_J;    /* K5 grid span above the ZPE (default 64 eV) */
    uint32_t reject_cap;    /* trials per LB sample before HCAO_EREJECT_LIMIT (default 2^20) */
    int max_rounds;         /* NTC pairing rounds per cell and step (default 2) */
    double capacity_factor; /* per-cell slots = count*factor + extra (default 2.0); a context
                               whose reactions neither create nor remove particles gives
                               each cell its count (rounded up to 8) */
    int capacity_extra;     /* (default 64) */
} hcao_config;

/* One species (Sec. "The polyatomic HCAO model").  Modes are numbered with the
   Morse stretches first (0..n_stretch-1), then the harmonic bends. */
typedef struct {
    double mass, d_ref, T_ref, omega; /* VHS: omega must be 0.5, 0.75 or 1.0 and
                                         equal for all species */
    double E_form;                    /* J, formation energy from the well bottom */
    int n_stretch;
    const double* we;                 /* host, n_stretch, m^-1 (Eq. energy-AHO) */
    const double* wexe;               /* host, n_stretch, m^-1 */
    const double* De;                 /* host, n_stretch, J (truncates the levels) */
    int n_bend;
    const double* theta;              /* host, n_bend, K (Theta form of Eq. energy-SHO) */
    int rot_dof;                      /* classical rotational degrees of freedom: 0 (none), 2
                                         (linear) or 3 (Sec. "Rotation coupling"); a rotating
                                         species has at most 12 modes in FP32 mode */
} hcao_species;

/* One reaction (Sec. "Polyatomic QK reaction modeling").
   HCAO_RECOMB (Sec. "Recombination reactions"): a colliding (B, C) pair forms
   A with a third body M with probability k_r(T_cell) n / (sigma_T g), n the
   third-body number density of the cell and k_r = k_f / K_eq: k_f is P times
   the VHS collision-rate coefficient of A and M, P the exact thermal average
   of Eq. recomb-correct over A's level combinations with the QK threshold of
   the reverse dissociation (the stretches in diss_mode_mask), and K_eq the
   equilibrium constant from translational and vibrational partition sums.
   k_r is tabulated per third-body species at T_i = 500 K * 2^(i/32),
   i = 0..224, and interpolated linearly in T (clamped at the ends); the
   tables are built on the host by hcao_set_reactions.  M is the particle at
   position 2 kmax + k of the round's pairing permutation (kmax pairs in the
   round, k the pair): a particle in no pair of the round; there is none when
   that position is past the cell's end.  C is removed at the end of the step
   (the survivors at the end of the cell fill the freed slots in increasing
   order).  At most HCAO_MAX_REMOVALS_PER_CELL removals per cell and step
   (HCAO_ECAPACITY beyond).  While a recombination reaction is set, a pairing
   round holds at most N/3 pairs (every pair needs a third body), so a cell
   needs about 1.5 times the rounds: raise hcao_config.max_rounds
   accordingly (HCAO_EROUNDS otherwise). */
#define HCAO_MAX_REMOVALS_PER_CELL 4096
#define HCAO_REC_NODES 225
typedef struct {
    int type;              /* HCAO_DISS: A + M -> B + C + M (Eq. Ecoll-diss);
                              HCAO_EXCH: A + B -> C + D (Eq. Ecoll-exch);
                              HCAO_RECOMB: B + C + M -> A + M */
    int reactants[2];      /* DISS: {A, -1}; EXCH: {A, B}; RECOMB: {B, C} (species indices) */
    int products[2];       /* DISS: {B, C}; EXCH: {C, D}; RECOMB: {A, -1} */
    uint32_t diss_mode_mask; /* DISS: stretches of A that may break; RECOMB: those of
                                the reverse dissociation (sets P's threshold) */
    double Ea;             /* EXCH: activation energy, J */
    double steric;         /* EXCH: steric factor in [0,1] */
    int alpha_mode;        /* EXCH: HCAO_ALPHA_PER_MODE or _ONE_RANDOM_STRETCH */
    const double* alpha;   /* host, n_modes of A, or NULL */
    int model;             /* DISS, EXCH: HCAO_MODEL_QK (0: the QK test of Eq. Ecoll-diss /
                              Eq. Ecoll-exch) or HCAO_MODEL_TCE (1: the total-collision-energy
                              probability of Eq. arrhenius, see below);
                              RECOMB: HCAO_RPROB_EXACT (0: P of Eq. recomb-correct summed over
                              every level combination) or HCAO_RPROB_WR (1: P from the sampled
                              sum with the Whitten-Rabinovitch density of states) */
    double arrhenius[3];   /* TCE: A (m^3/s K^-b), b, E_a (J) of k(T) = A T^b exp(-E_a/(k T)) */
    double tce_zeta;       /* TCE: internal degrees of freedom of the pair (half their sum)
                              whose energy counts in the collision energy; 0 = translational
                              energy only */
    int wr_samples;        /* RECOMB with HCAO_RPROB_WR: sample energies (<= 0: 1000) */
    double gamma;          /* DISS, EXCH (QK): rotation-vibration coupling in [0, 1]; the
                              collision energies of Eq. Ecoll-diss and Eq. Ecoll-exch add
                              gamma E_rot,A (Sec. "Rotation coupling") */
    int prod_split;        /* how the products' levels share the energy left (Sec. "Polyatomic
                              QK reaction modeling"), see below: HCAO_SPLIT_RELAX (0) or
                              HCAO_SPLIT_TCOLL (1) */
} hcao_reaction;
enum { HCAO_MODEL_QK = 0, HCAO_MODEL_TCE = 1 };
/* Product levels.  HCAO_SPLIT_RELAX: each product's levels follow the
   relaxation step's LB target (exponent 3/2 - omega), the first product at
   the available energy less the second's ZPE, the second at what the first
   left.  HCAO_SPLIT_TCOLL: equipartition at a collision temperature T_c,
   the root of xi_tr/2 k T_c + sum over the products of <E_vib>(T_c) = the
   energy above the products' ground states (xi_tr = 6 after a dissociation,
   3 after an exchange or a recombination; <E_vib> the Boltzmann mean of a
   stretch's levels, k Theta / (e^(Theta/T) - 1) for a bend); the first
   product's levels follow (E - E_state)^b1, b1 = (xi_tr + xi_vib,2(T_c))/2 - 1
   with xi_vib = 2 <E_vib> / (k T_c), the second's (E - E_state)^(xi_tr/2 - 1),
   a recombination's product (E - E_state)^(1/2).  Drawn exactly: a table
   draw at exponent 3/2 - omega (or 1/2, tables built for the products when
   the exponent is below 3/2 - omega) accepted with ((E - sum E)/(E - ZPE))
   to the power of the difference.  FP64 mode evaluates T_c by bisection
   with its own exponential; FP32 mode interpolates b1 from a per-reaction
   table over the energy above the ground states (4096 points per reaction,
   log-spaced). */
enum { HCAO_SPLIT_RELAX = 0, HCAO_SPLIT_TCOLL = 1 };
enum { HCAO_RPROB_EXACT = 0, HCAO_RPROB_WR = 1 };

/* One candidate pair of the last step (parity inspection). */
typedef struct {
    uint32_t step, cell, round_k, p, q;
    int32_t event;         /* -1 rejected candidate, 0 relaxed, 1+r reaction r */
    uint32_t aux;          /* DISS: broken stretch (+16 if partner q); EXCH: side;
                              RECOMB: side (B is p: 0, q: 1) + 2 x the third body's index */
} hcao_log_rec;

typedef struct {
    int64_t n[HCAO_MAX_SPECIES];        /* particles per species */
    double momentum[3];                 /* sum m v, kg m/s (times 1, not the weight) */
    double E_tr;                        /* sum 1/2 m v^2, J */
    double E_vib[HCAO_MAX_SPECIES];     /* sum of vibrational energies incl. ZPE, J */
    double E_form;                      /* sum of formation energies, J */
    double T_tr;                        /* from the peculiar translational energy, K */
    double T_vib[HCAO_MAX_SPECIES];     /* zero-point search (Sec. implementation), K */
    double E_rot[HCAO_MAX_SPECIES];     /* sum of rotational energies, J */
    double T_rot[HCAO_MAX_SPECIES];     /* 2 <E_rot> / (rot_dof k), K (0 without rotation) */
} hcao_moments;

typedef struct hcao_ctx hcao_ctx;

/* Create a context on config->device.  config may be NULL (defaults).  The
   context allocates its device memory from a stream-ordered memory pool of
   its own, which keeps up to 8 GiB of memory the context freed mapped for its
   later allocations (reloading reservoirs reuses it); hcao_destroy releases
   the pool.  HCAO_ECUDA if the device or the pool cannot be set up.  Every
   call on a context runs on its device and leaves the calling thread's
   current device as it found it; the serving engine's thread uses the
   context's device. */
hcao_status hcao_create(const hcao_config* config, hcao_ctx** out);
/* Free all device memory of the context (synchronises its stream). */
void hcao_destroy(hcao_ctx* ctx);
const char* hcao_last_error(const hcao_ctx* ctx);
/* Fill *config with the defaults. */
void hcao_default_config(hcao_config* config);

/* Species and their level / sampler tables: Morse stretch levels (Eq.
   energy-AHO), harmonic bends (Eq. energy-SHO), the K5 sampler tables.  Call
   once, before any reservoir is added.  Copies all arrays. */
hcao_status hcao_set_species(hcao_ctx* ctx, const hcao_species* species, int n);
/* Reactions (Sec. "Polyatomic QK reaction modeling").  Call after
   hcao_set_species, before any reservoir is added.  Copies all arrays. */
hcao_status hcao_set_reactions(hcao_ctx* ctx, const hcao_reaction* reactions, int n);

/* A 0D reservoir of n_cells independent cells of volume cell_volume with
   particle weight `weight` and time step dt (Sec. "Verification": single
   reservoir cell, closed system).  seed keys its Philox stream; T_sgmax sets
   the initial (sigma_T g)_max = 2 <sigma_T g>(T_sgmax).  *id receives the
   reservoir index. */
hcao_status hcao_add_reservoir(hcao_ctx* ctx, int n_cells, double cell_volume, double weight,
                               double dt, uint64_t seed, double T_sgmax, int* id);
/* The index of reservoir res's first cell in the random-number keys
   (default 0).  Every draw of a cell is keyed by (reservoir seed, step, cell
   index, round, pair), so a reservoir that holds cells [base, base +
   n_cells) of a larger workload -- same seed, same cell volume, weight and
   time step -- steps those cells exactly as the whole workload would: one
   workload split across GPUs or processes by contiguous cell ranges gives
   the same particles as the unsplit run (Multi-GPU split, no exchange between
   the ranges).  Call before hcao_load_particles (HCAO_EINVAL after it);
   base + n_cells must fit 32 bits. */
hcao_status hcao_set_cell_base(hcao_ctx* ctx, int res, uint32_t base);
/* Remove a reservoir and free its device memory. */
hcao_status hcao_remove_reservoir(hcao_ctx* ctx, int res);

/* Load n particles into reservoir res (host arrays: v n x 3 doubles, qn
   n x 16 bytes (mode j of particle i at qn[16 i + j]), species and cell
   n int32).  Sorts them into cells with the stable counting sort, keeping
   input order within a cell.  Replaces any earlier content.  Input that fails
   validation (HCAO_EINVAL, HCAO_ELEVEL_OVERFLOW) leaves the reservoir as it
   was.  A device allocation that fails after the earlier particles were
   released leaves the context refusing device work (step, init and reads
   return HCAO_EINVAL) until a load or a removal succeeds. */
hcao_status hcao_load_particles(hcao_ctx* ctx, int res, int64_t n, const double* host_v,
                                const uint8_t* host_qn, const int32_t* host_species,
                                const int32_t* host_cell);
/* hcao_load_particles with FP32 host velocities (n x 3 floats): 12 instead of
   24 bytes per particle cross the host-device link.  In FP32 mode the records
   equal those of hcao_load_particles with the same values rounded to float;
   in FP64 mode the floats are widened exactly. */
hcao_status hcao_load_particles_f32(hcao_ctx* ctx, int res, int64_t n, const float* host_v,
                                    const uint8_t* host_qn, const int32_t* host_species,
                                    const int32_t* host_cell);
/* Initial quantum numbers of all particles of res at T_vib on the device:
   bends i = floor(-ln(r) T_vib / Theta) (redrawn beyond the level list),
   stretches drawn uniformly over 0..i_diss and accepted with
   exp(-(E_i - E_0)/(k T_vib)) (Sec. implementation, Eq. accept-quant). */
hcao_status hcao_init_vibration(hcao_ctx* ctx, int res, double T_vib);

/* Rotation (Sec. "Rotation coupling"; the paper's verification runs leave it
   out).  Each molecule of a species with rot_dof > 0 carries a classical
   rotational energy, 0 after hcao_load_particles.  Every accepted collision
   that relaxes also relaxes the rotation of each rotating partner after the
   vibrational draws, P before Q, by the classical LB draw E_rot' = x (E_rel +
   E_rot), x ~ Beta(rot_dof/2, (5 - 2 omega)/2).  A reaction adds the
   reactants' rotational energy to the energy it redistributes; products start
   without rotation; a third body keeps its own.
   hcao_init_rotation draws every rotational energy of reservoir res from the
   equilibrium distribution at T_rot (kT times a Gamma(rot_dof/2) variate);
   hcao_load_erot / hcao_read_erot copy them in and out (host, n doubles in
   the order of hcao_read_particles; entries of non-rotating species are
   ignored / 0). */
hcao_status hcao_init_rotation(hcao_ctx* ctx, int res, double T_rot);
hcao_status hcao_load_erot(hcao_ctx* ctx, int res, const double* host_erot);
hcao_status hcao_read_erot(hcao_ctx* ctx, int res, double* host_erot);

/* Advance every reservoir by n_steps collision phases (NTC pair selection with
   VHS cross-sections, QK reaction test and execution, HCAO LB relaxation,
   isotropic scattering).  Asynchronous on the context's stream.  With
   profiling off, one step is captured as a CUDA graph on a private stream
   (again whenever the kernel arguments change, e.g. after a reservoir is
   added) and launched n_steps times on the context's stream. */
hcao_status hcao_step(hcao_ctx* ctx, int n_steps);
/* Wait for the stream; return the sticky device error status. */
hcao_status hcao_sync(hcao_ctx* ctx);

/* Number of particles of reservoir res (synchronises). */
hcao_status hcao_count(hcao_ctx* ctx, int res, int64_t* n);
/* Copy reservoir res back in canonical order (cell by cell, slot order):
   host arrays sized by hcao_count; any of them may be NULL. */
hcao_status hcao_read_particles(hcao_ctx* ctx, int res, double* host_v, uint8_t* host_qn,
                                int32_t* host_species, int32_t* host_cell);
/* Moments of reservoir res, reduced on the device; T_vib by the zero-point
   search on the host.  FP64 mode sums in FP64.  FP32 mode sums exact int64
   fixed point: E_vib from the level tables, momentum and E_tr from float
   products of each particle's velocity and its mass (the mass as a float
   pair, so unrounded): a few float roundings per particle (<= 3e-7
   relative), unbiased.  Synchronises. */
hcao_status hcao_read_moments(hcao_ctx* ctx, int res, hcao_moments* out);
/* Level populations of one mode of one species in reservoir res:
   counts[i] = particles with quantum number i (i < max_levels). */
hcao_status hcao_read_level_populations(hcao_ctx* ctx, int res, int species, int mode,
                                        uint64_t* host_counts, int max_levels);
/* Counters of reservoir res since load: [0] candidate pairs, [1] accepted
   collisions, [2] LB samples, [3] LB trials, [4] sampler table overflows,
   [5] degenerate samples, [6] reactions not executed, [7] steps,
   [8 + r] events of reaction r.  Returns the number written in *n_out. */
hcao_status hcao_read_counters(hcao_ctx* ctx, int res, uint64_t* host_out, int max, int* n_out);
/* Reaction event counts only (host_out[r], r < n). */
hcao_status hcao_read_reaction_counts(hcao_ctx* ctx, int res, uint64_t* host_out, int n);
/* (sigma_T g)_max of every cell of res (host, n_cells doubles). */
hcao_status hcao_read_cell_sgmax(hcao_ctx* ctx, int res, double* host_out);

/* Per-pair log of the most recent step, in canonical order (reservoir, cell,
   round, pair).  Enable before stepping; costs one 28-byte record per pair.
   With host_out == NULL, *n_out receives the number of records available. */
hcao_status hcao_set_log(hcao_ctx* ctx, int enable);
hcao_status hcao_read_log(hcao_ctx* ctx, hcao_log_rec* host_out, int64_t max, int64_t* n_out);

/* Stable counting sort by cell (the sort that places loaded particles in
   their cells): device keys[n] (cell ids < n_cells) -> device perm[n]
   (perm[j] = input index of the j-th particle in cell order, input order kept
   within a cell) and device offsets[n_cells+1] (start of each cell in perm).
   Every key must be < n_cells: a larger key is not counted in offsets, and
   its place in perm is unspecified (the radix passes read only the digits
   that n_cells needs).  Uses scratch from the context; asynchronous on the
   context's stream. */
hcao_status hcao_cell_sort(hcao_ctx* ctx, const uint32_t* keys, int64_t n, uint32_t n_cells,
                           uint32_t* perm, uint32_t* offsets);

/* The relaxation step's sampler alone (diagnostics, distribution tests):
   n independent post-collision vibrational states of species sp at collision
   energy Ec (J), drawn with the sampler of hcao_step in the context's
   precision (the joint LB acceptance of all modes, Sec. implementation of the
   HCAO model).  Sample i uses the Philox stream keyed by seed with counter
   (i, i >> 32, 0, 8 << 24 | block).  host_qn: n x 16 bytes; *host_trials
   (may be NULL) receives the total number of trials.  HCAO_EINVAL if Ec is
   outside the sampler's tables or sp has no vibrational modes. */
hcao_status hcao_sample_lb(hcao_ctx* ctx, int sp, double Ec, uint64_t seed, int64_t n,
                           uint8_t* host_qn, uint64_t* host_trials);

/* The stable cell sort of hcao_cell_sort for callers that cannot allocate
   device memory: code that must not call cudaMalloc once it is running, such
   as a host application whose own pool allocator owns the device memory, or
   a latency-bound loop that cannot take the device-wide synchronisation a
   cudaMalloc/cudaFree may cause.  Same arguments and results as
   hcao_cell_sort (device keys, perm and offsets; see there), on cuda_stream
   (NULL = the legacy default stream); no context is needed.
   - It allocates nothing: its scratch is one file-scope device array sized
     for HCAO_NOALLOC_SORT_MAX_KEYS keys (about 8.7 MB), which every GPU that
     loads the library holds until the process exits.
   - Every call looks up that array's device address with the calling
     thread's device current (a host-side query, no allocation of its own).
   - The array belongs to the library's sort module.  Under CUDA's lazy module
     loading (the default) the first call on each device loads that module,
     which allocates the array and may synchronise the device and fail for
     lack of memory (HCAO_ECUDA).  Callers that must never allocate should
     make one warm-up call on each device at start-up, before any stream
     capture and before their own allocator takes the device's memory.
   - n > HCAO_NOALLOC_SORT_MAX_KEYS returns HCAO_EINVAL; a failed CUDA call
     returns HCAO_ECUDA.
   - All calls share the one array: calls that may overlap on the GPU (other
     streams, other host threads) race and must be serialised by the caller.
   The paper has no counterpart of this entry point. */
#define HCAO_NOALLOC_SORT_MAX_KEYS (1 << 19)
hcao_status hcao_cell_sort_noalloc(const uint32_t* keys, int64_t n, uint32_t n_cells, uint32_t* perm,
                                   uint32_t* offsets, void* cuda_stream);

/* Level energy (J) of level `level` of mode `mode` of species sp, and the
   number of levels; host-side table lookups. */
hcao_status hcao_level_energy(const hcao_ctx* ctx, int sp, int mode, int level, double* out);
hcao_status hcao_n_levels(const hcao_ctx* ctx, int sp, int mode, int* out);

/* Collision-phase path.  HCAO_PATH_QUEUE: per pairing round, a selection,
   a relaxation and a reaction kernel that pass pairs through queues in
   global memory, then end-of-step kernels (about eleven launches a step; any
   context).  HCAO_PATH_FUSED: one kernel a step, one CTA per cell, the
   cell's records staged in shared memory; it needs FP32 mode, no reaction
   that creates or removes particles (dissociation, recombination), no
   per-pair log and cells of at most 4096 particle slots, and gives the same
   bits as the queue path.  HCAO_PATH_AUTO (the default) takes the queue
   path, the faster of the two on every workload measured (the fused kernel
   holds one cell's pairs per CTA and keeps fewer pairs in flight per SM).
   hcao_set_step_path(ctx, HCAO_PATH_FUSED)
   on a context that does not allow it makes the next hcao_step return
   HCAO_EINVAL.  hcao_get_step_path gives the path the next step takes
   (HCAO_PATH_QUEUE or HCAO_PATH_FUSED). */
enum { HCAO_PATH_AUTO = 0, HCAO_PATH_QUEUE = 1, HCAO_PATH_FUSED = 2 };
hcao_status hcao_set_step_path(hcao_ctx* ctx, int path);
hcao_status hcao_get_step_path(const hcao_ctx* ctx, int* path);

/* Kernel timing: with profiling on, hcao_step records CUDA events on the
   context's stream around each kernel.  hcao_read_profile accumulates and
   returns, for k = 0 (setup), 1 (select), 2 (relax), 3 (react), 4 (finish),
   5 (the fused per-cell kernel), the summed device time in ms (host_ms[k])
   and the number of launches (host_launches[k]); *n_out = min(max, 6).
   hcao_set_profiling resets the sums. */
hcao_status hcao_set_profiling(hcao_ctx* ctx, int enable);
hcao_status hcao_read_profile(hcao_ctx* ctx, double* host_ms, uint64_t* host_launches, int max,
                              int* n_out);

/* Launch-schedule autotuner: steps the reservoirs by 7 x steps_per_candidate
   steps while timing candidate grid sizes of the pair-acceptance and
   relaxation kernels (CUDA events), then keeps the fastest; in FP32 mode with
   more than one work class (species pairs whose molecules differ in mode
   counts) 2 x steps_per_candidate more, timing the relaxation queue with and
   without its placement by work class.  The simulation advances normally:
   results do not depend on the schedule (every draw is keyed by step, cell
   and pair).  chosen (may be NULL, else 3 ints) receives the two grid sizes
   and 1 if the queue is placed by work class. */
hcao_status hcao_autotune(hcao_ctx* ctx, int steps_per_candidate, int* chosen);

/* Algorithmic work of the FP32 relaxation kernel since create, counted on
   the steps taken with profiling on (hcao_set_profiling, and the autotuner's
   steps; other steps skip the counting, which costs the kernel ~4%):
   host_out[0] LB level evaluations (one weight of one level of one mode), [1]
   mode draws (one Philox uniform each), [2] molecule samples, [3] relaxed
   pairs; *n_out = 4.  Zero in FP64 mode.  (Instrumentation for the ALU
   roofline.) */
hcao_status hcao_read_work(hcao_ctx* ctx, uint64_t* host_out, int max, int* n_out);

/* ---------------------------------------------------------------- serving
   Continuous batching of 0D reservoir jobs (no counterpart in the paper: the
   serving form of the collision phase).  hcao_serve_start starts an engine
   thread on a context that has species/reactions but no reservoir.  Jobs
   submitted from any thread are admitted, between engine iterations, while
   their estimated HBM (particle slots, per-pair buffers, staging) fits the
   budget and fewer than max_active are resident.  A job larger than the
   budget runs alone.  Every iteration advances all resident jobs together by
   K steps, K the fewest steps any of them still needs (<= max_batch_steps).
   Finished jobs are read back and their memory freed.  Each job's results
   equal those of the same reservoir stepped alone: its draws are keyed by its
   own seed, cells and step count.  While serving, only the serve_* functions
   may be called on the context.  A device error during an iteration fails
   every job resident in it; the engine then clears the error and continues. */
typedef struct {
    int n_cells;
    double cell_volume, weight, dt;  /* as hcao_add_reservoir */
    uint64_t seed;
    double T_sgmax;
    int64_t n;                       /* particles; host arrays as hcao_load_particles */
    const double* v;
    const uint8_t* qn;               /* NULL = all ground state */
    const int32_t* species;
    const int32_t* cell;
    double T_vib;                    /* > 0: initial quantum numbers drawn at T_vib */
    int n_steps;
} hcao_job;

typedef struct {
    int status;                      /* hcao_status of the job */
    int steps;
    int64_t n_particles;             /* at the end */
    hcao_moments moments;            /* at the end */
    uint64_t counters[8 + HCAO_MAX_REACTIONS];  /* as hcao_read_counters */
    double t_submit, t_admit, t_done;           /* CLOCK_MONOTONIC, s */
} hcao_job_result;

/* hbm_budget_bytes <= 0: 80% of the free device memory; max_active <= 0: 256;
   max_batch_steps <= 0: 8.  HCAO_EBUSY if already serving. */
hcao_status hcao_serve_start(hcao_ctx* ctx, int64_t hbm_budget_bytes, int max_active,
                             int max_batch_steps);
/* Copies the job's host arrays; *job_id identifies it.  Thread-safe. */
hcao_status hcao_serve_submit(hcao_ctx* ctx, const hcao_job* job, uint64_t* job_id);
/* HCAO_EBUSY while queued or running; otherwise fills *out, releases the job
   and returns its status (HCAO_ENOTFOUND for an unknown or released id).
   Thread-safe. */
hcao_status hcao_serve_poll(hcao_ctx* ctx, uint64_t job_id, hcao_job_result* out);
/* Cancel a served job: a queued job is dropped at once; a resident job is
   retired at the end of the engine's current iteration (its reservoir
   removed, its steps so far discarded).  Either way the job's result reports
   HCAO_ECANCELLED with t_done set.  HCAO_ENOTFOUND for an unknown, finished
   or released id.  Thread-safe. */
hcao_status hcao_serve_cancel(hcao_ctx* ctx, uint64_t job_id);
/* Finishes the queued and resident jobs, then stops the engine thread. */
hcao_status hcao_serve_stop(hcao_ctx* ctx);
/* Queue length, resident jobs, budgeted bytes in use, engine iterations. */
hcao_status hcao_serve_stats(hcao_ctx* ctx, int64_t* queued, int64_t* active, int64_t* used_bytes,
                             uint64_t* iterations);
/* The engine thread's time since hcao_serve_start by activity, host clock in
   seconds, into seconds4[4]: [0] admission (reservoir set-up, the load from
   the job's host copy, initial levels), [1] stepping (the iterations' step
   launches and their synchronisation: the device busy with resident jobs),
   [2] retirement (moments, counters, release), [3] waiting for work.
   Thread-safe; HCAO_EINVAL for a null argument. */
hcao_status hcao_serve_timing(hcao_ctx* ctx, double* seconds4);
/* Clear the context's device error word.  Device-side conditions (a
   rejection loop at its cap, a cell out of slots, more rounds needed, a
   non-finite value) set a sticky word that every synchronising call reports
   until it is cleared; the particle state stays consistent (a failed draw
   keeps the molecule's state), so a caller may clear it and carry on. */
hcao_status hcao_clear_error(hcao_ctx* ctx);
/* Fault injection for tests (a host-side fault: no device fault, trap or
   hang): the context's next n device allocations of per-call buffers
   (staging, scratch, per-pair buffers, tables) fail as out of memory, so the
   calls that make them return HCAO_ENOMEM as a real shortage would.  n <= 0
   disarms it.  Thread-safe. */
hcao_status hcao_debug_fail_allocs(hcao_ctx* ctx, int n);

/* The tabulated recombination rate coefficient k_r (m^6/s) of reaction
   `reaction` (an HCAO_RECOMB) with a third body of species spM at temperature
   T, interpolated as the collision step does (host copy of the device table). */
hcao_status hcao_recomb_rate(hcao_ctx* ctx, int reaction, int spM, double T, double* out);

/* Whitten-Rabinovitch density of vibrational states (1/J) of n_osc harmonic
   oscillators with quanta hnu[0..n_osc-1] (J) at energy E (J) above the
   ground state: the approximation the paper gives beside Eq. recomb-correct
   for the sampled dissociation probability (decadic logarithm in the Omega
   correlation, E_z half the sum of the quanta).  Host computation: needs no
   context or GPU.  NaN for n_osc < 1, a non-positive quantum or E < 0. */
double hcao_wr_density(const double* hnu, int n_osc, double E);
/* The sampled form of the dissociation probability with the WR density:
   n_samp energies at the midpoints of equal intervals between the ground
   state and the threshold Dx (J above the ground state), weighted
   rho(E) exp(-E/kT); P = sum Q(5/2 - omega, (Dx - E_i)/kT) w_i / sum w_i, Q
   the regularised upper incomplete gamma.  Host computation.  NaN for bad
   arguments; 1 for Dx <= 0.  (The rate tables use the exact level sum.) */
double hcao_wr_diss_prob(const double* hnu, int n_osc, double Dx, double omega, double T, int n_samp);

/* Number of this library's kernels launched since create (instrumentation). */
uint64_t hcao_kernel_launches(const hcao_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
