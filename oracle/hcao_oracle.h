/*
 * hcao_oracle.h -- the oracle: a plain, slow, single-threaded FP64 CPU
 * implementation of the DSMC collision phase with the HCAO vibrational model
 * and QK-type chemistry of "A harmonically-coupled-anharmonic-oscillator
 * approach for polyatomic chemistry modeling in DSMC".
 *
 * THIS IS TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it. The product path (the CUDA
 * library) shares no code, header, table or constant generator with it.
 *
 * Paper sections followed:
 *   Eq. energy-SHO, the Theta form of the harmonic levels (Sec. "The polyatomic
 *   HCAO model")                                   -> harmonic bend levels
 *   Eq. energy-AHO                                  -> Morse stretch levels
 *   Sec. "Implementation of the polyatomic HCAO model": initial bend and
 *   stretch quantum numbers, Eq. accept-quant, the joint LB acceptance of all
 *   modes (the relaxation step)                     -> ora_init_vibration, samplers
 *   Sec. "Polyatomic QK reaction modeling", Eq. Ecoll-diss, Eq. Ecoll-exch,
 *   "Competing reactions"                           -> reaction test / execution
 *   Sec. "Verification": single reservoir cell, closed system, no rotation.
 * Readings where the paper is silent are stated beside each function.
 */
#ifndef HCAO_ORACLE_H
#define HCAO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORA_MAX_MODES 16
#define ORA_MAX_LEVELS 256

enum { ORA_OK = 0, ORA_EINVAL = -1, ORA_ENOMEM = -2, ORA_EREJECT = -4, ORA_ELEVEL = -5 };
enum { ORA_DISS = 1, ORA_EXCH = 2, ORA_RECOMB = 3 };
enum { ORA_ALPHA_PER_MODE = 0, ORA_ALPHA_ONE_RANDOM_STRETCH = 1 };
enum { ORA_SAMPLER_TABLE = 0, ORA_SAMPLER_LITERAL = 1 };

typedef struct {
    double mass;     /* kg */
    double d_ref;    /* m, VHS reference diameter */
    double T_ref;    /* K */
    double omega;    /* VHS viscosity index (0.5, 0.75 or 1.0) */
    double E_form;   /* J, formation energy measured from the well bottom */
    int n_stretch;   /* Morse local stretches, modes 0..n_stretch-1 */
    double we[ORA_MAX_MODES];    /* m^-1 */
    double wexe[ORA_MAX_MODES];  /* m^-1 (omega_e * chi_e) */
    double De[ORA_MAX_MODES];    /* J, from the well bottom */
    int n_bend;      /* harmonic bends, modes n_stretch..n_stretch+n_bend-1 */
    double theta[ORA_MAX_MODES]; /* K */
    int rot_dof;     /* classical rotational degrees of freedom: 0, 2 (linear) or 3 */
} ora_species_desc;

typedef struct {
    int type;             /* ORA_DISS: A + M -> B + C + M ; ORA_EXCH: A + B -> C + D ;
                             ORA_RECOMB: B + C + M -> A + M */
    int reactants[2];     /* DISS: {A, -1}; EXCH: {A, B}; RECOMB: {B, C} */
    int products[2];      /* DISS: {B, C};  EXCH: {C, D}; RECOMB: {A, -1} */
    uint32_t diss_mode_mask; /* DISS / RECOMB: stretch modes of A whose breaking gives B + C */
    double Ea;            /* EXCH: activation energy, J */
    double steric;        /* EXCH: steric factor in [0,1] */
    int alpha_mode;       /* EXCH: ORA_ALPHA_PER_MODE or ORA_ALPHA_ONE_RANDOM_STRETCH */
    double alpha[ORA_MAX_MODES];
    int model;            /* DISS / EXCH: ORA_MODEL_QK or ORA_MODEL_TCE;
                             RECOMB: ORA_RPROB_EXACT or ORA_RPROB_WR (the probability P) */
    double arrhenius[3];  /* TCE: A (m^3/s K^-b), b, E_a (J) of Eq. arrhenius */
    double tce_zeta;      /* TCE: internal degrees of freedom (half the pair's sum) in E_c */
    int wr_samples;       /* RECOMB, WR: sample energies (<= 0: 1000) */
    double gamma;         /* DISS / EXCH (QK): rotation-vibration coupling, gamma E_rot,A in E_coll */
    int prod_split;       /* products' vibrational states: ORA_SPLIT_RELAX (reading A13, the
                             relaxation target) or ORA_SPLIT_TCOLL (equipartition at the
                             collision temperature) */
} ora_reaction_desc;
enum { ORA_SPLIT_RELAX = 0, ORA_SPLIT_TCOLL = 1 };
enum { ORA_MODEL_QK = 0, ORA_MODEL_TCE = 1 };
enum { ORA_RPROB_EXACT = 0, ORA_RPROB_WR = 1 };

typedef struct {
    uint32_t step, cell, round_k, p, q;
    int32_t event;        /* -1: rejected candidate, 0: relaxed, 1+r: reaction r */
    uint32_t aux;         /* DISS: broken stretch mode (+16 if partner q); EXCH: 0/1 A is p/q;
                             RECOMB: 0/1 B is p/q, plus 2 x the third body's index in the cell */
} ora_log_rec;

typedef struct ora_ctx ora_ctx;

ora_ctx* ora_create(int table_points, double table_span_J, uint32_t reject_cap);
void     ora_destroy(ora_ctx*);
int      ora_add_species(ora_ctx*, const ora_species_desc*);
int      ora_add_reaction(ora_ctx*, const ora_reaction_desc*);
int      ora_add_reservoir(ora_ctx*, int n_cells, double cell_volume, double weight,
                           double dt, uint64_t seed, double T_sgmax);
int      ora_load(ora_ctx*, int res, int64_t n, const double* v, const uint8_t* qn,
                  const int32_t* species, const int32_t* cell);
int      ora_init_vibration(ora_ctx*, int res, double T_vib);
/* Rotation (Sec. "Rotation coupling"): per particle a classical rotational
   energy (0 after ora_load).  ora_init_rotation draws it at T_rot from the
   equilibrium distribution Gamma(rot_dof/2) kT; ora_load_erot and
   ora_read_erot copy it in and out in the order of ora_read_particles. */
int      ora_init_rotation(ora_ctx*, int res, double T_rot);
int      ora_load_erot(ora_ctx*, int res, const double* erot);
int      ora_read_erot(ora_ctx*, int res, double* erot);
/* the natural logarithm the oracle's rotation draws use (own series, see
   ora_ln in the source) */
double   ora_ln(double x);
double   ora_exp(double x);  /* own exponential (Taylor series after ln 2 reduction) */
/* n classical LB rotational fractions of species sp (Beta(rot_dof/2,
   (5 - 2 omega)/2)) from a Philox stream keyed by seed (test diagnostic) */
int      ora_sample_rot_fraction(ora_ctx*, int sp, uint64_t seed, int64_t n, double* out);
/* index of the reservoir's first cell in the random-number keys (default 0):
   a reservoir holding cells [base, base + n_cells) of a larger workload steps
   those cells exactly as the whole workload would */
int      ora_set_cell_base(ora_ctx*, int res, uint32_t base);
int      ora_step(ora_ctx*, int n_steps);
int      ora_set_log(ora_ctx*, int enable);
int64_t  ora_log_count(ora_ctx*);
int      ora_read_log(ora_ctx*, ora_log_rec* out, int64_t max);
int64_t  ora_count(ora_ctx*, int res);
int      ora_read_particles(ora_ctx*, int res, double* v, uint8_t* qn, int32_t* species,
                            int32_t* cell);
int      ora_read_cell_sgmax(ora_ctx*, int res, double* out);
/* counters: [0] candidate pairs, [1] accepted collisions, [2] LB samples,
   [3] LB trials, [4] table overflows, [5] degenerate (A6) samples,
   [6] not-executed reactions, [7] steps, [8..8+n_reactions) reaction events */
int      ora_read_counters(ora_ctx*, int res, uint64_t* out, int max);
int      ora_n_levels(ora_ctx*, int sp, int mode);
double   ora_level_energy(ora_ctx*, int sp, int mode, int level);
double   ora_table_value(ora_ctx*, int sp, int k, int m);
int      ora_table_entries(ora_ctx*, int sp);
double   ora_zpe(ora_ctx*, int sp);
/* draws n samples of the post-collision state of species sp at collision
   energy Ec with the chosen sampler; a Philox stream keyed by seed */
int      ora_sample_lb(ora_ctx*, int sp, double Ec, uint64_t seed, int64_t n, int method,
                       uint8_t* out_qn, uint64_t* trials);
/* Test diagnostic: n independent executions of reaction rx on one fixed set
   of reactants, event i with the random streams of pair i.  Reactants 1, 2
   (species, velocity, levels): dissociation A and its third body M; exchange
   A and B; recombination B and C, with reactant 3 its third body M (reactant
   3 is unused otherwise).  Per executed event out_v[9 i ..] receives three
   velocities and out_q[32 i ..] two level sets: dissociation B, C, M and the
   levels of B, C; exchange C, D, zeros and the levels of C, D; recombination
   A, zeros, M and the levels of A.  Returns the number of executed events (0
   when the reactants cannot react) or a negative error. */
int64_t  ora_sample_products(ora_ctx*, int rx, int sp1, const double* v1, const uint8_t* q1, int sp2,
                             const double* v2, const uint8_t* q2, int sp3, const double* v3, const uint8_t* q3,
                             uint64_t seed, int64_t n, double* out_v, uint8_t* out_q);
/* TCE probability of reaction rx (model ORA_MODEL_TCE) for a partner of
   species m at collision energy Ec (J), as the collision step evaluates it */
double   ora_tce_prob(ora_ctx*, int rx, int m, double Ec);
/* draws n initial states of species sp at T_vib (P6/P7) */
int      ora_sample_init(ora_ctx*, int sp, double T_vib, uint64_t seed, int64_t n,
                         uint8_t* out_qn);
/* keyed permutation of [0,N) that forms the disjoint NTC pairs */
uint32_t ora_pair_perm(uint32_t x, uint32_t N, const uint32_t key[4]);
void     ora_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* T_vib of one species in a reservoir by the zero-point search (P5) */
double   ora_tvib(ora_ctx*, int res, int sp);
double   ora_mean_sigma_g(ora_ctx*, int sp, int sq, double T);
/* Recombination rates (reading A14).  Nodes T_i = 500 K * 2^(i/32), i < ORA_REC_NODES. */
#define ORA_REC_NODES 225
double   ora_rec_node_T(int i);
/* Regularised upper incomplete gamma Q(a, x) (x <= 0 gives 1) */
double   ora_gamma_q(double a, double x);
/* thermal dissociation probability per collision of recombination rx's molecule A at T */
double   ora_diss_prob(ora_ctx*, int rx, double T);
/* Whitten-Rabinovitch density of states (1/J) of l oscillators with quanta
   hnu (J) at energy E (J) above the ground state */
double   ora_wr_density(const double* hnu, int l, double E);
/* the dissociation probability of recombination rx's molecule A at T by the
   WR sum over n_samp evenly spaced energies below the threshold */
double   ora_diss_prob_wr(ora_ctx*, int rx, double T, int n_samp);
/* equilibrium constant n_B n_C / n_A (m^-3) of recombination rx at T */
double   ora_keq(ora_ctx*, int rx, double T);
/* k_r (m^6/s) of recombination rx with a third body of species spM at node i / at T */
double   ora_rec_rate_node(ora_ctx*, int rx, int spM, int i);
double   ora_rec_rate(ora_ctx*, int rx, int spM, double T);
/* translational temperature of one cell as the collision step computes it */
double   ora_cell_temperature(ora_ctx*, int res, int cell);
const char* ora_last_error(ora_ctx*);

#ifdef __cplusplus
}
#endif
#endif
