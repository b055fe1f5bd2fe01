/*
 * hcao_oracle.c -- TEST INFRASTRUCTURE, not the product.
 *
 * A plain, slow, single-threaded FP64 reference DSMC for the collision phase of
 * the HCAO model ("A harmonically-coupled-anharmonic-oscillator approach for
 * polyatomic chemistry modeling in DSMC").  It is loaded only by the tests, by
 * the smoke check and by the CPU-baseline leg of the benchmark.  It shares no
 * code with the CUDA library; both follow the same written readings of the
 * paper, so that in FP64 every decision can be compared bit for bit.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC (no FMA
 * contraction, IEEE double everywhere).
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   philox            : pinned (published known-answer vectors)
 *   levels            : pinned (Morse closed-form spacing, D_e truncation by
 *                       brute force, harmonic spacing)
 *   K5 table sampler  : pinned (enumerated LB target, chi^2; equals literal P8)
 *   literal P8        : pinned (enumerated LB target, chi^2)
 *   init P6/P7        : pinned (Boltzmann populations, chi^2)
 *   pair_perm         : pinned (bijection, exhaustive; uniform image and partner offsets)
 *   NTC + VHS         : pinned (VHS closed-form collision frequency)
 *   relax + scatter   : pinned (per-collision momentum/energy conservation,
 *                       equilibrium Boltzmann populations, detailed balance)
 *   dissociation      : pinned (single-step probability vs level-sum quadrature)
 *   exchange          : pinned (single-step probability vs level-sum quadrature)
 *   product split     : pinned (reading A13: each product's levels vs the
 *                       enumerated LB target at its budget, Beta(3/2,3/2)
 *                       three-body split, isotropy, conservation; the same
 *                       for the recombination product, reading A14)
 *   T_c product split : pinned (each product's levels vs the enumerated
 *                       target at the exponent the collision temperature
 *                       gives, found independently with scipy; the
 *                       relaxation-table exponent rejected)
 *   recombination     : pinned (Q(a,x) vs scipy, P(T) vs binned convolution
 *                       and level sums, K_eq closed form, rate law)
 *   WR density / P    : pinned (exact harmonic state counts, quadrature for
 *                       one oscillator, convergence)
 *   TCE               : pinned (P(E_c) closed form, the Arrhenius rate from
 *                       the probability's thermal average by quadrature)
 *   competing choice  : pinned (channel frequencies vs E_excess shares)
 *   rotation          : pinned (own log vs libm, Beta fraction, Gamma
 *                       initialisation, equipartition, gamma-coupled
 *                       dissociation probability closed form)
 *   own exp           : pinned (vs libm within 2 ulp)
 *   cell_base split   : pinned (two cell ranges reproduce the whole run)
 */
#include "hcao_oracle.h"
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* SI constants (CODATA 2018 exact values, k_B, h, c). */
#define KB 1.380649e-23
#define HPLANCK 6.62607015e-34
#define CLIGHT 299792458.0
#define PI_D 3.14159265358979323846

/* Philox stream purposes (counter word 3 = purpose << 24 | block). */
enum { PU_NSEL = 1, PU_PERM = 2, PU_PAIR = 3, PU_LB_A = 4, PU_LB_B = 5, PU_SCAT = 6,
       PU_INIT = 7, PU_TEST = 8, PU_REC = 9, PU_TCE = 10, PU_ROT = 11, PU_ROTINIT = 12 };

#define MAX_SPECIES 16
#define MAX_REACTIONS 32
#define MAX_RES 4096
#define MAX_CHANNELS 80
#define TABLE_PAD 17

typedef struct {
    ora_species_desc d;
    int n_modes;
    int is_bend[ORA_MAX_MODES];
    int n_levels[ORA_MAX_MODES];
    double E[ORA_MAX_MODES][ORA_MAX_LEVELS];
    double ktheta[ORA_MAX_MODES];
    double zpe;
    /* K5 tables */
    double base[ORA_MAX_MODES + 1];
    double cq;          /* quadratic grid: g_m = base_k + cq * m^2 */
    double eps_min;     /* smallest single-quantum excitation of any mode */
    int MT;
    double* H[ORA_MAX_MODES];
    double* Hh[ORA_MAX_MODES]; /* the same tables at exponent 1/2 (built for the products of a
                                  reaction that redistributes at the collision temperature) */
    double rot_fmax;    /* rotation: the maximum of the LB fraction's density shape */
} o_species;

typedef struct {
    double v[3];
    int32_t sp;
    uint8_t qn[ORA_MAX_MODES];
    double erot;    /* classical rotational energy, J */
} o_part;

typedef struct {
    int n, cap;
    o_part* p;
    double sgmax;
} o_cell;

typedef struct {
    int n_cells;
    double Vc, w, dt, T_sgmax;
    uint64_t seed;
    uint32_t step;
    uint32_t cell_base;  /* index of the first cell in the random-number keys */
    o_cell* cells;
    uint64_t counters[8 + MAX_REACTIONS];
} o_res;

struct ora_ctx {
    int M;
    double span;
    uint32_t reject_cap;
    int n_species, n_reactions, n_res;
    o_species sp[MAX_SPECIES];
    ora_reaction_desc rx[MAX_REACTIONS];
    double rx_zpesum[MAX_REACTIONS];
    o_res* res[MAX_RES];
    int amode; /* 0: a=0.75, 1: a=1, 2: a=0.5 ; -1 unset */
    double omega;
    int log_on;
    ora_log_rec* log;
    int64_t log_n, log_cap;
    int error;
    char msg[256];
    /* recombination: thermal dissociation probability of A at the rate-table
       nodes, computed when first needed */
    double rec_P[MAX_REACTIONS][ORA_REC_NODES];
    unsigned char rec_P_done[MAX_REACTIONS][ORA_REC_NODES];
    /* TCE reactions: the probability tables per partner species (see
       tce_build), NULL for QK reactions */
    double* tce[MAX_REACTIONS][MAX_SPECIES];
};

static void set_err(ora_ctx* c, int code, const char* m) {
    if (!c->error) c->error = code;
    snprintf(c->msg, sizeof c->msg, "%s", m);
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random numbers:
   as easy as 1, 2, 3"): 10 rounds of two 32x32->64 multiplies with the
   published multipliers and Weyl key increments. */
void ora_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

typedef struct {
    uint32_t key[2];
    uint32_t c0, c1, c2, purpose;
    uint32_t block;
    int word;
    uint32_t buf[4];
} o_stream;

static void st_init(o_stream* s, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                    uint32_t purpose) {
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->c0 = c0; s->c1 = c1; s->c2 = c2; s->purpose = purpose;
    s->block = 0; s->word = 4;
}
static uint32_t st_word(o_stream* s) {
    if (s->word == 4) {
        uint32_t ctr[4] = { s->c0, s->c1, s->c2, (s->purpose << 24) | (s->block & 0xFFFFFFu) };
        ora_philox(ctr, s->key, s->buf);
        s->block++;
        s->word = 0;
    }
    return s->buf[s->word++];
}
/* uniform in [0,1): 27 bits of the first word, 26 of the second, times 2^-53 */
static double st_u01(o_stream* s) {
    uint32_t a = st_word(s) >> 5;
    uint32_t b = st_word(s) >> 6;
    uint64_t m = ((uint64_t)a << 26) | (uint64_t)b;
    return (double)m * 0x1p-53;
}

/* ------------------------------------------------------------------ */
/* Keyed bijection of [0,N) that forms the disjoint NTC pairs (reading A9:
   pair k of a round is (pi(2k), pi(2k+1))).  On b-bit words, b the smallest
   width with 2^b >= N, three rounds of
       x = ((x xor k_r) * M_r) mod 2^b,   x = x xor (x >> ceil(b/2)),
   each a bijection of [0, 2^b) (xor with a constant, multiplication by an
   odd number modulo 2^b, a right xorshift), repeated from the result until it
   falls in [0,N) (cycle walking keeps a bijection of [0,N)).  Round keys:
   the round's key words 0..2; multipliers: the odd constants 0x9E3779B1,
   0x85EBCA6B, 0xC2B2AE35. */
uint32_t ora_pair_perm(uint32_t x, uint32_t N, const uint32_t key[4]) {
    static const uint32_t mult[3] = {0x9E3779B1u, 0x85EBCA6Bu, 0xC2B2AE35u};
    if (N <= 1u) return 0u;
    int b = 1;
    while (((uint64_t)1 << b) < (uint64_t)N) b++;
    uint32_t mask = (uint32_t)(((uint64_t)1 << b) - 1);
    int h = (b + 1) / 2;
    do {
        for (int r = 0; r < 3; ++r) {
            x = ((x ^ (key[r] & mask)) * mult[r]) & mask;
            x = x ^ (x >> h);
        }
    } while (x >= N);
    return x;
}

/* ------------------------------------------------------------------ */
/* LB weight (E_coll - sum E_j)^(xi_rel/2 - 1), xi_rel = 5 - 2 omega:
   exponent 0.75, 1 or 0.5 for omega = 0.75, 0.5, 1 (written with sqrt). */
static double pw_mode(int amode, double x) {
    if (amode == 0) { double s = sqrt(x); return s * sqrt(s); }
    if (amode == 1) return x;
    return sqrt(x);
}
static double pw(const ora_ctx* c, double x) { return pw_mode(c->amode, x); }
/* g^(2 - 2 omega): sigma_T(g) g of the VHS model */
static double gpow(const ora_ctx* c, double g) {
    if (c->amode == 0) return sqrt(g);
    if (c->amode == 1) return g;
    return 1.0;
}

/* ------------------------------------------------------------------ */
/* Levels.  Stretch: Eq. energy-AHO, E(i) = hc we (i+1/2) - hc wexe (i+1/2)^2,
   kept while E(i) < De and E(i) increases (reading A2: we and wexe give the
   levels, De truncates them).  Bend: (i+1/2) k Theta (harmonic, Theta form),
   kept while i < 256 and E(i) < ZPE + table span. */
static void build_levels(ora_ctx* c, o_species* s) {
    const double hc = HPLANCK * CLIGHT;
    int n = s->d.n_stretch + s->d.n_bend;
    s->n_modes = n;
    for (int j = 0; j < s->d.n_stretch; ++j) {
        s->is_bend[j] = 0;
        int L = 0;
        double prev = -1.0;
        for (int i = 0; i < ORA_MAX_LEVELS; ++i) {
            double x = (double)i + 0.5;
            double E = hc * s->d.we[j] * x - hc * s->d.wexe[j] * (x * x);
            if (!(E < s->d.De[j])) break;
            if (i > 0 && !(E > prev)) break;
            s->E[j][L++] = E;
            prev = E;
        }
        s->n_levels[j] = L;
    }
    double zpe_bend = 0.0;
    for (int b = 0; b < s->d.n_bend; ++b) {
        int j = s->d.n_stretch + b;
        s->is_bend[j] = 1;
        s->ktheta[j] = KB * s->d.theta[b];
    }
    /* ZPE: sum of ground levels in mode order */
    double z = 0.0;
    for (int j = 0; j < n; ++j) {
        double e0 = s->is_bend[j] ? 0.5 * s->ktheta[j] : s->E[j][0];
        z = z + e0;
    }
    (void)zpe_bend;
    s->zpe = z;
    double top = z + c->span;
    for (int j = 0; j < n; ++j) {
        if (!s->is_bend[j]) continue;
        int L = 0;
        for (int i = 0; i < ORA_MAX_LEVELS; ++i) {
            double E = ((double)i + 0.5) * s->ktheta[j];
            if (!(E < top)) break;
            s->E[j][L++] = E;
        }
        s->n_levels[j] = L;
    }
}

/* K5 tables (reading A5).  H_k(g) bounds from above the LB weight sum of modes
   k..n-1 at budget g, on the quadratic grid g_m = base_k + cq m^2 (cq = span /
   M^2), base_k = sum_{j>=k} E_j(0):
     H_{n-1}(g) = sum_i pw(g - E_{n-1,i}),   H_k(g) = sum_i W_{k+1}(g - E_{k,i}),
     W_k(E) = H_k[idx_k(E)], idx_k(E) = the smallest m >= 1 with g_m >= E (0 if
   E <= base_k; MT if no grid point reaches E).  Found by bisection. */
static double grid_pt(const o_species* s, int k, int64_t m) {
    return s->base[k] + s->cq * (double)(m * m);
}
static int64_t grid_idx(const o_species* s, int k, double E) {
    if (!(E > s->base[k])) return 0;
    if (grid_pt(s, k, s->MT - 1) < E) return s->MT;
    int64_t lo = 0, hi = s->MT - 1; /* g_lo < E <= g_hi */
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (grid_pt(s, k, mid) < E) lo = mid; else hi = mid;
    }
    return hi;
}
static double W_tab(const o_species* s, double* const* H, int k, double E) {
    int64_t m = grid_idx(s, k, E);
    if (m == 0) return 0.0;
    if (m > s->MT - 1) m = s->MT - 1; /* only reached by table entries never queried */
    return H[k][m];
}
/* The tables H (s->H at the context's exponent, amode = c->amode; s->Hh at
   exponent 1/2, amode 2) on the species' grid. */
static int fill_tables(const o_species* s, int amode, double** H) {
    int n = s->n_modes;
    for (int k = n - 1; k >= 0; --k) {
        H[k] = (double*)malloc(sizeof(double) * (size_t)s->MT);
        if (!H[k]) return -1;
        for (int m = 0; m < s->MT; ++m) {
            double g = grid_pt(s, k, m);
            double sum = 0.0;
            for (int i = 0; i < s->n_levels[k]; ++i) {
                if (!(s->E[k][i] < g)) break;
                double x = g - s->E[k][i];
                double w = (k == n - 1) ? pw_mode(amode, x) : W_tab(s, H, k + 1, x);
                sum = sum + w;
            }
            H[k][m] = sum;
        }
    }
    return 0;
}
static int build_tables(ora_ctx* c, o_species* s) {
    int n = s->n_modes;
    if (n == 0) return 0;
    s->base[n] = 0.0;
    for (int k = n - 1; k >= 0; --k) s->base[k] = s->E[k][0] + s->base[k + 1];
    s->cq = c->span / ((double)c->M * (double)c->M);
    s->MT = c->M + TABLE_PAD;
    s->eps_min = INFINITY;
    for (int j = 0; j < n; ++j)
        if (s->n_levels[j] > 1 && s->E[j][1] - s->E[j][0] < s->eps_min) s->eps_min = s->E[j][1] - s->E[j][0];
    return fill_tables(s, c->amode, s->H);
}

static double evib(const o_species* s, const uint8_t* qn) {
    double e = 0.0;
    for (int j = 0; j < s->n_modes; ++j) e = e + s->E[j][qn[j]];
    return e;
}

/* ------------------------------------------------------------------ */
/* Samplers of the post-collision vibrational state at collision energy Ec.
   Target (relaxation step of the HCAO model, the joint acceptance of all
   modes): p(i) proportional to (Ec - sum_j E_j(i_j))^(xi_rel/2-1) over states
   with sum_j E_j(i_j) < Ec.  Return: 0 new state, 1 table overflow (state
   kept), 2 degenerate Ec (A6, state kept), -1 rejection cap (state kept). */
enum { S_OK = 0, S_OVER = 1, S_DEGEN = 2, S_CAP = -1 };

/* K5: sequential draw through the H tables; a draw that runs past the end of a
   mode's level list restarts the trial.  Accepted states follow the target
   exactly (each trial's acceptance probability is pw(..)/H_0).  Below the
   smallest single-quantum excitation only the ground state has sum E < Ec, so
   it is taken without a draw. */
static int sample_table_with(ora_ctx* c, const o_species* s, int amode, double* const* H, double Ec,
                             o_stream* st, uint8_t* qn_out, uint64_t* trials) {
    int n = s->n_modes;
    if (n == 0) return S_OK;
    int64_t m0 = grid_idx(s, 0, Ec);
    if (m0 > c->M) return S_OVER;
    if (m0 == 0 || !(H[0][m0] > 0.0)) return S_DEGEN;
    if (Ec - s->base[0] < s->eps_min) {
        memset(qn_out, 0, (size_t)n);
        return S_OK;
    }
    uint8_t qn[ORA_MAX_MODES];
    for (uint32_t trial = 0; trial < c->reject_cap; ++trial) {
        if (trials) (*trials)++;
        double E = Ec;
        int ok = 1;
        for (int k = 0; k < n; ++k) {
            int64_t m = (k == 0) ? m0 : grid_idx(s, k, E);
            double u = st_u01(st);
            double t = u * H[k][m];
            double cum = 0.0;
            int sel = -1;
            for (int i = 0; i < s->n_levels[k]; ++i) {
                if (!(s->E[k][i] < E)) break;
                double x = E - s->E[k][i];
                double w = (k == n - 1) ? pw_mode(amode, x) : W_tab(s, H, k + 1, x);
                cum = cum + w;
                if (t < cum) { sel = i; break; }
            }
            if (sel < 0) { ok = 0; break; }
            qn[k] = (uint8_t)sel;
            E = E - s->E[k][sel];
        }
        if (ok) {
            memcpy(qn_out, qn, (size_t)n);
            return S_OK;
        }
    }
    return S_CAP;
}
static int sample_table(ora_ctx* c, const o_species* s, double Ec, o_stream* st, uint8_t* qn_out,
                        uint64_t* trials) {
    return sample_table_with(c, s, c->amode, s->H, Ec, st, qn_out, trials);
}

/* Literal P8 (distribution reference): each mode drawn uniformly below Ec
   (bend: i_max = floor(Ec/(k Theta) - 1/2) + 1, i = floor(r i_max); stretch:
   i_max = highest level below Ec, i = floor(r (i_max+1)), reading A4), then
   all modes accepted jointly if r < pw(Ec - sum E)/pw(Ec - ZPE). */
static int sample_literal(ora_ctx* c, const o_species* s, double Ec, o_stream* st,
                          uint8_t* qn_out, uint64_t* trials) {
    int n = s->n_modes;
    if (n == 0) return S_OK;
    if (!(Ec > s->zpe)) return S_DEGEN;
    double denom = pw(c, Ec - s->zpe);
    uint8_t qn[ORA_MAX_MODES];
    for (uint32_t trial = 0; trial < c->reject_cap; ++trial) {
        if (trials) (*trials)++;
        double Esum = 0.0;
        int bad = 0;
        for (int j = 0; j < n; ++j) {
            double u = st_u01(st);
            int i;
            if (s->is_bend[j]) {
                int imax = (int)floor(Ec / s->ktheta[j] - 0.5) + 1;
                i = (int)floor(u * (double)imax);
            } else {
                int imax = 0;
                for (int l = 0; l < s->n_levels[j]; ++l)
                    if (s->E[j][l] < Ec) imax = l;
                i = (int)floor(u * (double)(imax + 1));
            }
            if (i >= s->n_levels[j]) { bad = 1; i = 0; }
            qn[j] = (uint8_t)i;
            Esum = Esum + s->E[j][i];
        }
        double u = st_u01(st);
        if (!bad && Esum < Ec && u < pw(c, Ec - Esum) / denom) {
            memcpy(qn_out, qn, (size_t)n);
            return S_OK;
        }
    }
    return S_CAP;
}

/* Initial quantum numbers at T_vib (P6 bends, P7 stretches with reading A7:
   i = floor(r (i_diss+1)), accepted if r < exp(-(E_i - E_0)/(k T_vib))).  A bend
   draw beyond the level list is redrawn (Boltzmann over the finite set). */
static int sample_init(ora_ctx* c, const o_species* s, double T, o_stream* st, uint8_t* qn) {
    for (int j = 0; j < s->n_modes; ++j) {
        int done = 0;
        for (uint32_t t = 0; t < c->reject_cap && !done; ++t) {
            if (s->is_bend[j]) {
                double u = st_u01(st);
                double x = floor(-log(u) * T / s->d.theta[j - s->d.n_stretch]);
                if (x < (double)s->n_levels[j]) { qn[j] = (uint8_t)x; done = 1; }
            } else {
                double u1 = st_u01(st);
                int i = (int)floor(u1 * (double)s->n_levels[j]);
                double u2 = st_u01(st);
                if (u2 < exp(-(s->E[j][i] - s->E[j][0]) / (KB * T))) { qn[j] = (uint8_t)i; done = 1; }
            }
        }
        if (!done) return S_CAP;
    }
    return S_OK;
}

/* ------------------------------------------------------------------ */
/* VHS pair constants (Bird's VHS model, cited for xi_rel = 5 - 2 omega):
   sigma_T(g) g = C g^(2-2 omega),
   C = pi d^2 (2 k T_ref / m_r)^(omega - 1/2) / Gamma(5/2 - omega),
   d and T_ref the means of the two species'.  Mean over a Maxwellian at T:
   <sigma_T g> = 2 d^2 sqrt(2 pi k T_ref / m_r) (T/T_ref)^(1-omega). */
typedef struct { double mr, C, mt, fp, fq; } o_pair;
static o_pair pair_consts(const ora_ctx* c, int a, int b) {
    const ora_species_desc* A = &c->sp[a].d;
    const ora_species_desc* B = &c->sp[b].d;
    o_pair p;
    p.mr = A->mass * B->mass / (A->mass + B->mass);
    double d = 0.5 * (A->d_ref + B->d_ref);
    double Tr = 0.5 * (A->T_ref + B->T_ref);
    p.C = PI_D * d * d * pow(2.0 * KB * Tr / p.mr, c->omega - 0.5) / tgamma(2.5 - c->omega);
    p.mt = A->mass + B->mass;
    p.fp = B->mass / p.mt; /* velocity share of particle a in the relative motion */
    p.fq = A->mass / p.mt;
    return p;
}
double ora_mean_sigma_g(ora_ctx* c, int a, int b, double T) {
    const ora_species_desc* A = &c->sp[a].d;
    const ora_species_desc* B = &c->sp[b].d;
    double mr = A->mass * B->mass / (A->mass + B->mass);
    double d = 0.5 * (A->d_ref + B->d_ref);
    double Tr = 0.5 * (A->T_ref + B->T_ref);
    return 2.0 * d * d * sqrt(2.0 * PI_D * KB * Tr / mr) * pow(T / Tr, 1.0 - c->omega);
}

/* ------------------------------------------------------------------ */
/* Recombination B + C + M -> A + M (Sec. "Recombination reactions").
   The rate coefficient is k_r = k_f / K_eq.  k_f is the forward (dissociation)
   rate of the paper's expression, P times the VHS collision-rate coefficient
   of A and M; P is the thermal average, over every vibrational level
   combination of A, of the probability that the collision-weighted VHS
   translational energy exceeds what the state lacks of the dissociation
   threshold (Eq. recomb-correct), with Gamma_inc the regularised upper
   incomplete gamma Q(5/2 - omega, .) (reading A16).  Readings (A14):
     - the threshold is the one the QK test applies, D = min over the
       breaking stretches j of (D_e,j + ZPE_A + ZPE_B + ZPE_C - E_j(0)), so
       that k_f is the rate the simulated dissociation produces;
     - the collision-rate factor is <sigma_T g>_{A,M}(T) for every M (no 1/2
       for M = A: either partner of an A-A pair may dissociate);
     - K_eq = n_B n_C / n_A from translational and HCAO vibrational
       partition sums (level sums over the tabulated levels, no rotation);
     - k_r is tabulated at T_i = 500 K * 2^(i/32) and interpolated linearly
       in T (clamped at the ends). */

double ora_rec_node_T(int i) { return 500.0 * pow(2.0, (double)i / 32.0); }

/* Q(a, x) = Gamma(a, x) / Gamma(a): for x < a + 1 as 1 - P(a, x) with the
   power series of P (Abramowitz & Stegun 6.5.29), otherwise the Legendre
   continued fraction of Q (A&S 6.5.31) evaluated by the modified Lentz
   method. */
double ora_gamma_q(double a, double x) {
    if (!(x > 0.0)) return 1.0;
    double lpre = a * log(x) - x - lgamma(a);
    if (x < a + 1.0) {
        double term = 1.0 / a, sum = term, an = a;
        for (int n = 1; n < 10000; ++n) {
            an += 1.0;
            term *= x / an;
            sum += term;
            if (fabs(term) < fabs(sum) * 1e-17) break;
        }
        return 1.0 - sum * exp(lpre);
    }
    const double tiny = 1e-300;
    double b = x + 1.0 - a;
    double C = 1.0 / tiny, D = 1.0 / b, h = D;
    for (int i = 1; i < 10000; ++i) {
        double an = -(double)i * ((double)i - a);
        b += 2.0;
        D = an * D + b;
        if (fabs(D) < tiny) D = tiny;
        C = b + an / C;
        if (fabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        double del = D * C;
        h *= del;
        if (fabs(del - 1.0) < 1e-17) break;
    }
    return exp(lpre) * h;
}

/* The recombination's molecule A and its QK dissociation threshold. */
static double rec_threshold(const ora_ctx* c, int rx) {
    const ora_reaction_desc* r = &c->rx[rx];
    const o_species* sA = &c->sp[r->products[0]];
    double D = INFINITY;
    for (int j = 0; j < sA->d.n_stretch; ++j) {
        if (!((r->diss_mode_mask >> j) & 1u)) continue;
        double Dj = (sA->d.De[j] + c->rx_zpesum[rx]) - sA->E[j][0];
        if (Dj < D) D = Dj;
    }
    return D;
}

/* Sum over the level combinations of modes k..n-1 given the excitation X of
   modes 0..k-1 (excitations x = E - E(0), so the ground state has X = 0):
   states below the threshold Dx contribute exp(-X/kT) Q(a, (Dx - X)/kT);
   every completion at or above it contributes exp(-X/kT), and once X >= Dx
   those completions are summed at once as exp(-X/kT) times the partition
   sums of the remaining modes (zr[k]); within a mode the levels increase,
   so the first level that reaches Dx starts a suffix summed by zs. */
typedef struct {
    const o_species* s;
    double kT, a, Dx;
    double zr[ORA_MAX_MODES + 1];        /* prod_{j >= k} sum_i exp(-x_ji / kT) */
    double zs[ORA_MAX_MODES][ORA_MAX_LEVELS + 1];  /* suffix sums per mode */
} o_penum;

static double penum(const o_penum* pe, int k, double X) {
    const o_species* s = pe->s;
    if (k == s->n_modes) return exp(-X / pe->kT) * ora_gamma_q(pe->a, (pe->Dx - X) / pe->kT);
    double sum = 0.0;
    for (int i = 0; i < s->n_levels[k]; ++i) {
        double Xi = X + (s->E[k][i] - s->E[k][0]);
        if (!(Xi < pe->Dx)) {
            sum += exp(-X / pe->kT) * pe->zs[k][i] * pe->zr[k + 1];
            break;
        }
        sum += penum(pe, k + 1, Xi);
    }
    return sum;
}

double ora_diss_prob(ora_ctx* c, int rx, double T) {
    const o_species* s = &c->sp[c->rx[rx].products[0]];
    o_penum* pe = (o_penum*)malloc(sizeof(o_penum));
    pe->s = s;
    pe->kT = KB * T;
    pe->a = 2.5 - c->omega;
    pe->Dx = rec_threshold(c, rx) - s->zpe;
    int n = s->n_modes;
    pe->zr[n] = 1.0;
    for (int k = n - 1; k >= 0; --k) {
        double acc = 0.0;
        pe->zs[k][s->n_levels[k]] = 0.0;
        for (int i = s->n_levels[k] - 1; i >= 0; --i) {
            acc += exp(-(s->E[k][i] - s->E[k][0]) / pe->kT);
            pe->zs[k][i] = acc;
        }
        pe->zr[k] = pe->zr[k + 1] * acc;
    }
    double P = penum(pe, 0, 0.0) / pe->zr[0];
    free(pe);
    return P;
}

/* Whitten-Rabinovitch density of vibrational states (the approximation the
   paper gives beside Eq. recomb-correct) of l oscillators with quanta hnu[k]
   (J) at energy E (J) above the ground state:
     rho(E) = [E + a(E) E_z]^(l-1) / ((l-1)! prod_k hnu_k),  a = 1 - beta Omega,
     E_z = sum_k hnu_k / 2,  beta = (l-1)^2 sum_k hnu_k^2 / (l (sum_k hnu_k)^2),
     Omega = 10^(-1.0506 (E/E_z)^(1/4)) for E >= E_z,
     1/Omega = 5 (E/E_z) + 2.73 (E/E_z)^(1/2) + 3.51 for E < E_z.
   Readings: the logarithm of the Omega correlation is decadic; E_z is the
   harmonic zero-point energy of the fundamentals. */
static double wr_a(const double* hnu, int l, double E) {
    double Ez = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < l; ++k) {
        Ez += 0.5 * hnu[k];
        s1 += hnu[k];
        s2 += hnu[k] * hnu[k];
    }
    const double beta = ((double)(l - 1) * (double)(l - 1)) * s2 / ((double)l * s1 * s1);
    const double x = E / Ez;
    const double Om = x >= 1.0 ? pow(10.0, -1.0506 * pow(x, 0.25)) : 1.0 / (5.0 * x + 2.73 * sqrt(x) + 3.51);
    return 1.0 - beta * Om;
}

double ora_wr_density(const double* hnu, int l, double E) {
    double Ez = 0.0, lden = 0.0;
    for (int k = 0; k < l; ++k) {
        Ez += 0.5 * hnu[k];
        lden += log(hnu[k]);
    }
    lden += lgamma((double)l);  /* log (l-1)! */
    return exp((double)(l - 1) * log(E + wr_a(hnu, l, E) * Ez) - lden);
}

/* The recombination's P by the WR sum: n_samp energies evenly spaced between
   the ground state and the threshold Dx above it, at the midpoints
   E_i = (i - 1/2) Dx / n_samp (reading), weighted rho(E_i) exp(-E_i/kT);
   P = sum_i Q(5/2 - omega, (Dx - E_i)/kT) w_i / sum_i w_i.  The quanta are
   the fundamentals E_j(1) - E_j(0) of A's modes (harmonic for bends,
   anharmonic for stretches).  The constant factor of rho cancels. */
double ora_diss_prob_wr(ora_ctx* c, int rx, double T, int n_samp) {
    const o_species* s = &c->sp[c->rx[rx].products[0]];
    const int l = s->n_modes;
    if (l < 1 || n_samp < 1) return NAN;
    double hnu[ORA_MAX_MODES], Ez = 0.0;
    for (int j = 0; j < l; ++j) {
        hnu[j] = s->E[j][1] - s->E[j][0];
        Ez += 0.5 * hnu[j];
    }
    const double kT = KB * T, a = 2.5 - c->omega;
    const double Dx = rec_threshold(c, rx) - s->zpe;
    if (!(Dx > 0.0)) return 1.0;
    /* log weights first, then the sums relative to their largest */
    double* lw = (double*)malloc(sizeof(double) * (size_t)n_samp);
    double mx = -INFINITY;
    for (int i = 0; i < n_samp; ++i) {
        const double E = ((double)i + 0.5) * Dx / (double)n_samp;
        lw[i] = (double)(l - 1) * log(E + wr_a(hnu, l, E) * Ez) - E / kT;
        if (lw[i] > mx) mx = lw[i];
    }
    double num = 0.0, den = 0.0;
    for (int i = 0; i < n_samp; ++i) {
        const double E = ((double)i + 0.5) * Dx / (double)n_samp;
        const double w = exp(lw[i] - mx);
        num += ora_gamma_q(a, (Dx - E) / kT) * w;
        den += w;
    }
    free(lw);
    return num / den;
}

/* vibrational partition sum with energies measured from the ground state */
static double zvib_x(const o_species* s, double T) {
    double z = 1.0;
    for (int j = 0; j < s->n_modes; ++j) {
        double m = 0.0;
        for (int i = 0; i < s->n_levels[j]; ++i) m += exp(-(s->E[j][i] - s->E[j][0]) / (KB * T));
        z *= m;
    }
    return z;
}

double ora_keq(ora_ctx* c, int rx, double T) {
    const ora_reaction_desc* r = &c->rx[rx];
    const o_species* sA = &c->sp[r->products[0]];
    const o_species* sB = &c->sp[r->reactants[0]];
    const o_species* sC = &c->sp[r->reactants[1]];
    /* translational partition functions per unit volume, (2 pi m k T / h^2)^(3/2) */
    double f = 2.0 * PI_D * KB * T / (HPLANCK * HPLANCK);
    double qtr = pow(f * sB->d.mass, 1.5) * pow(f * sC->d.mass, 1.5) / pow(f * sA->d.mass, 1.5);
    /* ground-state energies from the well bottoms, formation energies included */
    double dE0 = (sB->d.E_form + sB->zpe + sC->d.E_form + sC->zpe) - (sA->d.E_form + sA->zpe);
    return qtr * (zvib_x(sB, T) * zvib_x(sC, T) / zvib_x(sA, T)) * exp(-dE0 / (KB * T));
}

double ora_rec_rate_node(ora_ctx* c, int rx, int spM, int i) {
    double T = ora_rec_node_T(i);
    if (!c->rec_P_done[rx][i]) {
        /* P of Eq. recomb-correct: the exact level sum, or its sampled WR form */
        const ora_reaction_desc* r = &c->rx[rx];
        c->rec_P[rx][i] = r->model == ORA_RPROB_WR
                              ? ora_diss_prob_wr(c, rx, T, r->wr_samples > 0 ? r->wr_samples : 1000)
                              : ora_diss_prob(c, rx, T);
        c->rec_P_done[rx][i] = 1;
    }
    double kf = c->rec_P[rx][i] * ora_mean_sigma_g(c, c->rx[rx].products[0], spM, T);
    return kf / ora_keq(c, rx, T);
}

double ora_rec_rate(ora_ctx* c, int rx, int spM, double T) {
    const int last = ORA_REC_NODES - 1;
    if (!(T > ora_rec_node_T(0))) return ora_rec_rate_node(c, rx, spM, 0);
    if (!(T < ora_rec_node_T(last))) return ora_rec_rate_node(c, rx, spM, last);
    int lo = 0, hi = last; /* T_lo <= T < T_hi */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (ora_rec_node_T(mid) <= T) lo = mid; else hi = mid;
    }
    double T0 = ora_rec_node_T(lo), T1 = ora_rec_node_T(hi);
    double f = (T - T0) / (T1 - T0);
    double k0 = ora_rec_rate_node(c, rx, spM, lo), k1 = ora_rec_rate_node(c, rx, spM, hi);
    return k0 + f * (k1 - k0);
}

/* ------------------------------------------------------------------ */
/* The total-collision-energy (TCE) model, the paper's comparison model
   (Sec. "Polyatomic QK reaction modeling", Eq. arrhenius): a reaction with
   the Arrhenius rate coefficient k(T) = A T^b exp(-E_a/kT) occurs in a
   collision of total energy E_c with probability
       P(E_c) = C1 (E_c - E_a)^(zeta + b + 1/2) / E_c^(zeta + 3/2 - omega)
   (0 below E_a), the form whose average over the collision-energy
   distribution of a VHS gas at equilibrium -- E_c = E_tr + E_int with E_tr
   ~ Gamma(5/2 - omega) and E_int ~ Gamma(zeta), in units of kT -- is
   eps k(T) / <sigma_T g>(T).  Integrating gives
       C1 = eps A k^(1 - omega - b) Gamma(zeta + 5/2 - omega) /
            (Gamma(zeta + b + 3/2) C_sigma),
   with <sigma_T g>(T) = C_sigma T^(1 - omega) and eps = 2 for a pair of
   like species (each collision counted once), 1 otherwise.  Readings:
     - zeta (tce_zeta) is the number of internal degrees of freedom of the
       pair, halved, whose energy counts in E_c: 0 takes the relative
       translational energy alone; otherwise E_c adds both partners'
       vibrational energy above their zero-point energy;
     - P above 1 is taken as 1;
     - P is tabulated per partner species at x_i = X (i/NT)^2 above E_a,
       i = 0..NT (NT = 4096, X = the sampler span), and interpolated linearly
       in s = sqrt(x/X) (the table's own variable), constant beyond X;
     - TCE reactions are tested before the QK channels, in reaction order,
       with one uniform of their own stream laid against the running sum of
       their probabilities; a dissociation by TCE breaks the first stretch
       of its mask (the products do not depend on which). */
#define TCE_NT 4096
static int tce_build(ora_ctx* c, int r) {
    const ora_reaction_desc* d = &c->rx[r];
    const double A = d->arrhenius[0], b = d->arrhenius[1], Ea = d->arrhenius[2], z = d->tce_zeta;
    const double w = c->omega;
    if (!(z >= 0.0) || !(z + b + 1.5 > 0.0) || !(A >= 0.0) || !(Ea >= 0.0)) return ORA_EINVAL;
    const int a = d->reactants[0];
    for (int m = 0; m < c->n_species; ++m) {
        if (d->type == ORA_EXCH && m != d->reactants[1]) continue;
        const ora_species_desc* SA = &c->sp[a].d;
        const ora_species_desc* SM = &c->sp[m].d;
        const double Tr = 0.5 * (SA->T_ref + SM->T_ref);
        const double Csig = ora_mean_sigma_g(c, a, m, Tr) / pow(Tr, 1.0 - w);
        const double eps = m == a ? 2.0 : 1.0;
        const double C1 = eps * A * pow(KB, 1.0 - w - b) * exp(lgamma(z + 2.5 - w) - lgamma(z + b + 1.5)) / Csig;
        const double beta = z + b + 0.5, gam = z + 1.5 - w;
        double* t = (double*)malloc(sizeof(double) * (TCE_NT + 1));
        if (!t) return ORA_ENOMEM;
        for (int i = 0; i <= TCE_NT; ++i) {
            const double sv = (double)i / (double)TCE_NT;
            const double x = c->span * (sv * sv);
            double P = x > 0.0 ? C1 * pow(x, beta) * pow(Ea + x, -gam) : 0.0;
            t[i] = P < 1.0 ? P : 1.0;
        }
        c->tce[r][m] = t;
    }
    return ORA_OK;
}

/* TCE probability of reaction r for a pair whose partner has species m at
   collision energy Ec (linear interpolation in s = sqrt(x/X)) */
static double tce_prob(const ora_ctx* c, int r, int m, double Ec) {
    const double* t = c->tce[r][m];
    if (!t) return 0.0;
    const double x = Ec - c->rx[r].arrhenius[2];
    if (!(x > 0.0)) return 0.0;
    const double sv = sqrt(x / c->span);
    if (!(sv < 1.0)) return t[TCE_NT];
    const double tt = sv * (double)TCE_NT;
    const int i = (int)tt;
    const double f = tt - (double)i;
    return t[i] + f * (t[i + 1] - t[i]);
}

double ora_tce_prob(ora_ctx* c, int r, int m, double Ec) { return tce_prob(c, r, m, Ec); }

/* ------------------------------------------------------------------ */
ora_ctx* ora_create(int table_points, double table_span_J, uint32_t reject_cap) {
    ora_ctx* c = (ora_ctx*)calloc(1, sizeof(ora_ctx));
    if (!c) return NULL;
    c->M = table_points;
    c->span = table_span_J;
    c->reject_cap = reject_cap;
    c->amode = -1;
    return c;
}
void ora_destroy(ora_ctx* c) {
    if (!c) return;
    for (int r = 0; r < MAX_REACTIONS; ++r)
        for (int m = 0; m < MAX_SPECIES; ++m) free(c->tce[r][m]);
    for (int i = 0; i < c->n_species; ++i)
        for (int k = 0; k < ORA_MAX_MODES; ++k) { free(c->sp[i].H[k]); free(c->sp[i].Hh[k]); }
    for (int r = 0; r < c->n_res; ++r) {
        o_res* R = c->res[r];
        for (int j = 0; j < R->n_cells; ++j) free(R->cells[j].p);
        free(R->cells);
        free(R);
    }
    free(c->log);
    free(c);
}
const char* ora_last_error(ora_ctx* c) { return c->msg; }

int ora_add_species(ora_ctx* c, const ora_species_desc* d) {
    if (c->n_species >= MAX_SPECIES) return ORA_EINVAL;
    if (d->n_stretch + d->n_bend > ORA_MAX_MODES) return ORA_EINVAL;
    int am;
    if (d->omega == 0.75) am = 0; else if (d->omega == 0.5) am = 1; else if (d->omega == 1.0) am = 2;
    else return ORA_EINVAL;
    if (c->amode >= 0 && c->amode != am) return ORA_EINVAL;
    c->amode = am;
    c->omega = d->omega;
    o_species* s = &c->sp[c->n_species];
    memset(s, 0, sizeof *s);
    s->d = *d;
    build_levels(c, s);
    for (int j = 0; j < s->n_modes; ++j)
        if (s->n_levels[j] < 1) return ORA_EINVAL;
    if (build_tables(c, s)) return ORA_ENOMEM;
    if (d->rot_dof != 0 && d->rot_dof != 2 && d->rot_dof != 3) return ORA_EINVAL;
    if (d->rot_dof == 2) {
        s->rot_fmax = 1.0;  /* (1 - x)^(3/2 - omega) is largest at x = 0 */
    } else if (d->rot_dof == 3) {
        /* x^(1/2) (1 - x)^(3/2 - omega) peaks at x = 1/2 / (1/2 + 3/2 - omega) */
        const double bb = 1.5 - c->omega;
        const double xs = 0.5 / (0.5 + bb);
        s->rot_fmax = sqrt(xs) * pow(1.0 - xs, bb);
    }
    return c->n_species++;
}

int ora_add_reaction(ora_ctx* c, const ora_reaction_desc* r) {
    if (c->n_reactions >= MAX_REACTIONS) return ORA_EINVAL;
    int id = c->n_reactions;
    c->rx[id] = *r;
    if (r->type == ORA_DISS) {
        /* Eq. Ecoll-diss: the ZPEs of A, B and C are subtracted */
        c->rx_zpesum[id] = c->sp[r->reactants[0]].zpe + c->sp[r->products[0]].zpe +
                           c->sp[r->products[1]].zpe;
    } else if (r->type == ORA_RECOMB) {
        /* the reverse dissociation A + M -> B + C + M sets the threshold of P */
        int A = r->products[0], B = r->reactants[0], Cc = r->reactants[1];
        if (A < 0 || A >= c->n_species || B < 0 || B >= c->n_species || Cc < 0 ||
            Cc >= c->n_species || c->sp[A].d.n_stretch == 0 ||
            (r->diss_mode_mask & ((1u << c->sp[A].d.n_stretch) - 1u)) == 0u)
            return ORA_EINVAL;
        c->rx_zpesum[id] = c->sp[A].zpe + c->sp[B].zpe + c->sp[Cc].zpe;
    } else {
        c->rx_zpesum[id] = 0.0;
    }
    if (r->type != ORA_RECOMB && r->model == ORA_MODEL_TCE) {
        int e = tce_build(c, id);
        if (e != ORA_OK) return e;
    }
    if (r->prod_split == ORA_SPLIT_TCOLL) {
        for (int k = 0; k < 2; ++k) {
            const int p = r->products[k];
            if (p < 0 || p >= c->n_species) continue;
            o_species* sp = &c->sp[p];
            if (sp->n_modes == 0 || sp->Hh[0]) continue;
            if (fill_tables(sp, 2, sp->Hh)) return ORA_ENOMEM;
        }
    } else if (r->prod_split != ORA_SPLIT_RELAX) {
        return ORA_EINVAL;
    }
    return c->n_reactions++;
}

int ora_add_reservoir(ora_ctx* c, int n_cells, double Vc, double w, double dt,
                      uint64_t seed, double T_sgmax) {
    if (c->n_res >= MAX_RES || n_cells < 1) return ORA_EINVAL;
    o_res* R = (o_res*)calloc(1, sizeof(o_res));
    R->n_cells = n_cells;
    R->Vc = Vc; R->w = w; R->dt = dt; R->seed = seed; R->T_sgmax = T_sgmax;
    R->cells = (o_cell*)calloc((size_t)n_cells, sizeof(o_cell));
    c->res[c->n_res] = R;
    return c->n_res++;
}

static void cell_push(o_cell* cl, const o_part* p) {
    if (cl->n == cl->cap) {
        cl->cap = cl->cap ? 2 * cl->cap : 16;
        cl->p = (o_part*)realloc(cl->p, sizeof(o_part) * (size_t)cl->cap);
    }
    cl->p[cl->n++] = *p;
}

/* Load: particles go to their cells in input order (a stable counting sort by
   cell).  (sigma g)_max starts at 2 <sigma_T g>(T_sgmax), the largest over the
   species pairs present (reading A10). */
int ora_load(ora_ctx* c, int res, int64_t n, const double* v, const uint8_t* qn,
             const int32_t* species, const int32_t* cell) {
    o_res* R = c->res[res];
    int present[MAX_SPECIES] = {0};
    for (int64_t i = 0; i < n; ++i) {
        if (cell[i] < 0 || cell[i] >= R->n_cells) return ORA_EINVAL;
        if (species[i] < 0 || species[i] >= c->n_species) return ORA_EINVAL;
        o_part p;
        memset(&p, 0, sizeof p);
        p.v[0] = v[3 * i]; p.v[1] = v[3 * i + 1]; p.v[2] = v[3 * i + 2];
        p.sp = species[i];
        memcpy(p.qn, qn + 16 * i, 16);
        cell_push(&R->cells[cell[i]], &p);
        present[species[i]] = 1;
    }
    double mx = 0.0;
    for (int a = 0; a < c->n_species; ++a)
        for (int b = 0; b < c->n_species; ++b)
            if (present[a] && present[b]) {
                double m = ora_mean_sigma_g(c, a, b, R->T_sgmax);
                if (m > mx) mx = m;
            }
    for (int j = 0; j < R->n_cells; ++j) R->cells[j].sgmax = 2.0 * mx;
    return 0;
}

static double rot_fraction(const ora_ctx* c, const o_species* s, o_stream* st);
static double rot_init_energy(const o_species* s, double kT, o_stream* st);

int ora_init_rotation(ora_ctx* c, int res, double T_rot) {
    if (res < 0 || res >= c->n_res || !(T_rot >= 0.0)) return ORA_EINVAL;
    o_res* R = c->res[res];
    for (int j = 0; j < R->n_cells; ++j) {
        o_cell* cl = &R->cells[j];
        for (int i = 0; i < cl->n; ++i) {
            const o_species* s = &c->sp[cl->p[i].sp];
            cl->p[i].erot = 0.0;
            if (s->d.rot_dof == 0 || T_rot == 0.0) continue;
            o_stream st;
            st_init(&st, R->seed, 0xFFFFFFFEu, R->cell_base + (uint32_t)j, (uint32_t)i, PU_ROTINIT);
            cl->p[i].erot = rot_init_energy(s, KB * T_rot, &st);
        }
    }
    return 0;
}

int ora_load_erot(ora_ctx* c, int res, const double* erot) {
    if (res < 0 || res >= c->n_res) return ORA_EINVAL;
    o_res* R = c->res[res];
    int64_t o = 0;
    for (int j = 0; j < R->n_cells; ++j)
        for (int i = 0; i < R->cells[j].n; ++i, ++o)
            R->cells[j].p[i].erot = c->sp[R->cells[j].p[i].sp].d.rot_dof ? erot[o] : 0.0;
    return 0;
}

int ora_read_erot(ora_ctx* c, int res, double* erot) {
    if (res < 0 || res >= c->n_res) return ORA_EINVAL;
    o_res* R = c->res[res];
    int64_t o = 0;
    for (int j = 0; j < R->n_cells; ++j)
        for (int i = 0; i < R->cells[j].n; ++i, ++o) erot[o] = R->cells[j].p[i].erot;
    return 0;
}

int ora_sample_rot_fraction(ora_ctx* c, int sp, uint64_t seed, int64_t n, double* out) {
    if (sp < 0 || sp >= c->n_species || c->sp[sp].d.rot_dof == 0) return ORA_EINVAL;
    for (int64_t i = 0; i < n; ++i) {
        o_stream st;
        st_init(&st, seed, (uint32_t)i, (uint32_t)(i >> 32), 0u, PU_ROT);
        out[i] = rot_fraction(c, &c->sp[sp], &st);
    }
    return 0;
}

int ora_set_cell_base(ora_ctx* c, int res, uint32_t base) {
    if (res < 0 || res >= c->n_res) return ORA_EINVAL;
    c->res[res]->cell_base = base;
    return 0;
}

int ora_init_vibration(ora_ctx* c, int res, double T_vib) {
    o_res* R = c->res[res];
    for (int j = 0; j < R->n_cells; ++j) {
        o_cell* cl = &R->cells[j];
        for (int i = 0; i < cl->n; ++i) {
            o_stream st;
            st_init(&st, R->seed, 0xFFFFFFFFu, R->cell_base + (uint32_t)j, (uint32_t)i, PU_INIT);
            const o_species* s = &c->sp[cl->p[i].sp];
            memset(cl->p[i].qn, 0, 16);
            if (sample_init(c, s, T_vib, &st, cl->p[i].qn) != S_OK) {
                set_err(c, ORA_EREJECT, "init: rejection cap");
                return ORA_EREJECT;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
static void iso_dir(o_stream* st, double d[3]) {
    /* Marsaglia (1972): a point uniform in the unit disk mapped onto the sphere */
    for (;;) {
        double x1 = 2.0 * st_u01(st) - 1.0;
        double x2 = 2.0 * st_u01(st) - 1.0;
        double s = x1 * x1 + x2 * x2;
        if (s < 1.0) {
            double r = 2.0 * sqrt(1.0 - s);
            d[0] = x1 * r; d[1] = x2 * r; d[2] = 1.0 - 2.0 * s;
            return;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Rotation (Sec. "Rotation coupling"; the paper drops rotation in its
   verification runs).  Readings:
     - a molecule's rotation is one classical energy E_rot with rot_dof
       degrees of freedom (2 linear, 3 non-linear);
     - every accepted collision that relaxes (reading A8) also relaxes the
       rotation of each rotating partner, after the vibrational draws, P
       before Q: with E_c = E_rel + E_rot the classical LB draw gives
       E_rot' = x E_c, x ~ Beta(rot_dof/2, (5 - 2 omega)/2), and E_rel' =
       E_c - E_rot' (one stream PU_ROT per pair);
     - x is drawn by rejection under the maximum of its density shape
       x^(rot_dof/2 - 1) (1 - x)^(3/2 - omega), written with square roots only;
     - the QK collision energies add gamma E_rot,A (the paper's extended
       Eq. Ecoll-diss and Eq. Ecoll-exch), gamma per reaction;
     - a reaction puts the reactants' rotational energy into the energy it
       redistributes; products start with E_rot = 0 and take rotation in
       their next collisions; a third body keeps its rotation;
     - TCE with internal degrees of freedom counts E_rot of both partners;
     - initial rotation at T_rot: E_rot = kT Gamma(rot_dof/2), from
       -ln(u) (rot_dof 2) plus Marsaglia's polar normal squared over two
       (rot_dof 3), with the logarithm ora_ln. */

/* natural logarithm for x > 0 (normal doubles): x = m 2^e with m in
   [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s), s = (m - 1)/(m + 1), |s| < 0.172,
   by the atanh series to s^25 (remainder below 1e-19), plus e ln 2 */
double ora_ln(double x) {
    union { double d; uint64_t u; } b;
    b.d = x;
    int e = (int)((b.u >> 52) & 0x7FF) - 1022;
    b.u = (b.u & 0x000FFFFFFFFFFFFFull) | 0x3FE0000000000000ull;  /* m in [0.5, 1) */
    double m = b.d;
    if (m < 0.70710678118654752440) { m = m * 2.0; e = e - 1; }
    const double s = (m - 1.0) / (m + 1.0);
    const double s2 = s * s;
    double t = 1.0 / 25.0;
    for (int k = 23; k >= 1; k -= 2) t = 1.0 / (double)k + s2 * t;
    return 2.0 * s * t + (double)e * 0.69314718055994530942;
}

/* exponential for -708 <= x <= 709: x = k ln 2 + r with k the integer
   nearest x / ln 2 and |r| <= ln 2 / 2 + tiny; ln 2 split into L1 (29
   significant bits, so k L1 is exact) and L2 = ln 2 - L1; e^r by its Taylor
   series to r^18 in Horner form (remainder below 1e-25), times 2^k.  Below
   -708 the result is taken as 0. */
double ora_exp(double x) {
    if (x < -708.0) return 0.0;
    if (x > 709.0) return HUGE_VAL;
    const double L1 = 0x1.62e42ffp-1, L2 = -0x1.718432a1b0e26p-35;
    const int k = (int)floor(x * 0x1.71547652b82fep+0 + 0.5);
    const double r = (x - (double)k * L1) - (double)k * L2;
    double t = 1.0;
    for (int n = 18; n >= 1; --n) t = 1.0 + (r * t) / (double)n;
    return ldexp(t, k);
}

/* x^y for x > 0 from the two series above */
static double ora_pow(double x, double y) { return ora_exp(y * ora_ln(x)); }

/* the LB fraction's density shape (1 - x)^(3/2 - omega) times x^(1/2) for
   three rotational degrees of freedom */
static double rot_shape(const ora_ctx* c, int rot_dof, double x) {
    double f = pw(c, 1.0 - x);
    if (rot_dof == 3) f = f * sqrt(x);
    return f;
}

static double rot_fraction(const ora_ctx* c, const o_species* s, o_stream* st) {
    for (uint32_t it = 0; it < c->reject_cap; ++it) {
        const double x = st_u01(st);
        const double y = st_u01(st);
        if (y * s->rot_fmax < rot_shape(c, s->d.rot_dof, x)) return x;
    }
    return 0.5;
}

static double rot_init_energy(const o_species* s, double kT, o_stream* st) {
    double E = -ora_ln(1.0 - st_u01(st));
    if (s->d.rot_dof == 3) {
        for (;;) {
            const double x1 = 2.0 * st_u01(st) - 1.0;
            const double x2 = 2.0 * st_u01(st) - 1.0;
            const double q = x1 * x1 + x2 * x2;
            if (q > 0.0 && q < 1.0) {
                E = E + x1 * x1 * (-ora_ln(q) / q);
                break;
            }
        }
    }
    return E * kT;
}

typedef struct { int rx, side, mode; double ex; } o_chan;

/* sample a molecule's state; keeps it on overflow/degenerate/cap and counts */
static void relax_one(ora_ctx* c, o_res* R, const o_species* s, double Ec, o_stream* st,
                      uint8_t* qn) {
    uint8_t nq[ORA_MAX_MODES];
    memcpy(nq, qn, 16);
    R->counters[2]++;
    int r = sample_table(c, s, Ec, st, nq, &R->counters[3]);
    if (r == S_OK) memcpy(qn, nq, (size_t)s->n_modes);
    else if (r == S_OVER) R->counters[4]++;
    else if (r == S_DEGEN) R->counters[5]++;
    else set_err(c, ORA_EREJECT, "LB sampler: rejection cap");
}

/* Product state at budget Ec (reading A13): the same LB target as relaxation */
static void product_state(ora_ctx* c, o_res* R, const o_species* s, double Ec, o_stream* st,
                          uint8_t* qn) {
    memset(qn, 0, 16);
    if (s->n_modes == 0) return;
    R->counters[2]++;
    int r = sample_table(c, s, Ec, st, qn, &R->counters[3]);
    if (r != S_OK) { memset(qn, 0, 16); set_err(c, ORA_EREJECT, "product sampler failed"); }
}

/* ------------------------------------------------------------------ */
/* The second reading of the product redistribution (Sec. "Polyatomic QK
   reaction modeling": the energy left after the reaction is shared with LB
   over all available degrees of freedom by equipartition, the vibrational
   degrees of freedom found by root-finding at a collision temperature).
   Readings:
     - the products' translational degrees of freedom: 3 per relative
       motion (6 after a dissociation, 3 after an exchange or a
       recombination);
     - the collision temperature T_c solves E_x = xi_tr/2 k T_c + sum over
       the products of <E_vib>(T_c), E_x the available energy above the
       products' ground states and <E_vib> the Boltzmann mean over the
       levels above the ZPE; a product's vibrational degrees of freedom are
       xi_vib = 2 <E_vib>(T_c) / (k T_c);
     - the first product's levels follow p ~ (E - E_state)^b1 with
       b1 = (xi_tr + xi_vib,2(T_c))/2 - 1 (the rest shared by the
       translation and the second product's vibration), at the budget of
       reading A13 (the partner's ZPE reserved); the second product's with
       b2 = xi_tr/2 - 1 at what the first left; a recombination's single
       product with b = xi_tr/2 - 1;
     - drawn exactly: a table draw at exponent a_t accepted with
       ((E - sum E)/(E - ZPE))^(b - a_t), a_t the context's exponent
       3/2 - omega when b reaches it, else 1/2 (every b here is at least
       1/2, since xi_tr >= 3). */
/* <E_vib>(T) above the ground level with the exponential ora_exp: a
   stretch's Boltzmann mean over its level list, a bend's harmonic
   k Theta / (e^(Theta/T) - 1) (0 once Theta/T > 700) */
static double mean_evib_c(const o_species* s, double T) {
    const double kT = KB * T;
    double e = 0.0;
    for (int j = 0; j < s->n_modes; ++j) {
        if (s->is_bend[j]) {
            const double th = s->d.theta[j - s->d.n_stretch];
            const double x = th / T;
            if (x <= 700.0) e = e + (KB * th) / (ora_exp(x) - 1.0);
        } else {
            double num = 0.0, den = 0.0;
            for (int i = 0; i < s->n_levels[j]; ++i) {
                const double de = s->E[j][i] - s->E[j][0];
                const double b = ora_exp(-de / kT);
                num = num + de * b;
                den = den + b;
            }
            e = e + num / den;
        }
    }
    return e;
}

static double xi_vib_at(const o_species* s, double T) {
    return s->n_modes ? (2.0 * mean_evib_c(s, T)) / (KB * T) : 0.0;
}

/* T_c by bisection on [1 K, 1e7 K]; 100 halvings reach adjacent doubles */
static double tcoll_root(double xi_tr, const o_species* p1, const o_species* p2, double Ex) {
    double lo = 1.0, hi = 1.0e7;
    for (int it = 0; it < 100; ++it) {
        const double T = 0.5 * (lo + hi);
        double g = (0.5 * xi_tr) * (KB * T) - Ex;
        if (p1 && p1->n_modes) g = g + mean_evib_c(p1, T);
        if (p2 && p2->n_modes) g = g + mean_evib_c(p2, T);
        if (g < 0.0) lo = T; else hi = T;
    }
    return 0.5 * (lo + hi);
}

static int sample_exponent(ora_ctx* c, const o_species* s, double Ec, double b, o_stream* st, uint8_t* qn,
                           uint64_t* trials) {
    const int n = s->n_modes;
    memset(qn, 0, 16);
    if (n == 0) return S_OK;
    if (!(Ec > s->zpe)) return S_DEGEN;
    const double a = 1.5 - c->omega;
    const int use_main = b >= a;
    const double a_t = use_main ? a : 0.5;
    if (!use_main && (!(b >= 0.5) || !s->Hh[0])) return S_CAP;
    const double span = Ec - s->zpe;
    uint8_t nq[ORA_MAX_MODES];
    for (uint32_t trial = 0; trial < c->reject_cap; ++trial) {
        const int r = use_main ? sample_table_with(c, s, c->amode, s->H, Ec, st, nq, trials)
                               : sample_table_with(c, s, 2, s->Hh, Ec, st, nq, trials);
        if (r != S_OK) return r;
        const double Esum = evib(s, nq);
        if (b == a_t || st_u01(st) < ora_pow((Ec - Esum) / span, b - a_t)) {
            memcpy(qn, nq, (size_t)n);
            return S_OK;
        }
    }
    return S_CAP;
}

static void product_state_b(ora_ctx* c, o_res* R, const o_species* s, double Ec, double b, o_stream* st,
                            uint8_t* qn) {
    memset(qn, 0, 16);
    if (s->n_modes == 0) return;
    R->counters[2]++;
    int r = sample_exponent(c, s, Ec, b, st, qn, &R->counters[3]);
    if (r != S_OK) { memset(qn, 0, 16); set_err(c, ORA_EREJECT, "product sampler failed"); }
}

static double table_top(const o_species* s, const ora_ctx* c) {
    if (s->n_modes == 0) return INFINITY;
    return grid_pt(s, 0, c->M);
}

/* Dissociation A + M -> B + C + M (Sec. "Dissociation reactions"), energy kept
   exactly with well-bottom formation energies (reading A13). Returns 1 if done. */
static int do_diss(ora_ctx* c, o_res* R, int rx, o_part* A, o_part* M, double EvibA,
                   uint32_t cell, uint32_t rk, o_cell* cl, o_part* created, int* n_created) {
    const ora_reaction_desc* r = &c->rx[rx];
    const o_species* sA = &c->sp[A->sp];
    const o_species* sM = &c->sp[M->sp];
    const o_species* sB = &c->sp[r->products[0]];
    const o_species* sC = &c->sp[r->products[1]];
    double mA = sA->d.mass, mM = sM->d.mass, mB = sB->d.mass, mC = sC->d.mass;
    double mBC = mB + mC;
    double mt = mBC + mM;
    double P[3], V[3];
    for (int i = 0; i < 3; ++i) P[i] = mA * A->v[i] + mM * M->v[i];
    for (int i = 0; i < 3; ++i) V[i] = P[i] / mt;
    double vA2 = A->v[0] * A->v[0] + A->v[1] * A->v[1] + A->v[2] * A->v[2];
    double vM2 = M->v[0] * M->v[0] + M->v[1] * M->v[1] + M->v[2] * M->v[2];
    double V2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    double KEin = 0.5 * mA * vA2 + 0.5 * mM * vM2;
    double KEcm = 0.5 * mt * V2;
    double dEf = (sB->d.E_form + sC->d.E_form) - sA->d.E_form;
    double Eav = KEin - KEcm + EvibA - dEf + A->erot;  /* A's rotation joins the pool */
    if (!(Eav - sB->zpe - sC->zpe > 0.0) || Eav - sC->zpe > table_top(sB, c) ||
        Eav - sB->zpe > table_top(sC, c))
        return 0;
    o_stream sa, sb, ss;
    st_init(&sa, R->seed, R->step, cell, rk, PU_LB_A);
    st_init(&sb, R->seed, R->step, cell, rk, PU_LB_B);
    st_init(&ss, R->seed, R->step, cell, rk, PU_SCAT);
    uint8_t qB[16], qC[16];
    if (r->prod_split == ORA_SPLIT_TCOLL) {
        const double Tc = tcoll_root(6.0, sB, sC, Eav - sB->zpe - sC->zpe);
        product_state_b(c, R, sB, Eav - sC->zpe, (6.0 + xi_vib_at(sC, Tc)) / 2.0 - 1.0, &sa, qB);
    } else {
        product_state(c, R, sB, Eav - sC->zpe, &sa, qB);
    }
    double EvB = evib(sB, qB);
    if (r->prod_split == ORA_SPLIT_TCOLL) product_state_b(c, R, sC, Eav - EvB, 2.0, &sb, qC);
    else product_state(c, R, sC, Eav - EvB, &sb, qC);
    double EvC = evib(sC, qC);
    double Etr = (Eav - EvB) - EvC;
    double x;
    for (;;) { /* Beta(3/2,3/2) by rejection under the constant 1/2 */
        x = st_u01(&ss);
        double y = st_u01(&ss);
        if (y * y * 0.25 < x * (1.0 - x)) break;
    }
    double E1 = x * Etr;
    double E2 = Etr - E1;
    double mu1 = mB * mC / mBC;
    double mu2 = mBC * mM / mt;
    double g1 = sqrt(2.0 * E1 / mu1);
    double g2 = sqrt(2.0 * E2 / mu2);
    double d1[3], d2[3];
    iso_dir(&ss, d1);
    iso_dir(&ss, d2);
    double fM = mM / mt, fBC = mBC / mt, fC = mC / mBC, fB = mB / mBC;
    double VBC[3], vM[3], vB[3], vC[3];
    for (int i = 0; i < 3; ++i) {
        double G2 = g2 * d2[i];
        VBC[i] = V[i] + fM * G2;
        vM[i] = V[i] - fBC * G2;
    }
    for (int i = 0; i < 3; ++i) {
        double G1 = g1 * d1[i];
        vB[i] = VBC[i] + fC * G1;
        vC[i] = VBC[i] - fB * G1;
    }
    A->sp = r->products[0];
    memcpy(A->qn, qB, 16);
    A->erot = 0.0;  /* products start without rotation; M keeps its own */
    for (int i = 0; i < 3; ++i) { A->v[i] = vB[i]; M->v[i] = vM[i]; }
    o_part nc;
    memset(&nc, 0, sizeof nc);
    nc.sp = r->products[1];
    memcpy(nc.qn, qC, 16);
    for (int i = 0; i < 3; ++i) nc.v[i] = vC[i];
    created[(*n_created)++] = nc;
    (void)cl;
    return 1;
}

/* Exchange A + B -> C + D (Sec. "Exchange reactions"). Returns 1 if done. */
static int do_exch(ora_ctx* c, o_res* R, int rx, o_part* A, o_part* B, double EvA,
                   double EvB, uint32_t cell, uint32_t rk) {
    const ora_reaction_desc* r = &c->rx[rx];
    const o_species* sA = &c->sp[A->sp];
    const o_species* sB = &c->sp[B->sp];
    const o_species* sC = &c->sp[r->products[0]];
    const o_species* sD = &c->sp[r->products[1]];
    double mA = sA->d.mass, mB = sB->d.mass, mC = sC->d.mass, mD = sD->d.mass;
    double mt = mC + mD;
    double P[3], V[3];
    for (int i = 0; i < 3; ++i) P[i] = mA * A->v[i] + mB * B->v[i];
    for (int i = 0; i < 3; ++i) V[i] = P[i] / mt;
    double vA2 = A->v[0] * A->v[0] + A->v[1] * A->v[1] + A->v[2] * A->v[2];
    double vB2 = B->v[0] * B->v[0] + B->v[1] * B->v[1] + B->v[2] * B->v[2];
    double V2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    double KEin = 0.5 * mA * vA2 + 0.5 * mB * vB2;
    double KEcm = 0.5 * mt * V2;
    double dEf = (sC->d.E_form + sD->d.E_form) - (sA->d.E_form + sB->d.E_form);
    double Eav = (KEin - KEcm + EvA + EvB - dEf + A->erot) + B->erot;  /* rotation joins the pool */
    if (!(Eav - sC->zpe - sD->zpe > 0.0) || Eav - sD->zpe > table_top(sC, c) ||
        Eav - sC->zpe > table_top(sD, c))
        return 0;
    o_stream sa, sb, ss;
    st_init(&sa, R->seed, R->step, cell, rk, PU_LB_A);
    st_init(&sb, R->seed, R->step, cell, rk, PU_LB_B);
    st_init(&ss, R->seed, R->step, cell, rk, PU_SCAT);
    uint8_t qC[16], qD[16];
    if (r->prod_split == ORA_SPLIT_TCOLL) {
        const double Tc = tcoll_root(3.0, sC, sD, Eav - sC->zpe - sD->zpe);
        product_state_b(c, R, sC, Eav - sD->zpe, (3.0 + xi_vib_at(sD, Tc)) / 2.0 - 1.0, &sa, qC);
    } else {
        product_state(c, R, sC, Eav - sD->zpe, &sa, qC);
    }
    double EvC = evib(sC, qC);
    if (r->prod_split == ORA_SPLIT_TCOLL) product_state_b(c, R, sD, Eav - EvC, 0.5, &sb, qD);
    else product_state(c, R, sD, Eav - EvC, &sb, qD);
    double EvD = evib(sD, qD);
    double Etr = (Eav - EvC) - EvD;
    double mu = mC * mD / mt;
    double g = sqrt(2.0 * Etr / mu);
    double d[3];
    iso_dir(&ss, d);
    double fC = mD / mt, fD = mC / mt;
    for (int i = 0; i < 3; ++i) {
        double G = g * d[i];
        A->v[i] = V[i] + fC * G;
        B->v[i] = V[i] - fD * G;
    }
    A->sp = r->products[0];
    B->sp = r->products[1];
    memcpy(A->qn, qC, 16);
    memcpy(B->qn, qD, 16);
    A->erot = 0.0;
    B->erot = 0.0;
    return 1;
}

/* Recombination B + C + M -> A + M (Sec. "Recombination reactions").  B takes
   A's species; C is removed; the third body M keeps its species and levels.
   The energy available to A's vibration and the A-M relative motion is the
   translational energy of B, C and M in their centre-of-mass frame plus the
   vibrational energies of B and C plus the released formation energy; A's
   levels are drawn with the LB target at that budget (as for reaction
   products, reading A13) and the rest goes to A-M relative motion in a
   uniformly random direction, total momentum kept.  Returns 1 if done. */
static int do_recomb(ora_ctx* c, o_res* R, int rx, o_part* B, o_part* Cp, o_part* M,
                     double EvB, double EvC, uint32_t cell, uint32_t rk) {
    const ora_reaction_desc* r = &c->rx[rx];
    const o_species* sA = &c->sp[r->products[0]];
    const o_species* sB = &c->sp[B->sp];
    const o_species* sC = &c->sp[Cp->sp];
    const o_species* sM = &c->sp[M->sp];
    double mA = sA->d.mass, mB = sB->d.mass, mC = sC->d.mass, mM = sM->d.mass;
    double mt = mA + mM;
    double P[3], V[3];
    for (int i = 0; i < 3; ++i) P[i] = (mB * B->v[i] + mC * Cp->v[i]) + mM * M->v[i];
    for (int i = 0; i < 3; ++i) V[i] = P[i] / mt;
    double vB2 = B->v[0] * B->v[0] + B->v[1] * B->v[1] + B->v[2] * B->v[2];
    double vC2 = Cp->v[0] * Cp->v[0] + Cp->v[1] * Cp->v[1] + Cp->v[2] * Cp->v[2];
    double vM2 = M->v[0] * M->v[0] + M->v[1] * M->v[1] + M->v[2] * M->v[2];
    double V2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    double KEin = (0.5 * mB * vB2 + 0.5 * mC * vC2) + 0.5 * mM * vM2;
    double KEcm = 0.5 * mt * V2;
    double dEf = sA->d.E_form - (sB->d.E_form + sC->d.E_form);
    double Eav = (KEin - KEcm + EvB + EvC - dEf + B->erot) + Cp->erot;  /* rotation joins the pool */
    if (!(Eav - sA->zpe > 0.0) || Eav > table_top(sA, c)) return 0;
    o_stream sa, ss;
    st_init(&sa, R->seed, R->step, cell, rk, PU_LB_A);
    st_init(&ss, R->seed, R->step, cell, rk, PU_SCAT);
    uint8_t qA[16];
    if (r->prod_split == ORA_SPLIT_TCOLL) product_state_b(c, R, sA, Eav, 0.5, &sa, qA);
    else product_state(c, R, sA, Eav, &sa, qA);
    double Etr = Eav - evib(sA, qA);
    double mu = mA * mM / mt;
    double g = sqrt(2.0 * Etr / mu);
    double d[3];
    iso_dir(&ss, d);
    double fA = mM / mt, fM = mA / mt;
    for (int i = 0; i < 3; ++i) {
        double G = g * d[i];
        B->v[i] = V[i] + fA * G;
        M->v[i] = V[i] - fM * G;
    }
    B->sp = r->products[0];
    memcpy(B->qn, qA, 16);
    B->erot = 0.0;
    Cp->sp = -1;
    Cp->erot = 0.0;
    return 1;
}

/* Translational temperature of a cell at the start of a step: the kinetic
   energy in the cell's centre-of-mass frame, 3/2 N k T.  The per-particle
   energies, momenta and masses are summed as integers (units 2^-96 J,
   2^-104 kg m/s, 2^-120 kg) so that the sums do not depend on their order. */
static double cell_temperature(const ora_ctx* c, const o_cell* cl) {
    int64_t E = 0, px = 0, py = 0, pz = 0, Ms = 0;
    int N = cl->n;
    if (N < 2) return 0.0;
    for (int i = 0; i < N; ++i) {
        const o_part* p = &cl->p[i];
        double m = c->sp[p->sp].d.mass;
        double e = 0.5 * m * (p->v[0] * p->v[0] + p->v[1] * p->v[1] + p->v[2] * p->v[2]);
        E += llrint(ldexp(e, 96));
        px += llrint(ldexp(m * p->v[0], 104));
        py += llrint(ldexp(m * p->v[1], 104));
        pz += llrint(ldexp(m * p->v[2], 104));
        Ms += llrint(ldexp(m, 120));
    }
    double Ek = ldexp((double)E, -96);
    double P2 = ((double)px * (double)px + (double)py * (double)py) + (double)pz * (double)pz;
    double Ecm = ldexp(0.5 * (P2 / (double)Ms), -88);
    return (2.0 * (Ek - Ecm)) / (3.0 * (double)N * KB);
}

double ora_cell_temperature(ora_ctx* c, int res, int cell) {
    return cell_temperature(c, &c->res[res]->cells[cell]);
}

static void log_push(ora_ctx* c, const ora_log_rec* r) {
    if (!c->log_on) return;
    if (c->log_n == c->log_cap) {
        c->log_cap = c->log_cap ? 2 * c->log_cap : 4096;
        c->log = (ora_log_rec*)realloc(c->log, sizeof(ora_log_rec) * (size_t)c->log_cap);
    }
    c->log[c->log_n++] = *r;
}

/* One candidate pair: VHS acceptance (NTC), then the QK reaction test, then
   either the reaction or LB relaxation of molecule 1, then molecule 2, then
   isotropic VHS scattering. */
typedef struct {
    o_cell* cl;
    uint32_t N;        /* particles at the start of the step */
    int64_t kmax;      /* pairs of this round */
    const uint32_t* key;
    double T;          /* cell temperature at the start of the step */
} o_round;

static void process_pair(ora_ctx* c, o_res* R, uint32_t cell, uint32_t round, uint32_t k,
                         o_part* P, o_part* Q, uint32_t ip, uint32_t iq, double sgmax,
                         double* seen, o_part* created, int* n_created, const o_round* rd) {
    uint32_t rk = (round << 24) | k;
    R->counters[0]++;
    if (P->sp < 0 || Q->sp < 0) { /* a member removed earlier in this step */
        ora_log_rec lr0 = { R->step, cell, rk, ip, iq, -1, 0 };
        log_push(c, &lr0);
        return;
    }
    const o_species* sP = &c->sp[P->sp];
    const o_species* sQ = &c->sp[Q->sp];
    o_pair pc = pair_consts(c, P->sp, Q->sp);
    double gx = P->v[0] - Q->v[0], gy = P->v[1] - Q->v[1], gz = P->v[2] - Q->v[2];
    double g2 = gx * gx + gy * gy + gz * gz;
    double g = sqrt(g2);
    double sg = pc.C * gpow(c, g);
    if (sg > *seen) *seen = sg;
    o_stream sp;
    st_init(&sp, R->seed, R->step, cell, rk, PU_PAIR);
    double u_acc = st_u01(&sp);
    double u_ster = st_u01(&sp);
    double u_sel = st_u01(&sp);
    double u_ch = st_u01(&sp);
    ora_log_rec lr = { R->step, cell, rk, ip, iq, -1, 0 };
    if (!(u_acc < sg / sgmax)) { log_push(c, &lr); return; }
    R->counters[1]++;
    double Etr = 0.5 * pc.mr * g2;
    double EvP = evib(sP, P->qn);
    double EvQ = evib(sQ, Q->qn);

    /* Recombination (reading A14), tested before the QK channels: the pair
       (B, C) recombines with probability k_r(T_cell) n / (sigma_T g), n the
       number density of third bodies ((N - 2) w / V_c); k_r is that of the
       third body M, the particle at position 2 kmax + k of this round's
       permutation (a particle in no pair of the round, uniform over them;
       rounds hold at most N/3 pairs when a recombination exists, so every
       pair has one when N >= 3).  One recombination per pair type. */
    for (int r = 0; r < c->n_reactions; ++r) {
        const ora_reaction_desc* rx = &c->rx[r];
        if (rx->type != ORA_RECOMB) continue;
        int side;
        if (P->sp == rx->reactants[0] && Q->sp == rx->reactants[1]) side = 0;
        else if (Q->sp == rx->reactants[0] && P->sp == rx->reactants[1]) side = 1;
        else continue;
        int64_t m = 2 * rd->kmax + (int64_t)k;
        if (m >= (int64_t)rd->N) break;
        uint32_t iM = ora_pair_perm((uint32_t)m, rd->N, rd->key);
        o_part* M = &rd->cl->p[iM];
        if (M->sp < 0) break;
        double kr = ora_rec_rate(c, r, M->sp, rd->T);
        double n3 = ((double)(rd->N - 2) * R->w) / R->Vc;
        double prec = (kr * n3) / sg;
        o_stream sr;
        st_init(&sr, R->seed, R->step, cell, rk, PU_REC);
        if (!(st_u01(&sr) < prec)) break;
        o_part* B = side ? Q : P;
        o_part* Cp = side ? P : Q;
        if (do_recomb(c, R, r, B, Cp, M, side ? EvQ : EvP, side ? EvP : EvQ, cell, rk)) {
            R->counters[8 + r]++;
            lr.event = 1 + r;
            lr.aux = (uint32_t)side + 2u * iM;
            log_push(c, &lr);
            return;
        }
        R->counters[6]++; /* not executed: the pair relaxes */
        goto relax;
    }

    /* TCE reactions (the comparison model, Eq. arrhenius): tested before
       the QK channels, in reaction order, against one uniform of their own */
    {
        double u_t = -1.0, run = 0.0;
        for (int r = 0; r < c->n_reactions; ++r) {
            const ora_reaction_desc* rx = &c->rx[r];
            if (rx->model != ORA_MODEL_TCE || rx->type == ORA_RECOMB) continue;
            int side;
            if (rx->type == ORA_DISS) {
                if (P->sp == rx->reactants[0]) side = 0;
                else if (Q->sp == rx->reactants[0]) side = 1;
                else continue;
            } else {
                if (P->sp == rx->reactants[0] && Q->sp == rx->reactants[1]) side = 0;
                else if (Q->sp == rx->reactants[0] && P->sp == rx->reactants[1]) side = 1;
                else continue;
            }
            double Ec = Etr;
            if (rx->tce_zeta > 0.0) Ec = (((Ec + (EvP - sP->zpe)) + (EvQ - sQ->zpe)) + P->erot) + Q->erot;
            run = run + tce_prob(c, r, side ? P->sp : Q->sp, Ec);
            if (u_t < 0.0) {
                o_stream st;
                st_init(&st, R->seed, R->step, cell, rk, PU_TCE);
                u_t = st_u01(&st);
            }
            if (!(u_t < run)) continue;
            o_part* A = side ? Q : P;
            o_part* B = side ? P : Q;
            int done;
            if (rx->type == ORA_DISS) {
                int mode = 0;
                while (mode < 31 && !((rx->diss_mode_mask >> mode) & 1u)) mode++;
                done = do_diss(c, R, r, A, B, side ? EvQ : EvP, cell, rk, NULL, created, n_created);
                lr.aux = (uint32_t)mode + (side ? 16u : 0u);
            } else {
                done = do_exch(c, R, r, A, B, side ? EvQ : EvP, side ? EvP : EvQ, cell, rk);
                lr.aux = (uint32_t)side;
            }
            if (done) {
                R->counters[8 + r]++;
                lr.event = 1 + r;
                log_push(c, &lr);
                return;
            }
            R->counters[6]++;
            lr.aux = 0;
            goto relax;
        }
    }

    /* QK reaction test: channel list in fixed order (reading A21) */
    o_chan ch[MAX_CHANNELS];
    int nch = 0;
    for (int side = 0; side < 2; ++side) {
        const o_part* A = side ? Q : P;
        const o_species* sA = side ? sQ : sP;
        double EvA = side ? EvQ : EvP;
        for (int r = 0; r < c->n_reactions; ++r) {
            const ora_reaction_desc* rx = &c->rx[r];
            if (rx->type != ORA_DISS || rx->model == ORA_MODEL_TCE || rx->reactants[0] != A->sp) continue;
            for (int j = 0; j < sA->d.n_stretch; ++j) {
                if (!((rx->diss_mode_mask >> j) & 1u)) continue;
                /* Eq. Ecoll-diss (with gamma E_rot,A, Sec. "Rotation coupling") */
                double Ecoll = Etr + EvA - c->rx_zpesum[r] + sA->E[j][0];
                if (rx->gamma != 0.0) Ecoll = Ecoll + rx->gamma * A->erot;
                double Eex = Ecoll - sA->d.De[j];
                if (Eex > 0.0 && nch < MAX_CHANNELS) {
                    o_chan cc = { r, side, j, Eex };
                    ch[nch++] = cc;
                }
            }
        }
    }
    for (int r = 0; r < c->n_reactions; ++r) {
        const ora_reaction_desc* rx = &c->rx[r];
        if (rx->type != ORA_EXCH || rx->model == ORA_MODEL_TCE) continue;
        int side;
        if (P->sp == rx->reactants[0] && Q->sp == rx->reactants[1]) side = 0;
        else if (Q->sp == rx->reactants[0] && P->sp == rx->reactants[1]) side = 1;
        else continue;
        if (!(u_ster < rx->steric)) continue;
        const o_part* A = side ? Q : P;
        const o_species* sA = side ? sQ : sP;
        /* Eq. Ecoll-exch (reading A12: level energies include the ZPE) */
        double s = 0.0;
        if (rx->alpha_mode == ORA_ALPHA_ONE_RANDOM_STRETCH) {
            int js = (int)floor(u_sel * (double)sA->d.n_stretch);
            s = sA->E[js][A->qn[js]];
        } else {
            for (int j = 0; j < sA->n_modes; ++j) s = s + rx->alpha[j] * sA->E[j][A->qn[j]];
        }
        double Ecoll = Etr + s;
        if (rx->gamma != 0.0) Ecoll = Ecoll + rx->gamma * A->erot;  /* Sec. "Rotation coupling" */
        double Eex = Ecoll - rx->Ea;
        if (Eex > 0.0 && nch < MAX_CHANNELS) {
            o_chan cc = { r, side, 0, Eex };
            ch[nch++] = cc;
        }
    }
    if (nch > 0) {
        int pick = 0;
        if (nch > 1) { /* "Competing reactions": weighted by E_excess */
            double tot = 0.0;
            for (int i = 0; i < nch; ++i) tot = tot + ch[i].ex;
            double t = u_ch * tot;
            double pre = 0.0;
            pick = nch - 1;
            for (int i = 0; i < nch; ++i) {
                pre = pre + ch[i].ex;
                if (t < pre) { pick = i; break; }
            }
        }
        const o_chan* cc = &ch[pick];
        int done;
        if (c->rx[cc->rx].type == ORA_DISS) {
            o_part* A = cc->side ? Q : P;
            o_part* M = cc->side ? P : Q;
            done = do_diss(c, R, cc->rx, A, M, cc->side ? EvQ : EvP, cell, rk, NULL, created,
                           n_created);
            lr.aux = (uint32_t)cc->mode + (cc->side ? 16u : 0u);
        } else {
            o_part* A = cc->side ? Q : P;
            o_part* B = cc->side ? P : Q;
            done = do_exch(c, R, cc->rx, A, B, cc->side ? EvQ : EvP, cc->side ? EvP : EvQ,
                           cell, rk);
            lr.aux = (uint32_t)cc->side;
        }
        if (done) {
            R->counters[8 + cc->rx]++;
            lr.event = 1 + cc->rx;
            log_push(c, &lr);
            return;
        }
        R->counters[6]++;
        lr.aux = 0;
    }

    /* relaxation (HCAO LB): molecule 1, then molecule 2 with the updated E_rel */
relax:;
    double E = Etr;
    if (sP->n_modes > 0) {
        o_stream s1;
        st_init(&s1, R->seed, R->step, cell, rk, PU_LB_A);
        double Ec = E + EvP;
        relax_one(c, R, sP, Ec, &s1, P->qn);
        E = Ec - evib(sP, P->qn);
    }
    if (sQ->n_modes > 0) {
        o_stream s2;
        st_init(&s2, R->seed, R->step, cell, rk, PU_LB_B);
        double Ec = E + EvQ;
        relax_one(c, R, sQ, Ec, &s2, Q->qn);
        E = Ec - evib(sQ, Q->qn);
    }
    /* classical LB rotational relaxation, P then Q (one stream) */
    if (sP->d.rot_dof > 0 || sQ->d.rot_dof > 0) {
        o_stream sr;
        st_init(&sr, R->seed, R->step, cell, rk, PU_ROT);
        for (int m = 0; m < 2; ++m) {
            o_part* X = m ? Q : P;
            const o_species* sX = m ? sQ : sP;
            if (sX->d.rot_dof == 0) continue;
            const double Ec = E + X->erot;
            X->erot = rot_fraction(c, sX, &sr) * Ec;
            E = Ec - X->erot;
        }
    }
    /* isotropic VHS scattering; centre-of-mass velocity kept */
    o_stream ss;
    st_init(&ss, R->seed, R->step, cell, rk, PU_SCAT);
    double gn = sqrt(2.0 * E / pc.mr);
    double d[3];
    iso_dir(&ss, d);
    double mp = sP->d.mass, mq = sQ->d.mass;
    double V[3];
    for (int i = 0; i < 3; ++i) V[i] = (mp * P->v[i] + mq * Q->v[i]) / pc.mt;
    for (int i = 0; i < 3; ++i) {
        double G = gn * d[i];
        P->v[i] = V[i] + pc.fp * G;
        Q->v[i] = V[i] - pc.fq * G;
    }
    lr.event = 0;
    log_push(c, &lr);
}

static int step_reservoir(ora_ctx* c, o_res* R) {
    for (int ci = 0; ci < R->n_cells; ++ci) {
        o_cell* cl = &R->cells[ci];
        /* the cell's index in every random-number key: a reservoir may hold a
           contiguous range of a larger workload's cells */
        const uint32_t gc = R->cell_base + (uint32_t)ci;
        int N = cl->n;
        if (N < 2) continue;
        /* NTC: N_sel = 1/2 N (N-1) w (sigma g)_max dt / V_c, rounded stochastically */
        double x = 0.5 * (double)N * (double)(N - 1) * R->w * cl->sgmax * R->dt / R->Vc;
        double fl = floor(x);
        int64_t nsel = (int64_t)fl;
        o_stream sn;
        st_init(&sn, R->seed, R->step, gc, 0u, PU_NSEL);
        if (st_u01(&sn) < x - fl) nsel++;
        int has_rec = 0;
        for (int r = 0; r < c->n_reactions; ++r) has_rec |= c->rx[r].type == ORA_RECOMB;
        /* pairs per round: N/2, or N/3 with a recombination reaction, so that
           every pair of a round has a third body in no pair of the round */
        int64_t P = (has_rec && N >= 3) ? N / 3 : N / 2;
        int64_t rounds = (nsel + P - 1) / P;
        if (rounds > 255) { set_err(c, ORA_EINVAL, "more than 255 NTC rounds"); return ORA_EINVAL; }
        double seen = 0.0;
        o_part* created = (o_part*)malloc(sizeof(o_part) * (size_t)(nsel + 1));
        int n_created = 0;
        double Tcell = has_rec ? cell_temperature(c, cl) : 0.0;
        for (int64_t r = 0; r < rounds; ++r) {
            o_stream sf;
            st_init(&sf, R->seed, R->step, gc, (uint32_t)r << 24, PU_PERM);
            uint32_t key[4];
            for (int i = 0; i < 4; ++i) key[i] = st_word(&sf);
            int64_t kmax = nsel - r * P;
            if (kmax > P) kmax = P;
            o_round rd = { cl, (uint32_t)N, kmax, key, Tcell };
            for (int64_t k = 0; k < kmax; ++k) {
                uint32_t ip = ora_pair_perm((uint32_t)(2 * k), (uint32_t)N, key);
                uint32_t iq = ora_pair_perm((uint32_t)(2 * k + 1), (uint32_t)N, key);
                process_pair(c, R, gc, (uint32_t)r, (uint32_t)k, &cl->p[ip], &cl->p[iq],
                             ip, iq, cl->sgmax, &seen, created, &n_created, &rd);
            }
        }
        for (int i = 0; i < n_created; ++i) cell_push(cl, &created[i]);
        free(created);
        /* removed particles (recombination): with d removed among the n
           records, the surviving records at positions >= n - d move, in
           increasing position order, into the removed positions below n - d,
           taken in increasing order; the cell keeps n - d records */
        int d = 0;
        for (int i = 0; i < cl->n; ++i) d += cl->p[i].sp < 0;
        if (d > 0) {
            int t0 = cl->n - d, h = 0;
            for (int t = t0; t < cl->n; ++t) {
                if (cl->p[t].sp < 0) continue;
                while (cl->p[h].sp >= 0) h++;
                cl->p[h++] = cl->p[t];
            }
            cl->n = t0;
        }
        if (seen > cl->sgmax) cl->sgmax = seen;
    }
    R->step++;
    R->counters[7]++;
    return 0;
}

int ora_step(ora_ctx* c, int n_steps) {
    for (int s = 0; s < n_steps; ++s) {
        c->log_n = 0; /* the log keeps the last step only */
        for (int r = 0; r < c->n_res; ++r) {
            int e = step_reservoir(c, c->res[r]);
            if (e) return e;
        }
        if (c->error) return c->error;
    }
    return 0;
}

int ora_set_log(ora_ctx* c, int on) { c->log_on = on; c->log_n = 0; return 0; }
int64_t ora_log_count(ora_ctx* c) { return c->log_n; }
int ora_read_log(ora_ctx* c, ora_log_rec* out, int64_t max) {
    int64_t n = c->log_n < max ? c->log_n : max;
    memcpy(out, c->log, sizeof(ora_log_rec) * (size_t)n);
    return 0;
}

int64_t ora_count(ora_ctx* c, int res) {
    o_res* R = c->res[res];
    int64_t n = 0;
    for (int j = 0; j < R->n_cells; ++j) n += R->cells[j].n;
    return n;
}

int ora_read_particles(ora_ctx* c, int res, double* v, uint8_t* qn, int32_t* species,
                       int32_t* cell) {
    o_res* R = c->res[res];
    int64_t o = 0;
    for (int j = 0; j < R->n_cells; ++j) {
        o_cell* cl = &R->cells[j];
        for (int i = 0; i < cl->n; ++i, ++o) {
            for (int d = 0; d < 3; ++d) v[3 * o + d] = cl->p[i].v[d];
            memcpy(qn + 16 * o, cl->p[i].qn, 16);
            species[o] = cl->p[i].sp;
            cell[o] = j;
        }
    }
    return 0;
}

int ora_read_cell_sgmax(ora_ctx* c, int res, double* out) {
    o_res* R = c->res[res];
    for (int j = 0; j < R->n_cells; ++j) out[j] = R->cells[j].sgmax;
    return 0;
}

int ora_read_counters(ora_ctx* c, int res, uint64_t* out, int max) {
    o_res* R = c->res[res];
    int n = 8 + c->n_reactions;
    if (n > max) n = max;
    memcpy(out, R->counters, sizeof(uint64_t) * (size_t)n);
    return n;
}

int ora_n_levels(ora_ctx* c, int sp, int mode) { return c->sp[sp].n_levels[mode]; }
double ora_level_energy(ora_ctx* c, int sp, int mode, int level) { return c->sp[sp].E[mode][level]; }
double ora_table_value(ora_ctx* c, int sp, int k, int m) { return c->sp[sp].H[k][m]; }
int ora_table_entries(ora_ctx* c, int sp) { return c->sp[sp].MT; }
double ora_zpe(ora_ctx* c, int sp) { return c->sp[sp].zpe; }

int ora_sample_lb(ora_ctx* c, int sp, double Ec, uint64_t seed, int64_t n, int method,
                  uint8_t* out_qn, uint64_t* trials) {
    const o_species* s = &c->sp[sp];
    uint64_t tr = 0;
    for (int64_t i = 0; i < n; ++i) {
        o_stream st;
        st_init(&st, seed, (uint32_t)i, (uint32_t)(i >> 32), 0u, PU_TEST);
        uint8_t* q = out_qn + 16 * i;
        memset(q, 0, 16);
        int r = method == ORA_SAMPLER_LITERAL ? sample_literal(c, s, Ec, &st, q, &tr)
                                              : sample_table(c, s, Ec, &st, q, &tr);
        if (r != S_OK) return r == S_CAP ? ORA_EREJECT : ORA_EINVAL;
    }
    if (trials) *trials = tr;
    return 0;
}

int64_t ora_sample_products(ora_ctx* c, int rx, int sp1, const double* v1, const uint8_t* q1, int sp2,
                            const double* v2, const uint8_t* q2, int sp3, const double* v3, const uint8_t* q3,
                            uint64_t seed, int64_t n, double* out_v, uint8_t* out_q) {
    if (rx < 0 || rx >= c->n_reactions || sp1 < 0 || sp1 >= c->n_species || sp2 < 0 || sp2 >= c->n_species ||
        n < 0)
        return ORA_EINVAL;
    const int type = c->rx[rx].type;
    if (type == ORA_RECOMB && (sp3 < 0 || sp3 >= c->n_species || !v3 || !q3)) return ORA_EINVAL;
    o_res R;
    memset(&R, 0, sizeof R);
    R.seed = seed;
    int64_t done = 0;
    for (int64_t i = 0; i < n; ++i) {
        o_part P1, P2, P3, created[1];
        memset(&P1, 0, sizeof P1);
        memset(&P2, 0, sizeof P2);
        memset(&P3, 0, sizeof P3);
        P1.sp = sp1;
        P2.sp = sp2;
        for (int k = 0; k < 3; ++k) { P1.v[k] = v1[k]; P2.v[k] = v2[k]; }
        memcpy(P1.qn, q1, 16);
        memcpy(P2.qn, q2, 16);
        if (type == ORA_RECOMB) {
            P3.sp = sp3;
            for (int k = 0; k < 3; ++k) P3.v[k] = v3[k];
            memcpy(P3.qn, q3, 16);
        }
        const double Ev1 = evib(&c->sp[sp1], P1.qn), Ev2 = evib(&c->sp[sp2], P2.qn);
        const uint32_t cell = (uint32_t)(i >> 32), rk = (uint32_t)i;
        int nc = 0, ok;
        if (type == ORA_DISS)
            ok = do_diss(c, &R, rx, &P1, &P2, Ev1, cell, rk, NULL, created, &nc);
        else if (type == ORA_EXCH)
            ok = do_exch(c, &R, rx, &P1, &P2, Ev1, Ev2, cell, rk);
        else
            ok = do_recomb(c, &R, rx, &P1, &P2, &P3, Ev1, Ev2, cell, rk);
        if (c->error) return c->error;
        if (!ok) continue;
        double* v = out_v + 9 * done;
        uint8_t* q = out_q + 32 * done;
        memset(v, 0, 9 * sizeof(double));
        memset(q, 0, 32);
        for (int k = 0; k < 3; ++k) v[k] = P1.v[k];
        memcpy(q, P1.qn, 16);
        if (type == ORA_DISS) {
            for (int k = 0; k < 3; ++k) { v[3 + k] = created[0].v[k]; v[6 + k] = P2.v[k]; }
            memcpy(q + 16, created[0].qn, 16);
        } else if (type == ORA_EXCH) {
            for (int k = 0; k < 3; ++k) v[3 + k] = P2.v[k];
            memcpy(q + 16, P2.qn, 16);
        } else {
            for (int k = 0; k < 3; ++k) v[6 + k] = P3.v[k];
        }
        ++done;
    }
    return done;
}

int ora_sample_init(ora_ctx* c, int sp, double T, uint64_t seed, int64_t n, uint8_t* out_qn) {
    const o_species* s = &c->sp[sp];
    for (int64_t i = 0; i < n; ++i) {
        o_stream st;
        st_init(&st, seed, (uint32_t)i, (uint32_t)(i >> 32), 1u, PU_TEST);
        uint8_t* q = out_qn + 16 * i;
        memset(q, 0, 16);
        if (sample_init(c, s, T, &st, q) != S_OK) return ORA_EREJECT;
    }
    return 0;
}

/* P5: T_vib of species sp as the root of <E_vib>(T) = mean vibrational energy
   above the ZPE (bends: harmonic closed form; stretches: Boltzmann sum over the
   Morse levels), by bisection. */
static double mean_evib_T(const o_species* s, double T) {
    double e = 0.0;
    for (int j = 0; j < s->n_modes; ++j) {
        if (s->is_bend[j]) {
            double th = s->d.theta[j - s->d.n_stretch];
            e += KB * th / (exp(th / T) - 1.0);
        } else {
            double num = 0.0, den = 0.0;
            for (int i = 0; i < s->n_levels[j]; ++i) {
                double de = s->E[j][i] - s->E[j][0];
                double b = exp(-de / (KB * T));
                num += de * b;
                den += b;
            }
            e += num / den;
        }
    }
    return e;
}
double ora_tvib(ora_ctx* c, int res, int sp) {
    o_res* R = c->res[res];
    const o_species* s = &c->sp[sp];
    double sum = 0.0;
    int64_t n = 0;
    for (int j = 0; j < R->n_cells; ++j)
        for (int i = 0; i < R->cells[j].n; ++i)
            if (R->cells[j].p[i].sp == sp) {
                sum += evib(s, R->cells[j].p[i].qn) - s->zpe;
                n++;
            }
    if (n == 0 || s->n_modes == 0) return 0.0;
    double target = sum / (double)n;
    if (!(target > 0.0)) return 0.0;
    double lo = 1.0, hi = 1.0e6;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mean_evib_T(s, mid) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}
