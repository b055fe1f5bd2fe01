// hcao_internal.h -- data layout shared by the host side and the kernels of
// libhcao.  Particle state lives in HBM as one fixed-size record per particle,
// grouped cell by cell (each cell owns a contiguous run of slots), so that the
// two members of a candidate pair are fetched with 128-bit loads and a cell's
// pairs touch one contiguous region.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hcao.h"

namespace hcao {

constexpr int MAXM = 16;        // vibrational modes per species
constexpr int MAXS = 16;        // species
constexpr int MAXR = 8;         // reactions
constexpr int MAXL = 256;       // levels per mode (quantum numbers are bytes)
#ifndef HCAO_F32_BUCKET_BITS
#define HCAO_F32_BUCKET_BITS 8
#endif
constexpr int F32_BUCKET_BITS = HCAO_F32_BUCKET_BITS;  // FP32 K5 buckets: mantissa bits per octave (~0.4% wide)
constexpr int TABLE_PAD = 17;   // grid entries beyond M (one per mode + 1)
constexpr int MAX_ROUNDS = 4;   // NTC pairing rounds per cell and step (hard cap)
constexpr int REC_NODES = HCAO_REC_NODES;  // recombination rate table: T_i = 500 K * 2^(i/32)
constexpr int MAX_REMOVALS = HCAO_MAX_REMOVALS_PER_CELL;
constexpr int FINISH_CHUNK = 1024;  // pair slots per warp of the end-of-step kernels
constexpr uint64_t POOL_KEEP_BYTES = 8ull << 30;  // unused memory a context's pool keeps mapped
constexpr int NCLS = 16;        // work classes of the FP32 relaxation queue
constexpr int QCNT_OFF = 2 * MAX_ROUNDS;               // StepArgs::qsize: per-class counts
constexpr int QCUR_OFF = QCNT_OFF + MAX_ROUNDS * NCLS;  // StepArgs::qsize: per-class placement cursors
constexpr int QSIZE_WORDS = QCUR_OFF + MAX_ROUNDS * NCLS;  // queue counters (StepArgs::qsize)
constexpr int SETUP_TILE = 256;     // cells per CTA of the step set-up
// prefix arrays built by the set-up: pairs of rounds 0..MAX_ROUNDS-1, all
// pairs, FINISH_CHUNK chunks, particles
enum { SA_ALL = MAX_ROUNDS, SA_CHUNK, SA_PART, SETUP_ARRAYS };
inline int setup_tiles(int n_cells) { return n_cells <= SETUP_TILE ? 1 : (n_cells + SETUP_TILE - 1) / SETUP_TILE; }

// Philox stream purposes: counter word 3 = purpose << 24 | block index.
enum { PU_NSEL = 1, PU_PERM = 2, PU_PAIR = 3, PU_LB_A = 4, PU_LB_B = 5, PU_SCAT = 6,
       PU_INIT = 7, PU_REC = 9, PU_TCE = 10, PU_ROT = 11, PU_ROTINIT = 12 };
constexpr int TCE_NT = 4096;    // TCE probability tables: NT + 1 points per (reaction, partner species)

// per-reservoir counters
enum { CNT_CAND = 0, CNT_ACC, CNT_SAMPLES, CNT_TRIALS, CNT_OVER, CNT_DEGEN, CNT_NOTEXEC,
       CNT_STEPS, CNT_RX0 = 8, NCNT = 8 + MAXR };

// load-path validation bits
enum { LOAD_BAD_CELL = 1, LOAD_BAD_SPECIES = 2, LOAD_BAD_LEVEL = 4 };

// sticky device error bits
enum { ERR_REJECT = 1, ERR_CAPACITY = 2, ERR_ROUNDS = 4, ERR_LEVEL = 8, ERR_NONFINITE = 16 };

constexpr uint32_t SPECIES_NONE = 0xFFu;

// Particle records.  FP32: 32 bytes (one sector); FP64: 64 bytes (two sectors).
// A rotating species' classical rotational energy: FP32, the float in q[3]
// (such species have at most 12 modes); FP64, erot.
struct alignas(16) RecF {
    float v[3];
    uint32_t meta;        // species in bits 0..7
    uint32_t q[4];        // quantum numbers, mode j in byte j
};
struct alignas(16) RecD {
    double v[3];
    uint32_t meta;
    uint32_t pad;
    uint32_t q[4];
    double erot;
    uint32_t pad2[2];
};
static_assert(sizeof(RecF) == 32, "RecF layout");
static_assert(sizeof(RecD) == 64, "RecD layout");

struct DevSpecies {
    double mass, E_form, zpe, top;   // top: highest collision energy the sampler covers
    double De[MAXM];                 // Morse De per stretch
    double base[MAXM + 1];           // K5 grid base per table (sum of ground levels k..n-1)
    double cq, inv_cq;               // quadratic grid g_m = base_k + cq m^2
    double eps_min;                  // smallest single-quantum excitation
    float base_f[MAXM + 1];
    float cq_f, inv_cq_f, eps_min_f, pad_f;
    int gshift, gj0;                 // FP32 buckets: (bits(E - base) >> gshift) - gj0
    int n_modes, n_stretch, MT, M;
    int lev_off[MAXM];               // offset of mode j's levels in the level arrays
    int n_lev[MAXM];
    int tab_off;                     // offset of table 0; table k at tab_off + k * MT
    float mass_f;
    float mass_lo_f;                 // mass - mass_f rounded to float: mass_f + mass_lo_f carries ~48 bits
    int pad;
    // FP32-mode bookkeeping in int64 fixed point (1 unit = 2^-100 J)
    long long zpe_fix, top_fix;
    long long De_fix[MAXM];
    // rotation: classical degrees of freedom (0, 2, 3) and the maximum of the
    // LB fraction's density shape x^(rot_dof/2 - 1) (1 - x)^(3/2 - omega)
    int rot_dof, pad_r;
    double rot_fmax;
    float rot_fmax_f, pad_rf;
    // products of a reaction with the collision-temperature split: bend
    // temperatures (K) by mode index (0 for stretches) and the offset of the
    // exponent-1/2 tables (-1 if none)
    double theta[MAXM];
    int tab_off_h, pad_h;
};

// FP32 K5 table entry of (species, mode k, bucket m), parallel to the float
// tables: the table value at the bucket's upper edge, and the bucket's alias
// table (first slot, slots = levels below the edge; 0 if no level fits).
// Looking up the acceptance weight of mode k's draw also fetches mode k+1's
// alias table: both index the same bucket.
struct alignas(16) K5Ent {
    float H;
    uint32_t off, L, pad;
};

// One alias-table slot j of a bucket: threshold, alias, and level j's and
// its alias's weights at the bucket edge; 16 bytes on a 16-byte boundary.
// The levels' energies come from the (L1-resident) level lists.
struct alignas(16) AliasEnt {
    float prob;
    uint32_t alias;
    float wg_j, wg_a;
};

struct DevPair {
    double mr, C, mt, fp, fq;        // reduced mass, VHS constant, total mass, velocity shares
    float mr_f, C_f, fp_f, fq_f, inv2mr_f;
    uint32_t qk;                     // a QK dissociation or exchange exists for this species pair
    uint32_t cls;                    // FP32 relaxation-queue work class (assign_work_classes)
};

// DISS: A + M -> P0 + P1; EXCH: A + B -> P0 + P1; RECOMB: A + B (+ M) -> P0
struct DevReaction {
    int type, A, B, P0, P1;
    uint32_t mask;
    int alpha_mode;
    int rslot;                       // RECOMB: slot of its rate table
    int model;                       // DISS / EXCH: HCAO_MODEL_QK or HCAO_MODEL_TCE
    int tce_slot;                    // TCE: slot of its probability tables
    int tce_zeta_on;                 // TCE: the vibrational energies count in E_c
    int tce_mode;                    // TCE dissociation: the stretch reported as broken
    double tce_Ea;                   // TCE: E_a (J)
    double Ea, steric, zpesum, dEf;
    double alpha[MAXM];
    long long Ea_fix, zpesum_fix, dEf_fix;   // FP32 mode (2^-100 J units)
    double gamma;                    // rotation-vibration coupling: gamma E_rot,A in the QK E_coll
    float gamma_f, pad_gf;
    int prod_split;                  // HCAO_SPLIT_RELAX or HCAO_SPLIT_TCOLL
    int tcb_off;                     // FP32, DISS / EXCH with TCOLL: offset of its b1 table
};
// FP32 b1 tables of the collision-temperature split: b1 at E_x = 2^(TCB_L0 +
// i / TCB_PER_OCTAVE) J, i = 0..TCB_N-1, linear in log2 E_x (clamped)
#define TCB_N 4096
#define TCB_L0 (-80.0)
#define TCB_PER_OCTAVE 128.0

struct Consts {
    int n_species, n_reactions, amode, creates;
    int has_recomb, has_tce, has_rot, n_cls;  // n_cls: FP32 relaxation-queue work classes in use
    int rec_pair[MAXS * MAXS];       // species pair -> recombination | side << 3, or -1
    DevSpecies sp[MAXS];
    DevPair pair[MAXS * MAXS];
    DevReaction rx[MAXR];
};

struct DevCell {
    void* rec;                        // first record of the cell
    uint32_t n, cap;                  // particles at step start, slots
    uint32_t res, lcell;              // reservoir slot, reservoir-local cell index
    double sgmax;                     // (sigma_T g)_max
    unsigned long long seen;          // max sigma_T g of this step (bits of a double >= 0)
    uint32_t nsel, ncreated;
    float sgmax_f;                    // FP32 copy of sgmax for the step
    uint32_t nremoved;                // particles removed this step (recombination)
    uint32_t rmfill;                  // removed positions gathered into rmpos this step
    uint32_t pkey[MAX_ROUNDS][4];     // pairing-permutation keys per round of this step
};

struct DevRes {
    uint64_t seed;
    uint32_t step;
    uint32_t active;
    double w, dt, Vc;
};

struct StepArgs {
    const Consts* C;
    const double* lev64;
    const float* lev32;
    const long long* levfix;        // level energies in 2^-100 J units (FP32-mode bookkeeping)
    const double* H64;
    const float* H32;
    const K5Ent* k5e;               // FP32 K5 tables with their alias proposals, parallel to H32
    const AliasEnt* ae;             // FP32 alias-table slots
    const double* H64h;             // exponent-1/2 tables of the collision-temperature split:
    const K5Ent* k5eh;              //   FP64 tables, FP32 tables + alias slots (offsets DevSpecies
    const AliasEnt* aeh;            //   tab_off_h), FP32 b1 tables (DevReaction tcb_off)
    const float* tcb;
    DevCell* cells;
    int n_cells;
    DevRes* res;
    int n_res;
    unsigned long long* counters;   // [n_res][NCNT]
    uint32_t* pbase;                // [MAX_ROUNDS][n_cells + 1]: round-r pair prefix
    uint32_t* blkcell;              // [MAX_ROUNDS][blk_stride]: cell of round r's pair 256 b
    uint32_t blk_stride;
    uint32_t* abase;                // [n_cells + 1]: all-round pair prefix
    uint32_t* totals;               // [MAX_ROUNDS + 2]: pairs per round, all pairs, chunks
    uint32_t* chbase;               // [n_cells + 1]: prefix of FINISH_CHUNK chunks of each cell's pairs
    uint32_t* chcnt;                // [chunks]: particles created in each chunk
    uint32_t* cflag;                // per-pair event word (acceptance, reaction, creation, trials)
    uint32_t* rmpos;                // recombination: a cell's removed positions at its event
                                    // slots [abase, abase + nremoved), gathered by k_finish_count
    void* cscratch;                 // per-pair record of a particle created by a reaction
    uint4* qA;                      // [2 pair_cap] accepted pairs of the current round (cell, pair, ip, iq);
                                    // FP32: k_select stages them at qA[pair_cap + i] with the work
                                    // class in the pair word's top byte, k_qorder places them
                                    // class by class at qA[0 ..)
    uint4* qB;                      // reacting pairs (cell, pair, channel)
    uint32_t* qsize;                // [QSIZE_WORDS]: per round, relax-queue entries and
                                    // react-queue length; then per round and class the FP32
                                    // relax queue's counts (QCNT_OFF), then the placement
                                    // cursors (QCUR_OFF)
    int has_reactions;
    int has_recomb;
    int creates;                    // a reaction creates particles or removes them (scratch slots)
    const double* krec;             // [slot][MAXS][REC_NODES] recombination k_r at the nodes
    const double* Tnode;            // [REC_NODES]
    long long* csum;                // [n_cells][5] integer sums: E (2^-96 J), p (2^-104), m (2^-120)
    uint32_t* nbase;                // [n_cells + 1]: particle prefix at step start
    uint32_t* tsum;                 // [SETUP_ARRAYS][setup tiles + 1] tile totals, then a ticket
    unsigned long long* work;       // [4] K5 level evaluations, mode starts, molecule samples, pairs
    int grid_select, grid_relax, grid_react;  // launch shapes (host-side; results do not depend on them)
    int qorder;                     // FP32: the relaxation queue is staged and placed by work class
    uint64_t pair_cap;              // capacity of cflag / log
    hcao_log_rec* log;
    int log_on;
    uint32_t* err;
    int max_rounds;
    uint32_t reject_cap;
    const double* tce;              // [slot][MAXS][TCE_NT + 1] TCE probabilities (see tce_prob)
    double tce_span;                // TCE tables: energy span X above E_a (J)
    uint32_t* ticket;               // fused step: CTAs finished (the last one advances the reservoirs)
    int fused_recs;                 // fused step: records staged per CTA (0 on the queue path)
};

// The FP32 step as one kernel per step, one CTA per cell with its records in
// shared memory (hcao_fused.cuh, built in hcao_f32.cu).  It serves contexts
// whose reactions neither create nor remove particles and whose cells all
// hold at most FUSED_MAX_RECS particle slots.
constexpr int FUSED_MAX_RECS = 4096;
void launch_fused(const StepArgs& a, int smem_recs, cudaStream_t s);
cudaError_t fused_prepare(int smem_recs);  // the kernel's dynamic shared-memory limit

// launchers, one instantiation per precision (hcao_f64.cu / hcao_f32.cu)
template <class R> struct RecOf;
template <> struct RecOf<float> { using T = RecF; };
template <> struct RecOf<double> { using T = RecD; };

template <class R> void launch_step(const StepArgs& a, int grid_collide, int block_collide,
                                    cudaStream_t s, uint64_t* launches);
int launch_setup(const StepArgs& a, cudaStream_t s);  // precision-independent (hcao_f64.cu); returns launches
void launch_validate_load(const Consts* C, int n_cells, const int32_t* cell, const int32_t* sp,
                          const uint8_t* qn, int64_t n, uint32_t* flags, cudaStream_t s);
// precision-independent read-outs on the device: a reservoir's particle prefix
// over its cells (n_cells + 1 entries), and its counters summed over its cells
// into out (zeroed by the caller)
void launch_cell_prefix(const DevCell* cells, int cell0, int n_cells, uint64_t* off, cudaStream_t s);
void launch_sum_counters(const unsigned long long* cnt, int cell0, int n_cells, int n_cnt, unsigned long long* out,
                         cudaStream_t s);
template <class R> void launch_collide(const StepArgs& a, int r, int grid, int block, cudaStream_t s);
// phase k of round r: 0 select, 1 relax, 2 react (for per-kernel timing)
template <class R> void launch_phase(const StepArgs& a, int r, int phase, int grid, cudaStream_t s);
template <class R> void launch_finish(const StepArgs& a, cudaStream_t s);
// recombination: per-cell temperature sums before the rounds, removals after
template <class R> void launch_cellstats(const StepArgs& a, cudaStream_t s);
template <class R> void launch_compact(const StepArgs& a, cudaStream_t s);
template <class R> void launch_scatter_load(void* rec_base, const uint32_t* perm,
                                            const uint32_t* offsets, const uint64_t* cell_slot0,
                                            int n_cells, const double* v, const float* vf,
                                            const uint8_t* qn, const int32_t* sp, int64_t n,
                                            cudaStream_t s);
template <class R> void launch_pack(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,
                                    uint64_t total, const Consts* C, double* v, uint8_t* qn, int32_t* sp,
                                    int32_t* cell, cudaStream_t s);
// rotational energies out of / into the records (canonical order), and
// their initialisation at T_rot
template <class R> void launch_erot(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,
                                    uint64_t total, const Consts* C, double* host_order_erot, int to_records,
                                    cudaStream_t s);
template <class R> void launch_init_rot(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,
                                        uint64_t total, const DevRes* res, int res_slot, const Consts* C,
                                        double T_rot, cudaStream_t s);
template <class R> void launch_init_vib(const DevCell* cells, int cell0, int n_cells,
                                        const uint64_t* off, uint64_t total, const DevRes* res,
                                        int res_slot, const Consts* C, const double* bend_thr,
                                        const double* str_acc, const int* thr_off,
                                        uint32_t reject_cap, uint32_t* err, cudaStream_t s);
template <class R> void launch_moments(const DevCell* cells, int cell0, int n_cells,
                                       const uint64_t* off, uint64_t total, const Consts* C,
                                       const double* lev64, const long long* levfix, double* acc,
                                       unsigned long long* cnt, cudaStream_t s);
template <class R> void launch_sample_diag(const StepArgs& a, int sp, double Ec, uint64_t seed,
                                           int64_t n, uint8_t* out, unsigned long long* trials,
                                           int* status, cudaStream_t s);
template <class R> void launch_levelpop(const DevCell* cells, int cell0, int n_cells,
                                        const uint64_t* off, uint64_t total, int sp, int mode,
                                        unsigned long long* hist, cudaStream_t s);

}  // namespace hcao
