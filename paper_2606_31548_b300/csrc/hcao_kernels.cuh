// hcao_kernels.cuh -- the collision-phase kernels of libhcao (sm_103a).
//
// One step of the DSMC collision phase, per reservoir cell:
//   k_setup_cells  one thread per cell, CTAs of SETUP_TILE cells: NTC candidate
//                  count N_sel = 1/2 N(N-1) w (sigma g)_max dt / V_c with
//                  stochastic rounding, pairing-permutation keys per round, tile
//                  scans of the per-cell counts; the last CTA scans the tiles.
//   k_setup_fix    adds the tile offsets (flat pair index of every candidate)
//                  and tabulates the cell of every 256th candidate of each round.
//   k_cellstats    (recombination only) per-cell sums for the cell temperature.
//   per pairing round:
//   k_select       one thread per candidate pair: permuted pair draw, VHS
//                  acceptance; FP32 mode stages accepted pairs with their
//                  species pair's work class and counts them per class.
//   k_qorder       (FP32, more than one work class) places the staged queue
//                  class by class, so a warp's pairs run like mode-draw loops.
//   k_relax_fast   (FP32) one thread per accepted pair: recombination and QK
//                  reaction tests (Eq. Ecoll-diss, Eq. Ecoll-exch, competing
//                  reactions) -- reacting pairs go to a second queue -- else
//                  the HCAO Larsen-Borgnakke relaxation of each molecule (the
//                  joint acceptance of all modes, drawn exactly with the K5
//                  tables and alias proposals) and isotropic VHS scattering.
//   k_relax        (FP64) the same with the sequential K5 scan of the oracle.
//   k_react        one thread per reacting pair: dissociation, exchange,
//                  recombination.
//   end of step, one warp per FINISH_CHUNK pair slots of a cell:
//   k_finish_count per-cell counters; k_finish_append stable append of created
//   particles; k_cellupd (sigma g)_max, counts, step; k_compact removals.
// Read-outs run flat over a reservoir's particles in canonical order, on a
// particle prefix the device scans (k_cell_prefix): k_moments (momentum and
// energies; FP32 in int64 fixed point), k_levelpop, k_pack, k_erot; the
// counters are summed over the cells on the device (k_sum_counters).
// Queue order is irrelevant: pairs of one round are disjoint and every draw is
// keyed by (step, cell, round, pair), never by a thread or queue position.
// Randomness: Philox4x32-10 keyed by the reservoir seed, counter
// (step, cell, round<<24 | pair, purpose<<24 | block): draws do not depend on
// launch geometry, so results are identical for any grid or batching.
//
// Template parameter R: double = FP64 parity mode (the translation unit is
// compiled without FMA contraction; every expression follows the documented
// operation order), float = FP32 mode (velocities, relative speeds and the
// sampler in FP32; energies, reaction thresholds and bookkeeping in int64
// fixed point, 1 unit = 2^-100 J).
#pragma once
#include <cstdint>
#include <type_traits>

#include "hcao_internal.h"

namespace hcao {

// ------------------------------------------------------------- arithmetic
// Round-to-nearest intrinsics never contract into FMA: the sampler and its
// host-built tables then see bit-identical arithmetic in either precision.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float ceil_r(float a) { return ceilf(a); }
__device__ __forceinline__ double ceil_r(double a) { return ceil(a); }

// (E_coll - sum E)^(xi_rel/2 - 1), xi_rel = 5 - 2 omega: exponent 3/4, 1, 1/2
template <class R>
__device__ __forceinline__ R lb_pow(int amode, R x) {
    if (amode == 0) {
        R s = sqrt_rn(x);
        return mul_rn(s, sqrt_rn(s));
    }
    if (amode == 1) return x;
    return sqrt_rn(x);
}

// The same weight for the FP32 kernels with approximate reciprocal square
// roots (x > 0): its ~1e-7 relative difference from the host-built FP32
// tables only moves a draw whose uniform lies that close to a level boundary.
__device__ __forceinline__ float lb_pow_fast(int amode, float x) {
    if (amode == 1) return x;
    const float s = x * rsqrtf(x);  // sqrt(x)
    if (amode == 2) return s;
    return s * (s * rsqrtf(s));     // x^(3/4)
}

// ------------------------------------------------------------- Philox4x32-10
__device__ __forceinline__ void philox10(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                         uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
        uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
        uint32_t n0 = hi1 ^ x1 ^ k0;
        uint32_t n2 = hi0 ^ x3 ^ k1;
        x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
    }
}

// A counter-based stream of Philox blocks, consumed word by word: an FP64
// uniform takes words (0,1) then (2,3) of a block, an FP32 uniform one word
// (0, 1, 2, 3 in turn).  A stream is read at one precision only.
struct Stream {
    uint32_t k0, k1, c0, c1, c2, c3;
    uint32_t blk;
    uint32_t w0, w1, w2, w3;
    int pos;  // next unread word; 4 = block used up
};
__device__ __forceinline__ void st_init(Stream& s, uint64_t seed, uint32_t c0, uint32_t c1,
                                        uint32_t c2, uint32_t purpose) {
    s.k0 = (uint32_t)seed; s.k1 = (uint32_t)(seed >> 32);
    s.c0 = c0; s.c1 = c1; s.c2 = c2; s.c3 = purpose << 24;
    s.blk = 0; s.pos = 4;
}
__device__ __forceinline__ void st_block(Stream& s) {
    s.w0 = s.c0; s.w1 = s.c1; s.w2 = s.c2; s.w3 = s.c3 | (s.blk & 0xFFFFFFu);
    philox10(s.w0, s.w1, s.w2, s.w3, s.k0, s.k1);
    s.blk++;
}
__device__ __forceinline__ void st_pair(Stream& s, uint32_t& a, uint32_t& b) {
    if (s.pos > 2) { st_block(s); s.pos = 0; }
    if (s.pos == 0) { a = s.w0; b = s.w1; }
    else { a = s.w2; b = s.w3; }
    s.pos += 2;
}
// FP64 uniform: (27 bits of a, 26 bits of b) * 2^-53; FP32 uniform: 24 bits of one word * 2^-24
__device__ __forceinline__ double st_u64(Stream& s) {
    uint32_t a, b;
    st_pair(s, a, b);
    uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return (double)m * 0x1p-53;
}
// the next 32-bit word
__device__ __forceinline__ uint32_t st_word(Stream& s) {
    if (s.pos > 3) { st_block(s); s.pos = 0; }
    const uint32_t w = s.pos == 0 ? s.w0 : (s.pos == 1 ? s.w1 : (s.pos == 2 ? s.w2 : s.w3));
    s.pos++;
    return w;
}
__device__ __forceinline__ float st_u32(Stream& s) { return (float)(st_word(s) >> 8) * 0x1p-24f; }
// The same stream with its key and fixed counter words in shared memory (one
// column per thread of a CTA of at most 128 threads: k_relax_fast, launched
// with 128), so that a long loop of draws holds only the block counter and
// the buffered block in registers: the FP32 relaxation kernel's LB draws
// (the kernel spills under its 64-register bound; 6 fewer live registers in
// the draw loop made the exchange step 2% faster).  The words drawn are those
// of Stream.
static __shared__ uint32_t s_lbkey[6][128];
struct LbStream {
    uint32_t blk;
    uint32_t w0, w1, w2, w3;
    int pos;
};
__device__ __forceinline__ void st_init(LbStream& s, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                        uint32_t purpose) {
    const int t = threadIdx.x;
    s_lbkey[0][t] = (uint32_t)seed; s_lbkey[1][t] = (uint32_t)(seed >> 32);
    s_lbkey[2][t] = c0; s_lbkey[3][t] = c1; s_lbkey[4][t] = c2; s_lbkey[5][t] = purpose << 24;
    s.blk = 0; s.pos = 4;
}
__device__ __forceinline__ uint32_t st_word(LbStream& s) {
    if (s.pos > 3) {
        const int t = threadIdx.x;
        s.w0 = s_lbkey[2][t]; s.w1 = s_lbkey[3][t]; s.w2 = s_lbkey[4][t]; s.w3 = s_lbkey[5][t] | (s.blk & 0xFFFFFFu);
        philox10(s.w0, s.w1, s.w2, s.w3, s_lbkey[0][t], s_lbkey[1][t]);
        s.blk++;
        s.pos = 0;
    }
    const uint32_t w = s.pos == 0 ? s.w0 : (s.pos == 1 ? s.w1 : (s.pos == 2 ? s.w2 : s.w3));
    s.pos++;
    return w;
}
// the top 24 bits of the next word (the bits behind st_u32)
__device__ __forceinline__ uint32_t st_bits24(Stream& s) { return st_word(s) >> 8; }
template <class R> __device__ __forceinline__ R st_uni(Stream& s);
template <> __device__ __forceinline__ double st_uni<double>(Stream& s) { return st_u64(s); }
template <> __device__ __forceinline__ float st_uni<float>(Stream& s) { return st_u32(s); }

// ------------------------------------------------------------- pairing permutation
// Keyed bijection of [0,N) that forms the disjoint NTC pairs of a round (pair k
// = (pi(2k), pi(2k+1))).  On b-bit words, b the smallest width with 2^b >= N,
// three rounds of x = ((x ^ k_r) * M_r) mod 2^b, x ^= x >> ceil(b/2) -- each
// step a bijection of [0, 2^b) -- repeated from the result until it lands in
// [0,N) (at most 2 evaluations on average).  Round keys: the round's key
// words 0..2; multipliers: the odd constants 0x9E3779B1, 0x85EBCA6B,
// 0xC2B2AE35.
__device__ __forceinline__ uint32_t pair_perm(uint32_t x, uint32_t N, const uint32_t key[4]) {
    if (N <= 1u) return 0u;
    const int b = 32 - __clz(N - 1u);  // smallest b with 2^b >= N
    const uint32_t mask = (uint32_t)(((uint64_t)1 << b) - 1u);
    const int h = (b + 1) >> 1;
    const uint32_t k0 = key[0] & mask, k1 = key[1] & mask, k2 = key[2] & mask;
    for (int walk = 0; walk < (1 << 20); ++walk) {
        x = ((x ^ k0) * 0x9E3779B1u) & mask;
        x ^= x >> h;
        x = ((x ^ k1) * 0x85EBCA6Bu) & mask;
        x ^= x >> h;
        x = ((x ^ k2) * 0xC2B2AE35u) & mask;
        x ^= x >> h;
        if (x < N) return x;
    }
    return 0;  // unreachable: a cycle through x < N returns to [0,N)
}

// ------------------------------------------------------------- quantum numbers
__device__ __forceinline__ uint32_t get_q(const uint32_t q[4], int j) {
    uint32_t w = j < 4 ? q[0] : (j < 8 ? q[1] : (j < 12 ? q[2] : q[3]));
    return (w >> ((j & 3) * 8)) & 0xFFu;
}
__device__ __forceinline__ void set_q(uint32_t q[4], int j, uint32_t v) {
    uint32_t sh = (uint32_t)(j & 3) * 8u;
    uint32_t m = ~(0xFFu << sh), val = v << sh;
    switch (j >> 2) {
        case 0: q[0] = (q[0] & m) | val; break;
        case 1: q[1] = (q[1] & m) | val; break;
        case 2: q[2] = (q[2] & m) | val; break;
        default: q[3] = (q[3] & m) | val; break;
    }
}

// ------------------------------------------------------------- records
// Record traffic of the FP32 step kernels carries the evict-first (streaming)
// cache policy, so that the records a step touches (630 MB for 19.7M
// particles) push fewer sampler-table lines out of L2 (measured: step 3-6%
// faster on the exchange mixture and the heat bath).
#define REC_LD(p) __ldcs(p)
#define REC_ST(p, v) __stcs((p), (v))
#ifndef HCAO_RELAX_MINB
#define HCAO_RELAX_MINB 8
#endif
__device__ __forceinline__ void load_rec(const RecF* p, RecF& r) {
    const uint4* s = reinterpret_cast<const uint4*>(p);
    uint4 a = s[0], b = s[1];
    r.v[0] = __uint_as_float(a.x); r.v[1] = __uint_as_float(a.y); r.v[2] = __uint_as_float(a.z);
    r.meta = a.w;
    r.q[0] = b.x; r.q[1] = b.y; r.q[2] = b.z; r.q[3] = b.w;
}
__device__ __forceinline__ void store_rec(RecF* p, const RecF& r) {
    uint4* d = reinterpret_cast<uint4*>(p);
    d[0] = make_uint4(__float_as_uint(r.v[0]), __float_as_uint(r.v[1]), __float_as_uint(r.v[2]), r.meta);
    d[1] = make_uint4(r.q[0], r.q[1], r.q[2], r.q[3]);
}
__device__ __forceinline__ void load_rec(const RecD* p, RecD& r) {
    const uint4* s = reinterpret_cast<const uint4*>(p);
    uint4 a = s[0], b = s[1], c = s[2];
    r.v[0] = __hiloint2double((int)a.y, (int)a.x);
    r.v[1] = __hiloint2double((int)a.w, (int)a.z);
    r.v[2] = __hiloint2double((int)b.y, (int)b.x);
    r.meta = b.z; r.pad = 0;
    r.q[0] = c.x; r.q[1] = c.y; r.q[2] = c.z; r.q[3] = c.w;
    const uint4 e = s[3];
    r.erot = __hiloint2double((int)e.y, (int)e.x);
    r.pad2[0] = r.pad2[1] = 0u;
}
__device__ __forceinline__ void store_rec(RecD* p, const RecD& r) {
    uint4* d = reinterpret_cast<uint4*>(p);
    unsigned long long v0 = __double_as_longlong(r.v[0]), v1 = __double_as_longlong(r.v[1]),
                       v2 = __double_as_longlong(r.v[2]);
    d[0] = make_uint4((uint32_t)v0, (uint32_t)(v0 >> 32), (uint32_t)v1, (uint32_t)(v1 >> 32));
    d[1] = make_uint4((uint32_t)v2, (uint32_t)(v2 >> 32), r.meta, 0u);
    d[2] = make_uint4(r.q[0], r.q[1], r.q[2], r.q[3]);
    const unsigned long long e = __double_as_longlong(r.erot);
    d[3] = make_uint4((uint32_t)e, (uint32_t)(e >> 32), 0u, 0u);
}

// ------------------------------------------------------------- rotation
// A molecule's classical rotational energy (Sec. "Rotation coupling"): FP64
// records hold it as a double, FP32 records as the float in q[3] (rotating
// species have at most 12 modes).
__device__ __forceinline__ float erot_f(const uint32_t q[4]) { return __uint_as_float(q[3]); }
// the FP64 record's rotational energy (0 for a species that does not rotate);
// the FP32 overloads serve only code paths that FP32 mode never runs
__device__ __forceinline__ double rec_erot(const RecD& r) { return r.erot; }
__device__ __forceinline__ double rec_erot(const RecF&) { return 0.0; }
__device__ __forceinline__ void rec_set_erot(RecD& r, double e) { r.erot = e; }
__device__ __forceinline__ void rec_set_erot(RecF&, double) {}
// a record's rotational energy in either precision (readouts)
__device__ __forceinline__ double rec_erot_of(const RecD& r, const DevSpecies&) { return r.erot; }
__device__ __forceinline__ double rec_erot_of(const RecF& r, const DevSpecies& S) {
    return S.rot_dof ? (double)erot_f(r.q) : 0.0;
}
__device__ __forceinline__ void rec_put_erot(RecD& r, const DevSpecies& S, double e) { r.erot = S.rot_dof ? e : 0.0; }
__device__ __forceinline__ void rec_put_erot(RecF& r, const DevSpecies& S, double e) {
    if (S.rot_dof) r.q[3] = __float_as_uint((float)e);
}

// Natural logarithm for x > 0 (normal doubles), the draws of the initial
// rotation: x = m 2^e with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s),
// s = (m - 1)/(m + 1), by the atanh series to s^25, plus e ln 2; every
// operation rounded as written.
__device__ __forceinline__ double ln_series(double x) {
    unsigned long long u = (unsigned long long)__double_as_longlong(x);
    int e = (int)((u >> 52) & 0x7FF) - 1022;
    u = (u & 0x000FFFFFFFFFFFFFull) | 0x3FE0000000000000ull;
    double m = __longlong_as_double((long long)u);
    if (m < 0.70710678118654752440) { m = __dmul_rn(m, 2.0); e = e - 1; }
    const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double s2 = __dmul_rn(s, s);
    double t = __ddiv_rn(1.0, 25.0);
    for (int k = 23; k >= 1; k -= 2) t = __dadd_rn(__ddiv_rn(1.0, (double)k), __dmul_rn(s2, t));
    return __dadd_rn(__dmul_rn(__dmul_rn(2.0, s), t), __dmul_rn((double)e, 0.69314718055994530942));
}

// Exponential for -708 <= x <= 709 (0 below), every operation rounded as
// written: x = k ln 2 + r with k the integer nearest x / ln 2, ln 2 split into
// L1 (29 significant bits: k L1 is exact) and L2 = ln 2 - L1, e^r by its
// Taylor series to r^18 in Horner form, times 2^k built from its exponent bits.
__device__ __forceinline__ double exp_series(double x) {
    if (x < -708.0) return 0.0;
    if (x > 709.0) return __longlong_as_double(0x7FF0000000000000ll);
    const double L1 = 0x1.62e42ffp-1, L2 = -0x1.718432a1b0e26p-35;
    const int k = (int)floor(__dadd_rn(__dmul_rn(x, 0x1.71547652b82fep+0), 0.5));
    const double kd = (double)k;
    const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(kd, L1)), __dmul_rn(kd, L2));
    double t = 1.0;
    for (int n = 18; n >= 1; --n) t = __dadd_rn(1.0, __ddiv_rn(__dmul_rn(r, t), (double)n));
    return __dmul_rn(t, __longlong_as_double((long long)(k + 1023) << 52));
}
// x^y = e^(y ln x) for x > 0 from the two series
__device__ __forceinline__ double pow_series(double x, double y) { return exp_series(__dmul_rn(y, ln_series(x))); }

// The classical LB fraction x ~ Beta(rot_dof/2, (5 - 2 omega)/2) of the
// energy a rotating molecule keeps: rejection under the maximum of the
// density shape x^(rot_dof/2 - 1) (1 - x)^(3/2 - omega), square roots only.
template <class R>
__device__ __forceinline__ R rot_fraction(const StepArgs& A, const DevSpecies& S, int amode, Stream& st) {
    for (uint32_t it = 0; it < A.reject_cap; ++it) {
        const R x = st_uni<R>(st);
        const R y = st_uni<R>(st);
        R f = lb_pow<R>(amode, sub_rn((R)1, x));
        if (S.rot_dof == 3) f = mul_rn(f, sqrt_rn(x));
        R fm;
        if constexpr (std::is_same<R, double>::value) fm = S.rot_fmax;
        else fm = S.rot_fmax_f;
        if (mul_rn(y, fm) < f) return x;
    }
    return (R)0.5;
}

// ------------------------------------------------------------- tables
template <class R> __device__ __forceinline__ const R* lev_tab(const StepArgs& A);
template <> __device__ __forceinline__ const double* lev_tab<double>(const StepArgs& A) { return A.lev64; }
template <> __device__ __forceinline__ const float* lev_tab<float>(const StepArgs& A) { return A.lev32; }
template <class R> __device__ __forceinline__ const R* h_tab(const StepArgs& A);
template <> __device__ __forceinline__ const double* h_tab<double>(const StepArgs& A) { return A.H64; }
template <> __device__ __forceinline__ const float* h_tab<float>(const StepArgs& A) { return A.H32; }
template <class R> __device__ __forceinline__ R sp_base(const DevSpecies& S, int k);
template <> __device__ __forceinline__ double sp_base<double>(const DevSpecies& S, int k) { return S.base[k]; }
template <> __device__ __forceinline__ float sp_base<float>(const DevSpecies& S, int k) { return S.base_f[k]; }
template <class R> __device__ __forceinline__ R sp_cq(const DevSpecies& S);
template <> __device__ __forceinline__ double sp_cq<double>(const DevSpecies& S) { return S.cq; }
template <> __device__ __forceinline__ float sp_cq<float>(const DevSpecies& S) { return S.cq_f; }
template <class R> __device__ __forceinline__ R sp_inv(const DevSpecies& S);
template <> __device__ __forceinline__ double sp_inv<double>(const DevSpecies& S) { return S.inv_cq; }
template <> __device__ __forceinline__ float sp_inv<float>(const DevSpecies& S) { return S.inv_cq_f; }
template <class R> __device__ __forceinline__ R sp_eps(const DevSpecies& S);
template <> __device__ __forceinline__ double sp_eps<double>(const DevSpecies& S) { return S.eps_min; }
template <> __device__ __forceinline__ float sp_eps<float>(const DevSpecies& S) { return S.eps_min_f; }

// quadratic grid point g_m = base + cq m^2 (m^2 exact in either precision)
template <class R>
__device__ __forceinline__ R grid_pt(R base, R cq, int m) {
    return add_rn(base, mul_rn(cq, (R)(m * m)));
}
// smallest m in [1, MT) with g_m >= E; 0 if E <= base; MT if no grid point
// reaches E.  The candidate from sqrt is corrected against the grid points,
// so the result is the exact function the host tables were built with.
template <class R>
__device__ __forceinline__ int grid_idx(R base, R cq, R inv, int MT, R E) {
    if (!(E > base)) return 0;
    const float t = (float)mul_rn(sub_rn(E, base), inv);
    int m;
    if (!(t < (float)MT * (float)MT)) m = MT - 1;
    else {
        m = (int)ceilf(sqrtf(t));
        m = m < 1 ? 1 : (m > MT - 1 ? MT - 1 : m);
    }
    for (int it = 0; it < 64 && m > 1 && !(grid_pt<R>(base, cq, m - 1) < E); ++it) m--;
    for (int it = 0; it < 64 && grid_pt<R>(base, cq, m) < E; ++it) {
        if (m == MT - 1) return MT;
        m++;
    }
    return m;
}

// FP32 buckets: idx(E) = ceil(sqrt((E - base) * inv)) in IEEE float (0 if E <=
// base, MT if above the last bucket).  The host builds the FP32 tables at each
// bucket's upper edge (the largest float with that index), so the same exact
// bound holds without comparing against grid points.
// FP32 buckets: a geometric grid read off the float bit pattern of x = E - base:
// idx = (bits(x) >> shift) - j0, at least 1 (0 if E <= base, MT past the last
// bucket).  Monotone in E and exactly reproducible with integer operations; the
// host builds the FP32 tables at each bucket's upper edge.
__device__ __forceinline__ int grid_idx_f32(float base, int shift, int j0, int MT, float E) {
    if (!(E > base)) return 0;
    const int j = (int)(__float_as_uint(__fsub_rn(E, base)) >> shift) - j0;
    return j < 1 ? 1 : (j > MT - 1 ? MT : j);
}

// grid index of table k of species S in precision R (FP64: quadratic grid
// with exact correction; FP32: bit-pattern buckets)
template <class R> __device__ __forceinline__ int gidx(const DevSpecies& S, int k, R E);
template <> __device__ __forceinline__ int gidx<double>(const DevSpecies& S, int k, double E) {
    return grid_idx<double>(S.base[k], S.cq, S.inv_cq, S.MT, E);
}
template <> __device__ __forceinline__ int gidx<float>(const DevSpecies& S, int k, float E) {
    return grid_idx_f32(S.base_f[k], S.gshift, S.gj0, S.MT, E);
}

__device__ __forceinline__ double evib64(const double* lev, const DevSpecies& S, const uint32_t q[4]) {
    double e = 0.0;
    for (int j = 0; j < S.n_modes; ++j) e = e + __ldg(lev + S.lev_off[j] + get_q(q, j));
    return e;
}

// FP32-mode energy bookkeeping: int64 fixed point, 1 unit = 2^-100 J.  A
// float energy converts exactly (a power-of-two scale); sums are exact.
__device__ __forceinline__ long long f2fix(float x) { return __float2ll_rn(__fmul_rn(x, 0x1p100f)); }
__device__ __forceinline__ float fix2f(long long a) { return __fmul_rn(__ll2float_rn(a), 0x1p-100f); }
__device__ __forceinline__ double fix2d(long long a) { return __ll2double_rn(a) * 0x1p-100; }
// (unrolled over the 16 mode slots: each quantum number is a fixed byte of
// its word, and the integer sum does not depend on the order)
__device__ __forceinline__ long long evib_fix(const long long* lf, const DevSpecies& S, const uint32_t q[4]) {
    const int n = S.n_modes;
    long long e = 0;
#pragma unroll
    for (int j = 0; j < MAXM; ++j)
        if (j < n) e += __ldg(lf + S.lev_off[j] + ((q[j >> 2] >> ((j & 3) * 8)) & 0xFFu));
    return e;
}

enum { S_OK = 0, S_OVER = 1, S_DEGEN = 2, S_CAP = -1 };

// Post-collision vibrational state of one molecule at collision energy Ec:
// p(i) ~ (Ec - sum_j E_j(i_j))^(xi_rel/2-1) over states with sum E < Ec (the
// joint LB acceptance of all local modes).  Sequential draw through the H_k
// tables; a draw running past the end of a mode's levels restarts the trial.
// Every accepted state has probability lb_pow(..)/H_0: the target, exactly.
template <class R>
__device__ int sample_lb_tab(const StepArgs& A, const DevSpecies& S, int amode, const R* H, double Ec_d,
                             Stream& st, uint32_t q[4], uint32_t& trials) {
    const int n = S.n_modes;
    if (n == 0) return S_OK;
    const R* L = lev_tab<R>(A);
    const R cq = sp_cq<R>(S), inv = sp_inv<R>(S);
    const int MT = S.MT;
    const R Ec = (R)Ec_d;
    const R b0 = sp_base<R>(S, 0);
    const int m0 = gidx<R>(S, 0, Ec);
    if (m0 > S.M) return S_OVER;
    if (m0 == 0) return S_DEGEN;
    const R h0 = __ldg(H + m0);
    if (!(h0 > (R)0)) return S_DEGEN;
    // below the smallest single-quantum excitation only the ground state fits
    if (sub_rn(Ec, b0) < sp_eps<R>(S)) {
        q[0] = 0u; q[1] = 0u; q[2] = 0u; q[3] = 0u;
        return S_OK;
    }
    for (uint32_t trial = 0; trial < A.reject_cap; ++trial) {
        trials++;
        uint32_t nq[4] = {0u, 0u, 0u, 0u};
        R E = Ec;
        bool ok = true;
        for (int k = 0; k < n; ++k) {
            int m = (k == 0) ? m0 : gidx<R>(S, k, E);
            if (m > MT - 1) {  // cannot happen for budgets below the table top
                m = MT - 1;
                atomicOr(A.err, (uint32_t)ERR_LEVEL);
            }
            const R u = st_uni<R>(st);
            const R t = mul_rn(u, __ldg(H + k * MT + m));
            const R* Lk = L + S.lev_off[k];
            const int nl = S.n_lev[k];
            const bool last = (k == n - 1);
            const R bn = last ? (R)0 : sp_base<R>(S, k + 1);
            const R* Hn = H + (k + 1) * MT;
            R cum = (R)0;
            int sel = -1;
            for (int i = 0; i < nl; ++i) {
                const R e = __ldg(Lk + i);
                if (!(e < E)) break;
                const R x = sub_rn(E, e);
                R w;
                if (last) {
                    w = lb_pow<R>(amode, x);
                } else {
                    int mm = gidx<R>(S, k + 1, x);
                    if (mm > MT - 1) mm = MT - 1;
                    w = mm == 0 ? (R)0 : __ldg(Hn + mm);
                }
                cum = add_rn(cum, w);
                if (t < cum) { sel = i; break; }
            }
            if (sel < 0) { ok = false; break; }
            set_q(nq, k, (uint32_t)sel);
            E = sub_rn(E, __ldg(Lk + sel));
        }
        if (ok) {
            q[0] = nq[0]; q[1] = nq[1]; q[2] = nq[2]; q[3] = nq[3];
            return S_OK;
        }
    }
    return S_CAP;
}
template <class R>
__device__ __forceinline__ int sample_lb(const StepArgs& A, const DevSpecies& S, int amode, double Ec_d,
                                         Stream& st, uint32_t q[4], uint32_t& trials) {
    return sample_lb_tab<R>(A, S, amode, h_tab<R>(A) + S.tab_off, Ec_d, st, q, trials);
}

// ------------------------------------------------- collision-temperature split
// The second reading of the product redistribution (Sec. "Polyatomic QK
// reaction modeling"): equipartition at a collision temperature T_c, the root
// of xi_tr/2 k T_c + sum over the products of <E_vib>(T_c) = E_x (E_x the
// energy above the products' ground states); a product's levels then follow
// (E - sum E)^b with b = (the degrees of freedom left to share with)/2 - 1.
// FP64 mode, every operation rounded as written.
__device__ __forceinline__ double mean_evib_tc(const StepArgs& A, const DevSpecies& S, double T) {
    const double kT = __dmul_rn(1.380649e-23, T);
    double e = 0.0;
    for (int j = 0; j < S.n_modes; ++j) {
        if (j >= S.n_stretch) {  // bend: k Theta / (e^(Theta/T) - 1)
            const double th = S.theta[j];
            const double x = __ddiv_rn(th, T);
            if (x <= 700.0) e = __dadd_rn(e, __ddiv_rn(__dmul_rn(1.380649e-23, th), __dsub_rn(exp_series(x), 1.0)));
        } else {  // stretch: Boltzmann mean over its levels above the ground level
            const double* L = A.lev64 + S.lev_off[j];
            const double e0 = __ldg(L);
            double num = 0.0, den = 0.0;
            for (int i = 0; i < S.n_lev[j]; ++i) {
                const double de = __dsub_rn(__ldg(L + i), e0);
                const double b = exp_series(__ddiv_rn(-de, kT));
                num = __dadd_rn(num, __dmul_rn(de, b));
                den = __dadd_rn(den, b);
            }
            e = __dadd_rn(e, __ddiv_rn(num, den));
        }
    }
    return e;
}
__device__ __forceinline__ double xi_vib_tc(const StepArgs& A, const DevSpecies& S, double T) {
    return S.n_modes ? __ddiv_rn(__dmul_rn(2.0, mean_evib_tc(A, S, T)), __dmul_rn(1.380649e-23, T)) : 0.0;
}
// T_c by bisection on [1 K, 1e7 K]; 100 halvings reach adjacent doubles
static __device__ double tcoll_root(const StepArgs& A, double xi_tr, const DevSpecies& P1, const DevSpecies& P2,
                             double Ex) {
    double lo = 1.0, hi = 1.0e7;
    for (int it = 0; it < 100; ++it) {
        const double T = __dmul_rn(0.5, __dadd_rn(lo, hi));
        double g = __dsub_rn(__dmul_rn(__dmul_rn(0.5, xi_tr), __dmul_rn(1.380649e-23, T)), Ex);
        if (P1.n_modes) g = __dadd_rn(g, mean_evib_tc(A, P1, T));
        if (P2.n_modes) g = __dadd_rn(g, mean_evib_tc(A, P2, T));
        if (g < 0.0) lo = T; else hi = T;
    }
    return __dmul_rn(0.5, __dadd_rn(lo, hi));
}
// One product's levels with p ~ (Ec - sum E)^b, exactly: a table draw at
// exponent a_t (the context's 3/2 - omega when b reaches it, else 1/2 from
// the exponent-1/2 tables) accepted with ((Ec - sum E)/(Ec - ZPE))^(b - a_t)
static __device__ int sample_exponent(const StepArgs& A, const DevSpecies& S, int amode, double Ec, double b,
                               Stream& st, uint32_t q[4], uint32_t& trials) {
    q[0] = q[1] = q[2] = q[3] = 0u;
    if (S.n_modes == 0) return S_OK;
    if (!(Ec > S.zpe)) return S_DEGEN;
    const double a = amode == 0 ? 0.75 : (amode == 1 ? 1.0 : 0.5);
    const bool use_main = b >= a;
    const double a_t = use_main ? a : 0.5;
    if (!use_main && (!(b >= 0.5) || S.tab_off_h < 0)) return S_CAP;
    const double* H = use_main ? A.H64 + S.tab_off : A.H64h + S.tab_off_h;
    const int am = use_main ? amode : 2;
    const double span = __dsub_rn(Ec, S.zpe);
    for (uint32_t trial = 0; trial < A.reject_cap; ++trial) {
        uint32_t nq[4];
        const int r = sample_lb_tab<double>(A, S, am, H, Ec, st, nq, trials);
        if (r != S_OK) return r;
        const double Esum = evib64(A.lev64, S, nq);
        if (b == a_t || st_uni<double>(st) < pow_series(__ddiv_rn(__dsub_rn(Ec, Esum), span), __dsub_rn(b, a_t))) {
            q[0] = nq[0]; q[1] = nq[1]; q[2] = nq[2]; q[3] = nq[3];
            return S_OK;
        }
    }
    return S_CAP;
}

// Marsaglia (1972): a point uniform in the unit disk mapped onto the sphere
// (FP32: approximate square root, the direction's norm is 1 to ~1e-7)
template <class R>
__device__ __forceinline__ void iso_dir(Stream& st, R d[3]) {
    for (int it = 0; it < 4096; ++it) {
        R x1 = (R)2 * st_uni<R>(st) - (R)1;
        R x2 = (R)2 * st_uni<R>(st) - (R)1;
        R s;
        if constexpr (std::is_same<R, float>::value)
            s = __fadd_rn(__fmul_rn(x1, x1), __fmul_rn(x2, x2));  // no contraction: same bits in every kernel
        else
            s = x1 * x1 + x2 * x2;
        if (s < (R)1) {
            const R om = (R)1 - s;
            R r;
            if constexpr (std::is_same<R, float>::value) r = 2.0f * (om * rsqrtf(om));
            else r = (R)2 * sqrt_rn(om);
            d[0] = x1 * r; d[1] = x2 * r; d[2] = (R)1 - (R)2 * s;
            return;
        }
    }
    d[0] = 0; d[1] = 0; d[2] = 1;
}

// per-pair event word, reduced per cell by k_finish
enum : uint32_t {
    EV_ACC = 1u, EV_CREATED = 2u, EV_RX_SHIFT = 2, /* bits 2..7: reaction + 1 */
    EV_SAMP_SHIFT = 8, /* bits 8..9 */ EV_OVER_SHIFT = 10, EV_DEGEN_SHIFT = 12,
    EV_NOTEXEC = 1u << 14, EV_REMOVED = 1u << 15, EV_TRIAL_SHIFT = 16
};

struct PairOut {
    uint32_t ev;
    uint32_t trials;
};

// energy-conserving dissociation A + M -> B + C + M (Sec. "Dissociation
// reactions"; product split of reading A13).  FP64 arithmetic in both modes.
template <class R>
__device__ bool do_diss(const StepArgs& A, const Consts* C, const DevReaction& rx, double vA[3],
                        double vM[3], int spA, int spM, double EvA, const DevRes& rs, uint32_t lcell,
                        uint32_t rk, uint32_t qB[4], uint32_t qC[4], double vC[3], PairOut& o,
                        double erA = 0.0) {
    const DevSpecies& sA = C->sp[spA];
    const DevSpecies& sM = C->sp[spM];
    const DevSpecies& sB = C->sp[rx.P0];
    const DevSpecies& sC = C->sp[rx.P1];
    const double mA = sA.mass, mM = sM.mass, mB = sB.mass, mC = sC.mass;
    const double mBC = mB + mC;
    const double mt = mBC + mM;
    double V[3];
    for (int i = 0; i < 3; ++i) V[i] = (mA * vA[i] + mM * vM[i]) / mt;
    const double vA2 = vA[0] * vA[0] + vA[1] * vA[1] + vA[2] * vA[2];
    const double vM2 = vM[0] * vM[0] + vM[1] * vM[1] + vM[2] * vM[2];
    const double V2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const double KEin = 0.5 * mA * vA2 + 0.5 * mM * vM2;
    const double KEcm = 0.5 * mt * V2;
    const double Eav = KEin - KEcm + EvA - rx.dEf + erA;  // A's rotation joins the pool
    if (!(Eav - sB.zpe - sC.zpe > 0.0) || Eav - sC.zpe > sB.top || Eav - sB.zpe > sC.top)
        return false;
    Stream sa, sb, ss;
    st_init(sa, rs.seed, rs.step, lcell, rk, PU_LB_A);
    st_init(sb, rs.seed, rs.step, lcell, rk, PU_LB_B);
    st_init(ss, rs.seed, rs.step, lcell, rk, PU_SCAT);
    for (int j = 0; j < 4; ++j) { qB[j] = 0u; qC[j] = 0u; }
    uint32_t tr = 0;
    const bool tc = rx.prod_split == HCAO_SPLIT_TCOLL;
    if (sB.n_modes > 0) {
        o.ev += 1u << EV_SAMP_SHIFT;
        int rc;
        if (tc) {  // xi_tr = 6: B shares with the two relative motions and C's vibration
            const double Tc = tcoll_root(A, 6.0, sB, sC, Eav - sB.zpe - sC.zpe);
            rc = sample_exponent(A, sB, C->amode, Eav - sC.zpe, (6.0 + xi_vib_tc(A, sC, Tc)) / 2.0 - 1.0, sa, qB, tr);
        } else {
            rc = sample_lb<R>(A, sB, C->amode, Eav - sC.zpe, sa, qB, tr);
        }
        if (rc != S_OK) {
            for (int j = 0; j < 4; ++j) qB[j] = 0u;
            atomicOr(A.err, (uint32_t)ERR_REJECT);
        }
    }
    const double EvB = evib64(A.lev64, sB, qB);
    if (sC.n_modes > 0) {
        o.ev += 1u << EV_SAMP_SHIFT;
        const int rc = tc ? sample_exponent(A, sC, C->amode, Eav - EvB, 2.0, sb, qC, tr)
                          : sample_lb<R>(A, sC, C->amode, Eav - EvB, sb, qC, tr);
        if (rc != S_OK) {
            for (int j = 0; j < 4; ++j) qC[j] = 0u;
            atomicOr(A.err, (uint32_t)ERR_REJECT);
        }
    }
    o.trials += tr;
    const double EvC = evib64(A.lev64, sC, qC);
    const double Etr = (Eav - EvB) - EvC;
    double x = 0.5;
    for (int it = 0; it < 4096; ++it) {  // Beta(3/2,3/2) by rejection under 1/2
        x = st_u64(ss);
        const double y = st_u64(ss);
        if (y * y * 0.25 < x * (1.0 - x)) break;
    }
    const double E1 = x * Etr;
    const double E2 = Etr - E1;
    const double mu1 = mB * mC / mBC;
    const double mu2 = mBC * mM / mt;
    const double g1 = sqrt(2.0 * E1 / mu1);
    const double g2 = sqrt(2.0 * E2 / mu2);
    double d1[3], d2[3];
    iso_dir<double>(ss, d1);
    iso_dir<double>(ss, d2);
    const double fM = mM / mt, fBC = mBC / mt, fC = mC / mBC, fB = mB / mBC;
    double VBC[3];
    for (int i = 0; i < 3; ++i) {
        const double G2 = g2 * d2[i];
        VBC[i] = V[i] + fM * G2;
        vM[i] = V[i] - fBC * G2;
    }
    for (int i = 0; i < 3; ++i) {
        const double G1 = g1 * d1[i];
        vA[i] = VBC[i] + fC * G1;
        vC[i] = VBC[i] - fB * G1;
    }
    return true;
}

// exchange A + B -> C + D (Sec. "Exchange reactions")
template <class R>
__device__ bool do_exch(const StepArgs& A, const Consts* C, const DevReaction& rx, double vA[3],
                        double vB[3], int spA, int spB, double EvA, double EvB, const DevRes& rs,
                        uint32_t lcell, uint32_t rk, uint32_t qC[4], uint32_t qD[4], PairOut& o,
                        double erA = 0.0, double erB = 0.0) {
    const DevSpecies& sA = C->sp[spA];
    const DevSpecies& sB = C->sp[spB];
    const DevSpecies& sC = C->sp[rx.P0];
    const DevSpecies& sD = C->sp[rx.P1];
    const double mA = sA.mass, mB = sB.mass, mC = sC.mass, mD = sD.mass;
    const double mt = mC + mD;
    double V[3];
    for (int i = 0; i < 3; ++i) V[i] = (mA * vA[i] + mB * vB[i]) / mt;
    const double vA2 = vA[0] * vA[0] + vA[1] * vA[1] + vA[2] * vA[2];
    const double vB2 = vB[0] * vB[0] + vB[1] * vB[1] + vB[2] * vB[2];
    const double V2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const double KEin = 0.5 * mA * vA2 + 0.5 * mB * vB2;
    const double KEcm = 0.5 * mt * V2;
    const double Eav = (KEin - KEcm + EvA + EvB - rx.dEf + erA) + erB;  // rotation joins the pool
    if (!(Eav - sC.zpe - sD.zpe > 0.0) || Eav - sD.zpe > sC.top || Eav - sC.zpe > sD.top)
        return false;
    Stream sa, sb, ss;
    st_init(sa, rs.seed, rs.step, lcell, rk, PU_LB_A);
    st_init(sb, rs.seed, rs.step, lcell, rk, PU_LB_B);
    st_init(ss, rs.seed, rs.step, lcell, rk, PU_SCAT);
    for (int j = 0; j < 4; ++j) { qC[j] = 0u; qD[j] = 0u; }
    uint32_t tr = 0;
    const bool tc = rx.prod_split == HCAO_SPLIT_TCOLL;
    if (sC.n_modes > 0) {
        o.ev += 1u << EV_SAMP_SHIFT;
        int rc;
        if (tc) {  // xi_tr = 3: C shares with the relative motion and D's vibration
            const double Tc = tcoll_root(A, 3.0, sC, sD, Eav - sC.zpe - sD.zpe);
            rc = sample_exponent(A, sC, C->amode, Eav - sD.zpe, (3.0 + xi_vib_tc(A, sD, Tc)) / 2.0 - 1.0, sa, qC, tr);
        } else {
            rc = sample_lb<R>(A, sC, C->amode, Eav - sD.zpe, sa, qC, tr);
        }
        if (rc != S_OK) {
            for (int j = 0; j < 4; ++j) qC[j] = 0u;
            atomicOr(A.err, (uint32_t)ERR_REJECT);
        }
    }
    const double EvC = evib64(A.lev64, sC, qC);
    if (sD.n_modes > 0) {
        o.ev += 1u << EV_SAMP_SHIFT;
        const int rc = tc ? sample_exponent(A, sD, C->amode, Eav - EvC, 0.5, sb, qD, tr)
                          : sample_lb<R>(A, sD, C->amode, Eav - EvC, sb, qD, tr);
        if (rc != S_OK) {
            for (int j = 0; j < 4; ++j) qD[j] = 0u;
            atomicOr(A.err, (uint32_t)ERR_REJECT);
        }
    }
    o.trials += tr;
    const double EvD = evib64(A.lev64, sD, qD);
    const double Etr = (Eav - EvC) - EvD;
    const double mu = mC * mD / mt;
    const double g = sqrt(2.0 * Etr / mu);
    double d[3];
    iso_dir<double>(ss, d);
    const double fC = mD / mt, fD = mC / mt;
    for (int i = 0; i < 3; ++i) {
        const double G = g * d[i];
        vA[i] = V[i] + fC * G;
        vB[i] = V[i] - fD * G;
    }
    return true;
}

// recombination B + C + M -> A + M (Sec. "Recombination reactions"): B takes
// A's species, C is removed, M keeps its species and levels.  The budget of
// A's vibration and the A-M relative motion is the B, C, M translational
// energy in their centre-of-mass frame, the vibrational energies of B and C
// and the released formation energy; A's levels follow the LB target at that
// budget, the rest goes to A-M relative motion in a uniform direction.
template <class R>
__device__ bool do_recomb(const StepArgs& A, const Consts* C, const DevReaction& rx, double vB[3],
                          double vC[3], double vM[3], int spB, int spC, int spM, double EvB, double EvC,
                          const DevRes& rs, uint32_t lcell, uint32_t rk, uint32_t qA[4], PairOut& o,
                          double erB = 0.0, double erC = 0.0) {
    const DevSpecies& sA = C->sp[rx.P0];
    const DevSpecies& sB = C->sp[spB];
    const DevSpecies& sC = C->sp[spC];
    const DevSpecies& sM = C->sp[spM];
    const double mA = sA.mass, mB = sB.mass, mC = sC.mass, mM = sM.mass;
    const double mt = mA + mM;
    double V[3];
    for (int i = 0; i < 3; ++i) V[i] = ((mB * vB[i] + mC * vC[i]) + mM * vM[i]) / mt;
    const double vB2 = vB[0] * vB[0] + vB[1] * vB[1] + vB[2] * vB[2];
    const double vC2 = vC[0] * vC[0] + vC[1] * vC[1] + vC[2] * vC[2];
    const double vM2 = vM[0] * vM[0] + vM[1] * vM[1] + vM[2] * vM[2];
    const double V2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const double KEin = (0.5 * mB * vB2 + 0.5 * mC * vC2) + 0.5 * mM * vM2;
    const double KEcm = 0.5 * mt * V2;
    const double Eav = (KEin - KEcm + EvB + EvC - rx.dEf + erB) + erC;  // rotation joins the pool
    if (!(Eav - sA.zpe > 0.0) || Eav > sA.top) return false;
    Stream sa, ss;
    st_init(sa, rs.seed, rs.step, lcell, rk, PU_LB_A);
    st_init(ss, rs.seed, rs.step, lcell, rk, PU_SCAT);
    for (int j = 0; j < 4; ++j) qA[j] = 0u;
    uint32_t tr = 0;
    if (sA.n_modes > 0) {
        o.ev += 1u << EV_SAMP_SHIFT;
        const int rc = rx.prod_split == HCAO_SPLIT_TCOLL ? sample_exponent(A, sA, C->amode, Eav, 0.5, sa, qA, tr)
                                                        : sample_lb<R>(A, sA, C->amode, Eav, sa, qA, tr);
        if (rc != S_OK) {
            for (int j = 0; j < 4; ++j) qA[j] = 0u;
            atomicOr(A.err, (uint32_t)ERR_REJECT);
        }
    }
    o.trials += tr;
    const double Etr = Eav - evib64(A.lev64, sA, qA);
    const double mu = mA * mM / mt;
    const double g = sqrt(2.0 * Etr / mu);
    double d[3];
    iso_dir<double>(ss, d);
    const double fA = mM / mt, fM = mA / mt;
    for (int i = 0; i < 3; ++i) {
        const double G = g * d[i];
        vB[i] = V[i] + fA * G;
        vM[i] = V[i] - fM * G;
    }
    return true;
}

// ------------------------------------------------------------- one pair
// Pairs per NTC round: N/2, or N/3 when a recombination reaction exists, so
// that every pair of a round has a particle in no pair of the round (its
// third body, reading A14) at position 2 kmax + k of the permutation.
__device__ __forceinline__ uint32_t round_pairs(uint32_t N, int has_recomb) {
    return (has_recomb && N >= 3u) ? N / 3u : N >> 1;
}

// Where pair k of round r of cell c lives: its permuted members, its event slot.
struct PairLoc {
    uint32_t N, lcell, rk, ev_idx, ip, iq;
    void* recs;
    double sgmax;
};
__device__ __forceinline__ PairLoc locate(const StepArgs& A, int c, int r, uint32_t k) {
    const DevCell& cell = A.cells[c];
    PairLoc L;
    L.N = cell.n;
    L.lcell = cell.lcell;
    L.rk = ((uint32_t)r << 24) | k;
    L.ev_idx = A.abase[c] + (uint32_t)r * round_pairs(L.N, A.has_recomb) + k;
    const uint32_t key[4] = {cell.pkey[r][0], cell.pkey[r][1], cell.pkey[r][2], cell.pkey[r][3]};
    L.ip = pair_perm(2u * k, L.N, key);
    L.iq = pair_perm(2u * k + 1u, L.N, key);
    L.recs = cell.rec;
    L.sgmax = cell.sgmax;
    return L;
}

// the same as locate() with the members already known
__device__ __forceinline__ PairLoc locate_known(const StepArgs& A, int c, int r, uint32_t k, uint32_t ip,
                                                uint32_t iq) {
    const DevCell& cell = A.cells[c];
    PairLoc L;
    L.N = cell.n;
    L.lcell = cell.lcell;
    L.rk = ((uint32_t)r << 24) | k;
    L.ev_idx = A.abase[c] + (uint32_t)r * round_pairs(L.N, A.has_recomb) + k;
    L.ip = ip;
    L.iq = iq;
    L.recs = cell.rec;
    L.sgmax = cell.sgmax;
    return L;
}

// NTC set-up of one cell for this step: N_sel = 1/2 N (N-1) w (sigma g)_max
// dt / V_c, rounded stochastically (stream PU_NSEL), the number of pairing
// rounds of P pairs each, and each round's pairing-permutation key (stream PU_PERM).
// The FP64 product is written with explicit roundings so that every kernel
// computing it (compiled with or without FMA contraction) gets the same N_sel.
// More rounds than max_rounds, or a non-finite (sigma g)_max, leave the cell
// without pairs and set the error word.
__device__ __forceinline__ uint32_t ntc_setup(const StepArgs& A, const DevRes& rs, const DevCell& cl, uint32_t N,
                                              uint32_t P, uint32_t& rounds, uint32_t (*pkey)[4]) {
    rounds = 0;
    if (!rs.active || N < 2) return 0u;
    const double x = __ddiv_rn(
        __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(0.5, (double)N), (double)(N - 1)), rs.w), cl.sgmax), rs.dt),
        rs.Vc);
    long long ns = 0, rr = 0;
    if (x >= 0.0 && x < 4.0e9) {
        const double fl = floor(x);
        ns = (long long)fl;
        Stream st;
        st_init(st, rs.seed, rs.step, cl.lcell, 0u, PU_NSEL);
        if (st_u64(st) < x - fl) ns++;
        rr = (ns + P - 1) / P;
        if (rr > A.max_rounds) { atomicOr(A.err, (uint32_t)ERR_ROUNDS); ns = 0; rr = 0; }
    } else {  // a non-finite or absurd (sigma g)_max: no pairs, report
        atomicOr(A.err, (uint32_t)ERR_NONFINITE);
    }
    for (uint32_t r = 0; r < (uint32_t)rr; ++r) {
        Stream sf;
        st_init(sf, rs.seed, rs.step, cl.lcell, r << 24, PU_PERM);
        st_block(sf);
        pkey[r][0] = sf.w0; pkey[r][1] = sf.w1;
        pkey[r][2] = sf.w2; pkey[r][3] = sf.w3;
    }
    rounds = (uint32_t)rr;
    return (uint32_t)ns;
}

// channel id: reaction (3 bits) | side << 3 | broken stretch << 4
__device__ __forceinline__ uint32_t chan_pack(int rx, int side, int mode) {
    return (uint32_t)rx | ((uint32_t)side << 3) | ((uint32_t)mode << 4);
}

// TCE probability (the comparison model of Eq. arrhenius) of reaction rx for
// a partner of species m at collision energy Ec: the host table at
// x_i = X (i/NT)^2 above E_a, linear in s = sqrt(x/X), constant beyond X.
// Written with explicit roundings (the same bits in every kernel).
__device__ __forceinline__ double tce_prob(const StepArgs& A, const DevReaction& rx, int m, double Ec) {
    const double x = __dsub_rn(Ec, rx.tce_Ea);
    if (!(x > 0.0)) return 0.0;
    const double* t = A.tce + ((size_t)rx.tce_slot * MAXS + (size_t)m) * (TCE_NT + 1);
    const double sv = __dsqrt_rn(__ddiv_rn(x, A.tce_span));
    if (!(sv < 1.0)) return __ldg(t + TCE_NT);
    const double tt = __dmul_rn(sv, (double)TCE_NT);
    const int i = (int)tt;
    const double f = __dsub_rn(tt, (double)i);
    const double t0 = __ldg(t + i), t1 = __ldg(t + i + 1);
    return __dadd_rn(t0, __dmul_rn(f, __dsub_rn(t1, t0)));
}

// TCE reactions, tested before the QK channels in reaction order against one
// uniform of their own stream (PU_TCE) laid on the running sum of their
// probabilities.  E_c is the relative translational energy, plus both
// partners' vibrational energy above their ZPE when the reaction counts
// internal degrees of freedom.  Returns true with the channel in chan.
template <class R>
__device__ bool tce_test(const StepArgs& A, const Consts* __restrict__ C, const DevRes& rs, uint32_t lcell,
                         uint32_t rk, int sP, int sQ, double Etr, double EvP, double EvQ, uint32_t& chan,
                         double erP = 0.0, double erQ = 0.0) {
    double run = 0.0, u = -1.0;
    for (int ri = 0; ri < C->n_reactions; ++ri) {
        const DevReaction& rx = C->rx[ri];
        if (rx.model != HCAO_MODEL_TCE || rx.type == HCAO_RECOMB) continue;
        int side;
        if (rx.type == HCAO_DISS) {
            if (sP == rx.A) side = 0;
            else if (sQ == rx.A) side = 1;
            else continue;
        } else {
            if (sP == rx.A && sQ == rx.B) side = 0;
            else if (sQ == rx.A && sP == rx.B) side = 1;
            else continue;
        }
        double Ec = Etr;
        if (rx.tce_zeta_on)  // internal energy: vibration above the ZPE and rotation of both
            Ec = __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(Ec, __dsub_rn(EvP, C->sp[sP].zpe)),
                                               __dsub_rn(EvQ, C->sp[sQ].zpe)), erP), erQ);
        run = __dadd_rn(run, tce_prob(A, rx, side ? sP : sQ, Ec));
        if (u < 0.0) {
            Stream st;
            st_init(st, rs.seed, rs.step, lcell, rk, PU_TCE);
            u = (double)st_uni<R>(st);
        }
        if (!(u < run)) continue;
        chan = (uint32_t)ri | ((uint32_t)side << 3) | ((uint32_t)(rx.type == HCAO_DISS ? rx.tce_mode : 0) << 4);
        return true;
    }
    return false;
}

// QK reaction test: channels in fixed order (partner 1 stretches, partner 2
// stretches, exchange); one with E_excess > 0 is taken, several are chosen
// with probability proportional to E_excess ("Competing reactions").  Two
// passes over the same channel list instead of storing it.
template <class R>
__device__ int reaction_pick(const StepArgs& A, const Consts* __restrict__ C, int sP, int sQ,
                             const uint32_t qP[4], const uint32_t qQ[4], double Etr, double EvP,
                             double EvQ, double u_ster, double u_sel, double u_ch, uint32_t& chan,
                             double erP = 0.0, double erQ = 0.0) {
    const DevSpecies& SP = C->sp[sP];
    const DevSpecies& SQ = C->sp[sQ];
    int nch = 0;
    double tot = 0.0;
    uint32_t last = 0u;
    double t = 0.0, pre = 0.0;
    bool picked = false;
    for (int pass = 0; pass < 2 && !picked; ++pass) {
        if (pass == 1) {
            if (nch <= 1) break;
            t = u_ch * tot;
        }
        for (int side = 0; side < 2 && !picked; ++side) {
            const int spA = side ? sQ : sP;
            const DevSpecies& SA = side ? SQ : SP;
            const double EvA = side ? EvQ : EvP;
            for (int ri = 0; ri < C->n_reactions && !picked; ++ri) {
                const DevReaction& rx = C->rx[ri];
                if (rx.type != HCAO_DISS || rx.model == HCAO_MODEL_TCE || rx.A != spA) continue;
                for (int j = 0; j < SA.n_stretch; ++j) {
                    if (!((rx.mask >> j) & 1u)) continue;
                    // Eq. Ecoll-diss: ZPEs of A, B, C removed, the breaking mode's restored
                    const double E0j = __ldg(A.lev64 + SA.lev_off[j]);
                    double Ecoll = Etr + EvA - rx.zpesum + E0j;
                    // rotation coupling (Sec. "Rotation coupling"): gamma E_rot,A
                    if (rx.gamma != 0.0) Ecoll = Ecoll + rx.gamma * (side ? erQ : erP);
                    const double Eex = Ecoll - SA.De[j];
                    if (!(Eex > 0.0)) continue;
                    const uint32_t id = chan_pack(ri, side, j);
                    if (pass == 0) { nch++; tot = tot + Eex; last = id; }
                    else {
                        pre = pre + Eex;
                        if (t < pre) { chan = id; picked = true; break; }
                    }
                }
            }
        }
        for (int ri = 0; ri < C->n_reactions && !picked; ++ri) {
            const DevReaction& rx = C->rx[ri];
            if (rx.type != HCAO_EXCH || rx.model == HCAO_MODEL_TCE) continue;
            int side;
            if (sP == rx.A && sQ == rx.B) side = 0;
            else if (sQ == rx.A && sP == rx.B) side = 1;
            else continue;
            if (!(u_ster < rx.steric)) continue;
            const DevSpecies& SA = side ? SQ : SP;
            const uint32_t* qa = side ? qQ : qP;
            // Eq. Ecoll-exch; level energies include the ZPE (reading A12)
            double s = 0.0;
            if (rx.alpha_mode == HCAO_ALPHA_ONE_RANDOM_STRETCH) {
                const int js = (int)floor(u_sel * (double)SA.n_stretch);
                s = __ldg(A.lev64 + SA.lev_off[js] + get_q(qa, js));
            } else {
                for (int j = 0; j < SA.n_modes; ++j)
                    s = s + rx.alpha[j] * __ldg(A.lev64 + SA.lev_off[j] + get_q(qa, j));
            }
            double Ecoll = Etr + s;
            if (rx.gamma != 0.0) Ecoll = Ecoll + rx.gamma * (side ? erQ : erP);
            const double Eex = Ecoll - rx.Ea;
            if (!(Eex > 0.0)) continue;
            const uint32_t id = chan_pack(ri, side, 0);
            if (pass == 0) { nch++; tot = tot + Eex; last = id; }
            else {
                pre = pre + Eex;
                if (t < pre) { chan = id; picked = true; }
            }
        }
    }
    if (nch == 0) return 0;
    if (!picked) chan = last;  // one channel, or rounding left t >= the full sum
    if (nch == 1) chan = last;
    return nch;
}

// relative velocity, VHS sigma_T g and the pair's energies (shared by the phases)
template <class R>
__device__ __forceinline__ void pair_energy(const DevPair& pc, int amode, const R vP[3],
                                            const R vQ[3], double& g2d, double& sg) {
    if constexpr (std::is_same<R, double>::value) {
        const double gx = vP[0] - vQ[0], gy = vP[1] - vQ[1], gz = vP[2] - vQ[2];
        g2d = gx * gx + gy * gy + gz * gz;
        const double g = sqrt(g2d);
        const double gp = amode == 0 ? sqrt(g) : (amode == 1 ? g : 1.0);
        sg = pc.C * gp;
    } else {
        const float gx = vP[0] - vQ[0], gy = vP[1] - vQ[1], gz = vP[2] - vQ[2];
        const float g2 = gx * gx + gy * gy + gz * gz;
        g2d = (double)g2;
        const float g = sqrtf(g2);
        const float gp = amode == 0 ? sqrtf(g) : (amode == 1 ? g : 1.0f);
        sg = (double)(pc.C_f * gp);
    }
}

// FP32 pair kinematics with each operation's rounding written out, so that
// every kernel evaluating them -- the per-round queue kernels and the fused
// per-cell kernel -- gets the same bits whatever the compiler would contract.
// Squared relative speed of velocities a and b.
__device__ __forceinline__ float g2_f32(const float a[3], const float b[3]) {
    const float gx = __fsub_rn(a[0], b[0]), gy = __fsub_rn(a[1], b[1]), gz = __fsub_rn(a[2], b[2]);
    return __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
}
// VHS sigma_T g of a pair at squared relative speed g2 (g^(2-2 omega))
__device__ __forceinline__ float sg_f32(const DevPair& pc, int amode, float g2) {
    const float gr = __fsqrt_rn(g2);
    return __fmul_rn(pc.C_f, amode == 0 ? __fsqrt_rn(gr) : (amode == 1 ? gr : 1.0f));
}
// relative translational energy 1/2 m_r g^2 in fixed point
__device__ __forceinline__ long long etr_fix_f32(const DevPair& pc, float g2) {
    return f2fix(__fmul_rn(__fmul_rn(0.5f, pc.mr_f), g2));
}
// isotropic scattering with the centre-of-mass velocity kept: relative speed
// from the relative energy Erel, direction d
__device__ __forceinline__ float cm_velocity_f32(const DevPair& pc, float va, float vb) {
    return __fadd_rn(__fmul_rn(pc.fq_f, va), __fmul_rn(pc.fp_f, vb));
}
// the same from the centre-of-mass velocity V (cm_velocity_f32)
__device__ __forceinline__ void scatter_cm_f32(const DevPair& pc, long long Erel, const float d[3],
                                               const float V[3], float na[3], float nb[3]) {
    const float gn = __fsqrt_rn(__fmul_rn(fix2f(Erel), pc.inv2mr_f));
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) {
        const float G = __fmul_rn(gn, d[c3]);
        na[c3] = __fadd_rn(V[c3], __fmul_rn(pc.fp_f, G));
        nb[c3] = __fsub_rn(V[c3], __fmul_rn(pc.fq_f, G));
    }
}
__device__ __forceinline__ void scatter_f32(const DevPair& pc, long long Erel, const float d[3],
                                            const float va[3], const float vb[3], float na[3], float nb[3]) {
    const float V[3] = {cm_velocity_f32(pc, va[0], vb[0]), cm_velocity_f32(pc, va[1], vb[1]),
                        cm_velocity_f32(pc, va[2], vb[2])};
    scatter_cm_f32(pc, Erel, d, V, na, nb);
}

// FP32 K5 draw of one molecule's levels at collision energy Ec (float, from
// the fixed-point Ecd) with the alias proposals: per mode k, a level i is
// proposed from the alias table of the bucket holding the budget E (weights
// w_i at the bucket's upper edge) and accepted with probability
// w_i(E)/w_i(edge); a rejection restarts the trial.  That is the K5 mode
// draw (level i with probability w_i(E)/H_k[idx(E)], restart otherwise) in
// constant work per mode.  Per mode two dependent loads from the larger
// tables: the proposal's 16-byte slot (threshold, alias, both edge weights)
// and the table entry of the remaining budget, whose H is the acceptance
// weight and whose alias table serves the next mode; the level energy comes
// from the small level list.  Returns S_OK with the levels in q and their
// fixed-point energy in Esel, S_OVER, S_DEGEN or S_CAP.  Counts mode draws
// and level evaluations (one per draw).
template <class ST>
static __device__ int sample_alias_tab(const StepArgs& A, const K5Ent* __restrict__ T,
                                       const AliasEnt* __restrict__ AE, const DevSpecies& S, int amode,
                                       float Ec, ST& st, uint32_t (&q)[4], long long& Esel,
                                       uint32_t& trials, uint32_t& wlev, uint32_t& wmode) {
    const int n = S.n_modes, MT = S.MT, gsh = S.gshift, gj0 = S.gj0;
    q[0] = q[1] = q[2] = q[3] = 0u;
    Esel = S.zpe_fix;
    if (n == 0) return S_OK;
    const float b0 = S.base_f[0];
    const int m0 = grid_idx_f32(b0, gsh, gj0, MT, Ec);
    if (m0 > S.M) return S_OVER;
    if (m0 == 0) return S_DEGEN;
    const uint4 t0 = __ldg(reinterpret_cast<const uint4*>(T + m0));
    if (!(__uint_as_float(t0.x) > 0.f)) return S_DEGEN;
    if (__fsub_rn(Ec, b0) < S.eps_min_f) return S_OK;  // only the ground state fits
    // One mode draw per pass of a single loop: a rejection starts the next
    // trial at mode 0 in the next pass.  The draws and their random words are
    // those of a loop over trials around a loop over modes, but a lane that
    // restarts does not hold its warp's other lanes for a whole trial.
    uint32_t nq[4] = {0u, 0u, 0u, 0u};
    long long es = 0;
    float E = Ec;
    uint32_t off = t0.y, L = t0.z, trial = 0;
    int k = 0;
    trials++;
    for (;;) {
        wmode++;
        bool acc = false;
        uint32_t i = 0;
        float e = 0.f;
        if (L != 0u) {
            // one word: its top 24 bits give the slot (integer part of r L) and
            // the coin, its low 8 bits the top bits of the acceptance uniform
            const uint32_t rw = st_word(st);
            const uint32_t rbits = rw >> 8, u8 = rw & 0xFFu;
            const uint64_t rl = (uint64_t)rbits * L;
            const uint32_t j = (uint32_t)(rl >> 24);
            const float coin = (float)(uint32_t)(rl & 0xFFFFFFu) * 0x1p-24f;
            const float* lv = A.lev32 + S.lev_off[k];
            const float4 s0 = __ldg(reinterpret_cast<const float4*>(AE + off + j));
            const float ej = __ldg(lv + j);  // in parallel with the slot
            const bool own = coin < s0.x;
            i = own ? j : __float_as_uint(s0.y);
            const float wg = own ? s0.z : s0.w;
            e = own ? ej : __ldg(lv + i);
            // acceptance at the actual budget
            float wE = 0.f;
            if (e < E) {
                const float x = __fsub_rn(E, e);
                if (k == n - 1) {
                    wE = lb_pow_fast(amode, x);
                } else {
                    const int mm = grid_idx_f32(S.base_f[k + 1], gsh, gj0, MT, x);
                    if (mm != 0) {
                        const uint4 tn = __ldg(reinterpret_cast<const uint4*>(T + (k + 1) * MT + min(mm, MT - 1)));
                        wE = __uint_as_float(tn.x);
                        off = tn.y;
                        L = tn.z;
                    }
                }
            }
            wlev++;
            // accept if u wg < wE, u = (u8 2^16 + b) 2^-24 with 16 more bits b
            // drawn only when u8 leaves the test open: rounding is monotone, so
            // fl(u8 2^-8 wg) >= wE rejects and fl((u8+1) 2^-8 wg) < wE accepts
            // for every b, the decision of the full 24-bit test either way
            acc = true;
            if (!(__fmul_rn((float)(u8 + 1u) * 0x1p-8f, wg) < wE)) {
                if (!(__fmul_rn((float)u8 * 0x1p-8f, wg) < wE)) {
                    acc = false;
                } else {
                    const float u = (float)((u8 << 16) | (st_word(st) >> 16)) * 0x1p-24f;
                    acc = __fmul_rn(u, wg) < wE;
                }
            }
        }
        if (acc) {
            set_q(nq, k, i);
            E = __fsub_rn(E, e);
            es += __ldg(A.levfix + S.lev_off[k] + i);
            if (++k == n) break;
        } else {
            if (++trial >= A.reject_cap) return S_CAP;
            trials++;
            nq[0] = nq[1] = nq[2] = nq[3] = 0u;
            es = 0;
            E = Ec;
            off = t0.y;
            L = t0.z;
            k = 0;
        }
    }
    q[0] = nq[0]; q[1] = nq[1]; q[2] = nq[2]; q[3] = nq[3];
    Esel = es;
    return S_OK;
}
template <class ST>
static __device__ __forceinline__ int sample_alias_f32(const StepArgs& A, const DevSpecies& S, int amode,
                                                       float Ec, ST& st, uint32_t (&q)[4], long long& Esel,
                                                       uint32_t& trials, uint32_t& wlev, uint32_t& wmode) {
    return sample_alias_tab(A, A.k5e + S.tab_off, A.ae, S, amode, Ec, st, q, Esel, trials, wlev, wmode);
}

// FP32 LB relaxation of one molecule of species sp (levels q, fixed-point
// E_vib Evold) against the relative energy Erel; returns the relative energy
// left, and took = true when q was replaced by a new state.  sp < 0 or a
// species without modes keeps everything.
template <class ST>
static __device__ __forceinline__ long long relax_one(const StepArgs& A, const Consts* __restrict__ C, int sp,
                                                      uint32_t (&q)[4], long long Evold, ST& st,
                                                      long long Erel, PairOut& o, uint32_t& wl, uint32_t& wm,
                                                      bool& took) {
    took = false;
    if (sp < 0 || C->sp[sp].n_modes == 0) return Erel;
    const DevSpecies& S = C->sp[sp];
    const long long Ecd = Erel + Evold;
    o.ev += 1u << EV_SAMP_SHIFT;
    uint32_t nq[4];
    long long Esel;
    uint32_t tr = 0;
    const int rc = sample_alias_f32(A, S, C->amode, fix2f(Ecd), st, nq, Esel, tr, wl, wm);
    o.trials += tr;
    if (rc == S_OK) {
        const long long En = Ecd - Esel;
        if (En >= 0) {
            q[0] = nq[0]; q[1] = nq[1]; q[2] = nq[2]; q[3] = nq[3];
            took = true;
            return En;
        }
        o.ev += 1u << EV_DEGEN_SHIFT;
    } else if (rc == S_OVER) {
        o.ev += 1u << EV_OVER_SHIFT;
    } else if (rc == S_DEGEN) {
        o.ev += 1u << EV_DEGEN_SHIFT;
    } else {
        atomicOr(A.err, (uint32_t)ERR_REJECT);
    }
    return Ecd - Evold;  // the state is kept
}

// FP32 LB relaxation of up to two molecules: molecule 1, then molecule 2
// with the updated relative energy, in int64 fixed point.  Returns the
// relative energy left for scattering.
static __device__ __forceinline__ long long relax_flat(const StepArgs& A, const Consts* __restrict__ C, int spA,
                                                       uint32_t (&qA)[4], long long EvA, Stream stA, int spB,
                                                       uint32_t (&qB)[4], long long EvB, Stream stB, long long Erel,
                                                       PairOut& o, uint32_t* work = nullptr) {
    uint32_t wl = 0, wm = 0;
    bool took;
    Erel = relax_one(A, C, spA, qA, EvA, stA, Erel, o, wl, wm, took);
    Erel = relax_one(A, C, spB, qB, EvB, stB, Erel, o, wl, wm, took);
    if (work) { work[0] += wl; work[1] += wm; }
    return Erel;
}

// FP32 mode, the collision-temperature split: one product's levels with
// p ~ (E - sum E)^b (E = Erel + Evold, Evold its ground state): alias draws at
// exponent a_t (the context's 3/2 - omega when b reaches it, else 1/2 from
// the exponent-1/2 tables) accepted with ((E - sum E)/(E - ZPE))^(b - a_t).
// Returns the relative energy left; a failed draw keeps the ground state.
static __device__ long long relax_one_b(const StepArgs& A, const Consts* __restrict__ C, int sp,
                                        uint32_t (&q)[4], long long Evold, Stream& st, long long Erel,
                                        float b, PairOut& o) {
    if (sp < 0 || C->sp[sp].n_modes == 0) return Erel;
    const DevSpecies& S = C->sp[sp];
    const long long Ecd = Erel + Evold;
    o.ev += 1u << EV_SAMP_SHIFT;
    const float a = C->amode == 0 ? 0.75f : (C->amode == 1 ? 1.0f : 0.5f);
    const bool use_main = b >= a;
    const float a_t = use_main ? a : 0.5f;
    if (!use_main && S.tab_off_h < 0) {
        atomicOr(A.err, (uint32_t)ERR_REJECT);
        return Erel;
    }
    const K5Ent* T = use_main ? A.k5e + S.tab_off : A.k5eh + S.tab_off_h;
    const AliasEnt* AE = use_main ? A.ae : A.aeh;
    const int am = use_main ? C->amode : 2;
    const double span = (double)(Ecd - S.zpe_fix);
    uint32_t tr = 0, wl = 0, wm = 0;
    for (uint32_t trial = 0; trial < A.reject_cap; ++trial) {
        uint32_t nq[4];
        long long Esel;
        const int rc = sample_alias_tab(A, T, AE, S, am, fix2f(Ecd), st, nq, Esel, tr, wl, wm);
        if (rc != S_OK) {
            o.trials += tr;
            if (rc == S_OVER) o.ev += 1u << EV_OVER_SHIFT;
            else if (rc == S_DEGEN) o.ev += 1u << EV_DEGEN_SHIFT;
            else atomicOr(A.err, (uint32_t)ERR_REJECT);
            return Erel;
        }
        const long long En = Ecd - Esel;
        if (En < 0) {
            o.trials += tr;
            o.ev += 1u << EV_DEGEN_SHIFT;
            return Erel;
        }
        if (b == a_t || st_u32(st) < powf((float)((double)En / span), b - a_t)) {
            o.trials += tr;
            q[0] = nq[0]; q[1] = nq[1]; q[2] = nq[2]; q[3] = nq[3];
            return En;
        }
    }
    o.trials += tr;
    atomicOr(A.err, (uint32_t)ERR_REJECT);
    return Erel;
}
// FP32 mode: b1 of the collision-temperature split at E_x (J) from the
// reaction's table, linear in log2 E_x and clamped at the ends
static __device__ __forceinline__ float tcb_b1(const StepArgs& A, const DevReaction& rx, double Ex) {
    const float* t = A.tcb + rx.tcb_off;
    float u = (log2f((float)Ex) - (float)TCB_L0) * (float)TCB_PER_OCTAVE;
    u = fminf(fmaxf(u, 0.0f), (float)(TCB_N - 1));
    const int i = min((int)u, TCB_N - 2);
    const float f = u - (float)i;
    return t[i] + f * (t[i + 1] - t[i]);
}

// FP32 mode: QK reaction test in fixed point (exact thresholds), the same
// channel order and E_excess-weighted choice as reaction_pick.
static __device__ __forceinline__ int reaction_pick_fix(const StepArgs& A, const Consts* __restrict__ C, int sP, int sQ,
                                 const uint32_t qP[4], const uint32_t qQ[4], long long Etr,
                                 long long EvP, long long EvQ, float u_ster, float u_sel, float u_ch,
                                 uint32_t& chan, float erP = 0.f, float erQ = 0.f) {
    const DevSpecies& SP = C->sp[sP];
    const DevSpecies& SQ = C->sp[sQ];
    int nch = 0;
    long long tot = 0;
    uint32_t last = 0u;
    double t = 0.0;
    long long pre = 0;
    bool picked = false;
    for (int pass = 0; pass < 2 && !picked; ++pass) {
        if (pass == 1) {
            if (nch <= 1) break;
            t = (double)u_ch * (double)tot;
        }
        for (int side = 0; side < 2 && !picked; ++side) {
            const int spA = side ? sQ : sP;
            const DevSpecies& SA = side ? SQ : SP;
            const long long EvA = side ? EvQ : EvP;
            for (int ri = 0; ri < C->n_reactions && !picked; ++ri) {
                const DevReaction& rx = C->rx[ri];
                if (rx.type != HCAO_DISS || rx.model == HCAO_MODEL_TCE || rx.A != spA) continue;
                const long long base = Etr + EvA - rx.zpesum_fix;
                for (int j = 0; j < SA.n_stretch; ++j) {
                    if (!((rx.mask >> j) & 1u)) continue;
                    long long Eex = base + __ldg(A.levfix + SA.lev_off[j]) - SA.De_fix[j];
                    if (rx.gamma != 0.0) Eex += f2fix(__fmul_rn(rx.gamma_f, side ? erQ : erP));
                    if (Eex <= 0) continue;
                    const uint32_t id = chan_pack(ri, side, j);
                    if (pass == 0) { nch++; tot += Eex; last = id; }
                    else {
                        pre += Eex;
                        if (t < (double)pre) { chan = id; picked = true; break; }
                    }
                }
            }
        }
        for (int ri = 0; ri < C->n_reactions && !picked; ++ri) {
            const DevReaction& rx = C->rx[ri];
            if (rx.type != HCAO_EXCH || rx.model == HCAO_MODEL_TCE) continue;
            int side;
            if (sP == rx.A && sQ == rx.B) side = 0;
            else if (sQ == rx.A && sP == rx.B) side = 1;
            else continue;
            if (!(u_ster < (float)rx.steric)) continue;
            const DevSpecies& SA = side ? SQ : SP;
            uint32_t qa[4];  // the words themselves: a pointer chosen at run time puts both arrays in memory
#pragma unroll
            for (int w = 0; w < 4; ++w) qa[w] = side ? qQ[w] : qP[w];
            long long s = 0;
            if (rx.alpha_mode == HCAO_ALPHA_ONE_RANDOM_STRETCH) {
                const int js = min((int)(u_sel * (float)SA.n_stretch), SA.n_stretch - 1);
                s = __ldg(A.levfix + SA.lev_off[js] + get_q(qa, js));
            } else {
                double sd = 0.0;
                for (int j = 0; j < SA.n_modes; ++j)
                    sd = sd + rx.alpha[j] * (double)__ldg(A.levfix + SA.lev_off[j] + get_q(qa, j));
                s = __double2ll_rn(sd);
            }
            long long Eex = Etr + s - rx.Ea_fix;
            if (rx.gamma != 0.0) Eex += f2fix(__fmul_rn(rx.gamma_f, side ? erQ : erP));
            if (Eex <= 0) continue;
            const uint32_t id = chan_pack(ri, side, 0);
            if (pass == 0) { nch++; tot += Eex; last = id; }
            else {
                pre += Eex;
                if (t < (double)pre) { chan = id; picked = true; }
            }
        }
    }
    if (nch == 0) return 0;
    if (!picked || nch == 1) chan = last;
    return nch;
}

// FP32 mode, dissociation A + M -> B + C + M: float kinematics, fixed-point
// energies (the same product split as do_diss, reading A13).
static __device__ bool do_diss_fix(const StepArgs& A, const Consts* __restrict__ C, const DevReaction& rx,
                            float vA[3], float vM[3], int spA, int spM, long long EvA, const DevRes& rs,
                            uint32_t lcell, uint32_t rk, uint32_t (&qB)[4], uint32_t (&qC)[4],
                            float vC[3], PairOut& o, float erA = 0.f) {
    const DevSpecies& sA = C->sp[spA];
    const DevSpecies& sM = C->sp[spM];
    const DevSpecies& sB = C->sp[rx.P0];
    const DevSpecies& sC = C->sp[rx.P1];
    // masses ~1e-26 kg: a product of two underflows FP32, so reduced masses
    // come from the host-built pair table and only ratios are formed here
    const float mA = sA.mass_f, mM = sM.mass_f, mB = sB.mass_f, mC = sC.mass_f;
    const float mAM = mA + mM, mBC = mB + mC, mt = mBC + mM;
    float V[3], g[3];
    for (int i = 0; i < 3; ++i) {
        V[i] = (mA * vA[i] + mM * vM[i]) / mAM;
        g[i] = vA[i] - vM[i];
    }
    const float g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const long long Ein = f2fix(0.5f * C->pair[spA * MAXS + spM].mr_f * g2);
    const long long Eav = Ein + EvA - rx.dEf_fix + f2fix(erA);  // A's rotation joins the pool
    if (!(Eav - sB.zpe_fix - sC.zpe_fix > 0) || Eav - sC.zpe_fix > sB.top_fix ||
        Eav - sB.zpe_fix > sC.top_fix)
        return false;
    Stream sa, sb, ss;
    st_init(sa, rs.seed, rs.step, lcell, rk, PU_LB_A);
    st_init(sb, rs.seed, rs.step, lcell, rk, PU_LB_B);
    st_init(ss, rs.seed, rs.step, lcell, rk, PU_SCAT);
    for (int j = 0; j < 4; ++j) { qB[j] = 0u; qC[j] = 0u; }
    // products start in their ground states: B is drawn at Eav - ZPE_C, then C
    // at Eav - E_vib,B; what is left is translational
    long long Etr;
    if (rx.prod_split == HCAO_SPLIT_TCOLL) {
        const long long Ex = Eav - sB.zpe_fix - sC.zpe_fix;
        Etr = relax_one_b(A, C, rx.P0, qB, sB.zpe_fix, sa, Ex, tcb_b1(A, rx, fix2d(Ex)), o);
        Etr = relax_one_b(A, C, rx.P1, qC, sC.zpe_fix, sb, Etr, 2.0f, o);
    } else {
        Etr = relax_flat(A, C, rx.P0, qB, sB.zpe_fix, sa, rx.P1, qC, sC.zpe_fix, sb,
                         Eav - sB.zpe_fix - sC.zpe_fix, o);
    }
    if (Etr < 0) { Etr = 0; o.ev += 1u << EV_DEGEN_SHIFT; }
    float x = 0.5f;
    for (int it = 0; it < 4096; ++it) {  // Beta(3/2,3/2) by rejection under 1/2
        x = st_u32(ss);
        const float y = st_u32(ss);
        if (y * y * 0.25f < x * (1.0f - x)) break;
    }
    const float Et = fix2f(Etr);
    const float E1 = x * Et;
    const float E2 = Et - E1;
    const float mu1 = C->pair[rx.P0 * MAXS + rx.P1].mr_f;
    const float mu2 = mBC * (mM / mt);
    const float g1 = sqrtf(2.0f * E1 / mu1);
    const float g2n = sqrtf(2.0f * E2 / mu2);
    float d1[3], d2[3];
    iso_dir<float>(ss, d1);
    iso_dir<float>(ss, d2);
    const float fM = mM / mt, fBC = mBC / mt, fC = mC / mBC, fB = mB / mBC;
    for (int i = 0; i < 3; ++i) {
        const float G2 = g2n * d2[i];
        const float VBC = V[i] + fM * G2;
        vM[i] = V[i] - fBC * G2;
        const float G1 = g1 * d1[i];
        vA[i] = VBC + fC * G1;
        vC[i] = VBC - fB * G1;
    }
    return true;
}

// FP32 mode, exchange A + B -> C + D: float kinematics, fixed-point energies
static __device__ bool do_exch_fix(const StepArgs& A, const Consts* __restrict__ C, const DevReaction& rx,
                            float vA[3], float vB[3], int spA, int spB, long long EvA, long long EvB,
                            const DevRes& rs, uint32_t lcell, uint32_t rk, uint32_t (&qC)[4],
                            uint32_t (&qD)[4], PairOut& o, float erA = 0.f, float erB = 0.f) {
    const DevSpecies& sA = C->sp[spA];
    const DevSpecies& sB = C->sp[spB];
    const DevSpecies& sC = C->sp[rx.P0];
    const DevSpecies& sD = C->sp[rx.P1];
    const float mA = sA.mass_f, mB = sB.mass_f, mC = sC.mass_f, mD = sD.mass_f;
    const float mAB = mA + mB, mt = mC + mD;
    float V[3];
    for (int i = 0; i < 3; ++i) V[i] = __fdiv_rn(__fadd_rn(__fmul_rn(mA, vA[i]), __fmul_rn(mB, vB[i])), mAB);
    const long long Ein = etr_fix_f32(C->pair[spA * MAXS + spB], g2_f32(vA, vB));
    const long long Eav = Ein + EvA + EvB - rx.dEf_fix + f2fix(erA) + f2fix(erB);
    if (!(Eav - sC.zpe_fix - sD.zpe_fix > 0) || Eav - sD.zpe_fix > sC.top_fix ||
        Eav - sC.zpe_fix > sD.top_fix)
        return false;
    Stream sa, sb, ss;
    st_init(sa, rs.seed, rs.step, lcell, rk, PU_LB_A);
    st_init(sb, rs.seed, rs.step, lcell, rk, PU_LB_B);
    st_init(ss, rs.seed, rs.step, lcell, rk, PU_SCAT);
    for (int j = 0; j < 4; ++j) { qC[j] = 0u; qD[j] = 0u; }
    long long Etr;
    if (rx.prod_split == HCAO_SPLIT_TCOLL) {
        const long long Ex = Eav - sC.zpe_fix - sD.zpe_fix;
        Etr = relax_one_b(A, C, rx.P0, qC, sC.zpe_fix, sa, Ex, tcb_b1(A, rx, fix2d(Ex)), o);
        Etr = relax_one_b(A, C, rx.P1, qD, sD.zpe_fix, sb, Etr, 0.5f, o);
    } else {
        Etr = relax_flat(A, C, rx.P0, qC, sC.zpe_fix, sa, rx.P1, qD, sD.zpe_fix, sb,
                         Eav - sC.zpe_fix - sD.zpe_fix, o);
    }
    if (Etr < 0) { Etr = 0; o.ev += 1u << EV_DEGEN_SHIFT; }
    const float gn = __fsqrt_rn(__fdiv_rn(__fmul_rn(2.0f, fix2f(Etr)), C->pair[rx.P0 * MAXS + rx.P1].mr_f));
    float d[3];
    iso_dir<float>(ss, d);
    const float fC = __fdiv_rn(mD, mt), fD = __fdiv_rn(mC, mt);
    for (int i = 0; i < 3; ++i) {
        const float G = __fmul_rn(gn, d[i]);
        vA[i] = __fadd_rn(V[i], __fmul_rn(fC, G));
        vB[i] = __fsub_rn(V[i], __fmul_rn(fD, G));
    }
    return true;
}

// FP32 mode, recombination B + C + M -> A + M: float kinematics, fixed-point
// energies (the three bodies' energies in their centre-of-mass frame are
// converted one by one; no product of two masses is formed)
static __device__ bool do_recomb_fix(const StepArgs& A, const Consts* __restrict__ C,
                                     const DevReaction& rx, float vB[3], float vC[3], float vM[3],
                                     int spB, int spC, int spM, long long EvB, long long EvC,
                                     const DevRes& rs, uint32_t lcell, uint32_t rk,
                                     uint32_t (&qA)[4], PairOut& o, float erB = 0.f, float erC = 0.f) {
    const DevSpecies& sA = C->sp[rx.P0];
    const float mB = C->sp[spB].mass_f, mC = C->sp[spC].mass_f, mM = C->sp[spM].mass_f;
    const float m3 = (mB + mC) + mM;
    float V[3];
    for (int i = 0; i < 3; ++i) V[i] = ((mB / m3) * vB[i] + (mC / m3) * vC[i]) + (mM / m3) * vM[i];
    float eB = 0.f, eC = 0.f, eM = 0.f;
    for (int i = 0; i < 3; ++i) {
        const float b = vB[i] - V[i], c = vC[i] - V[i], m = vM[i] - V[i];
        eB += b * b;
        eC += c * c;
        eM += m * m;
    }
    const long long Ein = f2fix(0.5f * mB * eB) + f2fix(0.5f * mC * eC) + f2fix(0.5f * mM * eM);
    const long long Eav = Ein + EvB + EvC - rx.dEf_fix + f2fix(erB) + f2fix(erC);
    if (!(Eav - sA.zpe_fix > 0) || Eav > sA.top_fix) return false;
    Stream sa, sb, ss;
    st_init(sa, rs.seed, rs.step, lcell, rk, PU_LB_A);
    st_init(sb, rs.seed, rs.step, lcell, rk, PU_LB_B);
    st_init(ss, rs.seed, rs.step, lcell, rk, PU_SCAT);
    for (int j = 0; j < 4; ++j) qA[j] = 0u;
    uint32_t qn[4] = {0u, 0u, 0u, 0u};
    long long Etr = rx.prod_split == HCAO_SPLIT_TCOLL
                        ? relax_one_b(A, C, rx.P0, qA, sA.zpe_fix, sa, Eav - sA.zpe_fix, 0.5f, o)
                        : relax_flat(A, C, rx.P0, qA, sA.zpe_fix, sa, -1, qn, 0, sb, Eav - sA.zpe_fix, o);
    if (Etr < 0) { Etr = 0; o.ev += 1u << EV_DEGEN_SHIFT; }
    const DevPair& pam = C->pair[rx.P0 * MAXS + spM];
    const float gn = sqrtf(fix2f(Etr) * pam.inv2mr_f);
    float d[3];
    iso_dir<float>(ss, d);
    for (int i = 0; i < 3; ++i) {
        const float G = gn * d[i];
        vB[i] = V[i] + pam.fp_f * G;
        vM[i] = V[i] - pam.fq_f * G;
    }
    return true;
}

// recombination: cell temperature at the step start from the integer sums
// (units 2^-96 J, 2^-104 kg m/s, 2^-120 kg): kinetic energy in the cell's
// centre-of-mass frame = 3/2 N k T
__device__ __forceinline__ double cell_temperature(const StepArgs& A, int c, uint32_t N) {
    if (N < 2u) return 0.0;
    const long long* s = A.csum + 5 * (size_t)c;
    const double Ek = (double)s[0] * 0x1p-96;
    const double px = (double)s[1], py = (double)s[2], pz = (double)s[3];
    const double P2 = (px * px + py * py) + pz * pz;
    const double Ecm = (0.5 * (P2 / (double)s[4])) * 0x1p-88;
    return (2.0 * (Ek - Ecm)) / (3.0 * (double)N * 1.380649e-23);
}

// k_r of rate-table slot `slot` with a third body of species sM at T: linear
// in T between the nodes T_i = 500 K * 2^(i/32), clamped at the ends
__device__ __forceinline__ double rec_rate(const StepArgs& A, int slot, int sM, double T) {
    const double* Tn = A.Tnode;
    const double* k = A.krec + ((size_t)slot * MAXS + sM) * REC_NODES;
    const int last = REC_NODES - 1;
    if (!(T > __ldg(Tn))) return __ldg(k);
    if (!(T < __ldg(Tn + last))) return __ldg(k + last);
    int lo = 0, hi = last;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(Tn + mid) <= T) lo = mid; else hi = mid;
    }
    const double T0 = __ldg(Tn + lo), T1 = __ldg(Tn + hi);
    const double f = (T - T0) / (T1 - T0);
    const double k0 = __ldg(k + lo), k1 = __ldg(k + hi);
    return k0 + f * (k1 - k0);
}

// Recombination test of an accepted pair (reading A14), before the QK
// channels: a (B, C) pair recombines with probability k_r(T_cell) n / (sigma_T g),
// n = (N - 2) w / V_c, k_r that of the third body M = the particle at position
// 2 kmax + k of the round's permutation (in no pair of this round); no third
// body (past the cell's end, or removed earlier this step), no recombination.
template <class R>
__device__ bool recomb_test(const StepArgs& A, const Consts* __restrict__ C, int c, int r, uint32_t k,
                            int sP, int sQ, double sg, uint32_t& chan, uint32_t& iM) {
    using Rec = typename RecOf<R>::T;
    const int code = C->rec_pair[sP * MAXS + sQ];
    if (code < 0) return false;
    const DevCell& cell = A.cells[c];
    const uint32_t N = cell.n;
    const uint32_t* pb = A.pbase + r * (A.n_cells + 1);
    const uint64_t m = 2ull * (uint64_t)(__ldg(pb + c + 1) - __ldg(pb + c)) + k;
    if (m >= N) return false;
    const uint32_t key[4] = {cell.pkey[r][0], cell.pkey[r][1], cell.pkey[r][2], cell.pkey[r][3]};
    iM = pair_perm((uint32_t)m, N, key);
    const Rec* recs = reinterpret_cast<const Rec*>(cell.rec);
    const uint32_t meta = reinterpret_cast<const uint32_t*>(recs + iM)[std::is_same<R, double>::value ? 6 : 3];
    const int sM = (int)(meta & 0xFFu);
    if (sM >= MAXS) return false;
    const int ri = code & 7;
    const double kr = rec_rate(A, C->rx[ri].rslot, sM, cell_temperature(A, c, N));
    const DevRes& rs = A.res[cell.res];
    const double n3 = ((double)(N - 2u) * rs.w) / rs.Vc;
    const double prec = (kr * n3) / sg;
    Stream st;
    st_init(st, rs.seed, rs.step, cell.lcell, ((uint32_t)r << 24) | k, PU_REC);
    const double u = std::is_same<R, double>::value ? st_u64(st) : (double)st_u32(st);
    if (!(u < prec)) return false;
    chan = chan_pack(ri, (code >> 3) & 1, 0);
    return true;
}

// HCAO LB relaxation of molecule 1 then molecule 2 (with the updated E_rel),
// then isotropic VHS scattering with the centre-of-mass velocity kept.
template <class R, class Rec>
__device__ void relax_scatter(const StepArgs& A, const Consts* __restrict__ C, const DevRes& rs,
                              const PairLoc& L, Rec& Pr, Rec& Qr, const DevPair& pc, double Etr,
                              double EvP, double EvQ, PairOut& o) {
    constexpr bool F64 = std::is_same<R, double>::value;
    const int sP = (int)(Pr.meta & 0xFFu), sQ = (int)(Qr.meta & 0xFFu);
    const DevSpecies& SP = C->sp[sP];
    const DevSpecies& SQ = C->sp[sQ];
    const int amode = C->amode;
    double E = Etr;
    uint32_t tr = 0;
    if constexpr (!F64) {
        // FP32 mode goes through relax_scatter_fix
    } else {
    if (SP.n_modes > 0) {
        Stream s1;
        st_init(s1, rs.seed, rs.step, L.lcell, L.rk, PU_LB_A);
        const double Ec = E + EvP;
        uint32_t nq[4] = {Pr.q[0], Pr.q[1], Pr.q[2], Pr.q[3]};
        o.ev += 1u << EV_SAMP_SHIFT;
        const int st = sample_lb<R>(A, SP, amode, Ec, s1, nq, tr);
        if (st == S_OK) {
            const double En = Ec - evib64(A.lev64, SP, nq);
            if (F64 || En >= 0.0) {
                for (int j = 0; j < 4; ++j) Pr.q[j] = nq[j];
                E = En;
            } else {
                o.ev += 1u << EV_DEGEN_SHIFT;
                E = Ec - EvP;
            }
        } else {
            if (st == S_OVER) o.ev += 1u << EV_OVER_SHIFT;
            else if (st == S_DEGEN) o.ev += 1u << EV_DEGEN_SHIFT;
            else atomicOr(A.err, (uint32_t)ERR_REJECT);
            E = Ec - EvP;
        }
    }
    if (SQ.n_modes > 0) {
        Stream s2;
        st_init(s2, rs.seed, rs.step, L.lcell, L.rk, PU_LB_B);
        const double Ec = E + EvQ;
        uint32_t nq[4] = {Qr.q[0], Qr.q[1], Qr.q[2], Qr.q[3]};
        o.ev += 1u << EV_SAMP_SHIFT;
        const int st = sample_lb<R>(A, SQ, amode, Ec, s2, nq, tr);
        if (st == S_OK) {
            const double En = Ec - evib64(A.lev64, SQ, nq);
            if (F64 || En >= 0.0) {
                for (int j = 0; j < 4; ++j) Qr.q[j] = nq[j];
                E = En;
            } else {
                o.ev += 1u << EV_DEGEN_SHIFT;
                E = Ec - EvQ;
            }
        } else {
            if (st == S_OVER) o.ev += 1u << EV_OVER_SHIFT;
            else if (st == S_DEGEN) o.ev += 1u << EV_DEGEN_SHIFT;
            else atomicOr(A.err, (uint32_t)ERR_REJECT);
            E = Ec - EvQ;
        }
    }
    o.trials += tr;
    // classical LB rotational relaxation, P then Q, one stream per pair
    if (SP.rot_dof > 0 || SQ.rot_dof > 0) {
        Stream sr;
        st_init(sr, rs.seed, rs.step, L.lcell, L.rk, PU_ROT);
        for (int m = 0; m < 2; ++m) {
            Rec& X = m ? Qr : Pr;
            const DevSpecies& SX = m ? SQ : SP;
            if (SX.rot_dof == 0) continue;
            const double Ec = E + rec_erot(X);
            const double er = rot_fraction<double>(A, SX, amode, sr) * Ec;
            rec_set_erot(X, er);
            E = Ec - er;
        }
    }
    }
    Stream ss;
    st_init(ss, rs.seed, rs.step, L.lcell, L.rk, PU_SCAT);
    if constexpr (F64) {
        const double gn = sqrt(2.0 * E / pc.mr);
        double d[3];
        iso_dir<double>(ss, d);
        const double mp = SP.mass, mq = SQ.mass;
        double V[3];
        for (int i = 0; i < 3; ++i) V[i] = (mp * Pr.v[i] + mq * Qr.v[i]) / pc.mt;
        for (int i = 0; i < 3; ++i) {
            const double G = gn * d[i];
            Pr.v[i] = V[i] + pc.fp * G;
            Qr.v[i] = V[i] - pc.fq * G;
        }
    } else {
        const float gn = sqrtf((float)E * pc.inv2mr_f);
        float d[3];
        iso_dir<float>(ss, d);
        float V[3];
        for (int i = 0; i < 3; ++i) V[i] = pc.fq_f * Pr.v[i] + pc.fp_f * Qr.v[i];
        for (int i = 0; i < 3; ++i) {
            const float G = gn * d[i];
            Pr.v[i] = V[i] + pc.fp_f * G;
            Qr.v[i] = V[i] - pc.fq_f * G;
        }
    }
}

// FP32 mode: relaxation (flattened sampler, fixed-point bookkeeping) and
// isotropic scattering with the centre-of-mass velocity kept.
// FP32 classical LB rotational relaxation of a pair's rotating molecules, P
// then Q (one stream): energies in fixed point, the new rotational energy a
// float stored in q[3]; erP, erQ the rotational energies before the
// collision.  Returns the relative energy left.
__device__ __forceinline__ long long rot_relax_fix(const StepArgs& A, const Consts* __restrict__ C, uint64_t seed,
                                                   uint32_t step, uint32_t lcell, uint32_t rk, int sP, int sQ,
                                                   float erP, float erQ, uint32_t (&qP)[4], uint32_t (&qQ)[4],
                                                   long long E) {
    const DevSpecies& SP = C->sp[sP];
    const DevSpecies& SQ = C->sp[sQ];
    if (SP.rot_dof == 0 && SQ.rot_dof == 0) return E;
    Stream sr;
    st_init(sr, seed, step, lcell, rk, PU_ROT);
    if (SP.rot_dof > 0) {
        const long long Ec = E + f2fix(erP);
        const float e = __fmul_rn(rot_fraction<float>(A, SP, C->amode, sr), fix2f(Ec));
        qP[3] = __float_as_uint(e);
        E = Ec - f2fix(e);
    }
    if (SQ.rot_dof > 0) {
        const long long Ec = E + f2fix(erQ);
        const float e = __fmul_rn(rot_fraction<float>(A, SQ, C->amode, sr), fix2f(Ec));
        qQ[3] = __float_as_uint(e);
        E = Ec - f2fix(e);
    }
    return E;
}

__device__ __forceinline__ void relax_scatter_fix(const StepArgs& A, const Consts* __restrict__ C,
                                                  const DevRes& rs, const PairLoc& L, RecF& Pr,
                                                  RecF& Qr, const DevPair& pc, long long Etr,
                                                  long long EvP, long long EvQ, PairOut& o) {
    const int sP = (int)(Pr.meta & 0xFFu), sQ = (int)(Qr.meta & 0xFFu);
    const float erP = C->sp[sP].rot_dof ? erot_f(Pr.q) : 0.f, erQ = C->sp[sQ].rot_dof ? erot_f(Qr.q) : 0.f;
    Stream s1, s2;
    st_init(s1, rs.seed, rs.step, L.lcell, L.rk, PU_LB_A);
    st_init(s2, rs.seed, rs.step, L.lcell, L.rk, PU_LB_B);
    long long E = relax_flat(A, C, sP, Pr.q, EvP, s1, sQ, Qr.q, EvQ, s2, Etr, o);
    E = rot_relax_fix(A, C, rs.seed, rs.step, L.lcell, L.rk, sP, sQ, erP, erQ, Pr.q, Qr.q, E);
    Stream ss;
    st_init(ss, rs.seed, rs.step, L.lcell, L.rk, PU_SCAT);
    float d[3];
    iso_dir<float>(ss, d);
    const float va[3] = {Pr.v[0], Pr.v[1], Pr.v[2]}, vb[3] = {Qr.v[0], Qr.v[1], Qr.v[2]};
    scatter_f32(pc, E, d, va, vb, Pr.v, Qr.v);
}

__device__ __forceinline__ uint32_t ev_final(const PairOut& o) {
    return o.ev | ((o.trials > 0xFFFFu ? 0xFFFFu : o.trials) << EV_TRIAL_SHIFT);
}

// warp-aggregated append of one entry per lane with `want` to a queue
__device__ __forceinline__ uint32_t queue_slot(uint32_t* size, bool want) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, want);
    if (!want) return 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(size, (uint32_t)__popc(m));
    base = __shfl_sync(m, base, leader);
    return base + (uint32_t)__popc(m & ((1u << lane) - 1u));
}

// A cell's max sigma_T g of the step (bits of a double >= 0, which order as
// integers).  In a large cell (a single-cell reservoir of millions) the
// atomic only when the value could raise the max: the max only grows during
// the step, so a value not above one already read changes nothing, and a
// stale read merely costs an atomic; without the test the cell's warps queue
// on one word.  A small cell takes the atomic without the read (few warps
// share its word, and the read would add its latency).
constexpr uint32_t SEEN_READ_MIN_N = 8192;
__device__ __forceinline__ void seen_max(unsigned long long* seen, double v, uint32_t N) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if (N < SEEN_READ_MIN_N || b > __ldcg(seen)) atomicMax(seen, b);
}

// cell of flat pair index g in a prefix array (largest c with pb[c] <= g)
__device__ __forceinline__ int cell_of(const uint32_t* pb, int n_cells, uint32_t g) {
    int lo = 0, hi = n_cells;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pb + mid) <= g) lo = mid; else hi = mid;
    }
    return lo;
}
// The same for a whole warp with one g (all 32 lanes active, g < pb[n_cells]):
// a 32-way search, each round's lanes probing evenly spaced cells, so a few
// dependent loads replace the bisection's log2(n_cells).
__device__ __forceinline__ int cell_of_warp(const uint32_t* pb, int n_cells, uint32_t g) {
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = n_cells;  // pb[lo] <= g < pb[hi]
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int idx = lo + (lane + 1) * step;
        const bool le = idx < hi && __ldg(pb + idx) <= g;
        const int c = __popc(__ballot_sync(0xFFFFFFFFu, le));
        const int nlo = lo + c * step;
        hi = min(hi, nlo + step);
        lo = nlo;
    }
    return lo;
}

// ------------------------------------------------------------- kernels
#ifdef HCAO_COMMON_KERNELS

// Per-cell step set-up, one thread per cell, SETUP_TILE cells per CTA: the
// NTC candidate count N_sel (stochastically rounded), the rounds and their
// pairing-permutation keys, and the counts behind the step's prefix arrays -- pairs per
// round, all pairs, FINISH_CHUNK chunks and (with recombination) particles.
// Each CTA writes the inclusive scans of its tile into the arrays and the
// tile's totals into tsum; the last CTA to finish (a ticket counter, no
// waiting) scans the tile totals, which k_setup_fix then adds to the tiles.
static __global__ void __launch_bounds__(SETUP_TILE) k_setup_cells(StepArgs A) {
    const int nc = A.n_cells, R = A.max_rounds, nt = (int)gridDim.x;
    const int c = blockIdx.x * SETUP_TILE + threadIdx.x;
    uint32_t v[SETUP_ARRAYS];
#pragma unroll
    for (int q = 0; q < SETUP_ARRAYS; ++q) v[q] = 0u;
    if (c < nc) {
        DevCell& cl = A.cells[c];
        const DevRes rs = A.res[cl.res];
        const uint32_t N = cl.n;
        uint32_t rounds = 0;
        const uint32_t P = round_pairs(N, A.has_recomb);
        // a round's pair index is a 24-bit field of the pair's Philox key (and
        // of the FP32 queue's pair word): at most 2^24 pairs a round
        if (P > (1u << 24)) atomicOr(A.err, (uint32_t)ERR_CAPACITY);
        const uint32_t nsel = ntc_setup(A, rs, cl, N, P, rounds, cl.pkey);
        cl.nsel = nsel;
        cl.ncreated = 0;
        cl.seen = 0ull;
        cl.sgmax_f = (float)cl.sgmax;
        cl.nremoved = 0u;
#pragma unroll
        for (int r = 0; r < MAX_ROUNDS; ++r)
            if ((uint32_t)r < rounds) {
                const uint32_t left = nsel - (uint32_t)r * P;
                v[r] = left < P ? left : P;
            }
        v[SA_ALL] = nsel;
        v[SA_CHUNK] = (nsel + (uint32_t)FINISH_CHUNK - 1u) / (uint32_t)FINISH_CHUNK;
        if (A.has_recomb) {
            v[SA_PART] = N;
            for (int q = 0; q < 5; ++q) A.csum[5 * (size_t)c + q] = 0ll;
        }
    }
    // tile-local inclusive scans of all arrays at once
    __shared__ uint32_t ws[SETUP_ARRAYS][SETUP_TILE / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < SETUP_ARRAYS; ++q) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v[q], o);
            if (lane >= o) v[q] += t;
        }
        if (lane == 31) ws[q][wid] = v[q];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < SETUP_ARRAYS; ++q) {
            uint32_t w = lane < SETUP_TILE / 32 ? ws[q][lane] : 0u;
#pragma unroll
            for (int o = 1; o < SETUP_TILE / 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, w, o);
                if (lane >= o) w += t;
            }
            if (lane < SETUP_TILE / 32) ws[q][lane] = w;
        }
    }
    __syncthreads();
    if (wid > 0) {
#pragma unroll
        for (int q = 0; q < SETUP_ARRAYS; ++q) v[q] += ws[q][wid - 1];
    }
    if (c < nc) {
#pragma unroll
        for (int r = 0; r < MAX_ROUNDS; ++r)
            if (r < R) A.pbase[r * (nc + 1) + c + 1] = v[r];
        A.abase[c + 1] = v[SA_ALL];
        A.chbase[c + 1] = v[SA_CHUNK];
        if (A.has_recomb) A.nbase[c + 1] = v[SA_PART];
    }
    // tile totals: tsum[q][t + 1]; the exclusive prefix of tile t ends up at tsum[q][t]
    if (threadIdx.x < SETUP_ARRAYS) A.tsum[threadIdx.x * (nt + 1) + blockIdx.x + 1] = ws[threadIdx.x][SETUP_TILE / 32 - 1];
    __threadfence();
    __shared__ uint32_t last;
    if (threadIdx.x == 0) last = atomicAdd(A.tsum + SETUP_ARRAYS * (nt + 1), 1u) == (uint32_t)(nt - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    // warp q scans array q's tile totals in place: tsum[q][t] becomes the
    // exclusive prefix of tile t, tsum[q][nt] the array's total
    for (int q = wid; q < SETUP_ARRAYS; q += SETUP_TILE / 32) {
        uint32_t* ts = A.tsum + q * (nt + 1);
        uint32_t carry = 0u;
        for (int b = 0; b < nt; b += 32) {
            const int t = b + lane;
            uint32_t x = t < nt ? __ldcg(ts + t + 1) : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            if (t < nt) ts[t + 1] = carry + x;
            carry += __shfl_sync(0xFFFFFFFFu, x, 31);
        }
        if (lane == 0) ts[0] = 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int r = 0; r < R; ++r) {
            A.pbase[r * (nc + 1)] = 0;
            A.totals[r] = A.tsum[r * (nt + 1) + nt];
        }
        A.abase[0] = 0;
        A.chbase[0] = 0;
        if (A.has_recomb) A.nbase[0] = 0;
        A.totals[MAX_ROUNDS] = A.tsum[SA_ALL * (nt + 1) + nt];
        A.totals[MAX_ROUNDS + 1] = A.tsum[SA_CHUNK * (nt + 1) + nt];
        A.tsum[SETUP_ARRAYS * (nt + 1)] = 0u;  // ticket, for the next step
    }
    for (int i = threadIdx.x; i < QSIZE_WORDS; i += SETUP_TILE) A.qsize[i] = 0u;
}

// Adds the scanned tile totals to every tile (tile 0's are zero) and
// tabulates the cell of every 256th candidate pair of each round, entries b =
// 0 .. ceil(total / 256): cell c writes the entries with pb[c] <= 256 b <
// pb[c + 1], the last cell also the entry past the end (the largest c with
// pb[c] <= 256 b, as a bisection would find it).  The selection then searches
// only the cells between two entries (one or two for cells of hundreds of
// pairs) instead of all cells.
static __global__ void __launch_bounds__(SETUP_TILE) k_setup_fix(StepArgs A) {
    const int nc = A.n_cells, R = A.max_rounds, nt = (int)gridDim.x;
    const int t = blockIdx.x;
    const int c = t * SETUP_TILE + threadIdx.x;
    const bool in = c < nc;
    uint32_t lo[MAX_ROUNDS], hi[MAX_ROUNDS];
#pragma unroll
    for (int r = 0; r < MAX_ROUNDS; ++r) {
        lo[r] = hi[r] = 0u;
        if (in && r < R) {
            const uint32_t off = __ldcg(A.tsum + r * (nt + 1) + t);
            const uint32_t* pb = A.pbase + r * (nc + 1);
            hi[r] = pb[c + 1] + off;
            // the tile's first cell starts at the tile's offset; the others
            // at their left neighbour's end, read before it is offset
            lo[r] = threadIdx.x == 0 ? off : pb[c] + off;
        }
    }
    __syncthreads();
    if (!in) return;
#pragma unroll
    for (int r = 0; r < MAX_ROUNDS; ++r) {
        if (r >= R) break;
        A.pbase[r * (nc + 1) + c + 1] = hi[r];
        uint32_t* bc = A.blkcell + (size_t)r * A.blk_stride;
        const uint32_t bend = (hi[r] + 255u) / 256u + (c == nc - 1 ? 1u : 0u);
        for (uint32_t b = (lo[r] + 255u) / 256u; b < bend && b < A.blk_stride; ++b) bc[b] = (uint32_t)c;
    }
    A.abase[c + 1] += __ldcg(A.tsum + SA_ALL * (nt + 1) + t);
    A.chbase[c + 1] += __ldcg(A.tsum + SA_CHUNK * (nt + 1) + t);
    if (A.has_recomb) A.nbase[c + 1] += __ldcg(A.tsum + SA_PART * (nt + 1) + t);
}

int launch_setup(const StepArgs& a, cudaStream_t s) {
    const int nt = setup_tiles(a.n_cells);
    k_setup_cells<<<nt, SETUP_TILE, 0, s>>>(a);
    k_setup_fix<<<nt, SETUP_TILE, 0, s>>>(a);
    return 2;
}

// Load-path validation of staged host arrays: cell and species in range,
// every quantum number inside its mode's level list (0 beyond the species'
// modes).  flags[0] collects LOAD_BAD_* bits, flags[1] the species present.
static __global__ void __launch_bounds__(256) k_validate_load(const Consts* C, int n_cells, const int32_t* cell,
                                                              const int32_t* sp, const uint8_t* qn, int64_t n,
                                                              uint32_t* flags) {
    uint32_t bad = 0u, present = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell[i], s = sp[i];
        if (c < 0 || c >= n_cells) bad |= LOAD_BAD_CELL;
        if (s < 0 || s >= C->n_species) {
            bad |= LOAD_BAD_SPECIES;
            continue;
        }
        present |= 1u << s;
        const uint4 q4 = reinterpret_cast<const uint4*>(qn)[i];
        const uint32_t q[4] = {q4.x, q4.y, q4.z, q4.w};
        const DevSpecies& S = C->sp[s];
        for (int j = 0; j < MAXM; ++j) {
            const uint32_t v = get_q(q, j);
            if (j < S.n_modes ? v >= (uint32_t)S.n_lev[j] : v != 0u) bad |= LOAD_BAD_LEVEL;
        }
    }
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
    present = __reduce_or_sync(0xFFFFFFFFu, present);
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(flags, bad);
        if (present) atomicOr(flags + 1, present);
    }
}

void launch_validate_load(const Consts* C, int n_cells, const int32_t* cell, const int32_t* sp, const uint8_t* qn,
                          int64_t n, uint32_t* flags, cudaStream_t s) {
    if (n <= 0) return;
    int64_t g = (n + 255) / 256;
    if (g > 2368) g = 2368;
    k_validate_load<<<(int)g, 256, 0, s>>>(C, n_cells, cell, sp, qn, n, flags);
}

// off[c] = the particles of cells cell0 .. cell0 + c - 1 (c = 0 .. n_cells),
// the canonical-order prefix of a reservoir, on the device (no copy of the
// cell table to the host): one CTA, each thread a contiguous run of cells.
static __global__ void __launch_bounds__(1024) k_cell_prefix(const DevCell* cells, int cell0, int n_cells,
                                                             uint64_t* off) {
    __shared__ uint64_t wtot[32];
    const int per = (n_cells + 1023) / 1024;
    const int c0 = min((int)threadIdx.x * per, n_cells), c1 = min(c0 + per, n_cells);
    uint64_t s = 0;
    for (int c = c0; c < c1; ++c) s += cells[cell0 + c].n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t x = s;  // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint64_t t = wtot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        wtot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    uint64_t run = (wid ? wtot[wid - 1] : 0ull) + x - s;  // exclusive prefix of this thread's run
    for (int c = c0; c < c1; ++c) {
        off[c] = run;
        run += cells[cell0 + c].n;
    }
    if (threadIdx.x == 0) off[n_cells] = wtot[31];
}

void launch_cell_prefix(const DevCell* cells, int cell0, int n_cells, uint64_t* off, cudaStream_t s) {
    k_cell_prefix<<<1, 1024, 0, s>>>(cells, cell0, n_cells, off);
}

// out[i] = the sum over cells cell0 .. cell0 + n_cells - 1 of counter i
// (n_cnt counters a cell): a warp per counter and CTA, one atomic each.
static __global__ void __launch_bounds__(256) k_sum_counters(const unsigned long long* cnt, int cell0, int n_cells,
                                                              int n_cnt, unsigned long long* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = wid; i < n_cnt; i += 8) {
        unsigned long long s = 0;
        for (int c = blockIdx.x * 32 + lane; c < n_cells; c += gridDim.x * 32)
            s += cnt[(size_t)(cell0 + c) * n_cnt + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if (lane == 0 && s) atomicAdd(out + i, s);
    }
}

void launch_sum_counters(const unsigned long long* cnt, int cell0, int n_cells, int n_cnt, unsigned long long* out,
                         cudaStream_t s) {
    const int g = (n_cells + 31) / 32 < 148 ? (n_cells + 31) / 32 : 148;
    k_sum_counters<<<g < 1 ? 1 : g, 256, 0, s>>>(cnt, cell0, n_cells, n_cnt, out);
}
#endif

// Phase 1 of a round: every candidate pair's VHS acceptance (NTC).  Rejected
// pairs are finished here; accepted ones go to the relaxation queue (in FP32
// mode staged with their work class, for k_qorder).
constexpr int SELECT_THREADS = 256;

template <class R>
__global__ void __launch_bounds__(SELECT_THREADS) k_select(StepArgs A, int r) {
    using Rec = typename RecOf<R>::T;
    const uint32_t total = A.totals[r];
    const uint32_t* pb = A.pbase + r * (A.n_cells + 1);
    const uint32_t stride = gridDim.x * blockDim.x;
    const Consts* __restrict__ C = A.C;
    const int amode = C->amode;
    uint32_t* qsize = A.qsize + 2 * r;
    if constexpr (std::is_same<R, float>::value) {
        // FP32 mode: no FP64 arithmetic; the second half of a record (the
        // quantum numbers) is read only for accepted pairs when reactions exist
        // staging counts, double-buffered by pass: a pass writes the set the
        // previous pass did not read, so it needs two barriers, not three
        __shared__ uint32_t sel_cnt[2][SELECT_THREADS / 32], sel_base[2], cls_cnt[2][NCLS];
        if (threadIdx.x < 2 * NCLS) cls_cnt[threadIdx.x / NCLS][threadIdx.x % NCLS] = 0u;
        __syncthreads();
        int par = 0;
        for (uint32_t g0 = blockIdx.x * blockDim.x; g0 < total; g0 += stride) {
            const uint32_t g = g0 + threadIdx.x;
            const bool valid = g < total;
            int c = 0;
            bool accept = false;
            uint32_t cls = 0u;
            float sgf = 0.f;
            uint32_t k = 0, ip = 0, iq = 0, N = 0;
            if (valid) {
                {  // the cell of g: bisection between the cells of g's 256-pair block and the next
                    const uint32_t* bc = A.blkcell + (size_t)r * A.blk_stride + (g >> 8);
                    int lo = (int)__ldg(bc), hi = (int)__ldg(bc + 1) + 1;
                    if (hi > A.n_cells) hi = A.n_cells;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (__ldg(pb + mid) <= g) lo = mid; else hi = mid;
                    }
                    c = lo;
                }
                k = g - __ldg(pb + c);
                const DevCell& cell = A.cells[c];
                N = cell.n;
                const uint32_t rk = ((uint32_t)r << 24) | k;
                const uint32_t key[4] = {cell.pkey[r][0], cell.pkey[r][1], cell.pkey[r][2], cell.pkey[r][3]};
                ip = pair_perm(2u * k, N, key);
                iq = pair_perm(2u * k + 1u, N, key);
                const uint4* recs = reinterpret_cast<const uint4*>(cell.rec);
                const uint4 a = REC_LD(recs + 2 * ip), b = REC_LD(recs + 2 * iq);
                const int sP = (int)(a.w & 0xFFu), sQ = (int)(b.w & 0xFFu);
                const DevRes& rs = A.res[cell.res];
                const uint32_t ev_idx = A.abase[c] + (uint32_t)r * round_pairs(N, A.has_recomb) + k;
                // a member removed earlier in this step (recombination): no collision
                if (sP < MAXS && sQ < MAXS) {
                const float va[3] = {__uint_as_float(a.x), __uint_as_float(a.y), __uint_as_float(a.z)};
                const float vb[3] = {__uint_as_float(b.x), __uint_as_float(b.y), __uint_as_float(b.z)};
                sgf = sg_f32(C->pair[sP * MAXS + sQ], amode, g2_f32(va, vb));
                if (!(sgf <= 3.0e38f)) {
                    atomicOr(A.err, (uint32_t)ERR_NONFINITE);
                    sgf = 0.f;
                }
                Stream sp;
                st_init(sp, rs.seed, rs.step, cell.lcell, rk, PU_PAIR);
                accept = st_u32(sp) < __fdiv_rn(sgf, cell.sgmax_f);
                cls = C->pair[sP * MAXS + sQ].cls;
                }
                if (!accept) {
                    A.cflag[ev_idx] = 0u;
                    if (A.log_on) A.log[ev_idx] = hcao_log_rec{rs.step, cell.lcell, rk, ip, iq, -1, 0u};
                }
            }
            // the relaxation queue, staged at qA[cap + i] in arrival order with
            // the pair's work class in the top byte of the pair word (k < 2^24,
            // as in the pair's Philox key); k_qorder then places the entries
            // class by class, so that the lanes of a warp of the relaxation
            // kernel run mode-draw loops of like length (with a single class in
            // use: straight to qA[i], no placement).  One atomic per CTA for
            // the staging slots, one per CTA and present class for the counts.
            {
                const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
                const unsigned m = __ballot_sync(0xFFFFFFFFu, accept);
                if (lane == 0) sel_cnt[par][wid] = (uint32_t)__popc(m);
                if (accept && A.qorder) atomicAdd(&cls_cnt[par][cls], 1u);
                __syncthreads();
                if (threadIdx.x == 0) {
                    uint32_t tot = 0u;
                    for (int w2 = 0; w2 < SELECT_THREADS / 32; ++w2) {
                        const uint32_t n = sel_cnt[par][w2];
                        sel_cnt[par][w2] = tot;
                        tot += n;
                    }
                    sel_base[par] = tot ? atomicAdd(qsize, tot) : 0u;
                }
                if (threadIdx.x < NCLS) {
                    const uint32_t n = cls_cnt[par][threadIdx.x];
                    if (n) {
                        atomicAdd(A.qsize + QCNT_OFF + r * NCLS + threadIdx.x, n);
                        cls_cnt[par][threadIdx.x] = 0u;
                    }
                }
                __syncthreads();
                if (accept) {
                    const uint64_t i = sel_base[par] + sel_cnt[par][wid] + (uint32_t)__popc(m & ((1u << lane) - 1u));
                    A.qA[(A.qorder ? A.pair_cap : 0u) + i] = make_uint4((uint32_t)c, (k & 0xFFFFFFu) | (cls << 24), ip, iq);
                }
                par ^= 1;
            }
            // per-cell max of sigma_T g: lanes of one cell combine before the atomic
            const unsigned act = __activemask();
            const int lane = threadIdx.x & 31;
            const int key = valid ? c : -1;
            unsigned left = __ballot_sync(act, valid);
            while (left) {
                const int leader = __ffs(left) - 1;
                const int cl = __shfl_sync(act, key, leader);
                const unsigned grp = __ballot_sync(act, key == cl);
                float mx = key == cl ? sgf : 0.f;
                for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(act, mx, o));
                if (lane == leader) seen_max(&A.cells[cl].seen, (double)mx, N);  // the leader's cell is cl
                left &= ~grp;
            }
        }
    } else {
    for (uint32_t g0 = blockIdx.x * blockDim.x; g0 < total; g0 += stride) {
        const uint32_t g = g0 + threadIdx.x;
        const bool valid = g < total;
        int c = 0;
        bool accept = false, react = false;
        double sg = 0.0;
        uint32_t k = 0, ip = 0, iq = 0, chan = 0, N = 0;
        if (valid) {
            c = cell_of(pb, A.n_cells, g);
            k = g - __ldg(pb + c);
            const PairLoc L = locate(A, c, r, k);
            ip = L.ip;
            N = L.N;
            iq = L.iq;
            const DevRes& rs = A.res[A.cells[c].res];
            const Rec* recs = reinterpret_cast<const Rec*>(L.recs);
            Rec Pr, Qr;
            load_rec(recs + L.ip, Pr);
            load_rec(recs + L.iq, Qr);
            const int sP = (int)(Pr.meta & 0xFFu), sQ = (int)(Qr.meta & 0xFFu);
            // a member removed earlier in this step (recombination): no collision
            if (sP < MAXS && sQ < MAXS) {
            double g2d;
            pair_energy<R>(C->pair[sP * MAXS + sQ], amode, Pr.v, Qr.v, g2d, sg);
            if (!(sg <= 1.0e300)) {  // non-finite velocities: report, keep (sigma g)_max
                atomicOr(A.err, (uint32_t)ERR_NONFINITE);
                sg = 0.0;
            }
            Stream sp;
            st_init(sp, rs.seed, rs.step, L.lcell, L.rk, PU_PAIR);
            if constexpr (std::is_same<R, double>::value) {
                accept = st_u64(sp) < sg / L.sgmax;
            } else {
                accept = st_u32(sp) < (float)sg / (float)L.sgmax;
                if (accept && C->n_reactions > 0) {
                    // FP32 mode: the QK reaction test here, in fixed point
                    const DevPair& pc = C->pair[sP * MAXS + sQ];
                    const long long Etr = f2fix(0.5f * pc.mr_f * (float)g2d);
                    const long long EvP = evib_fix(A.levfix, C->sp[sP], Pr.q);
                    const long long EvQ = evib_fix(A.levfix, C->sp[sQ], Qr.q);
                    const float u_ster = st_u32(sp);
                    const float u_sel = st_u32(sp);
                    const float u_ch = st_u32(sp);
                    react = reaction_pick_fix(A, C, sP, sQ, Pr.q, Qr.q, Etr, EvP, EvQ, u_ster, u_sel,
                                              u_ch, chan) > 0;
                }
            }
            }
            if (!accept) {
                A.cflag[L.ev_idx] = 0u;
                if (A.log_on) A.log[L.ev_idx] = hcao_log_rec{rs.step, L.lcell, L.rk, L.ip, L.iq, -1, 0u};
            }
        }
        const uint32_t slot = queue_slot(qsize, accept && !react);
        if (accept && !react) A.qA[slot] = make_uint4((uint32_t)c, k, ip, iq);
        const uint32_t rslot = queue_slot(qsize + 1, react);
        if (react) A.qB[rslot] = make_uint4((uint32_t)c, k, chan, 0u);
        // per-cell max of sigma_T g: lanes of one cell combine before the atomic
        const unsigned act = __activemask();
        const int lane = threadIdx.x & 31;
        const int key = valid ? c : -1;
        unsigned left = __ballot_sync(act, valid);
        while (left) {
            const int leader = __ffs(left) - 1;
            const int cl = __shfl_sync(act, key, leader);
            const unsigned grp = __ballot_sync(act, key == cl);
            double mx = 0.0;
            unsigned g2 = grp;
            while (g2) {
                const double v = __shfl_sync(act, sg, __ffs(g2) - 1);
                if (v > mx) mx = v;
                g2 &= g2 - 1;
            }
            if (lane == leader) seen_max(&A.cells[cl].seen, mx, N);  // the leader's cell is cl
            left &= ~grp;
        }
    }
    }
}

// FP32: the staged relaxation queue (qA[cap + i], arrival order) placed class
// by class at qA[0 ..): class c starts at the sum of the counts of classes
// below c (heaviest work first).  A CTA takes a chunk of 2048 staged entries,
// ranks them per class in shared memory, reserves each class's share of the
// chunk with one atomic on the class cursor and writes them out, so a chunk's
// entries of one class stay together (and near the cells they came from).
// The order within a class is free: every draw of a pair is keyed by the
// pair, not by its queue slot.
constexpr int QORDER_GRID = 592;  // 148 SMs x 4 CTAs of 256 threads, grid-stride over chunks
constexpr int QORDER_PER = 8;     // entries per thread and chunk
static __global__ void __launch_bounds__(256) k_qorder(StepArgs A, int r) {
    __shared__ uint32_t start[NCLS], cnt[NCLS], base[NCLS];
    const uint32_t total = A.qsize[2 * r];
    if (threadIdx.x < NCLS) {
        uint32_t s0 = 0u;
        for (int c = 0; c < (int)threadIdx.x; ++c) s0 += A.qsize[QCNT_OFF + r * NCLS + c];
        start[threadIdx.x] = s0;
    }
    uint32_t* cur = A.qsize + QCUR_OFF + r * NCLS;
    const uint4* stage = A.qA + A.pair_cap;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    constexpr uint32_t CH = 256u * QORDER_PER;
    for (uint32_t c0 = blockIdx.x * CH; c0 < total; c0 += gridDim.x * CH) {
        if (threadIdx.x < NCLS) cnt[threadIdx.x] = 0u;
        __syncthreads();
        uint4 e[QORDER_PER];
        uint32_t rank[QORDER_PER];
#pragma unroll
        for (int j = 0; j < QORDER_PER; ++j) {
            const uint32_t i = c0 + (uint32_t)j * 256u + threadIdx.x;
            const bool v = i < total;
            e[j] = v ? stage[i] : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t cls = v ? e[j].y >> 24 : 0xFFFFFFFFu;  // no class: lanes past the end
            const unsigned grp = __match_any_sync(0xFFFFFFFFu, cls);
            const int leader = __ffs(grp) - 1;
            uint32_t b0 = 0u;
            if (v && lane == leader) b0 = atomicAdd(&cnt[cls], (uint32_t)__popc(grp));
            rank[j] = __shfl_sync(0xFFFFFFFFu, b0, leader) + (uint32_t)__popc(grp & lt);
        }
        __syncthreads();
        if (threadIdx.x < NCLS) {
            const uint32_t n = cnt[threadIdx.x];
            base[threadIdx.x] = n ? start[threadIdx.x] + atomicAdd(cur + threadIdx.x, n) : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < QORDER_PER; ++j) {
            const uint32_t i = c0 + (uint32_t)j * 256u + threadIdx.x;
            if (i < total) A.qA[base[e[j].y >> 24] + rank[j]] = e[j];
        }
        __syncthreads();  // base and cnt are rewritten for the next chunk
    }
}

// Phase 2: accepted pairs.  QK reaction test; reacting pairs go to the
// reaction queue, the others are relaxed and scattered here.
template <class R>
__global__ void __launch_bounds__(128) k_relax(StepArgs A, int r) {
    using Rec = typename RecOf<R>::T;
    const uint32_t total = A.qsize[2 * r];
    const uint32_t stride = gridDim.x * blockDim.x;
    const Consts* __restrict__ C = A.C;
    const int amode = C->amode;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const uint4 e = A.qA[g];
        const int c = (int)e.x;
        const PairLoc L = locate_known(A, c, r, e.y, e.z, e.w);
        const DevRes& rs = A.res[A.cells[c].res];
        Rec* recs = reinterpret_cast<Rec*>(L.recs);
        Rec Pr, Qr;
        load_rec(recs + L.ip, Pr);
        load_rec(recs + L.iq, Qr);
        const int sP = (int)(Pr.meta & 0xFFu), sQ = (int)(Qr.meta & 0xFFu);
        const DevPair& pc = C->pair[sP * MAXS + sQ];
        if constexpr (!std::is_same<R, double>::value) {
            // FP32 mode: fixed-point energies, no FP64 arithmetic
            const long long Etr = etr_fix_f32(pc, g2_f32(Pr.v, Qr.v));
            const long long EvP = evib_fix(A.levfix, C->sp[sP], Pr.q);
            const long long EvQ = evib_fix(A.levfix, C->sp[sQ], Qr.q);
            if (C->n_reactions > 0) {
                Stream sp;
                st_init(sp, rs.seed, rs.step, L.lcell, L.rk, PU_PAIR);
                st_u32(sp);
                const float u_ster = st_u32(sp);
                const float u_sel = st_u32(sp);
                const float u_ch = st_u32(sp);
                uint32_t chan = 0u;
                if (reaction_pick_fix(A, C, sP, sQ, Pr.q, Qr.q, Etr, EvP, EvQ, u_ster, u_sel, u_ch, chan) > 0) {
                    const uint32_t slot = queue_slot(A.qsize + 2 * r + 1, true);
                    A.qB[slot] = make_uint4((uint32_t)c, e.y, chan, 0u);
                    continue;
                }
            }
            PairOut o{EV_ACC, 0u};
            relax_scatter_fix(A, C, rs, L, Pr, Qr, pc, Etr, EvP, EvQ, o);
            store_rec(recs + L.ip, Pr);
            store_rec(recs + L.iq, Qr);
            A.cflag[L.ev_idx] = ev_final(o);
            if (A.log_on) A.log[L.ev_idx] = hcao_log_rec{rs.step, L.lcell, L.rk, L.ip, L.iq, 0, 0u};
            continue;
        }
        double g2d, sg;
        pair_energy<R>(pc, amode, Pr.v, Qr.v, g2d, sg);
        const double Etr = 0.5 * pc.mr * g2d;
        const double EvP = evib64(A.lev64, C->sp[sP], Pr.q);
        const double EvQ = evib64(A.lev64, C->sp[sQ], Qr.q);
        if (C->n_reactions > 0) {
            uint32_t rchan = 0u, mpos = 0u;
            if (C->has_recomb && recomb_test<R>(A, C, c, r, e.y, sP, sQ, sg, rchan, mpos)) {
                const uint32_t slot = queue_slot(A.qsize + 2 * r + 1, true);
                A.qB[slot] = make_uint4((uint32_t)c, e.y, rchan, mpos);
                continue;
            }
            if (C->has_tce && tce_test<R>(A, C, rs, L.lcell, L.rk, sP, sQ, Etr, EvP, EvQ, rchan, rec_erot(Pr),
                                          rec_erot(Qr))) {
                const uint32_t slot = queue_slot(A.qsize + 2 * r + 1, true);
                A.qB[slot] = make_uint4((uint32_t)c, e.y, rchan, 0u);
                continue;
            }
            Stream sp;
            st_init(sp, rs.seed, rs.step, L.lcell, L.rk, PU_PAIR);
            st_u64(sp);
            const double u_ster = st_u64(sp);
            const double u_sel = st_u64(sp);
            const double u_ch = st_u64(sp);
            uint32_t chan = 0u;
            const int nch = reaction_pick<R>(A, C, sP, sQ, Pr.q, Qr.q, Etr, EvP, EvQ, u_ster, u_sel,
                                             u_ch, chan, rec_erot(Pr), rec_erot(Qr));
            if (nch > 0) {
                const uint32_t slot = queue_slot(A.qsize + 2 * r + 1, true);
                A.qB[slot] = make_uint4((uint32_t)c, e.y, chan, 0u);
                continue;
            }
        }
        PairOut o{EV_ACC, 0u};
        relax_scatter<R>(A, C, rs, L, Pr, Qr, pc, Etr, EvP, EvQ, o);
        store_rec(recs + L.ip, Pr);
        store_rec(recs + L.iq, Qr);
        A.cflag[L.ev_idx] = ev_final(o);
        if (A.log_on) A.log[L.ev_idx] = hcao_log_rec{rs.step, L.lcell, L.rk, L.ip, L.iq, 0, 0u};
    }
}

// FP32 phase 2: one thread per accepted pair (grid-stride over the queue in
// work-class order, heaviest class first).  The molecules with
// modes, P before Q, with the alias K5 draw (relative energy in int64 fixed
// point), then isotropic scattering with the centre-of-mass velocity kept.
// COUNT: the K5 work counters (profiled steps only: four more live registers
// under the 64-register bound cost the kernel ~4%).
template <class R, bool COUNT>
__global__ void __launch_bounds__(128, HCAO_RELAX_MINB) k_relax_fast(StepArgs A, int r) {
    static_assert(std::is_same<R, float>::value, "FP32 mode only");
    const Consts* __restrict__ C = A.C;
    // the queue in work classes (k_qorder); the pair word's top byte is the class
    const uint32_t total = A.qsize[2 * r];
    const uint32_t stride = gridDim.x * blockDim.x;
    uint32_t w[2] = {0u, 0u};
    uint32_t w_samp = 0, w_pair = 0;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const uint4 e = A.qA[g];
        const uint32_t kp = e.y & 0xFFFFFFu;
        const int cidx = (int)e.x;
        const DevCell& cell = A.cells[cidx];
        const DevRes& rs = A.res[cell.res];
        const uint32_t step = rs.step, lcell = cell.lcell;
        const uint32_t rk = ((uint32_t)r << 24) | kp;
        const uint32_t ev_idx = A.abase[cidx] + (uint32_t)r * round_pairs(cell.n, A.has_recomb) + kp;
        const uint32_t ip = e.z, iq = e.w;
        uint4* recs = reinterpret_cast<uint4*>(cell.rec);
        const uint4 a = REC_LD(recs + 2 * ip), b = REC_LD(recs + 2 * iq);
        const uint4 qa = REC_LD(recs + 2 * ip + 1), qb = REC_LD(recs + 2 * iq + 1);
        const int sP = (int)(a.w & 0xFFu), sQ = (int)(b.w & 0xFFu);
        const DevPair& pc = C->pair[sP * MAXS + sQ];
        // what the pair keeps across its draws is held small (the sampler's
        // own state needs the registers): the centre-of-mass velocity instead
        // of both velocities, and the species as the records' meta words.
        // (Storing a relaxed molecule's levels as soon as they are drawn, to
        // drop the pair's level words too, measured slower.)
        float V[3];
        float g2;
        {
            const float va[3] = {__uint_as_float(a.x), __uint_as_float(a.y), __uint_as_float(a.z)};
            const float vb[3] = {__uint_as_float(b.x), __uint_as_float(b.y), __uint_as_float(b.z)};
            g2 = g2_f32(va, vb);
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3) V[c3] = cm_velocity_f32(pc, va[c3], vb[c3]);
        }
        const long long Etr = etr_fix_f32(pc, g2);
        long long EvP, EvQ;
        float erP, erQ;
        uint32_t qP[4] = {qa.x, qa.y, qa.z, qa.w}, qQ[4] = {qb.x, qb.y, qb.z, qb.w};
        {
            EvP = evib_fix(A.levfix, C->sp[sP], qP);
            EvQ = evib_fix(A.levfix, C->sp[sQ], qQ);
            erP = C->sp[sP].rot_dof ? __uint_as_float(qa.w) : 0.f;
            erQ = C->sp[sQ].rot_dof ? __uint_as_float(qb.w) : 0.f;
            // reaction tests (recombination, then the QK channels in fixed
            // point); a reacting pair goes to the reaction queue instead
            bool react = false;
            uint32_t chan = 0u, mpos = 0u;
            if (C->n_reactions > 0) {
                if (C->has_recomb &&
                    recomb_test<float>(A, C, cidx, r, kp, sP, sQ, (double)sg_f32(pc, C->amode, g2), chan, mpos)) {
                    react = true;
                } else if (C->has_tce && tce_test<float>(A, C, rs, lcell, rk, sP, sQ, fix2d(Etr), fix2d(EvP),
                                                         fix2d(EvQ), chan, (double)erP, (double)erQ)) {
                    react = true;
                } else if (pc.qk) {  // a pair no QK reaction can take draws nothing from this stream
                    Stream sp;
                    st_init(sp, rs.seed, step, lcell, rk, PU_PAIR);
                    st_u32(sp);  // the acceptance draw
                    const float u_ster = st_u32(sp);
                    const float u_sel = st_u32(sp);
                    const float u_ch = st_u32(sp);
                    react = reaction_pick_fix(A, C, sP, sQ, qP, qQ, Etr, EvP, EvQ, u_ster, u_sel, u_ch, chan, erP,
                                              erQ) > 0;
                }
            }
            const uint32_t rslot = queue_slot(A.qsize + 2 * r + 1, react);
            if (react) {
                A.qB[rslot] = make_uint4((uint32_t)cidx, kp, chan, mpos);
                continue;
            }
        }
        // the molecules with modes, P before Q, in one loop: a lane relaxing
        // its pair's first molecule and a lane relaxing its second (an H-CH3
        // next to a CH3-H pair) run the same code at the same time
        PairOut o{EV_ACC, 0u};
        long long Erel = Etr;
        const bool relP = C->sp[sP].n_modes > 0;
        const int nmol = (int)relP + (int)(C->sp[sQ].n_modes > 0);
        for (int m = 0; m < nmol; ++m) {
            const bool isQ = !relP || m == 1;
            LbStream st;
            st_init(st, rs.seed, step, lcell, rk, isQ ? PU_LB_B : PU_LB_A);
            uint32_t nq[4];
            bool took;
            uint32_t wl_ = 0, wm_ = 0;  // unread (and dropped) without COUNT
            Erel = relax_one(A, C, isQ ? sQ : sP, nq, isQ ? EvQ : EvP, st, Erel, o, COUNT ? w[0] : wl_,
                             COUNT ? w[1] : wm_, took);
            if (took) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    qP[i] = isQ ? qP[i] : nq[i];
                    qQ[i] = isQ ? nq[i] : qQ[i];
                }
            }
        }
        if (COUNT) {
            w_samp += (uint32_t)nmol;
            w_pair++;
        }
        if (C->has_rot) Erel = rot_relax_fix(A, C, rs.seed, step, lcell, rk, sP, sQ, erP, erQ, qP, qQ, Erel);
        Stream ss;
        st_init(ss, rs.seed, step, lcell, rk, PU_SCAT);
        float d[3];
        iso_dir<float>(ss, d);
        float na[3], nb[3];
        scatter_cm_f32(pc, Erel, d, V, na, nb);
        // the meta word is the species (the selection admits no removed member)
        REC_ST(recs + 2 * ip, make_uint4(__float_as_uint(na[0]), __float_as_uint(na[1]), __float_as_uint(na[2]),
                                         (uint32_t)sP));
        REC_ST(recs + 2 * iq, make_uint4(__float_as_uint(nb[0]), __float_as_uint(nb[1]), __float_as_uint(nb[2]),
                                         (uint32_t)sQ));
        REC_ST(recs + 2 * ip + 1, make_uint4(qP[0], qP[1], qP[2], qP[3]));
        REC_ST(recs + 2 * iq + 1, make_uint4(qQ[0], qQ[1], qQ[2], qQ[3]));
        A.cflag[ev_idx] = ev_final(o);
        if (A.log_on) A.log[ev_idx] = hcao_log_rec{step, lcell, rk, ip, iq, 0, 0u};
    }
    // work counters: reduced over the CTA, one atomic per CTA and counter
    // (none for a CTA without work: an empty round's launch stays cheap)
    if (!COUNT) return;
    __shared__ unsigned long long wred[4][4];
    unsigned long long wv[4] = {w[0], w[1], w_samp, w_pair};
#pragma unroll
    for (int i = 0; i < 4; ++i)
        for (int o2 = 16; o2 > 0; o2 >>= 1) wv[i] += __shfl_xor_sync(0xFFFFFFFFu, wv[i], o2);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) wred[threadIdx.x >> 5][i] = wv[i];
    }
    __syncthreads();
    if (threadIdx.x < 4 && A.work) {
        const unsigned long long t = wred[0][threadIdx.x] + wred[1][threadIdx.x] + wred[2][threadIdx.x] +
                                     wred[3][threadIdx.x];
        if (t) atomicAdd(A.work + threadIdx.x, t);
    }
}

// Phase 3: pairs whose reaction test picked a channel: dissociation or
// exchange; a reaction whose products cannot be formed falls back to
// relaxation.
// FP32: at least 3 CTAs an SM (168 registers, small spills) so that a step's
// reacting pairs run in one wave rather than two (2 CTAs at 178 registers):
// the exchange step 1% faster
template <class R>
__global__ void __launch_bounds__(128, (std::is_same<R, float>::value ? 3 : 1)) k_react(StepArgs A, int r) {
    using Rec = typename RecOf<R>::T;
    const uint32_t total = A.qsize[2 * r + 1];
    const uint32_t stride = gridDim.x * blockDim.x;
    const Consts* __restrict__ C = A.C;
    const int amode = C->amode;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const uint4 e = A.qB[g];
        const int c = (int)e.x;
        const PairLoc L = locate(A, c, r, e.y);
        const DevRes& rs = A.res[A.cells[c].res];
        Rec* recs = reinterpret_cast<Rec*>(L.recs);
        Rec Pr, Qr;
        load_rec(recs + L.ip, Pr);
        load_rec(recs + L.iq, Qr);
        const int sP = (int)(Pr.meta & 0xFFu), sQ = (int)(Qr.meta & 0xFFu);
        const DevPair& pc = C->pair[sP * MAXS + sQ];
        const int rxi = (int)(e.z & 7u), side = (int)((e.z >> 3) & 1u), mode = (int)(e.z >> 4);
        if constexpr (!std::is_same<R, double>::value) {
            const long long Etr = etr_fix_f32(pc, g2_f32(Pr.v, Qr.v));
            const long long EvP = evib_fix(A.levfix, C->sp[sP], Pr.q);
            const long long EvQ = evib_fix(A.levfix, C->sp[sQ], Qr.q);
            const DevReaction& rx = C->rx[rxi];
            PairOut o{EV_ACC, 0u};
            hcao_log_rec lr{rs.step, L.lcell, L.rk, L.ip, L.iq, 0, 0u};
            float vA[3], vB[3], vN[3];
            RecF& RA = side ? Qr : Pr;
            RecF& RB = side ? Pr : Qr;
            for (int i = 0; i < 3; ++i) { vA[i] = RA.v[i]; vB[i] = RB.v[i]; }
            const int spA = (int)(RA.meta & 0xFFu), spB = (int)(RB.meta & 0xFFu);
            const float erA = C->sp[spA].rot_dof ? erot_f(RA.q) : 0.f, erB = C->sp[spB].rot_dof ? erot_f(RB.q) : 0.f;
            uint32_t q1[4], q2[4];
            bool done;
            if (rx.type == HCAO_RECOMB) {
                // RA is B, RB is C; the third body's position came with the queue entry
                const uint32_t iM = e.w;
                RecF Mr;
                load_rec(recs + iM, Mr);
                float vM[3] = {Mr.v[0], Mr.v[1], Mr.v[2]};
                done = do_recomb_fix(A, C, rx, vA, vB, vM, spA, spB, (int)(Mr.meta & 0xFFu),
                                     side ? EvQ : EvP, side ? EvP : EvQ, rs, L.lcell, L.rk, q1, o, erA, erB);
                lr.aux = (uint32_t)side + 2u * iM;
                if (done) {
                    for (int i = 0; i < 3; ++i) { RA.v[i] = vA[i]; Mr.v[i] = vM[i]; }
                    RA.meta = (uint32_t)rx.P0;
                    for (int j = 0; j < 4; ++j) RA.q[j] = q1[j];
                    RB.meta = SPECIES_NONE;
                    store_rec(recs + iM, Mr);
                    reinterpret_cast<uint32_t*>(reinterpret_cast<RecF*>(A.cscratch) + L.ev_idx)[0] =
                        side ? L.ip : L.iq;
                    o.ev |= EV_REMOVED;
                }
            } else if (rx.type == HCAO_DISS) {
                done = do_diss_fix(A, C, rx, vA, vB, spA, spB, side ? EvQ : EvP, rs, L.lcell, L.rk, q1, q2,
                                   vN, o, erA);
                lr.aux = (uint32_t)mode + (side ? 16u : 0u);
                if (done) {
                    for (int i = 0; i < 3; ++i) { RA.v[i] = vA[i]; RB.v[i] = vB[i]; }
                    RA.meta = (uint32_t)rx.P0;
                    for (int j = 0; j < 4; ++j) RA.q[j] = q1[j];
                    RecF RN;
                    for (int i = 0; i < 3; ++i) RN.v[i] = vN[i];
                    RN.meta = (uint32_t)rx.P1;
                    for (int j = 0; j < 4; ++j) RN.q[j] = q2[j];
                    store_rec(reinterpret_cast<RecF*>(A.cscratch) + L.ev_idx, RN);
                    o.ev |= EV_CREATED;
                }
            } else {
                done = do_exch_fix(A, C, rx, vA, vB, spA, spB, side ? EvQ : EvP, side ? EvP : EvQ, rs,
                                   L.lcell, L.rk, q1, q2, o, erA, erB);
                lr.aux = (uint32_t)side;
                if (done) {
                    for (int i = 0; i < 3; ++i) { RA.v[i] = vA[i]; RB.v[i] = vB[i]; }
                    RA.meta = (uint32_t)rx.P0;
                    RB.meta = (uint32_t)rx.P1;
                    for (int j = 0; j < 4; ++j) { RA.q[j] = q1[j]; RB.q[j] = q2[j]; }
                }
            }
            if (done) {
                o.ev |= (uint32_t)(rxi + 1) << EV_RX_SHIFT;
                lr.event = 1 + rxi;
            } else {
                o.ev |= EV_NOTEXEC;
                lr.aux = 0u;
                relax_scatter_fix(A, C, rs, L, Pr, Qr, pc, Etr, EvP, EvQ, o);
            }
            store_rec(recs + L.ip, Pr);
            store_rec(recs + L.iq, Qr);
            A.cflag[L.ev_idx] = ev_final(o);
            if (A.log_on) A.log[L.ev_idx] = lr;
            continue;
        }
        double g2d, sg;
        pair_energy<R>(pc, amode, Pr.v, Qr.v, g2d, sg);
        const double Etr = 0.5 * pc.mr * g2d;
        const double EvP = evib64(A.lev64, C->sp[sP], Pr.q);
        const double EvQ = evib64(A.lev64, C->sp[sQ], Qr.q);
        const DevReaction& rx = C->rx[rxi];
        PairOut o{EV_ACC, 0u};
        hcao_log_rec lr{rs.step, L.lcell, L.rk, L.ip, L.iq, 0, 0u};
        double vA[3], vB[3], vN[3];
        Rec& RA = side ? Qr : Pr;
        Rec& RB = side ? Pr : Qr;
        for (int i = 0; i < 3; ++i) { vA[i] = (double)RA.v[i]; vB[i] = (double)RB.v[i]; }
        const int spA = (int)(RA.meta & 0xFFu), spB = (int)(RB.meta & 0xFFu);
        const double erA = rec_erot(RA), erB = rec_erot(RB);
        uint32_t q1[4], q2[4];
        bool done;
        if (rx.type == HCAO_RECOMB) {
            // RA is B, RB is C; the third body's position came with the queue entry
            const uint32_t iM = e.w;
            Rec Mr;
            load_rec(recs + iM, Mr);
            double vM[3] = {(double)Mr.v[0], (double)Mr.v[1], (double)Mr.v[2]};
            done = do_recomb<R>(A, C, rx, vA, vB, vM, spA, spB, (int)(Mr.meta & 0xFFu), side ? EvQ : EvP,
                                side ? EvP : EvQ, rs, L.lcell, L.rk, q1, o, erA, erB);
            lr.aux = (uint32_t)side + 2u * iM;
            if (done) {
                for (int i = 0; i < 3; ++i) { RA.v[i] = (R)vA[i]; Mr.v[i] = (R)vM[i]; }
                RA.meta = (uint32_t)rx.P0;
                for (int j = 0; j < 4; ++j) RA.q[j] = q1[j];
                rec_set_erot(RA, 0.0);  // products start without rotation; M keeps its own
                RB.meta = SPECIES_NONE;
                rec_set_erot(RB, 0.0);
                store_rec(recs + iM, Mr);
                reinterpret_cast<uint32_t*>(reinterpret_cast<Rec*>(A.cscratch) + L.ev_idx)[0] =
                    side ? L.ip : L.iq;
                o.ev |= EV_REMOVED;
            }
        } else if (rx.type == HCAO_DISS) {
            done = do_diss<R>(A, C, rx, vA, vB, spA, spB, side ? EvQ : EvP, rs, L.lcell, L.rk, q1, q2,
                              vN, o, erA);
            lr.aux = (uint32_t)mode + (side ? 16u : 0u);
            if (done) {
                // A becomes B in place; M keeps its state; C goes to the pair's
                // scratch slot and is appended to the cell by k_finish
                for (int i = 0; i < 3; ++i) { RA.v[i] = (R)vA[i]; RB.v[i] = (R)vB[i]; }
                RA.meta = (uint32_t)rx.P0;
                for (int j = 0; j < 4; ++j) RA.q[j] = q1[j];
                rec_set_erot(RA, 0.0);
                Rec RN;
                for (int i = 0; i < 3; ++i) RN.v[i] = (R)vN[i];
                RN.meta = (uint32_t)rx.P1;
                for (int j = 0; j < 4; ++j) RN.q[j] = q2[j];
                if constexpr (std::is_same<R, double>::value) { RN.pad = 0; RN.erot = 0.0; }
                store_rec(reinterpret_cast<Rec*>(A.cscratch) + L.ev_idx, RN);
                o.ev |= EV_CREATED;
            }
        } else {
            done = do_exch<R>(A, C, rx, vA, vB, spA, spB, side ? EvQ : EvP, side ? EvP : EvQ, rs,
                              L.lcell, L.rk, q1, q2, o, erA, erB);
            lr.aux = (uint32_t)side;
            if (done) {
                for (int i = 0; i < 3; ++i) { RA.v[i] = (R)vA[i]; RB.v[i] = (R)vB[i]; }
                RA.meta = (uint32_t)rx.P0;
                RB.meta = (uint32_t)rx.P1;
                for (int j = 0; j < 4; ++j) { RA.q[j] = q1[j]; RB.q[j] = q2[j]; }
                rec_set_erot(RA, 0.0);
                rec_set_erot(RB, 0.0);
            }
        }
        if (done) {
            o.ev |= (uint32_t)(rxi + 1) << EV_RX_SHIFT;
            lr.event = 1 + rxi;
        } else {
            o.ev |= EV_NOTEXEC;
            lr.aux = 0u;
            relax_scatter<R>(A, C, rs, L, Pr, Qr, pc, Etr, EvP, EvQ, o);
        }
        store_rec(recs + L.ip, Pr);
        store_rec(recs + L.iq, Qr);
        A.cflag[L.ev_idx] = ev_final(o);
        if (A.log_on) A.log[L.ev_idx] = lr;
    }
}

// End of step, in three kernels so that a cell of any size is spread over
// many warps.  The pair slots of each cell are cut into FINISH_CHUNK-slot
// chunks (prefix chbase, built by k_setup); one warp takes one chunk, so a
// cell of 500 particles costs one warp and a cell of 4M about a thousand.
// k_finish_count: per chunk, the event words reduced into the cell's
// counters, and the number of particles the chunk's reactions created; the
// positions of particles removed by recombination gathered into the cell's
// list (rmpos at the cell's event slots, in no particular order).
template <class R>
__global__ void __launch_bounds__(256) k_finish_count(StepArgs A) {
    using Rec = typename RecOf<R>::T;
    const int lane = threadIdx.x & 31;
    const uint32_t nch = A.totals[MAX_ROUNDS + 1];
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long* cellcnt = reinterpret_cast<unsigned long long*>(A.counters);
    for (uint32_t ch = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < nch; ch += warps) {
        const int c = cell_of_warp(A.chbase, A.n_cells, ch);
        DevCell& cl = A.cells[c];
        const uint32_t j0 = (ch - A.chbase[c]) * (uint32_t)FINISH_CHUNK;
        const uint32_t j1 = min(j0 + (uint32_t)FINISH_CHUNK, cl.nsel);
        const uint32_t base = A.abase[c];
        uint32_t acc = 0, samp = 0, over = 0, degen = 0, notex = 0, removed = 0, created = 0, trials = 0;
        uint32_t rxc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        // four event words a lane in flight at once (the words are read-only
        // here); a slot past the chunk reads as 0, which counts nothing.  A
        // chunk's trials fit 32 bits (at most 1024 x 65535)
        for (uint32_t j = j0 + lane; j < j1; j += 128) {
            uint32_t evs[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t jj = j + 32u * (uint32_t)u;
                evs[u] = jj < j1 ? __ldg(A.cflag + base + jj) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t ev = evs[u];
                acc += ev & EV_ACC;
                samp += (ev >> EV_SAMP_SHIFT) & 3u;
                over += (ev >> EV_OVER_SHIFT) & 3u;
                degen += (ev >> EV_DEGEN_SHIFT) & 3u;
                notex += (ev & EV_NOTEXEC) ? 1u : 0u;
                if (ev & EV_REMOVED) {
                    removed++;
                    const uint32_t slot = atomicAdd(&cl.rmfill, 1u);
                    A.rmpos[base + slot] = reinterpret_cast<const uint32_t*>(
                        reinterpret_cast<const Rec*>(A.cscratch) + base + j + 32u * (uint32_t)u)[0];
                }
                created += (ev & EV_CREATED) ? 1u : 0u;
                trials += ev >> EV_TRIAL_SHIFT;
                const uint32_t rxid = (ev >> EV_RX_SHIFT) & 63u;
                if (rxid > 0 && rxid <= 8) rxc[rxid - 1]++;
            }
        }
        acc = __reduce_add_sync(0xFFFFFFFFu, acc);
        samp = __reduce_add_sync(0xFFFFFFFFu, samp);
        over = __reduce_add_sync(0xFFFFFFFFu, over);
        degen = __reduce_add_sync(0xFFFFFFFFu, degen);
        notex = __reduce_add_sync(0xFFFFFFFFu, notex);
        removed = __reduce_add_sync(0xFFFFFFFFu, removed);
        created = __reduce_add_sync(0xFFFFFFFFu, created);
        trials = __reduce_add_sync(0xFFFFFFFFu, trials);
#pragma unroll
        for (int i = 0; i < 8; ++i) rxc[i] = __reduce_add_sync(0xFFFFFFFFu, rxc[i]);
        unsigned long long* cc = cellcnt + (size_t)c * NCNT;
        // one lane per counter; a cell of one chunk needs no atomics, but its
        // counters may also receive other chunks' atomics, so all use them
        switch (lane) {
            case 0: if (acc) atomicAdd(cc + CNT_ACC, (unsigned long long)acc); break;
            case 1: if (samp) atomicAdd(cc + CNT_SAMPLES, (unsigned long long)samp); break;
            case 2: if (over) atomicAdd(cc + CNT_OVER, (unsigned long long)over); break;
            case 3: if (degen) atomicAdd(cc + CNT_DEGEN, (unsigned long long)degen); break;
            case 4: if (notex) atomicAdd(cc + CNT_NOTEXEC, (unsigned long long)notex); break;
            case 5: if (removed) atomicAdd(&cl.nremoved, removed); break;
            case 6:
                A.chcnt[ch] = created;
                if (created) atomicAdd(&cl.ncreated, created);
                break;
            case 7: if (trials) atomicAdd(cc + CNT_TRIALS, (unsigned long long)trials); break;
            default:
                if (lane < 16 && rxc[lane - 8] && lane - 8 < NCNT - CNT_RX0)
                    atomicAdd(cc + CNT_RX0 + (lane - 8), (unsigned long long)rxc[lane - 8]);
        }
    }
}

// k_finish_append: particles created by dissociation, appended after the
// cell's step-start particles in pair order: a warp scan per chunk on top of
// the created counts of the cell's earlier chunks.
template <class R>
__global__ void __launch_bounds__(256) k_finish_append(StepArgs A) {
    using Rec = typename RecOf<R>::T;
    const int lane = threadIdx.x & 31;
    const uint32_t nch = A.totals[MAX_ROUNDS + 1];
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t ch = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < nch; ch += warps) {
        if (A.chcnt[ch] == 0u) continue;  // uniform over the warp
        const int c = cell_of_warp(A.chbase, A.n_cells, ch);
        const DevCell& cl = A.cells[c];
        const uint32_t j0 = (ch - A.chbase[c]) * (uint32_t)FINISH_CHUNK;
        const uint32_t j1 = min(j0 + (uint32_t)FINISH_CHUNK, cl.nsel);
        const uint32_t base = A.abase[c];
        uint32_t run = 0;  // created in the cell's earlier chunks
        for (uint32_t q = A.chbase[c] + lane; q < ch; q += 32) run += A.chcnt[q];
        for (int o = 16; o > 0; o >>= 1) run += __shfl_xor_sync(0xFFFFFFFFu, run, o);
        const uint32_t N = cl.n;
        Rec* recs = reinterpret_cast<Rec*>(cl.rec);
        for (uint32_t t0 = j0; t0 < j1; t0 += 32) {
            const uint32_t j = t0 + lane;
            const bool cr = j < j1 && (A.cflag[base + j] & EV_CREATED) != 0u;
            const unsigned m = __ballot_sync(0xFFFFFFFFu, cr);
            if (cr) {
                const uint32_t dst = N + run + (uint32_t)__popc(m & ((1u << lane) - 1u));
                if (dst < cl.cap) {
                    Rec t;
                    load_rec(reinterpret_cast<const Rec*>(A.cscratch) + base + j, t);
                    store_rec(recs + dst, t);
                } else {
                    atomicOr(A.err, (uint32_t)ERR_CAPACITY);
                }
            }
            run += (uint32_t)__popc(m);
        }
    }
}

// k_cellupd: per cell, candidate count, (sigma g)_max update and the new
// particle count; per reservoir, the step counter.
static __global__ void __launch_bounds__(256) k_cellupd(StepArgs A) {
    unsigned long long* cellcnt = reinterpret_cast<unsigned long long*>(A.counters);
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < A.n_res; i += blockDim.x)
            if (A.res[i].active) A.res[i].step++;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < A.n_cells; c += gridDim.x * blockDim.x) {
        DevCell& cl = A.cells[c];
        cellcnt[(size_t)c * NCNT + CNT_CAND] += cl.nsel;
        const double seen = __longlong_as_double((long long)cl.seen);
        if (seen > cl.sgmax) cl.sgmax = seen;
        const uint32_t n = cl.n + cl.ncreated;
        cl.n = n < cl.cap ? n : cl.cap;
    }
}

// Recombination, before the rounds: per-cell integer sums of the kinetic
// energy (2^-96 J), momentum (2^-104 kg m/s) and mass (2^-120 kg) of the
// particles present at the step start, for the cell temperature.  Flat over
// particles in chunks; a chunk inside one cell reduces over the CTA, lanes of
// one cell otherwise combine per warp before the atomics.
template <class R>
__global__ void __launch_bounds__(256) k_cellstats(StepArgs A) {
    using Rec = typename RecOf<R>::T;
    constexpr uint32_t CH = 4096;
    __shared__ long long red[8][5];
    const uint32_t total = A.nbase[A.n_cells];
    const Consts* __restrict__ C = A.C;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t b0 = blockIdx.x * CH; b0 < total; b0 += gridDim.x * CH) {
        const uint32_t end = min(b0 + CH, total);
        const int c_lo = cell_of(A.nbase, A.n_cells, b0);
        const int c_hi = cell_of(A.nbase, A.n_cells, end - 1);
        long long acc[5] = {0ll, 0ll, 0ll, 0ll, 0ll};
        for (uint32_t j0 = b0; j0 < end; j0 += blockDim.x) {
            const uint32_t j = j0 + threadIdx.x;
            const bool valid = j < end;
            int c = c_lo;
            long long v5[5] = {0ll, 0ll, 0ll, 0ll, 0ll};
            if (valid) {
                if (c_lo != c_hi) c = cell_of(A.nbase, A.n_cells, j);
                const Rec* recs = reinterpret_cast<const Rec*>(A.cells[c].rec);
                Rec rr;
                load_rec(recs + (j - __ldg(A.nbase + c)), rr);
                const DevSpecies& S = C->sp[min(rr.meta & 0xFFu, (uint32_t)(MAXS - 1))];
                if constexpr (std::is_same<R, double>::value) {
                    const double m = S.mass;
                    const double e = 0.5 * m * (rr.v[0] * rr.v[0] + rr.v[1] * rr.v[1] + rr.v[2] * rr.v[2]);
                    v5[0] = __double2ll_rn(e * 0x1p96);
                    v5[1] = __double2ll_rn((m * rr.v[0]) * 0x1p104);
                    v5[2] = __double2ll_rn((m * rr.v[1]) * 0x1p104);
                    v5[3] = __double2ll_rn((m * rr.v[2]) * 0x1p104);
                    v5[4] = __double2ll_rn(m * 0x1p120);
                } else {
                    const float m = S.mass_f;
                    const float e = 0.5f * m * (rr.v[0] * rr.v[0] + rr.v[1] * rr.v[1] + rr.v[2] * rr.v[2]);
                    v5[0] = __float2ll_rn(e * 0x1p96f);
                    v5[1] = __float2ll_rn((m * rr.v[0]) * 0x1p104f);
                    v5[2] = __float2ll_rn((m * rr.v[1]) * 0x1p104f);
                    v5[3] = __float2ll_rn((m * rr.v[2]) * 0x1p104f);
                    v5[4] = __float2ll_rn(m * 0x1p120f);
                }
            }
            if (c_lo == c_hi) {
#pragma unroll
                for (int q = 0; q < 5; ++q) acc[q] += v5[q];
                continue;
            }
            // several cells in the chunk: lanes of one cell combine, then one atomic each
            const unsigned act = __activemask();
            const int key = valid ? c : -1;
            unsigned left = __ballot_sync(act, valid);
            while (left) {
                const int leader = __ffs(left) - 1;
                const int cl = __shfl_sync(act, key, leader);
                const unsigned grp = __ballot_sync(act, key == cl);
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    long long x = key == cl ? v5[q] : 0ll;
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(act, x, o);
                    if (lane == leader)
                        atomicAdd(reinterpret_cast<unsigned long long*>(A.csum + 5 * (size_t)cl + q),
                                  (unsigned long long)x);
                }
                left &= ~grp;
            }
        }
        if (c_lo == c_hi) {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                long long x = acc[q];
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
                if (lane == 0) red[wid][q] = x;
            }
            __syncthreads();
            if (threadIdx.x < 5) {
                long long x = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[w][threadIdx.x];
                atomicAdd(reinterpret_cast<unsigned long long*>(A.csum + 5 * (size_t)c_lo + threadIdx.x),
                          (unsigned long long)x);
            }
            __syncthreads();
        }
    }
}

// Recombination, after k_finish: remove the particles marked removed.  With
// d removed among a cell's n records, the surviving records at positions
// >= n - d move, in increasing position order, into the removed positions
// below n - d, taken in increasing order.  One CTA per cell with removals:
// the removed positions (gathered by k_finish_count, over all the cell's
// chunks) are sorted in shared memory.
template <class R>
__global__ void __launch_bounds__(256) k_compact(StepArgs A) {
    using Rec = typename RecOf<R>::T;
    __shared__ uint32_t pos[MAX_REMOVALS];
    for (int c = blockIdx.x; c < A.n_cells; c += gridDim.x) {
        DevCell& cl = A.cells[c];
        const uint32_t d = cl.nremoved;
        if (d == 0u) continue;
        __syncthreads();
        if (d > (uint32_t)MAX_REMOVALS) {
            if (threadIdx.x == 0) {
                atomicOr(A.err, (uint32_t)ERR_CAPACITY);
                cl.rmfill = 0u;
            }
            continue;
        }
        const uint32_t base = A.abase[c];
        for (uint32_t j = threadIdx.x; j < d; j += blockDim.x) pos[j] = A.rmpos[base + j];
        __syncthreads();
        uint32_t P = 1;
        while (P < d) P <<= 1;
        for (uint32_t i = d + threadIdx.x; i < P; i += blockDim.x) pos[i] = 0xFFFFFFFFu;
        __syncthreads();
        // bitonic sort of pos[0, P)
        for (uint32_t kk = 2; kk <= P; kk <<= 1)
            for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
                for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                    const uint32_t l = i ^ jj;
                    if (l > i) {
                        const uint32_t a = pos[i], b = pos[l];
                        const bool up = (i & kk) == 0;
                        if ((a > b) == up) { pos[i] = b; pos[l] = a; }
                    }
                }
                __syncthreads();
            }
        const uint32_t n = cl.n, t0 = n - d;
        // holes: removed positions below t0 (the first h0 sorted entries)
        uint32_t lo = 0, hi = d;
        while (lo < hi) { const uint32_t mid = (lo + hi) >> 1; if (pos[mid] < t0) lo = mid + 1; else hi = mid; }
        const uint32_t h0 = lo;
        Rec* recs = reinterpret_cast<Rec*>(cl.rec);
        for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
            const uint32_t t = t0 + i;
            uint32_t a = 0, b = d;  // removed positions < t
            while (a < b) { const uint32_t mid = (a + b) >> 1; if (pos[mid] < t) a = mid + 1; else b = mid; }
            if (a < d && pos[a] == t) continue;
            const uint32_t rank = i - (a - h0);
            if (rank < h0) {
                Rec tmp;
                load_rec(recs + t, tmp);
                store_rec(recs + pos[rank], tmp);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            cl.n = t0;
            cl.nremoved = 0u;
            cl.rmfill = 0u;
        }
    }
}

template <class R>
void launch_phase_impl(const StepArgs& a, int r, int phase, int grid, cudaStream_t s) {
    const int gs = a.grid_select > 0 ? a.grid_select : grid;
    const int gr = a.grid_relax > 0 ? a.grid_relax : grid;
    const int gx = a.grid_react > 0 ? a.grid_react : grid;
    if (phase == 0) {
        k_select<R><<<gs, SELECT_THREADS, 0, s>>>(a, r);
        if constexpr (std::is_same<R, float>::value)
            if (a.qorder) k_qorder<<<QORDER_GRID, 256, 0, s>>>(a, r);
    } else if (phase == 1) {
        if constexpr (std::is_same<R, float>::value) {
            if (a.work) k_relax_fast<R, true><<<gr, 128, 0, s>>>(a, r);
            else k_relax_fast<R, false><<<gr, 128, 0, s>>>(a, r);
        }
        else k_relax<R><<<gr, 128, 0, s>>>(a, r);
    } else if (a.has_reactions) k_react<R><<<gx, 128, 0, s>>>(a, r);
}
template <class R>
void launch_collide_impl(const StepArgs& a, int r, int grid, int block, cudaStream_t s) {
    (void)block;
    launch_phase_impl<R>(a, r, 0, grid, s);
    launch_phase_impl<R>(a, r, 1, grid, s);
    launch_phase_impl<R>(a, r, 2, grid, s);
}
template <class R>
void launch_finish_impl(const StepArgs& a, cudaStream_t s) {
    k_finish_count<R><<<1184, 256, 0, s>>>(a);
    if (a.creates) k_finish_append<R><<<592, 256, 0, s>>>(a);
    const int g = (a.n_cells + 255) / 256 < 148 ? (a.n_cells + 255) / 256 : 148;
    k_cellupd<<<g < 1 ? 1 : g, 256, 0, s>>>(a);
}
template <class R>
void launch_cellstats_impl(const StepArgs& a, cudaStream_t s) {
    if (a.has_recomb) k_cellstats<R><<<1184, 256, 0, s>>>(a);
}
template <class R>
void launch_compact_impl(const StepArgs& a, cudaStream_t s) {
    if (!a.has_recomb) return;
    const int g = a.n_cells < 1184 ? a.n_cells : 1184;
    k_compact<R><<<g < 1 ? 1 : g, 256, 0, s>>>(a);
}
template <class R>
void launch_step_impl(const StepArgs& a, int grid, int block, cudaStream_t s, uint64_t* launches) {
    const int ns = launch_setup(a, s);
    launch_cellstats_impl<R>(a, s);
    for (int r = 0; r < a.max_rounds; ++r) launch_collide_impl<R>(a, r, grid, block, s);
    launch_finish_impl<R>(a, s);
    launch_compact_impl<R>(a, s);
    if (launches)
        *launches += ns + 2 + a.max_rounds * ((a.has_reactions ? 3 : 2) + (std::is_same<R, float>::value && a.qorder ? 1 : 0)) +
                     (a.has_recomb ? 2 : 0) + (a.creates ? 1 : 0);
}

// ------------------------------------------------------------- sampler diagnostics
// n independent post-collision states of species sp at collision energy Ec,
// sample i on the Philox stream (seed; i, i >> 32, 0; purpose 8).  FP64: the
// sequential K5 sampler of the collision kernels; FP32: the flattened one.
template <class R>
__global__ void k_sample_diag(StepArgs A, int sp, double Ec, uint64_t seed, int64_t n, uint8_t* out,
                              unsigned long long* trials, int* status) {
    const Consts* __restrict__ C = A.C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        Stream st;
        st_init(st, seed, (uint32_t)i, (uint32_t)(i >> 32), 0u, 8u);
        uint32_t q[4] = {0u, 0u, 0u, 0u};
        PairOut o{0u, 0u};
        int rc = S_OK;
        if constexpr (std::is_same<R, double>::value) {
            uint32_t tr = 0;
            rc = sample_lb<double>(A, C->sp[sp], C->amode, Ec, st, q, tr);
            o.trials = tr;
        } else {
            // the relative energy plus the ground state's energy is Ec
            const long long Ev0 = evib_fix(A.levfix, C->sp[sp], q);
            uint32_t qdummy[4] = {0u, 0u, 0u, 0u};
            relax_flat(A, C, sp, q, Ev0, st, -1, qdummy, 0, st, __double2ll_rn(Ec * 0x1p100) - Ev0, o);
            if ((o.ev >> EV_OVER_SHIFT) & 3u) rc = S_OVER;
            if ((o.ev >> EV_DEGEN_SHIFT) & 3u) rc = S_DEGEN;
        }
        uint32_t* d = reinterpret_cast<uint32_t*>(out + 16 * i);
        for (int w = 0; w < 4; ++w) d[w] = q[w];
        atomicAdd(trials, (unsigned long long)o.trials);
        if (rc != S_OK) atomicExch(status, rc);
    }
}

// ------------------------------------------------------------- load / read kernels
template <class R>
__global__ void k_scatter_load(typename RecOf<R>::T* recs, const uint32_t* perm,
                               const uint32_t* offsets, const uint64_t* slot0, int n_cells,
                               const double* v, const float* vf, const uint8_t* qn, const int32_t* sp,
                               int64_t n) {
    using Rec = typename RecOf<R>::T;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        // cell of sorted position j: largest c with offsets[c] <= j
        int lo = 0, hi = n_cells;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (offsets[mid] <= (uint32_t)j) lo = mid; else hi = mid;
        }
        const uint32_t i = perm[j];
        Rec r;
        for (int d = 0; d < 3; ++d) r.v[d] = vf ? (R)vf[3 * (int64_t)i + d] : (R)v[3 * (int64_t)i + d];
        r.meta = (uint32_t)sp[i];
        const uint32_t* q = reinterpret_cast<const uint32_t*>(qn + 16 * (int64_t)i);
        for (int w = 0; w < 4; ++w) r.q[w] = q[w];
        if constexpr (std::is_same<R, double>::value) { r.pad = 0; }
        store_rec(recs + slot0[lo] + (j - offsets[lo]), r);
    }
}

// Readout and initialisation kernels run flat over a reservoir's particles
// (off[c] = first particle of cell c in canonical order, off[n_cells] = total),
// so one very large cell spreads over the whole GPU.
__device__ __forceinline__ int cell_of64(const uint64_t* off, int n_cells, uint64_t j) {
    int lo = 0, hi = n_cells;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= j) lo = mid; else hi = mid;
    }
    return lo;
}
// the same for a whole warp with one j (all lanes active, j < off[n_cells]): a
// 32-way search, each round's lanes probing evenly spaced cells
__device__ __forceinline__ int cell_of64_warp(const uint64_t* off, int n_cells, uint64_t j) {
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = n_cells;  // off[lo] <= j < off[hi]
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int idx = lo + (lane + 1) * step;
        const bool le = idx < hi && off[idx] <= j;
        const int c = __popc(__ballot_sync(0xFFFFFFFFu, le));
        const int nlo = lo + c * step;
        hi = min(hi, nlo + step);
        lo = nlo;
    }
    return lo;
}

template <class R>
__global__ void k_pack(const DevCell* cells, int cell0, int n_cells, const uint64_t* off, const Consts* C,
                       double* v, uint8_t* qn, int32_t* sp, int32_t* cell) {
    using Rec = typename RecOf<R>::T;
    const uint64_t total = off[n_cells];
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < total;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const int c = cell_of64(off, n_cells, j);
        const Rec* recs = reinterpret_cast<const Rec*>(cells[cell0 + c].rec);
        Rec r;
        load_rec(recs + (j - off[c]), r);
        if (v) for (int d = 0; d < 3; ++d) v[3 * j + d] = (double)r.v[d];
        if (qn) {
            uint32_t* q = reinterpret_cast<uint32_t*>(qn + 16 * j);
            const int s = (int)(r.meta & 0xFFu);
            // an FP32 record's q[3] holds a rotating species' rotational energy
            const bool rot_word = std::is_same<R, float>::value && s < MAXS && C->sp[s].rot_dof;
            for (int w = 0; w < 4; ++w) q[w] = (w == 3 && rot_word) ? 0u : r.q[w];
        }
        if (sp) sp[j] = (int32_t)(r.meta & 0xFFu);
        if (cell) cell[j] = c;
    }
}

// P6/P7 initial quantum numbers (double draws in both precisions)
template <class R>
__global__ void k_init_vib(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,
                           const DevRes* res, int rslot, const Consts* C, const double* bend_thr,
                           const double* str_acc, const int* thr_off, uint32_t reject_cap,
                           uint32_t* err) {
    using Rec = typename RecOf<R>::T;
    const DevRes rs = res[rslot];
    const uint64_t total = off[n_cells];
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < total;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const int c = cell_of64(off, n_cells, j);
        const uint32_t i = (uint32_t)(j - off[c]);
        const DevCell& cl = cells[cell0 + c];
        Rec* recs = reinterpret_cast<Rec*>(cl.rec);
        Rec r;
        load_rec(recs + i, r);
        const int s = (int)(r.meta & 0xFFu);
        if (s >= MAXS) continue;  // a removed particle left by a failed compaction (error reported)
        const DevSpecies& S = C->sp[s];
        Stream st;
        st_init(st, rs.seed, 0xFFFFFFFFu, cl.lcell, i, PU_INIT);
        uint32_t q[4] = {0u, 0u, 0u, 0u};
        for (int m = 0; m < S.n_modes; ++m) {
            const int L = S.n_lev[m];
            const int to = thr_off[s * MAXM + m];
            bool done = false;
            for (uint32_t t = 0; t < reject_cap && !done; ++t) {
                if (m >= S.n_stretch) {
                    // bend: i = floor(-ln(u) T / Theta) >= k  <=>  u <= exp(-k Theta / T)
                    const double u = st_u64(st);
                    int lv = 0;
                    while (lv < L && u <= bend_thr[to + lv]) lv++;
                    if (lv < L) { set_q(q, m, (uint32_t)lv); done = true; }
                } else {
                    const double u1 = st_u64(st);
                    const int lv = (int)floor(u1 * (double)L);
                    const double u2 = st_u64(st);
                    if (u2 < str_acc[to + lv]) { set_q(q, m, (uint32_t)lv); done = true; }
                }
            }
            if (!done) atomicOr(err, (uint32_t)ERR_REJECT);
        }
        for (int w = 0; w < 4; ++w) r.q[w] = q[w];
        store_rec(recs + i, r);
    }
}

// moments: acc[0..2] momentum, [3] E_tr, [4] E_form, [5 + s] E_vib of species s.
// Each thread sums its particles in registers (species by an unrolled
// compare, so no array is indexed at run time); warps then reduce by shuffles
// and one lane per warp adds into shared memory, once per kernel.  Atomics
// per particle into a few shared words serialised the block.  A warp finds
// the cell of its 32 consecutive particles once (warp search, then each lane
// steps forward).  FP32 mode sums each species' vibrational energy in the
// fixed point of its bookkeeping (exact integer sums per thread; B300's FP64
// rate made the per-species FP64 sums most of the kernel's time).
template <class R>
__global__ void __launch_bounds__(256) k_moments(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,
                                                 const Consts* C, const double* lev64, const long long* levfix,
                                                 double* acc, unsigned long long* cnt) {
    using Rec = typename RecOf<R>::T;
    __shared__ double sacc[5 + 2 * MAXS];
    __shared__ unsigned long long scnt[MAXS];
    for (int i = threadIdx.x; i < 5 + 2 * MAXS; i += blockDim.x) sacc[i] = 0.0;
    for (int i = threadIdx.x; i < MAXS; i += blockDim.x) scnt[i] = 0ull;
    __syncthreads();
    constexpr bool f32 = std::is_same<R, float>::value;
    double px = 0.0, py = 0.0, pz = 0.0, etr = 0.0, ef = 0.0;
    // FP32 mode: momentum (2^-110 kg m/s) and translational energy (2^-100
    // J) in int64 fixed point from float products, exact integer sums (no
    // FP64 work per particle); the mass as the float pair mass_f + mass_lo_f,
    // so that only the float rounding of each particle's v and v^2 products
    // remains (unbiased), not that of the mass; E_form from the species counts
    long long pxx = 0, pyx = 0, pzx = 0, etx = 0;
    double ev[MAXS], er[MAXS];
    long long evx[MAXS];
    uint32_t nc[MAXS];
#pragma unroll
    for (int k = 0; k < MAXS; ++k) { ev[k] = 0.0; er[k] = 0.0; evx[k] = 0ll; nc[k] = 0u; }
    const bool rot = C->has_rot != 0;
    const int lane = threadIdx.x & 31;
    const uint64_t total = off[n_cells];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j0 = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); j0 < total; j0 += stride) {
        int c = cell_of64_warp(off, n_cells, j0);  // j0 is the same for the warp's lanes
        const uint64_t j = j0 + (uint64_t)lane;
        if (j >= total) continue;
        while (off[c + 1] <= j) ++c;
        const Rec* recs = reinterpret_cast<const Rec*>(cells[cell0 + c].rec);
        Rec r;
        load_rec(recs + (j - off[c]), r);
        const int s = (int)(r.meta & 0xFFu);
        if (s >= MAXS) continue;  // a removed particle left by a failed compaction (error reported)
        const DevSpecies& S = C->sp[s];
        if constexpr (f32) {
            const float mf = S.mass_f, ml = S.mass_lo_f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const long long p = __float2ll_rn(__fmul_rn(__fmul_rn(mf, r.v[d]), 0x1p110f)) +
                                    __float2ll_rn(__fmul_rn(__fmul_rn(ml, r.v[d]), 0x1p110f));
                if (d == 0) pxx += p; else if (d == 1) pyx += p; else pzx += p;
            }
            const float v2 = __fadd_rn(__fadd_rn(__fmul_rn(r.v[0], r.v[0]), __fmul_rn(r.v[1], r.v[1])),
                                       __fmul_rn(r.v[2], r.v[2]));
            etx += f2fix(__fmul_rn(__fmul_rn(0.5f, mf), v2)) + f2fix(__fmul_rn(__fmul_rn(0.5f, ml), v2));
        } else {
            const double m = S.mass;
            const double vx = r.v[0], vy = r.v[1], vz = r.v[2];
            px += m * vx;
            py += m * vy;
            pz += m * vz;
            etr += 0.5 * m * (vx * vx + vy * vy + vz * vz);
            ef += S.E_form;
        }
        if constexpr (f32) {
            const long long e = evib_fix(levfix, S, r.q);
#pragma unroll
            for (int k = 0; k < MAXS; ++k)
                if (s == k) { evx[k] += e; nc[k]++; }
        } else {
            const double e = evib64(lev64, S, r.q);
#pragma unroll
            for (int k = 0; k < MAXS; ++k)
                if (s == k) { ev[k] += e; nc[k]++; }
        }
        if (rot) {
            const double erot = rec_erot_of(r, S);
#pragma unroll
            for (int k = 0; k < MAXS; ++k)
                if (s == k) er[k] += erot;
        }
    }
    if constexpr (f32) {
        // a thread's sums stay below 2^53 units up to ~1e9 particles a
        // launch, where the conversions are exact
#pragma unroll
        for (int k = 0; k < MAXS; ++k) {
            ev[k] = (double)evx[k] * 0x1p-100;
            if (nc[k]) ef += (double)nc[k] * C->sp[k].E_form;
        }
        px = (double)pxx * 0x1p-110;
        py = (double)pyx * 0x1p-110;
        pz = (double)pzx * 0x1p-110;
        etr = (double)etx * 0x1p-100;
    }
    auto wsum = [](double x) {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        return x;
    };
    px = wsum(px); py = wsum(py); pz = wsum(pz); etr = wsum(etr); ef = wsum(ef);
    if (lane == 0) {
        atomicAdd(&sacc[0], px); atomicAdd(&sacc[1], py); atomicAdd(&sacc[2], pz);
        atomicAdd(&sacc[3], etr); atomicAdd(&sacc[4], ef);
    }
#pragma unroll
    for (int k = 0; k < MAXS; ++k) {
        const unsigned any = __ballot_sync(0xFFFFFFFFu, nc[k] != 0u);
        if (any == 0u) continue;  // uniform over the warp
        const double x = wsum(ev[k]);
        const double y = wsum(er[k]);
        const uint32_t n = __reduce_add_sync(0xFFFFFFFFu, nc[k]);
        if (lane == 0) {
            atomicAdd(&sacc[5 + k], x);
            if (y != 0.0) atomicAdd(&sacc[5 + MAXS + k], y);
            atomicAdd(&scnt[k], (unsigned long long)n);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 5 + 2 * MAXS; i += blockDim.x) atomicAdd(&acc[i], sacc[i]);
    for (int i = threadIdx.x; i < MAXS; i += blockDim.x) atomicAdd(&cnt[i], scnt[i]);
}

// rotational energies out of the records (to_records = 0) or into them (1),
// in canonical order
template <class R>
__global__ void k_erot(const DevCell* cells, int cell0, int n_cells, const uint64_t* off, const Consts* C,
                       double* e, int to_records) {
    using Rec = typename RecOf<R>::T;
    const uint64_t total = off[n_cells];
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < total;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const int c = cell_of64(off, n_cells, j);
        Rec* recs = reinterpret_cast<Rec*>(cells[cell0 + c].rec);
        Rec r;
        load_rec(recs + (j - off[c]), r);
        const int s = (int)(r.meta & 0xFFu);
        if (s >= MAXS) continue;
        if (to_records) {
            rec_put_erot(r, C->sp[s], e[j]);
            store_rec(recs + (j - off[c]), r);
        } else {
            e[j] = rec_erot_of(r, C->sp[s]);
        }
    }
}

// Initial rotational energies at T_rot: kT Gamma(rot_dof/2), -ln(u) plus,
// for three degrees of freedom, Marsaglia's polar normal squared over two;
// keyed by (seed, 0xFFFFFFFE, cell, particle) as the oracle's
template <class R>
__global__ void k_init_rot(const DevCell* cells, int cell0, int n_cells, const uint64_t* off, const DevRes* res,
                           int rslot, const Consts* C, double kT) {
    using Rec = typename RecOf<R>::T;
    const DevRes rs = res[rslot];
    const uint64_t total = off[n_cells];
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < total;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const int c = cell_of64(off, n_cells, j);
        const uint32_t i = (uint32_t)(j - off[c]);
        const DevCell& cl = cells[cell0 + c];
        Rec* recs = reinterpret_cast<Rec*>(cl.rec);
        Rec r;
        load_rec(recs + i, r);
        const int s = (int)(r.meta & 0xFFu);
        if (s >= MAXS) continue;
        const DevSpecies& S = C->sp[s];
        double E = 0.0;
        if (S.rot_dof > 0 && kT > 0.0) {
            Stream st;
            st_init(st, rs.seed, 0xFFFFFFFEu, cl.lcell, i, PU_ROTINIT);
            E = -ln_series(__dsub_rn(1.0, st_u64(st)));
            if (S.rot_dof == 3) {
                for (int it = 0; it < 4096; ++it) {
                    const double x1 = __dsub_rn(__dmul_rn(2.0, st_u64(st)), 1.0);
                    const double x2 = __dsub_rn(__dmul_rn(2.0, st_u64(st)), 1.0);
                    const double q = __dadd_rn(__dmul_rn(x1, x1), __dmul_rn(x2, x2));
                    if (q > 0.0 && q < 1.0) {
                        E = __dadd_rn(E, __dmul_rn(__dmul_rn(x1, x1), __ddiv_rn(-ln_series(q), q)));
                        break;
                    }
                }
            }
            E = __dmul_rn(E, kT);
        }
        rec_put_erot(r, S, E);
        store_rec(recs + i, r);
    }
}

template <class R>
__global__ void k_levelpop(const DevCell* cells, int cell0, int n_cells, const uint64_t* off, int sp,
                           int mode, unsigned long long* hist) {
    using Rec = typename RecOf<R>::T;
    __shared__ unsigned int sh[MAXL];
    for (int i = threadIdx.x; i < MAXL; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const uint64_t total = off[n_cells];
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < total;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const int c = cell_of64(off, n_cells, j);
        const Rec* recs = reinterpret_cast<const Rec*>(cells[cell0 + c].rec);
        Rec r;
        load_rec(recs + (j - off[c]), r);
        if ((int)(r.meta & 0xFFu) == sp) atomicAdd(&sh[get_q(r.q, mode)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < MAXL; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

// ------------------------------------------------------------- launchers
#define HCAO_INSTANTIATE(R)                                                                      \
    template <>                                                                                  \
    void launch_step<R>(const StepArgs& a, int grid, int block, cudaStream_t s,                  \
                        uint64_t* launches) {                                                    \
        launch_step_impl<R>(a, grid, block, s, launches);                                        \
    }                                                                                            \
    template <>                                                                                  \
    void launch_collide<R>(const StepArgs& a, int r, int grid, int block, cudaStream_t s) {      \
        launch_collide_impl<R>(a, r, grid, block, s);                                            \
    }                                                                                            \
    template <>                                                                                  \
    void launch_finish<R>(const StepArgs& a, cudaStream_t s) { launch_finish_impl<R>(a, s); }    \
    template <>                                                                                  \
    void launch_cellstats<R>(const StepArgs& a, cudaStream_t s) { launch_cellstats_impl<R>(a, s); } \
    template <>                                                                                  \
    void launch_compact<R>(const StepArgs& a, cudaStream_t s) { launch_compact_impl<R>(a, s); }  \
    template <>                                                                                  \
    void launch_phase<R>(const StepArgs& a, int r, int phase, int grid, cudaStream_t s) {        \
        launch_phase_impl<R>(a, r, phase, grid, s);                                              \
    }                                                                                            \
    template <>                                                                                  \
    void launch_scatter_load<R>(void* rec_base, const uint32_t* perm, const uint32_t* offsets,   \
                                const uint64_t* slot0, int n_cells, const double* v,             \
                                const float* vf, const uint8_t* qn, const int32_t* sp, int64_t n, \
                                cudaStream_t s) {                                                \
        if (n <= 0) return;                                                                      \
        int grid = (int)((n + 255) / 256);                                                       \
        if (grid > 4096) grid = 4096;                                                            \
        k_scatter_load<R><<<grid, 256, 0, s>>>(reinterpret_cast<typename RecOf<R>::T*>(rec_base), \
                                               perm, offsets, slot0, n_cells, v, vf, qn, sp, n); \
    }                                                                                            \
    template <>                                                                                  \
    void launch_pack<R>(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,       \
                        uint64_t total, const Consts* C, double* v, uint8_t* qn, int32_t* sp,    \
                        int32_t* cell, cudaStream_t s) {                                         \
        if (total == 0) return;                                                                  \
        const int grid = (int)(total / 256 + 1 < 4096 ? total / 256 + 1 : 4096);                \
        k_pack<R><<<grid, 256, 0, s>>>(cells, cell0, n_cells, off, C, v, qn, sp, cell);          \
    }                                                                                            \
    template <>                                                                                  \
    void launch_erot<R>(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,       \
                        uint64_t total, const Consts* C, double* e, int to_records,              \
                        cudaStream_t s) {                                                        \
        if (total == 0) return;                                                                  \
        const int grid = (int)(total / 256 + 1 < 4096 ? total / 256 + 1 : 4096);                \
        k_erot<R><<<grid, 256, 0, s>>>(cells, cell0, n_cells, off, C, e, to_records);            \
    }                                                                                            \
    template <>                                                                                  \
    void launch_init_rot<R>(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,   \
                            uint64_t total, const DevRes* res, int rslot, const Consts* C,       \
                            double T_rot, cudaStream_t s) {                                      \
        if (total == 0) return;                                                                  \
        const int grid = (int)(total / 256 + 1 < 4096 ? total / 256 + 1 : 4096);                \
        k_init_rot<R><<<grid, 256, 0, s>>>(cells, cell0, n_cells, off, res, rslot, C,            \
                                           1.380649e-23 * T_rot);                                \
    }                                                                                            \
    template <>                                                                                  \
    void launch_init_vib<R>(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,   \
                            uint64_t total, const DevRes* res, int rslot, const Consts* C,       \
                            const double* bt, const double* sa, const int* to, uint32_t cap,     \
                            uint32_t* err, cudaStream_t s) {                                     \
        if (total == 0) return;                                                                  \
        const int grid = (int)(total / 256 + 1 < 4096 ? total / 256 + 1 : 4096);                \
        k_init_vib<R><<<grid, 256, 0, s>>>(cells, cell0, n_cells, off, res, rslot, C, bt, sa, to, \
                                           cap, err);                                            \
    }                                                                                            \
    template <>                                                                                  \
    void launch_moments<R>(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,    \
                           uint64_t total, const Consts* C, const double* lev64,                 \
                           const long long* levfix, double* acc, unsigned long long* cnt,        \
                           cudaStream_t s) {                                                     \
        if (total == 0) return;                                                                  \
        const int grid = (int)(total / 256 + 1 < 1184 ? total / 256 + 1 : 1184);                \
        k_moments<R><<<grid, 256, 0, s>>>(cells, cell0, n_cells, off, C, lev64, levfix, acc, cnt); \
    }                                                                                            \
    template <>                                                                                  \
    void launch_sample_diag<R>(const StepArgs& a, int sp, double Ec, uint64_t seed, int64_t n,   \
                               uint8_t* out, unsigned long long* trials, int* status,            \
                               cudaStream_t s) {                                                 \
        int grid = (int)((n + 127) / 128);                                                       \
        if (grid > 4096) grid = 4096;                                                            \
        if (grid < 1) return;                                                                    \
        k_sample_diag<R><<<grid, 128, 0, s>>>(a, sp, Ec, seed, n, out, trials, status);         \
    }                                                                                            \
    template <>                                                                                  \
    void launch_levelpop<R>(const DevCell* cells, int cell0, int n_cells, const uint64_t* off,   \
                            uint64_t total, int sp, int mode, unsigned long long* hist,          \
                            cudaStream_t s) {                                                    \
        if (total == 0) return;                                                                  \
        const int grid = (int)(total / 256 + 1 < 1184 ? total / 256 + 1 : 1184);                \
        k_levelpop<R><<<grid, 256, 0, s>>>(cells, cell0, n_cells, off, sp, mode, hist);          \
    }

}  // namespace hcao
