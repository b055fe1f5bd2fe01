// hcao_fused.cuh -- the FP32 collision phase of a step as one kernel: one
// CTA per cell (persistent over the cells), the cell's records staged in
// shared memory.
//
// The per-round queue kernels (k_setup_cells ... k_cellupd) run a step as
// about eleven launches that hand candidate and accepted pairs to each other
// through queues in global memory, and gather each pair's records from HBM
// twice.  For the common case -- cells that fit in shared memory and no
// reaction that creates or removes particles (relaxation, exchange) -- this
// kernel does the whole step of a cell in one CTA:
//   1. the NTC set-up (N_sel, rounds, permutation keys: ntc_setup, shared with
//      k_setup_cells);
//   2. the cell's records (32 B each) copied into shared memory with
//      coalesced 128-bit loads;
//   3. per round and per batch of candidate pairs: the permuted pair draw and
//      the VHS acceptance from shared memory; accepted pairs queued in shared
//      memory in three regions by the number of molecules to relax (coarser
//      than the queue path's work classes: a cell has only a few hundred
//      pairs a round, too few to fill warps class by class);
//   4. per accepted pair: the QK reaction test (Eq. Ecoll-diss, Eq.
//      Ecoll-exch, competing reactions), then the exchange or the HCAO LB
//      relaxation (the K5 alias draw) and isotropic scattering; the new
//      records go to shared memory (later rounds see them) and to HBM (only
//      the records of accepted pairs are written back);
//   5. the cell's counters, (sigma g)_max and candidate count; the last CTA
//      advances the reservoirs' step counters.
// Every random draw is keyed by (step, cell, round, pair) exactly as in the
// queue kernels, and every floating-point expression is the same function
// with explicit roundings, so the two paths give identical bits.
#pragma once
#include "hcao_kernels.cuh"

namespace hcao {

constexpr int FUSED_THREADS = 128;
constexpr int FUSED_BATCH = 512;   // candidate pairs selected before they are processed

// per-CTA counters of one cell, reduced in shared memory
enum { FC_ACC = 0, FC_SAMP, FC_OVER, FC_DEGEN, FC_NOTEX, FC_RX0, FC_N = FC_RX0 + MAXR };

static __global__ void __launch_bounds__(FUSED_THREADS, 4) k_collide_fused(StepArgs A, int smem_recs) {
    extern __shared__ uint4 s_rec[];                  // 2 per particle: (v, meta), q
    __shared__ uint2 s_q[2 * FUSED_BATCH];             // accepted pairs: (k, ip | iq << 16)
    __shared__ uint32_t s_n[3];                        // queue regions: two, one, no molecules
    __shared__ uint32_t s_key[MAX_ROUNDS][4];
    __shared__ uint32_t s_nsel, s_rounds, s_seen;
    __shared__ uint32_t s_cnt[FC_N];
    __shared__ unsigned long long s_trials;
    const Consts* __restrict__ C = A.C;
    const int amode = C->amode;
    const int tid = threadIdx.x;
    uint32_t w_lev = 0, w_mode = 0, w_samp = 0, w_pair = 0;

    for (int c = blockIdx.x; c < A.n_cells; c += gridDim.x) {
        DevCell& cl = A.cells[c];
        const DevRes& rs = A.res[cl.res];
        const uint32_t N = cl.n, step = rs.step, lcell = cl.lcell;
        const float sgmax_f = (float)cl.sgmax;
        const uint32_t P = round_pairs(N, 0);
        if (tid == 0) {
            uint32_t rounds = 0;
            s_nsel = ntc_setup(A, rs, cl, N, P, rounds, s_key);
            s_rounds = rounds;
            s_seen = 0u;
            s_trials = 0ull;
        }
        if (tid < FC_N) s_cnt[tid] = 0u;
        if (tid < 3) s_n[tid] = 0u;
        // the cell's records: in shared memory if they fit, else used in place
        uint4* grec = reinterpret_cast<uint4*>(cl.rec);
        if (N > 65535u) {  // pair entries hold 16-bit positions; the host never sends such a cell
            if (tid == 0) atomicOr(A.err, (uint32_t)ERR_CAPACITY);
            __syncthreads();
            continue;
        }
        const bool staged = N <= (uint32_t)smem_recs;
        if (staged)
            for (uint32_t i = tid; i < 2u * N; i += FUSED_THREADS) s_rec[i] = grec[i];
        uint4* R = staged ? s_rec : grec;
        __syncthreads();
        const uint32_t nsel = s_nsel, rounds = s_rounds;
        float seen = 0.f;
        unsigned long long trials = 0ull;
        for (uint32_t r = 0; r < rounds; ++r) {
            const uint32_t left = nsel - r * P, npairs = left < P ? left : P;
            const uint32_t key[4] = {s_key[r][0], s_key[r][1], s_key[r][2], s_key[r][3]};
            for (uint32_t kb = 0; kb < npairs; kb += FUSED_BATCH) {
                const uint32_t ke = min(npairs, kb + (uint32_t)FUSED_BATCH);
                // select: permuted members, VHS acceptance; accepted pairs to
                // the queue region of their number of molecules to relax
                for (uint32_t k = kb + tid; k < ke; k += FUSED_THREADS) {
                    const uint32_t ip = pair_perm(2u * k, N, key), iq = pair_perm(2u * k + 1u, N, key);
                    const uint4 a = R[2 * ip], b = R[2 * iq];
                    const int sP = (int)(a.w & 0xFFu), sQ = (int)(b.w & 0xFFu);
                    if (sP >= MAXS || sQ >= MAXS) continue;
                    const float va[3] = {__uint_as_float(a.x), __uint_as_float(a.y), __uint_as_float(a.z)};
                    const float vb[3] = {__uint_as_float(b.x), __uint_as_float(b.y), __uint_as_float(b.z)};
                    float sgf = sg_f32(C->pair[sP * MAXS + sQ], amode, g2_f32(va, vb));
                    if (!(sgf <= 3.0e38f)) {
                        atomicOr(A.err, (uint32_t)ERR_NONFINITE);
                        sgf = 0.f;
                    }
                    seen = fmaxf(seen, sgf);
                    Stream sp;
                    st_init(sp, rs.seed, step, lcell, (r << 24) | k, PU_PAIR);
                    if (!(st_u32(sp) < __fdiv_rn(sgf, sgmax_f))) continue;
                    const int nm = (int)(C->sp[sP].n_modes > 0) + (int)(C->sp[sQ].n_modes > 0);
                    const int q = 2 - nm;
                    const uint32_t i = atomicAdd(&s_n[q], 1u);
                    const uint2 ent = make_uint2(k, ip | (iq << 16));
                    s_q[q == 0 ? i : (q == 1 ? 2u * FUSED_BATCH - 1u - i : FUSED_BATCH + i)] = ent;
                }
                __syncthreads();
                const uint32_t n2 = s_n[0], n21 = n2 + s_n[1], total = n21 + s_n[2];
                // process: reaction test, exchange or relaxation, scattering
                for (uint32_t g = tid; g < total; g += FUSED_THREADS) {
                    const uint2 e = s_q[g < n2 ? g : (g < n21 ? 2u * FUSED_BATCH - 1u - (g - n2) : FUSED_BATCH + (g - n21))];
                    const uint32_t k = e.x, ip = e.y & 0xFFFFu, iq = e.y >> 16;
                    const uint32_t rk = (r << 24) | k;
                    RecF Pr, Qr;
                    load_rec(reinterpret_cast<const RecF*>(R) + ip, Pr);
                    load_rec(reinterpret_cast<const RecF*>(R) + iq, Qr);
                    const int sP = (int)(Pr.meta & 0xFFu), sQ = (int)(Qr.meta & 0xFFu);
                    const DevPair& pc = C->pair[sP * MAXS + sQ];
                    const long long Etr = etr_fix_f32(pc, g2_f32(Pr.v, Qr.v));
                    const long long EvP = evib_fix(A.levfix, C->sp[sP], Pr.q);
                    const long long EvQ = evib_fix(A.levfix, C->sp[sQ], Qr.q);
                    PairOut o{EV_ACC, 0u};
                    uint32_t chan = 0u;
                    bool react = false;
                    if (C->n_reactions > 0) {
                        Stream sp;
                        st_init(sp, rs.seed, step, lcell, rk, PU_PAIR);
                        st_u32(sp);  // the acceptance draw
                        const float u_ster = st_u32(sp);
                        const float u_sel = st_u32(sp);
                        const float u_ch = st_u32(sp);
                        react = reaction_pick_fix(A, C, sP, sQ, Pr.q, Qr.q, Etr, EvP, EvQ, u_ster, u_sel, u_ch, chan) > 0;
                    }
                    if (react) {
                        // exchange A + B -> C + D (no reaction that creates or
                        // removes particles reaches this kernel)
                        const int rxi = (int)(chan & 7u), side = (int)((chan >> 3) & 1u);
                        const DevReaction& rx = C->rx[rxi];
                        RecF& RA = side ? Qr : Pr;
                        RecF& RB = side ? Pr : Qr;
                        float vA[3], vB[3];
                        for (int i = 0; i < 3; ++i) { vA[i] = RA.v[i]; vB[i] = RB.v[i]; }
                        uint32_t q1[4], q2[4];
                        const bool done = rx.type == HCAO_EXCH &&
                                          do_exch_fix(A, C, rx, vA, vB, (int)(RA.meta & 0xFFu), (int)(RB.meta & 0xFFu),
                                                      side ? EvQ : EvP, side ? EvP : EvQ, rs, lcell, rk, q1, q2, o);
                        if (done) {
                            for (int i = 0; i < 3; ++i) { RA.v[i] = vA[i]; RB.v[i] = vB[i]; }
                            RA.meta = (uint32_t)rx.P0;
                            RB.meta = (uint32_t)rx.P1;
                            for (int j = 0; j < 4; ++j) { RA.q[j] = q1[j]; RB.q[j] = q2[j]; }
                            o.ev |= (uint32_t)(rxi + 1) << EV_RX_SHIFT;
                        } else {
                            o.ev |= EV_NOTEXEC;
                            PairLoc L;
                            L.lcell = lcell;
                            L.rk = rk;
                            relax_scatter_fix(A, C, rs, L, Pr, Qr, pc, Etr, EvP, EvQ, o);
                        }
                    } else {
                        // the molecules with modes, P before Q, in one loop
                        long long Erel = Etr;
                        const bool relP = C->sp[sP].n_modes > 0;
                        const int nmol = (int)relP + (int)(C->sp[sQ].n_modes > 0);
                        for (int m = 0; m < nmol; ++m) {
                            const bool isQ = !relP || m == 1;
                            Stream st;
                            st_init(st, rs.seed, step, lcell, rk, isQ ? PU_LB_B : PU_LB_A);
                            uint32_t nq[4];
                            bool took;
                            Erel = relax_one(A, C, isQ ? sQ : sP, nq, isQ ? EvQ : EvP, st, Erel, o, w_lev, w_mode, took);
                            if (took) {
#pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    Pr.q[i] = isQ ? Pr.q[i] : nq[i];
                                    Qr.q[i] = isQ ? nq[i] : Qr.q[i];
                                }
                            }
                        }
                        w_samp += (uint32_t)nmol;
                        w_pair++;
                        Stream ss;
                        st_init(ss, rs.seed, step, lcell, rk, PU_SCAT);
                        float d[3];
                        iso_dir<float>(ss, d);
                        const float va[3] = {Pr.v[0], Pr.v[1], Pr.v[2]}, vb[3] = {Qr.v[0], Qr.v[1], Qr.v[2]};
                        scatter_f32(pc, Erel, d, va, vb, Pr.v, Qr.v);
                    }
                    store_rec(reinterpret_cast<RecF*>(R) + ip, Pr);
                    store_rec(reinterpret_cast<RecF*>(R) + iq, Qr);
                    if (staged) {
                        store_rec(reinterpret_cast<RecF*>(grec) + ip, Pr);
                        store_rec(reinterpret_cast<RecF*>(grec) + iq, Qr);
                    }
                    // the pair's event word, as the queue kernels' end-of-step
                    // reduction reads it (trials saturate at 0xFFFF per pair)
                    const uint32_t ev = ev_final(o);
                    atomicAdd(&s_cnt[FC_ACC], ev & EV_ACC);
                    const uint32_t samp = (ev >> EV_SAMP_SHIFT) & 3u, over = (ev >> EV_OVER_SHIFT) & 3u,
                                   degen = (ev >> EV_DEGEN_SHIFT) & 3u;
                    if (samp) atomicAdd(&s_cnt[FC_SAMP], samp);
                    if (over) atomicAdd(&s_cnt[FC_OVER], over);
                    if (degen) atomicAdd(&s_cnt[FC_DEGEN], degen);
                    if (ev & EV_NOTEXEC) atomicAdd(&s_cnt[FC_NOTEX], 1u);
                    const uint32_t rxid = (ev >> EV_RX_SHIFT) & 63u;
                    if (rxid > 0 && rxid <= MAXR) atomicAdd(&s_cnt[FC_RX0 + rxid - 1], 1u);
                    trials += ev >> EV_TRIAL_SHIFT;
                }
                __syncthreads();
                if (tid < 3) s_n[tid] = 0u;
                __syncthreads();
            }
        }
        // the cell's (sigma g)_max seen this step and its trial count
        atomicMax(&s_seen, __float_as_uint(seen));  // non-negative floats order as their bits
        if (trials) atomicAdd(&s_trials, trials);
        __syncthreads();
        if (tid == 0) {
            unsigned long long* cc = A.counters + (size_t)c * NCNT;
            cc[CNT_CAND] += nsel;
            cc[CNT_ACC] += s_cnt[FC_ACC];
            cc[CNT_SAMPLES] += s_cnt[FC_SAMP];
            cc[CNT_TRIALS] += s_trials;
            cc[CNT_OVER] += s_cnt[FC_OVER];
            cc[CNT_DEGEN] += s_cnt[FC_DEGEN];
            cc[CNT_NOTEXEC] += s_cnt[FC_NOTEX];
            for (int i = 0; i < MAXR && i < NCNT - CNT_RX0; ++i) cc[CNT_RX0 + i] += s_cnt[FC_RX0 + i];
            const double sd = (double)__uint_as_float(s_seen);
            if (sd > cl.sgmax) cl.sgmax = sd;
            cl.nsel = nsel;
            cl.ncreated = 0u;
            cl.nremoved = 0u;
        }
        __syncthreads();  // shared memory is reused by the next cell
    }
    // algorithmic-work counters: one atomic per warp and counter
    unsigned long long wl = w_lev, wm = w_mode, wsmp = w_samp, wp = w_pair;
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        wl += __shfl_xor_sync(0xFFFFFFFFu, wl, o2);
        wm += __shfl_xor_sync(0xFFFFFFFFu, wm, o2);
        wsmp += __shfl_xor_sync(0xFFFFFFFFu, wsmp, o2);
        wp += __shfl_xor_sync(0xFFFFFFFFu, wp, o2);
    }
    if ((tid & 31) == 0 && A.work) {
        atomicAdd(A.work + 0, wl);
        atomicAdd(A.work + 1, wm);
        atomicAdd(A.work + 2, wsmp);
        atomicAdd(A.work + 3, wp);
    }
    // the last CTA to finish advances the reservoirs' step counters (every
    // CTA has read them before it takes its ticket)
    __shared__ bool s_last;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(A.ticket, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int i = tid; i < A.n_res; i += FUSED_THREADS)
            if (A.res[i].active) A.res[i].step++;
        if (tid == 0) *A.ticket = 0u;
    }
}

// One CTA per cell; dynamic shared memory holds smem_recs records (32 B
// each) beside the static queue.
void launch_fused(const StepArgs& a, int smem_recs, cudaStream_t s) {
    const size_t dyn = (size_t)smem_recs * sizeof(RecF);
    const int grid = a.n_cells > 0 ? a.n_cells : 1;
    k_collide_fused<<<grid, FUSED_THREADS, dyn, s>>>(a, smem_recs);
}

cudaError_t fused_prepare(int smem_recs) {
    if (smem_recs < 0 || smem_recs > FUSED_MAX_RECS) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_collide_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((size_t)smem_recs * sizeof(RecF)));
}

}  // namespace hcao
