// hcao_api.cu -- host side of libhcao: the C ABI, species level tables and
// the K5 sampler tables (FP32: alias tables), recombination rate tables,
// reservoir layout in HBM from a per-context memory pool, launches and the
// CUDA graph of a step, the continuous-batching serving engine.
//
// Host arithmetic that feeds device decisions (level energies, grid bases,
// K5 tables, VHS pair constants) is evaluated in IEEE double without FMA
// contraction (-ffp-contract=off) in the operation order documented beside
// each formula.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <ctime>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hcao_internal.h"
#include "hcao_rates.h"
#include "hcao_sort.h"

using namespace hcao;

namespace {

constexpr double KB = 1.380649e-23;
constexpr double HPLANCK = 6.62607015e-34;
constexpr double CLIGHT = 299792458.0;
constexpr double PI_D = 3.14159265358979323846;

struct HostSpecies {
    hcao_species d;
    std::vector<double> we, wexe, De, theta;
    int n_modes = 0;
    bool bend[MAXM] = {};
    double ktheta[MAXM] = {};
    std::vector<double> lev[MAXM];
    double zpe = 0.0;
};

struct Reservoir {
    bool live = false, loaded = false;
    int n_cells = 0;
    double Vc = 0, w = 0, dt = 0, T_sgmax = 0;
    uint64_t seed = 0;
    int cell0 = 0;                 // first global cell index
    void* recs = nullptr;
    size_t rec_bytes = 0;
    uint64_t total_cap = 0;
    uint32_t max_cap = 0;          // largest cell capacity (slots)
    uint32_t cell_base = 0;        // index of the first cell in the random-number keys
};

// one served job: its copied inputs, state and result
struct Job {
    uint64_t id = 0;
    hcao_job spec{};
    std::vector<double> v;
    std::vector<uint8_t> qn;
    std::vector<int32_t> sp, cell;
    int res = -1;          // reservoir while resident
    int steps_left = 0;
    int64_t est_bytes = 0;
    int state = 0;         // 0 queued, 1 resident, 2 done, 3 failed
    bool cancel = false;   // resident and cancelled: retired at the iteration's end
    hcao_job_result result{};
};

double now_s() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

}  // namespace

struct hcao_ctx {
    hcao_config cfg{};
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;  // this context's device memory (see hcao_create)
    int sm_count = 148;
    std::string err;
    uint64_t launches = 0;

    int n_species = 0;
    HostSpecies sp[MAXS];
    int n_reactions = 0;
    // per reaction: the host-side choices of hcao_reaction (model, TCE
    // parameters, WR sample count)
    hcao_reaction rx_host[MAXR] = {};
    Consts hc{};
    Consts* d_consts = nullptr;
    double* d_lev64 = nullptr;
    float* d_lev32 = nullptr;
    long long* d_levfix = nullptr;
    double* d_H64 = nullptr;
    float* d_H32 = nullptr;
    K5Ent* d_k5e = nullptr;
    AliasEnt* d_ae = nullptr;
    // collision-temperature product split: exponent-1/2 tables, FP32 b1 tables
    double* d_H64h = nullptr;
    K5Ent* d_k5eh = nullptr;
    AliasEnt* d_aeh = nullptr;
    float* d_tcb = nullptr;
    int amode = -1;
    double omega = 0.75;

    std::vector<Reservoir> res;
    DevRes* d_res = nullptr;
    int d_res_cap = 0;
    DevCell* d_cells = nullptr;
    unsigned long long* d_cellcnt = nullptr;
    int n_cells_total = 0;
    uint32_t* d_pbase = nullptr;
    uint32_t* d_abase = nullptr;
    uint32_t* d_totals = nullptr;
    uint32_t* d_cflag = nullptr;
    uint32_t* d_rmpos = nullptr;
    uint32_t* d_blkcell = nullptr;  // per round, the cell of every 256th candidate pair
    uint32_t blk_stride = 0;
    void* d_cscratch = nullptr;
    uint4* d_qA = nullptr;
    uint4* d_qB = nullptr;
    uint32_t* d_qsize = nullptr;
    unsigned long long* d_work = nullptr;
    // recombination: rate tables (host copy + device), per-cell sums, particle prefix
    int n_recomb = 0;
    std::vector<double> h_krec, h_Tnode;
    double* d_krec = nullptr;
    // TCE reactions: probability tables [slot][MAXS][TCE_NT + 1]
    std::vector<double> h_tce;
    double* d_tce = nullptr;
    double* d_Tnode = nullptr;
    long long* d_csum = nullptr;
    uint32_t* d_nbase = nullptr;
    uint32_t* d_chbase = nullptr;
    uint32_t* d_tsum = nullptr;
    uint32_t* d_chcnt = nullptr;
    // launch shapes (autotuned; results do not depend on them)
    int grid_select = 0, grid_relax = 0, grid_react = 0;
    bool qorder_off = false;  // the autotuner found the FP32 work-class placement not paying
    // CUDA graph of one step, captured on a private stream, re-captured when
    // the kernel arguments change
    cudaStream_t cap_stream = nullptr;
    // the load path's second stream (copies overlapping the cell sort) and its events
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_aux0 = nullptr, ev_aux1 = nullptr;
    cudaGraphExec_t graph = nullptr;
    StepArgs graph_args{};
    uint64_t graph_launches = 0;     // kernels launched by one replay of the step graph
    bool use_graph = true;
    // serving engine: thread-safe queue in, results out; the engine thread is
    // the only caller of the context's other functions while it runs
    std::mutex serve_mu;
    std::condition_variable serve_cv;
    std::deque<std::shared_ptr<Job>> serve_queue;
    std::vector<std::shared_ptr<Job>> serve_active;
    std::map<uint64_t, std::shared_ptr<Job>> serve_jobs;
    std::thread serve_thread;
    bool serve_running = false, serve_stop = false;
    uint64_t serve_next_id = 1;
    int64_t serve_budget = 0, serve_used = 0;
    int serve_max_active = 256, serve_max_batch_steps = 64;
    uint64_t serve_iterations = 0;
    // engine time by activity (host clock, s): admission (reservoir set-up,
    // load, initial levels), stepping (the iterations' graph launches and
    // their synchronisation), retirement (read-back, release), waiting
    double serve_t[4] = {0.0, 0.0, 0.0, 0.0};
    std::atomic<int> fail_allocs{0};  // test fault injection: device allocations left to fail
    hcao_log_rec* d_log = nullptr;
    uint64_t pair_cap = 0;
    uint64_t pairs_need = 0;        // pair slots the current layout needs (set by relayout)
    bool layout_ok = true;          // false from a layout change until it completed
    size_t chcnt_cap = 0;
    uint32_t* d_err = nullptr;
    uint32_t* d_ticket = nullptr;   // fused step: CTAs finished
    int step_path = HCAO_PATH_AUTO; // requested collision-phase path (hcao_set_step_path)
    int fused_smem_set = -1;        // dynamic shared memory the fused kernel was prepared for (records)
    bool log_on = false;
    uint32_t* d_scratch = nullptr;
    int64_t scratch_words = 0;
    // kernel timing: events recorded on the stream around each kernel class
    bool prof_on = false;
    static constexpr int NPROF = 6;  // setup, select, relax, react, finish, fused collide
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[NPROF];
    size_t prof_used[NPROF] = {};
    double prof_ms[NPROF] = {};
    uint64_t prof_n[NPROF] = {};
};

namespace {

hcao_status fail(hcao_ctx* c, hcao_status s, const std::string& m) {
    if (c) c->err = m;
    return s;
}

// Every entry point runs on the context's device and gives the calling
// thread its previous current device back on return.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(const hcao_ctx* c);
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// device work needs a complete layout: after a load or removal failed part
// way, the cell table may be stale until a load or removal succeeds
#define LAYOUT_GUARD(ctx)                                                                     \
    do {                                                                                      \
        if ((ctx) && !(ctx)->layout_ok)                                                       \
            return fail((ctx), HCAO_EINVAL, "the last load or removal failed; load again first"); \
    } while (0)

// set on the serving engine thread: while a context serves, its state-changing
// entry points are refused on every other thread
thread_local bool tl_serve_engine = false;
#define SERVE_GUARD(ctx)                                                  \
    do {                                                                  \
        if ((ctx) && (ctx)->serve_running && !tl_serve_engine) return HCAO_EBUSY; \
    } while (0)
DeviceScope::DeviceScope(const hcao_ctx* c) {
    int cur = -1;
    if (c && cudaGetDevice(&cur) == cudaSuccess && cur != c->cfg.device && cudaSetDevice(c->cfg.device) == cudaSuccess)
        prev = cur;
}

#define CU(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? HCAO_ENOMEM : HCAO_ECUDA,     \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

template <class T>
cudaError_t dalloc(hcao_ctx* ctx, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (ctx->fail_allocs.load() > 0 && ctx->fail_allocs.fetch_sub(1) > 0)  // test fault injection
        return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), count * sizeof(T), ctx->pool, ctx->stream);
}
template <class T>
void dfree(hcao_ctx* ctx, T*& p) {
    if (p) cudaFreeAsync(p, ctx->stream);
    p = nullptr;
}

// A temporary device buffer of one entry point, released on every exit path
// (stream-ordered, like dfree).
template <class T>
struct DevTemp {
    hcao_ctx* ctx;
    T* p = nullptr;
    explicit DevTemp(hcao_ctx* c) : ctx(c) {}
    ~DevTemp() { dfree(ctx, p); }
    DevTemp(const DevTemp&) = delete;
    DevTemp& operator=(const DevTemp&) = delete;
};

// FP32-mode energy bookkeeping unit: 2^-100 J (int64 range +-7e-12 J,
// resolution 8e-31 J)
long long to_fix(double E) { return std::llround(std::ldexp(E, 100)); }

size_t rec_size(const hcao_ctx* c) { return c->cfg.precision == HCAO_FP64 ? sizeof(RecD) : sizeof(RecF); }

// ---- levels: Morse stretches (Eq. energy-AHO) E(i) = hc we (i+1/2) - hc wexe (i+1/2)^2,
// kept while E < De and increasing; bends (i+1/2) k Theta, kept while i < 256 and
// E < ZPE + table span.  Operation order: ((hc*we)*x) - ((hc*wexe)*(x*x)).
void build_levels(const hcao_ctx* ctx, HostSpecies& s) {
    const double hc = HPLANCK * CLIGHT;
    const int ns = s.d.n_stretch, nb = s.d.n_bend;
    s.n_modes = ns + nb;
    for (int j = 0; j < ns; ++j) {
        s.bend[j] = false;
        s.lev[j].clear();
        double prev = -1.0;
        for (int i = 0; i < MAXL; ++i) {
            const double x = (double)i + 0.5;
            const double E = hc * s.we[j] * x - hc * s.wexe[j] * (x * x);
            if (!(E < s.De[j])) break;
            if (i > 0 && !(E > prev)) break;
            s.lev[j].push_back(E);
            prev = E;
        }
    }
    for (int b = 0; b < nb; ++b) {
        s.bend[ns + b] = true;
        s.ktheta[ns + b] = KB * s.theta[b];
    }
    double z = 0.0;
    for (int j = 0; j < s.n_modes; ++j) {
        const double e0 = s.bend[j] ? 0.5 * s.ktheta[j] : (s.lev[j].empty() ? 0.0 : s.lev[j][0]);
        z = z + e0;
    }
    s.zpe = z;
    const double top = z + ctx->cfg.table_span_J;
    for (int j = ns; j < s.n_modes; ++j) {
        s.lev[j].clear();
        for (int i = 0; i < MAXL; ++i) {
            const double E = ((double)i + 0.5) * s.ktheta[j];
            if (!(E < top)) break;
            s.lev[j].push_back(E);
        }
    }
}

template <class R>
R lbpow_host(int amode, R x) {
    if (amode == 0) {
        const R s = std::sqrt(x);
        return s * std::sqrt(s);
    }
    if (amode == 1) return x;
    return std::sqrt(x);
}

// K5 tables in precision R over the levels `lev` (already in R), quadratic grid
// g_m = base_k + cq m^2:  H_{n-1}(g_m) = sum_i pw(g_m - E_i),
// H_k(g_m) = sum_i W_{k+1}(g_m - E_{k,i}),  W_k(E) = H_k[idx_k(E)],
// idx_k(E) = smallest m >= 1 with g_m >= E (0 if E <= base_k, MT if none).
template <class R>
R grid_pt_host(R base, R cq, int64_t m) {
    return base + cq * (R)(m * m);
}
template <class R>
int64_t grid_idx_host(R base, R cq, int MT, R E) {
    if (!(E > base)) return 0;
    if (grid_pt_host<R>(base, cq, MT - 1) < E) return MT;
    int64_t lo = 0, hi = MT - 1;  // g_lo < E <= g_hi
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) / 2;
        if (grid_pt_host<R>(base, cq, mid) < E) lo = mid; else hi = mid;
    }
    return hi;
}
template <class R>
void build_tables(int amode, int n, const std::vector<R>* lev, const R* base, R cq, int MT,
                  std::vector<R>& out) {
    out.assign((size_t)n * MT, (R)0);
    for (int k = n - 1; k >= 0; --k) {
        for (int m = 0; m < MT; ++m) {
            const R g = grid_pt_host<R>(base[k], cq, m);
            R sum = (R)0;
            for (size_t i = 0; i < lev[k].size(); ++i) {
                if (!(lev[k][i] < g)) break;
                const R x = g - lev[k][i];
                R w;
                if (k == n - 1) {
                    w = lbpow_host<R>(amode, x);
                } else {
                    int64_t mm = grid_idx_host<R>(base[k + 1], cq, MT, x);
                    if (mm > MT - 1) mm = MT - 1;
                    w = mm == 0 ? (R)0 : out[(size_t)(k + 1) * MT + mm];
                }
                sum = sum + w;
            }
            out[(size_t)k * MT + m] = sum;
        }
    }
}

// FP32 tables on geometric buckets read off the float bit pattern of
// x = E - base: idx = (bits(x) >> shift) - j0, at least 1 (0 if E <= base, MT
// past the last bucket), as on the device.  Entry m is evaluated at the
// bucket's upper edge G_m, the largest float whose index is <= m (bisection
// over the ordered bit patterns of positive floats), so every budget in the
// bucket is bounded.
int idx_f32(float base, int shift, int j0, int MT, float E) {
    if (!(E > base)) return 0;
    const float x = E - base;
    uint32_t b;
    std::memcpy(&b, &x, 4);
    const int j = (int)(b >> shift) - j0;
    return j < 1 ? 1 : (j > MT - 1 ? MT : j);
}
float bucket_top_f32(float base, int shift, int j0, int MT, int m) {
    if (m <= 0) return base;
    uint32_t lo, hi;
    float fb = base, fmax = 3.4028234663852886e38f;
    std::memcpy(&lo, &fb, 4);
    std::memcpy(&hi, &fmax, 4);
    while (hi - lo > 1) {  // idx(lo) <= m < idx(hi)
        const uint32_t mid = lo + (hi - lo) / 2;
        float f;
        std::memcpy(&f, &mid, 4);
        if (idx_f32(base, shift, j0, MT, f) <= m) lo = mid; else hi = mid;
    }
    float r;
    std::memcpy(&r, &lo, 4);
    return r;
}
void build_tables_f32(int amode, int n, const std::vector<float>* lev, const float* base, int shift, int j0,
                      int MT, std::vector<float>& out) {
    out.assign((size_t)n * MT, 0.0f);
    for (int k = n - 1; k >= 0; --k) {
        for (int m = 0; m < MT; ++m) {
            const float g = bucket_top_f32(base[k], shift, j0, MT, m);
            float sum = 0.0f;
            for (size_t i = 0; i < lev[k].size(); ++i) {
                if (!(lev[k][i] < g)) break;
                const float x = g - lev[k][i];
                float w;
                if (k == n - 1) {
                    w = lbpow_host<float>(amode, x);
                } else {
                    int mm = idx_f32(base[k + 1], shift, j0, MT, x);
                    if (mm > MT - 1) mm = MT - 1;
                    w = mm == 0 ? 0.0f : out[(size_t)(k + 1) * MT + mm];
                }
                sum = sum + w;
            }
            out[(size_t)k * MT + m] = sum;
        }
    }
}

// FP32 alias proposals of the K5 draw.  For table entry (mode k, bucket m),
// the levels i of mode k below the bucket's upper edge G_m with their weights
// w_i(G_m) (the summands of H_k[m]) as a Walker/Vose alias table.  Drawing i
// from it with probability w_i(G_m)/H_k[m] and accepting with probability
// w_i(E)/w_i(G_m) (E <= G_m, weights increase with the budget) takes level i
// with probability w_i(E)/H_k[idx(E)] and rejects with the rest: the K5 mode
// draw exactly, in constant work instead of a scan of the levels.
// Output: one K5Ent per (k, m) with H_k[m] and the bucket's slots, appended
// to ents; the slots appended to ae (offsets are global in ae).
void build_alias_f32(int amode, int n, const std::vector<float>* lev, const float* base, int shift, int j0,
                     int MT, const std::vector<float>& H, std::vector<K5Ent>& ents, std::vector<AliasEnt>& ae) {
    const size_t e0 = ents.size();
    ents.resize(e0 + (size_t)n * MT);
    for (int k = 0; k < n; ++k)
        for (int m = 0; m < MT; ++m) ents[e0 + (size_t)k * MT + m] = K5Ent{H[(size_t)k * MT + m], 0u, 0u, 0u};
    std::vector<double> w, q;
    std::vector<int> small, large, alias;
    for (int k = 0; k < n; ++k) {
        for (int m = 0; m < MT; ++m) {
            const float g = bucket_top_f32(base[k], shift, j0, MT, m);
            w.clear();
            for (size_t i = 0; i < lev[k].size() && i < 256; ++i) {
                if (!(lev[k][i] < g)) break;
                const float x = g - lev[k][i];
                float wi;
                if (k == n - 1) {
                    wi = lbpow_host<float>(amode, x);
                } else {
                    int mm = idx_f32(base[k + 1], shift, j0, MT, x);
                    if (mm > MT - 1) mm = MT - 1;
                    wi = mm == 0 ? 0.0f : H[(size_t)(k + 1) * MT + mm];
                }
                w.push_back(wi);
            }
            double tot = 0.0;
            for (double x : w) tot += x;
            const int L = tot > 0.0 ? (int)w.size() : 0;
            ents[e0 + (size_t)k * MT + m].off = (uint32_t)ae.size();
            ents[e0 + (size_t)k * MT + m].L = (uint32_t)L;
            if (L == 0) continue;
            // Vose: scaled probabilities L w_i / W, split into small and large
            q.assign(L, 0.0);
            alias.assign(L, 0);
            small.clear();
            large.clear();
            for (int i = 0; i < L; ++i) {
                q[i] = w[i] * L / tot;
                alias[i] = i;
                (q[i] < 1.0 ? small : large).push_back(i);
            }
            while (!small.empty() && !large.empty()) {
                const int a = small.back(), b = large.back();
                small.pop_back();
                alias[a] = b;
                q[b] = (q[b] + q[a]) - 1.0;
                if (q[b] < 1.0) { large.pop_back(); small.push_back(b); }
            }
            for (int i : large) q[i] = 1.0;
            for (int i : small) q[i] = 1.0;  // rounding leftovers
            for (int i = 0; i < L; ++i) {
                AliasEnt a{};
                a.prob = (float)q[i];
                a.alias = (uint32_t)alias[i];
                a.wg_j = (float)w[i];
                a.wg_a = (float)w[alias[i]];
                ae.push_back(a);
            }
        }
    }
}

// VHS pair constants: sigma_T g = C g^(2 - 2 omega),
// C = ((pi*d)*d) * (2 k T_ref / m_r)^(omega-1/2) / Gamma(5/2 - omega),
// d, T_ref the means of both species', m_r = (mA*mB)/(mA+mB).
DevPair pair_consts(const hcao_ctx* ctx, int a, int b) {
    const hcao_species& A = ctx->sp[a].d;
    const hcao_species& B = ctx->sp[b].d;
    DevPair p{};
    p.mr = A.mass * B.mass / (A.mass + B.mass);
    const double d = 0.5 * (A.d_ref + B.d_ref);
    const double Tr = 0.5 * (A.T_ref + B.T_ref);
    p.C = PI_D * d * d * std::pow(2.0 * KB * Tr / p.mr, ctx->omega - 0.5) / std::tgamma(2.5 - ctx->omega);
    p.mt = A.mass + B.mass;
    p.fp = B.mass / p.mt;
    p.fq = A.mass / p.mt;
    p.mr_f = (float)p.mr;
    p.C_f = (float)p.C;
    p.fp_f = (float)p.fp;
    p.fq_f = (float)p.fq;
    p.inv2mr_f = (float)(2.0 / p.mr);
    return p;
}

// <sigma_T g> over a Maxwellian at T: 2 d^2 sqrt(2 pi k T_ref / m_r) (T/T_ref)^(1-omega)
double mean_sigma_g(const hcao_ctx* ctx, int a, int b, double T) {
    const hcao_species& A = ctx->sp[a].d;
    const hcao_species& B = ctx->sp[b].d;
    const double mr = A.mass * B.mass / (A.mass + B.mass);
    const double d = 0.5 * (A.d_ref + B.d_ref);
    const double Tr = 0.5 * (A.T_ref + B.T_ref);
    return 2.0 * d * d * std::sqrt(2.0 * PI_D * KB * Tr / mr) * std::pow(T / Tr, 1.0 - ctx->omega);
}

// Work classes of the FP32 relaxation queue.  A species pair's work key is
// the mode counts of the molecules it relaxes, in order (P first when it has
// modes), and whether it takes the QK test; its class is the rank of its key
// among the distinct keys of the species present, heaviest work (most modes)
// first, the keys past the NCLS - 1 heaviest sharing the last class.  Pairs of
// one class run mode-draw loops of like length, so the lanes of a warp that
// holds them stay busy together.
static void assign_work_classes(Consts& C) {
    const int S = C.n_species;
    struct Key { int first, second, qk; };
    std::vector<Key> keys;
    auto key_of = [&](int a, int b) {
        const int ma = C.sp[a].n_modes, mb = C.sp[b].n_modes;
        return Key{ma > 0 ? ma : mb, ma > 0 ? mb : 0, (int)C.pair[a * MAXS + b].qk};
    };
    auto same = [](const Key& x, const Key& y) { return x.first == y.first && x.second == y.second && x.qk == y.qk; };
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
            const Key k = key_of(a, b);
            bool seen = false;
            for (const Key& x : keys) seen = seen || same(x, k);
            if (!seen) keys.push_back(k);
        }
    std::sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) {
        if (x.first + x.second != y.first + y.second) return x.first + x.second > y.first + y.second;
        if (x.first != y.first) return x.first > y.first;
        return x.qk > y.qk;
    });
    for (int i = 0; i < MAXS * MAXS; ++i) C.pair[i].cls = NCLS - 1;
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
            const Key k = key_of(a, b);
            int rank = 0;
            while (!same(keys[rank], k)) ++rank;
            C.pair[a * MAXS + b].cls = (uint32_t)std::min(rank, NCLS - 1);
        }
    C.n_cls = std::min((int)keys.size(), NCLS);
}

hcao_status upload_consts(hcao_ctx* ctx) {
    assign_work_classes(ctx->hc);
    if (!ctx->d_consts) CU(dalloc(ctx, &ctx->d_consts, 1));
    CU(cudaMemcpyAsync(ctx->d_consts, &ctx->hc, sizeof(Consts), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return HCAO_OK;
}

hcao_status ensure_scratch(hcao_ctx* ctx, int64_t words) {
    if (words <= ctx->scratch_words) return HCAO_OK;
    dfree(ctx, ctx->d_scratch);
    CU(dalloc(ctx, &ctx->d_scratch, (size_t)words));
    ctx->scratch_words = words;
    return HCAO_OK;
}

hcao_status map_err(hcao_ctx* ctx) {
    uint32_t e = 0;
    CU(cudaMemcpyAsync(&e, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (e & ERR_REJECT) return fail(ctx, HCAO_EREJECT_LIMIT, "a rejection loop hit its cap");
    if (e & ERR_CAPACITY) return fail(ctx, HCAO_ECAPACITY, "a cell ran out of particle slots");
    if (e & ERR_ROUNDS) return fail(ctx, HCAO_EROUNDS, "NTC needed more pairing rounds than max_rounds");
    if (e & ERR_LEVEL) return fail(ctx, HCAO_ELEVEL_OVERFLOW, "quantum number outside the level list");
    if (e & ERR_NONFINITE) return fail(ctx, HCAO_ENONFINITE, "non-finite velocity or (sigma g)_max");
    return HCAO_OK;
}

// (Re)build the global cell table after reservoirs change: cells of live,
// loaded reservoirs in reservoir order, with the prefix arrays of the step
// set-up; records the per-pair slots the layout needs (max_rounds * slots / 2
// + cells), which the next step's ensure_pair_buffers provides.
hcao_status relayout(hcao_ctx* ctx, int new_res, const std::vector<DevCell>* new_cells) {
    ctx->layout_ok = false;  // until every table below exists again
    int total = 0;
    uint64_t pairs = 0;
    for (auto& r : ctx->res)
        if (r.live && r.loaded) {
            total += r.n_cells;
            pairs += (uint64_t)ctx->cfg.max_rounds * (r.total_cap / 2) + (uint64_t)r.n_cells;
        }
    DevCell* cells = nullptr;
    unsigned long long* cnt = nullptr;
    const size_t cells_alloc = (size_t)std::max(total, 1);
    CU(dalloc(ctx, &cells, cells_alloc));
    CU(dalloc(ctx, &cnt, cells_alloc * NCNT));
    CU(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * cells_alloc * NCNT, ctx->stream));
    // kept reservoirs' cells and counters move in runs that are contiguous in
    // the old table: one copy per run, not per reservoir (loading R reservoirs
    // one by one would otherwise issue O(R^2) copies)
    int at = 0, run_src = 0, run_dst = 0, run_len = 0;
    auto flush = [&]() -> cudaError_t {
        if (run_len == 0) return cudaSuccess;
        cudaError_t e = cudaMemcpyAsync(cells + run_dst, ctx->d_cells + run_src, sizeof(DevCell) * run_len,
                                        cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cnt + (size_t)run_dst * NCNT, ctx->d_cellcnt + (size_t)run_src * NCNT,
                                sizeof(unsigned long long) * run_len * NCNT, cudaMemcpyDeviceToDevice, ctx->stream);
        run_len = 0;
        return e;
    };
    for (int id = 0; id < (int)ctx->res.size(); ++id) {
        Reservoir& r = ctx->res[id];
        if (!(r.live && r.loaded)) continue;
        if (id == new_res) {
            CU(flush());
            CU(cudaMemcpyAsync(cells + at, new_cells->data(), sizeof(DevCell) * r.n_cells,
                               cudaMemcpyHostToDevice, ctx->stream));
        } else if (run_len > 0 && r.cell0 == run_src + run_len) {
            run_len += r.n_cells;
        } else {
            CU(flush());
            run_src = r.cell0;
            run_dst = at;
            run_len = r.n_cells;
        }
        r.cell0 = at;
        at += r.n_cells;
    }
    CU(flush());
    dfree(ctx, ctx->d_cells);
    dfree(ctx, ctx->d_cellcnt);
    ctx->d_cells = cells;
    ctx->d_cellcnt = cnt;
    ctx->n_cells_total = total;
    dfree(ctx, ctx->d_pbase);
    dfree(ctx, ctx->d_abase);
    dfree(ctx, ctx->d_nbase);
    dfree(ctx, ctx->d_csum);
    dfree(ctx, ctx->d_chbase);
    CU(dalloc(ctx, &ctx->d_chbase, (size_t)total + 1));
    CU(dalloc(ctx, &ctx->d_pbase, (size_t)MAX_ROUNDS * (total + 1)));
    CU(dalloc(ctx, &ctx->d_abase, (size_t)total + 1));
    CU(dalloc(ctx, &ctx->d_nbase, (size_t)total + 1));
    dfree(ctx, ctx->d_tsum);
    {
        const size_t nts = (size_t)SETUP_ARRAYS * (setup_tiles(total) + 1) + 1;
        CU(dalloc(ctx, &ctx->d_tsum, nts));
        CU(cudaMemsetAsync(ctx->d_tsum, 0, sizeof(uint32_t) * nts, ctx->stream));
    }
    CU(dalloc(ctx, &ctx->d_csum, (size_t)5 * cells_alloc));
    // the per-pair buffers are sized at the next step (ensure_pair_buffers):
    // loading many reservoirs one by one then grows them once, not per load
    ctx->pairs_need = pairs;
    // reservoir table
    if ((int)ctx->res.size() > ctx->d_res_cap) {
        DevRes* nr = nullptr;
        const int cap = std::max<int>(64, 2 * (int)ctx->res.size());
        CU(dalloc(ctx, &nr, (size_t)cap));
        if (ctx->d_res)
            CU(cudaMemcpyAsync(nr, ctx->d_res, sizeof(DevRes) * ctx->d_res_cap, cudaMemcpyDeviceToDevice,
                               ctx->stream));
        dfree(ctx, ctx->d_res);
        ctx->d_res = nr;
        ctx->d_res_cap = cap;
    }
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->layout_ok = true;
    return HCAO_OK;
}

hcao_status read_cells(hcao_ctx* ctx, const Reservoir& r, std::vector<DevCell>& out) {
    out.resize(r.n_cells);
    CU(cudaMemcpyAsync(out.data(), ctx->d_cells + r.cell0, sizeof(DevCell) * r.n_cells,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return HCAO_OK;
}

// off[c] = first particle of cell c in canonical order, off[n_cells] = total,
// in a fresh device buffer the caller frees: scanned on the device, only the
// total comes back (synchronises)
hcao_status particle_prefix(hcao_ctx* ctx, const Reservoir& r, uint64_t** d_off, uint64_t* total) {
    CU(dalloc(ctx, d_off, (size_t)r.n_cells + 1));
    launch_cell_prefix(ctx->d_cells, r.cell0, r.n_cells, *d_off, ctx->stream);
    ctx->launches++;
    CU(cudaMemcpyAsync(total, *d_off + r.n_cells, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return HCAO_OK;
}

Reservoir* get_res(hcao_ctx* ctx, int id) {
    if (id < 0 || id >= (int)ctx->res.size() || !ctx->res[id].live) return nullptr;
    return &ctx->res[id];
}

// P5 zero-point search for T_vib: root of <E_vib>(T) (bends: harmonic closed
// form k Theta / (exp(Theta/T) - 1); stretches: Boltzmann mean over the Morse
// levels) = mean vibrational energy above the ZPE, by bisection.
double tvib_host(const HostSpecies& s, double target) {
    if (!(target > 0.0) || s.n_modes == 0) return 0.0;
    auto mean = [&](double T) {
        double e = 0.0;
        for (int j = 0; j < s.n_modes; ++j) {
            if (s.bend[j]) {
                const double th = s.theta[j - s.d.n_stretch];
                e += KB * th / (std::exp(th / T) - 1.0);
            } else {
                double num = 0.0, den = 0.0;
                for (double Ei : s.lev[j]) {
                    const double de = Ei - s.lev[j][0];
                    const double b = std::exp(-de / (KB * T));
                    num += de * b;
                    den += b;
                }
                e += num / den;
            }
        }
        return e;
    };
    double lo = 1.0, hi = 1.0e6;
    for (int it = 0; it < 200; ++it) {
        const double plo = lo, phi = hi;
        const double mid = 0.5 * (lo + hi);
        if (mean(mid) < target) lo = mid; else hi = mid;
        // a pass is a function of (lo, hi) alone: once it changes neither,
        // the remaining passes would not either (the same result, ~60 passes)
        if (lo == plo && hi == phi) break;
    }
    return 0.5 * (lo + hi);
}

// Rate tables of the recombination reactions (Sec. "Recombination
// reactions", reading A14): at every node T_i and for every third-body
// species M, k_r = P_A(T) <sigma_T g>_{A,M}(T) / K_eq(T), with P_A the exact
// thermal dissociation probability of the product A (threshold of the reverse
// QK dissociation: min over the masked stretches of De_j + ZPE_A + ZPE_B +
// ZPE_C - E_j(0)) and K_eq = n_B n_C / n_A from translational and vibrational
// partition sums with the formation energies.  Nodes are independent: they are
// computed on host threads.
// TCE probability tables (the comparison model, Eq. arrhenius): for a
// reaction with k(T) = A T^b exp(-E_a/kT), the probability in a collision of
// total energy E_c is P = C1 (E_c - E_a)^(zeta + b + 1/2) / E_c^(zeta + 3/2 -
// omega), the form whose average over the equilibrium collision-energy
// distribution of a VHS gas (E_tr ~ Gamma(5/2 - omega), internal energy ~
// Gamma(zeta), in units of kT) is eps k(T) / <sigma_T g>(T); integrating,
//   C1 = eps A k^(1 - omega - b) Gamma(zeta + 5/2 - omega) / (Gamma(zeta + b + 3/2) C_sigma),
// <sigma_T g>(T) = C_sigma T^(1 - omega), eps = 2 for like partners.  P is
// capped at 1 and tabulated per partner species at x_i = X (i/NT)^2 above
// E_a (X the sampler span), i = 0..NT.
hcao_status build_tce_tables(hcao_ctx* ctx) {
    Consts& C = ctx->hc;
    const double w = ctx->omega;
    int slots = 0;
    for (int i = 0; i < C.n_reactions; ++i)
        if (C.rx[i].model == HCAO_MODEL_TCE) C.rx[i].tce_slot = slots++;
    C.has_tce = slots > 0 ? 1 : 0;
    ctx->h_tce.assign((size_t)std::max(slots, 1) * MAXS * (TCE_NT + 1), 0.0);
    const double span = ctx->cfg.table_span_J;
    for (int i = 0; i < C.n_reactions; ++i) {
        DevReaction& D = C.rx[i];
        if (D.model != HCAO_MODEL_TCE) continue;
        const double A = ctx->rx_host[i].arrhenius[0], b = ctx->rx_host[i].arrhenius[1];
        const double Ea = ctx->rx_host[i].arrhenius[2], z = ctx->rx_host[i].tce_zeta;
        for (int m = 0; m < ctx->n_species; ++m) {
            if (D.type == HCAO_EXCH && m != D.B) continue;
            const hcao_species& SA = ctx->sp[D.A].d;
            const hcao_species& SM = ctx->sp[m].d;
            const double Tr = 0.5 * (SA.T_ref + SM.T_ref);
            const double Csig = mean_sigma_g(ctx, D.A, m, Tr) / std::pow(Tr, 1.0 - w);
            const double eps = m == D.A ? 2.0 : 1.0;
            const double C1 = eps * A * std::pow(KB, 1.0 - w - b) *
                              std::exp(std::lgamma(z + 2.5 - w) - std::lgamma(z + b + 1.5)) / Csig;
            const double beta = z + b + 0.5, gam = z + 1.5 - w;
            double* t = ctx->h_tce.data() + ((size_t)D.tce_slot * MAXS + (size_t)m) * (TCE_NT + 1);
            for (int k = 0; k <= TCE_NT; ++k) {
                const double sv = (double)k / (double)TCE_NT;
                const double x = span * (sv * sv);
                const double P = x > 0.0 ? C1 * std::pow(x, beta) * std::pow(Ea + x, -gam) : 0.0;
                t[k] = P < 1.0 ? P : 1.0;
            }
        }
    }
    dfree(ctx, ctx->d_tce);
    CU(dalloc(ctx, &ctx->d_tce, ctx->h_tce.size()));
    CU(cudaMemcpyAsync(ctx->d_tce, ctx->h_tce.data(), sizeof(double) * ctx->h_tce.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return HCAO_OK;
}

hcao_status build_recomb_tables(hcao_ctx* ctx) {
    const Consts& C = ctx->hc;
    const int S = ctx->n_species;
    ctx->h_Tnode.resize(REC_NODES);
    for (int i = 0; i < REC_NODES; ++i) ctx->h_Tnode[i] = rec_node_T(i);
    ctx->h_krec.assign((size_t)ctx->n_recomb * MAXS * REC_NODES, 0.0);
    const double a = 2.5 - ctx->omega;
    std::vector<int> rxs;
    for (int i = 0; i < C.n_reactions; ++i)
        if (C.rx[i].type == HCAO_RECOMB) rxs.push_back(i);
    auto levels = [&](int sp) {
        std::vector<std::vector<double>> l;
        for (int j = 0; j < ctx->sp[sp].n_modes; ++j) l.push_back(ctx->sp[sp].lev[j]);
        return l;
    };
    auto work = [&](int node) {
        const double T = ctx->h_Tnode[node];
        for (int ri : rxs) {
            const DevReaction& D = C.rx[ri];
            const HostSpecies& sA = ctx->sp[D.P0];
            const HostSpecies& sB = ctx->sp[D.A];
            const HostSpecies& sC = ctx->sp[D.B];
            double Dthr = INFINITY;
            for (int j = 0; j < sA.d.n_stretch; ++j)
                if ((D.mask >> j) & 1u) Dthr = std::min(Dthr, (sA.De[j] + D.zpesum) - sA.lev[j][0]);
            double P;
            if (ctx->rx_host[ri].model == HCAO_RPROB_WR) {
                // the sampled sum with the WR density: the quanta are the
                // fundamentals E_j(1) - E_j(0) of A's modes, the threshold is
                // taken above A's ground state
                double hnu[MAXM];
                for (int j = 0; j < sA.n_modes; ++j) hnu[j] = sA.lev[j][1] - sA.lev[j][0];
                const int ns = ctx->rx_host[ri].wr_samples > 0 ? ctx->rx_host[ri].wr_samples : 1000;
                P = wr_diss_prob(hnu, sA.n_modes, Dthr - sA.zpe, a, T, ns);
            } else {
                P = thermal_diss_prob(levels(D.P0), Dthr, a, T);
            }
            const double f = 2.0 * PI_D * KB * T / (HPLANCK * HPLANCK);
            const double qtr = std::pow(f * sB.d.mass, 1.5) * std::pow(f * sC.d.mass, 1.5) /
                               std::pow(f * sA.d.mass, 1.5);
            const double dE0 = (sB.d.E_form + sB.zpe + sC.d.E_form + sC.zpe) - (sA.d.E_form + sA.zpe);
            const double keq = qtr * (zvib_excited(levels(D.A), T) * zvib_excited(levels(D.B), T) /
                                      zvib_excited(levels(D.P0), T)) * std::exp(-dE0 / (KB * T));
            for (int m = 0; m < S; ++m)
                ctx->h_krec[((size_t)D.rslot * MAXS + m) * REC_NODES + node] =
                    P * mean_sigma_g(ctx, D.P0, m, T) / keq;
        }
    };
    const int nth = std::max(1, std::min<int>(32, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t)
        th.emplace_back([&, t] {
            for (int node = t; node < REC_NODES; node += nth) work(node);
        });
    for (auto& x : th) x.join();
    dfree(ctx, ctx->d_krec);
    dfree(ctx, ctx->d_Tnode);
    CU(dalloc(ctx, &ctx->d_krec, ctx->h_krec.size()));
    CU(dalloc(ctx, &ctx->d_Tnode, ctx->h_Tnode.size()));
    CU(cudaMemcpyAsync(ctx->d_krec, ctx->h_krec.data(), sizeof(double) * ctx->h_krec.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->d_Tnode, ctx->h_Tnode.data(), sizeof(double) * ctx->h_Tnode.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return HCAO_OK;
}

// Per-pair buffers for the current layout: event words, the relaxation queue
// (two entries per slot), the reaction queue, the log, the chunk counters and
// the created-particle scratch; grown (by at least half) only when too small.
hcao_status ensure_pair_buffers(hcao_ctx* ctx) {
    const uint64_t pairs = ctx->pairs_need;
    // a capacity is recorded only once its buffers exist, so a failed
    // allocation leaves the next call to retry, never a null buffer in use
    if (pairs > ctx->pair_cap || (ctx->log_on && !ctx->d_log) || !ctx->d_cflag) {
        const uint64_t cap = std::max<uint64_t>({pairs, (uint64_t)1024, ctx->pair_cap + ctx->pair_cap / 2});
        ctx->pair_cap = 0;
        dfree(ctx, ctx->d_cflag);
        dfree(ctx, ctx->d_rmpos);
        dfree(ctx, ctx->d_log);
        if (ctx->d_cscratch) cudaFreeAsync(ctx->d_cscratch, ctx->stream);
        ctx->d_cscratch = nullptr;
        dfree(ctx, ctx->d_qA);
        dfree(ctx, ctx->d_qB);
        CU(dalloc(ctx, &ctx->d_qA, 2 * (size_t)cap));  // FP32: class-ordered half + staging half
        CU(dalloc(ctx, &ctx->d_qB, (size_t)cap));
        if (ctx->log_on) CU(dalloc(ctx, &ctx->d_log, (size_t)cap));
        CU(dalloc(ctx, &ctx->d_rmpos, (size_t)cap));
        dfree(ctx, ctx->d_blkcell);
        CU(dalloc(ctx, &ctx->d_blkcell, (size_t)MAX_ROUNDS * (size_t)(cap / 256 + 2)));
        ctx->blk_stride = (uint32_t)(cap / 256 + 2);
        CU(dalloc(ctx, &ctx->d_cflag, (size_t)cap));  // last: its presence marks a complete set
        ctx->pair_cap = cap;
    }
    // chunk counters: at most pairs / FINISH_CHUNK + one partial chunk per cell
    const size_t nch = (size_t)(ctx->pair_cap / FINISH_CHUNK) + (size_t)ctx->n_cells_total + 1;
    if (nch > ctx->chcnt_cap || !ctx->d_chcnt) {
        ctx->chcnt_cap = 0;
        dfree(ctx, ctx->d_chcnt);
        CU(dalloc(ctx, &ctx->d_chcnt, nch));
        ctx->chcnt_cap = nch;
    }
    if (ctx->hc.creates && !ctx->d_cscratch)
        CU(cudaMallocFromPoolAsync(&ctx->d_cscratch, (size_t)ctx->pair_cap * rec_size(ctx), ctx->pool, ctx->stream));
    return HCAO_OK;
}

StepArgs make_args(hcao_ctx* ctx) {
    StepArgs a{};
    a.C = ctx->d_consts;
    a.lev64 = ctx->d_lev64;
    a.lev32 = ctx->d_lev32;
    a.levfix = ctx->d_levfix;
    a.H64 = ctx->d_H64;
    a.H32 = ctx->d_H32;
    a.k5e = ctx->d_k5e;
    a.ae = ctx->d_ae;
    a.H64h = ctx->d_H64h;
    a.k5eh = ctx->d_k5eh;
    a.aeh = ctx->d_aeh;
    a.tcb = ctx->d_tcb;
    a.cells = ctx->d_cells;
    a.n_cells = ctx->n_cells_total;
    a.res = ctx->d_res;
    a.n_res = (int)ctx->res.size();
    a.counters = ctx->d_cellcnt;
    a.pbase = ctx->d_pbase;
    a.abase = ctx->d_abase;
    a.totals = ctx->d_totals;
    a.cflag = ctx->d_cflag;
    a.rmpos = ctx->d_rmpos;
    a.blkcell = ctx->d_blkcell;
    a.blk_stride = ctx->blk_stride;
    a.cscratch = ctx->d_cscratch;
    a.qA = ctx->d_qA;
    a.qB = ctx->d_qB;
    a.qsize = ctx->d_qsize;
    a.has_reactions = ctx->n_reactions > 0 ? 1 : 0;
    a.has_recomb = ctx->n_recomb > 0 ? 1 : 0;
    a.creates = ctx->hc.creates;
    a.krec = ctx->d_krec;
    a.Tnode = ctx->d_Tnode;
    a.csum = ctx->d_csum;
    a.nbase = ctx->d_nbase;
    a.tsum = ctx->d_tsum;
    a.chbase = ctx->d_chbase;
    a.chcnt = ctx->d_chcnt;
    a.work = ctx->prof_on ? ctx->d_work : nullptr;  // the K5 work is counted on profiled steps
    a.grid_select = ctx->grid_select;
    a.grid_relax = ctx->grid_relax;
    a.grid_react = ctx->grid_react;
    a.qorder = (ctx->hc.n_cls > 1 && !ctx->qorder_off) ? 1 : 0;
    a.pair_cap = ctx->pair_cap;
    a.log = ctx->d_log;
    a.log_on = ctx->log_on ? 1 : 0;
    a.err = ctx->d_err;
    a.max_rounds = ctx->cfg.max_rounds;
    a.reject_cap = ctx->cfg.reject_cap;
    a.ticket = ctx->d_ticket;
    a.tce = ctx->d_tce;
    a.tce_span = ctx->cfg.table_span_J;
    return a;
}

// The collision-phase path of the next step: the fused per-cell kernel when
// the context allows it (FP32, no reaction that creates or removes particles,
// no per-pair log, every cell within FUSED_MAX_RECS slots), else the
// per-round queue kernels.  *smem_recs: the records the fused kernel stages.
bool fused_eligible(const hcao_ctx* ctx, int* smem_recs) {
    if (ctx->cfg.precision != HCAO_FP32 || ctx->hc.creates || ctx->n_recomb > 0 || ctx->hc.has_tce ||
        ctx->hc.has_rot || ctx->log_on)
        return false;
    uint32_t mx = 0;
    for (const auto& r : ctx->res)
        if (r.live && r.loaded && r.max_cap > mx) mx = r.max_cap;
    if (mx > (uint32_t)FUSED_MAX_RECS) return false;
    if (smem_recs) *smem_recs = (int)mx;
    return true;
}
bool use_fused(const hcao_ctx* ctx, int* smem_recs) {
    // the queue kernels are the faster path on every workload measured (the
    // fused kernel keeps fewer pairs in flight per SM), so the fused kernel
    // runs only when asked for
    if (ctx->step_path != HCAO_PATH_FUSED) return false;
    return fused_eligible(ctx, smem_recs);
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

void hcao_default_config(hcao_config* c) {
    std::memset(c, 0, sizeof *c);
    c->precision = HCAO_FP64;
    c->device = 0;
    c->cuda_stream = nullptr;
    c->table_points = 2048;
    c->table_span_J = 64.0 * 1.602176634e-19;
    c->reject_cap = 1u << 20;
    c->max_rounds = 2;
    c->capacity_factor = 2.0;
    c->capacity_extra = 64;
}

hcao_status hcao_create(const hcao_config* config, hcao_ctx** out) {
    if (!out) return HCAO_EINVAL;
    *out = nullptr;
    hcao_ctx* ctx = new hcao_ctx();
    hcao_default_config(&ctx->cfg);
    if (config) ctx->cfg = *config;
    if (ctx->cfg.table_points < 16 || ctx->cfg.table_points > 4000 || !(ctx->cfg.table_span_J > 0) ||
        ctx->cfg.max_rounds < 1 || ctx->cfg.max_rounds > MAX_ROUNDS || ctx->cfg.reject_cap < 1 ||
        (ctx->cfg.precision != HCAO_FP64 && ctx->cfg.precision != HCAO_FP32) ||
        ctx->cfg.capacity_factor < 1.0 || ctx->cfg.capacity_extra < 0) {
        delete ctx;
        return HCAO_EINVAL;
    }
    DeviceScope ds_(ctx);  // the caller's current device is given back on return
    cudaError_t e = cudaSetDevice(ctx->cfg.device);
    if (e != cudaSuccess) {
        delete ctx;
        return HCAO_ECUDA;
    }
    int dev = ctx->cfg.device;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, dev);
    ctx->stream = static_cast<cudaStream_t>(ctx->cfg.cuda_stream);
    // A pool of the context's own: memory it frees stays mapped for its next
    // allocations (up to POOL_KEEP_BYTES unused), so reloading a reservoir
    // does not map and unmap its staging buffers and records each time.  The
    // default pool would return freed memory to the system at every
    // synchronisation.  Destroyed with the context.
    {
        cudaMemPoolProps pp{};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.handleTypes = cudaMemHandleTypeNone;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = dev;
        uint64_t keep = POOL_KEEP_BYTES;
        if (cudaMemPoolCreate(&ctx->pool, &pp) != cudaSuccess) {
            delete ctx;
            return HCAO_ECUDA;
        }
        if (cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaMemPoolDestroy(ctx->pool);
            delete ctx;
            return HCAO_ECUDA;
        }
    }
    if (dalloc(ctx, &ctx->d_err, 1) != cudaSuccess || dalloc(ctx, &ctx->d_totals, MAX_ROUNDS + 2) != cudaSuccess ||
        dalloc(ctx, &ctx->d_qsize, QSIZE_WORDS) != cudaSuccess || dalloc(ctx, &ctx->d_work, 4) != cudaSuccess ||
        dalloc(ctx, &ctx->d_ticket, 1) != cudaSuccess) {
        hcao_destroy(ctx);  // frees what was allocated and the pool
        return HCAO_ENOMEM;
    }
    cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream);
    cudaMemsetAsync(ctx->d_ticket, 0, sizeof(uint32_t), ctx->stream);
    cudaMemsetAsync(ctx->d_totals, 0, sizeof(uint32_t) * (MAX_ROUNDS + 2), ctx->stream);
    cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long) * 4, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        hcao_destroy(ctx);
        return HCAO_ECUDA;
    }
    *out = ctx;
    return HCAO_OK;
}

void hcao_destroy(hcao_ctx* ctx) {
    DeviceScope ds_(ctx);
    if (!ctx) return;
    hcao_serve_stop(ctx);
    cudaStreamSynchronize(ctx->stream);
    for (auto& r : ctx->res)
        if (r.recs) cudaFreeAsync(r.recs, ctx->stream);
    dfree(ctx, ctx->d_consts);
    dfree(ctx, ctx->d_lev64);
    dfree(ctx, ctx->d_lev32);
    dfree(ctx, ctx->d_levfix);
    dfree(ctx, ctx->d_H64);
    dfree(ctx, ctx->d_H32);
    dfree(ctx, ctx->d_k5e);
    dfree(ctx, ctx->d_ae);
    dfree(ctx, ctx->d_H64h);
    dfree(ctx, ctx->d_k5eh);
    dfree(ctx, ctx->d_aeh);
    dfree(ctx, ctx->d_tcb);
    dfree(ctx, ctx->d_res);
    dfree(ctx, ctx->d_cells);
    dfree(ctx, ctx->d_cellcnt);
    dfree(ctx, ctx->d_pbase);
    dfree(ctx, ctx->d_abase);
    dfree(ctx, ctx->d_totals);
    dfree(ctx, ctx->d_cflag);
    dfree(ctx, ctx->d_rmpos);
    dfree(ctx, ctx->d_blkcell);
    if (ctx->d_cscratch) cudaFreeAsync(ctx->d_cscratch, ctx->stream);
    dfree(ctx, ctx->d_log);
    dfree(ctx, ctx->d_qA);
    dfree(ctx, ctx->d_qB);
    dfree(ctx, ctx->d_qsize);
    dfree(ctx, ctx->d_work);
    dfree(ctx, ctx->d_krec);
    dfree(ctx, ctx->d_Tnode);
    dfree(ctx, ctx->d_csum);
    dfree(ctx, ctx->d_nbase);
    dfree(ctx, ctx->d_chbase);
    dfree(ctx, ctx->d_tsum);
    dfree(ctx, ctx->d_chcnt);
    dfree(ctx, ctx->d_err);
    dfree(ctx, ctx->d_ticket);
    dfree(ctx, ctx->d_tce);
    dfree(ctx, ctx->d_scratch);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    if (ctx->ev_aux0) cudaEventDestroy(ctx->ev_aux0);
    if (ctx->ev_aux1) cudaEventDestroy(ctx->ev_aux1);
    for (int k = 0; k < hcao_ctx::NPROF; ++k)
        for (auto& e : ctx->prof_ev[k]) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    delete ctx;
}

const char* hcao_last_error(const hcao_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

double hcao_wr_density(const double* hnu, int n_osc, double E) { return wr_density(hnu, n_osc, E); }

double hcao_wr_diss_prob(const double* hnu, int n_osc, double Dx, double omega, double T, int n_samp) {
    return wr_diss_prob(hnu, n_osc, Dx, 2.5 - omega, T, n_samp);
}

hcao_status hcao_recomb_rate(hcao_ctx* ctx, int reaction, int spM, double T, double* out) {
    DeviceScope ds_(ctx);
    if (!ctx || !out || reaction < 0 || reaction >= ctx->n_reactions || spM < 0 || spM >= ctx->n_species)
        return fail(ctx, HCAO_EINVAL, "recomb_rate: bad arguments");
    const DevReaction& D = ctx->hc.rx[reaction];
    if (D.type != HCAO_RECOMB) return fail(ctx, HCAO_EINVAL, "recomb_rate: not a recombination");
    const double* Tn = ctx->h_Tnode.data();
    const double* k = ctx->h_krec.data() + ((size_t)D.rslot * MAXS + spM) * REC_NODES;
    const int last = REC_NODES - 1;
    if (!(T > Tn[0])) { *out = k[0]; return HCAO_OK; }
    if (!(T < Tn[last])) { *out = k[last]; return HCAO_OK; }
    int lo = 0, hi = last;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (Tn[mid] <= T) lo = mid; else hi = mid;
    }
    const double f = (T - Tn[lo]) / (Tn[hi] - Tn[lo]);
    *out = k[lo] + f * (k[hi] - k[lo]);
    return HCAO_OK;
}

uint64_t hcao_kernel_launches(const hcao_ctx* ctx) { return ctx ? ctx->launches : 0; }

hcao_status hcao_set_species(hcao_ctx* ctx, const hcao_species* species, int n) {
    DeviceScope ds_(ctx);
    if (!ctx || !species || n < 1 || n > MAXS) return fail(ctx, HCAO_EINVAL, "set_species: bad arguments");
    if (ctx->n_species > 0) return fail(ctx, HCAO_EINVAL, "set_species: already set");
    int amode = -1;
    for (int i = 0; i < n; ++i) {
        const hcao_species& d = species[i];
        int am;
        if (d.omega == 0.75) am = 0;
        else if (d.omega == 0.5) am = 1;
        else if (d.omega == 1.0) am = 2;
        else return fail(ctx, HCAO_EINVAL, "set_species: omega must be 0.5, 0.75 or 1");
        if (amode >= 0 && am != amode) return fail(ctx, HCAO_EINVAL, "set_species: omega differs between species");
        amode = am;
        if (d.n_stretch < 0 || d.n_bend < 0 || d.n_stretch + d.n_bend > MAXM || !(d.mass > 0) ||
            !(d.d_ref > 0) || !(d.T_ref > 0))
            return fail(ctx, HCAO_EINVAL, "set_species: bad species parameters");
        if ((d.n_stretch > 0 && (!d.we || !d.wexe || !d.De)) || (d.n_bend > 0 && !d.theta))
            return fail(ctx, HCAO_EINVAL, "set_species: missing mode arrays");
        if (d.rot_dof != 0 && d.rot_dof != 2 && d.rot_dof != 3)
            return fail(ctx, HCAO_EINVAL, "set_species: rot_dof must be 0, 2 or 3");
        if (d.rot_dof != 0 && ctx->cfg.precision == HCAO_FP32 && d.n_stretch + d.n_bend > 12)
            return fail(ctx, HCAO_EINVAL, "set_species: a rotating species has at most 12 modes in FP32 mode");
    }
    ctx->amode = amode;
    ctx->omega = species[0].omega;
    // levels
    std::vector<double> lev64;
    std::vector<float> lev32;
    std::vector<long long> levfix;
    for (int i = 0; i < n; ++i) {
        HostSpecies& s = ctx->sp[i];
        s.d = species[i];
        s.we.assign(species[i].we, species[i].we + species[i].n_stretch);
        s.wexe.assign(species[i].wexe, species[i].wexe + species[i].n_stretch);
        s.De.assign(species[i].De, species[i].De + species[i].n_stretch);
        s.theta.assign(species[i].theta, species[i].theta + species[i].n_bend);
        s.d.we = s.we.data(); s.d.wexe = s.wexe.data(); s.d.De = s.De.data(); s.d.theta = s.theta.data();
        build_levels(ctx, s);
        for (int j = 0; j < s.n_modes; ++j)
            if (s.lev[j].empty()) return fail(ctx, HCAO_EINVAL, "set_species: a stretch has no level below De");
    }
    ctx->n_species = n;
    Consts& C = ctx->hc;
    std::memset(&C, 0, sizeof C);
    C.n_species = n;
    C.amode = amode;
    // FP64: table_points quadratic grid points.  FP32: geometric buckets of
    // F32_BUCKET_BITS mantissa bits over the same table_points / 128 octaves
    // below the span (finer buckets: fewer rejected draws, larger tables)
    const int M = ctx->cfg.precision == HCAO_FP32 ? ctx->cfg.table_points << (F32_BUCKET_BITS - 7)
                                                  : ctx->cfg.table_points;
    const int MT = M + TABLE_PAD;
    std::vector<double> H64;
    std::vector<float> H32;
    std::vector<K5Ent> k5e;
    std::vector<AliasEnt> ae;
    for (int i = 0; i < n; ++i) {
        HostSpecies& s = ctx->sp[i];
        DevSpecies& D = C.sp[i];
        D.mass = s.d.mass;
        D.mass_f = (float)s.d.mass;
        D.mass_lo_f = (float)(s.d.mass - (double)D.mass_f);
        D.E_form = s.d.E_form;
        // rotation: the maximum of the LB fraction's density shape,
        // x^(rot_dof/2 - 1) (1 - x)^(3/2 - omega): 1 at x = 0 for two degrees
        // of freedom, at x = 1/2 / (1/2 + 3/2 - omega) for three
        D.rot_dof = s.d.rot_dof;
        if (s.d.rot_dof == 2) {
            D.rot_fmax = 1.0;
        } else if (s.d.rot_dof == 3) {
            const double bb = 1.5 - ctx->omega;
            const double xs = 0.5 / (0.5 + bb);
            D.rot_fmax = std::sqrt(xs) * std::pow(1.0 - xs, bb);
        }
        D.rot_fmax_f = (float)D.rot_fmax;
        if (s.d.rot_dof) C.has_rot = 1;
        D.zpe = s.zpe;
        D.n_modes = s.n_modes;
        D.n_stretch = s.d.n_stretch;
        D.tab_off_h = -1;
        for (int b = 0; b < s.d.n_bend; ++b) D.theta[s.d.n_stretch + b] = s.theta[b];
        D.M = M;
        D.MT = MT;
        for (int j = 0; j < s.d.n_stretch; ++j) {
            D.De[j] = s.De[j];
            D.De_fix[j] = to_fix(s.De[j]);
        }
        for (int j = 0; j < s.n_modes; ++j) {
            D.lev_off[j] = (int)lev64.size();
            D.n_lev[j] = (int)s.lev[j].size();
            for (double e : s.lev[j]) {
                lev64.push_back(e);
                lev32.push_back((float)e);
                levfix.push_back(to_fix(e));
            }
        }
        // K5 grid: base_k = E_k(0) + base_{k+1}; delta = span / M
        const int nm = s.n_modes;
        D.base[nm] = 0.0;
        D.base_f[nm] = 0.0f;
        for (int k = nm - 1; k >= 0; --k) {
            D.base[k] = s.lev[k][0] + D.base[k + 1];
            D.base_f[k] = (float)s.lev[k][0] + D.base_f[k + 1];
        }
        D.cq = ctx->cfg.table_span_J / ((double)M * (double)M);
        D.inv_cq = 1.0 / D.cq;
        D.cq_f = (float)D.cq;
        D.inv_cq_f = 1.0f / D.cq_f;
        D.top = nm > 0 ? D.base[0] + D.cq * (double)((int64_t)M * M) : INFINITY;
        D.eps_min = INFINITY;
        D.eps_min_f = INFINITY;
        for (int j = 0; j < nm; ++j)
            if (s.lev[j].size() > 1) {
                const double e = s.lev[j][1] - s.lev[j][0];
                const float ef = (float)s.lev[j][1] - (float)s.lev[j][0];
                if (e < D.eps_min) D.eps_min = e;
                if (ef < D.eps_min_f) D.eps_min_f = ef;
            }
        if (nm > 0) {
            if (ctx->cfg.precision == HCAO_FP64) {
                std::vector<double> L[MAXM];
                for (int j = 0; j < nm; ++j) L[j] = s.lev[j];
                std::vector<double> t;
                build_tables<double>(amode, nm, L, D.base, D.cq, MT, t);
                D.tab_off = (int)H64.size();
                H64.insert(H64.end(), t.begin(), t.end());
            } else {
                std::vector<float> L[MAXM];
                for (int j = 0; j < nm; ++j) {
                    L[j].resize(s.lev[j].size());
                    for (size_t l = 0; l < s.lev[j].size(); ++l) L[j][l] = (float)s.lev[j][l];
                }
                // F32_BUCKET_BITS mantissa bits per octave; x = span maps to M
                D.gshift = 23 - F32_BUCKET_BITS;
                const float span = (float)ctx->cfg.table_span_J;
                uint32_t sb;
                std::memcpy(&sb, &span, 4);
                D.gj0 = (int)(sb >> D.gshift) - M;
                std::vector<float> t;
                build_tables_f32(amode, nm, L, D.base_f, D.gshift, D.gj0, MT, t);
                D.tab_off = (int)H32.size();
                build_alias_f32(amode, nm, L, D.base_f, D.gshift, D.gj0, MT, t, k5e, ae);
                H32.insert(H32.end(), t.begin(), t.end());
                D.top = (double)bucket_top_f32(D.base_f[0], D.gshift, D.gj0, MT, M);
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        DevSpecies& D = C.sp[i];
        long long z = 0;  // ZPE in fixed point: the exact sum of the ground levels
        for (int j = 0; j < D.n_modes; ++j) z += levfix[D.lev_off[j]];
        D.zpe_fix = z;
        D.top_fix = std::isfinite(D.top) ? to_fix(D.top) : (long long)0x7FFFFFFFFFFFFFFFll;
    }
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) C.pair[a * MAXS + b] = pair_consts(ctx, a, b);
    CU(dalloc(ctx, &ctx->d_lev64, lev64.size()));
    CU(dalloc(ctx, &ctx->d_lev32, lev32.size()));
    CU(dalloc(ctx, &ctx->d_levfix, levfix.size()));
    CU(cudaMemcpyAsync(ctx->d_levfix, levfix.data(), sizeof(long long) * levfix.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaMemcpyAsync(ctx->d_lev64, lev64.data(), sizeof(double) * lev64.size(), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->d_lev32, lev32.data(), sizeof(float) * lev32.size(), cudaMemcpyHostToDevice, ctx->stream));
    if (!H64.empty()) {
        CU(dalloc(ctx, &ctx->d_H64, H64.size()));
        CU(cudaMemcpyAsync(ctx->d_H64, H64.data(), sizeof(double) * H64.size(), cudaMemcpyHostToDevice, ctx->stream));
    }
    if (!H32.empty()) {
        dfree(ctx, ctx->d_H32);
        dfree(ctx, ctx->d_k5e);
        dfree(ctx, ctx->d_ae);
        CU(dalloc(ctx, &ctx->d_H32, H32.size()));
        CU(cudaMemcpyAsync(ctx->d_H32, H32.data(), sizeof(float) * H32.size(), cudaMemcpyHostToDevice, ctx->stream));
        CU(dalloc(ctx, &ctx->d_k5e, k5e.size()));
        CU(cudaMemcpyAsync(ctx->d_k5e, k5e.data(), sizeof(K5Ent) * k5e.size(), cudaMemcpyHostToDevice, ctx->stream));
        CU(dalloc(ctx, &ctx->d_ae, std::max<size_t>(ae.size(), 1)));
        if (!ae.empty())
            CU(cudaMemcpyAsync(ctx->d_ae, ae.data(), sizeof(AliasEnt) * ae.size(), cudaMemcpyHostToDevice, ctx->stream));
    }
    return upload_consts(ctx);
}

// Collision-temperature product split (host side).  <E_vib>(T) of species i
// above its ground level: Boltzmann mean of each stretch's levels, k Theta /
// (e^(Theta/T) - 1) for a bend; T_c by bisection; b1 of the first product.
static double mean_evib_host(const HostSpecies& s, double T) {
    const double kT = KB * T;
    double e = 0.0;
    for (int j = 0; j < s.n_modes; ++j) {
        if (j >= s.d.n_stretch) {
            const double x = s.theta[j - s.d.n_stretch] / T;
            if (x <= 700.0) e += KB * s.theta[j - s.d.n_stretch] / std::expm1(x);
        } else {
            double num = 0.0, den = 0.0;
            for (double l : s.lev[j]) {
                const double de = l - s.lev[j][0];
                const double b = std::exp(-de / kT);
                num += de * b;
                den += b;
            }
            e += num / den;
        }
    }
    return e;
}
static double b1_host(const HostSpecies& p1, const HostSpecies& p2, double xi_tr, double Ex) {
    double lo = 1.0, hi = 1.0e7;
    for (int it = 0; it < 100; ++it) {
        const double T = 0.5 * (lo + hi);
        const double g = 0.5 * xi_tr * KB * T + mean_evib_host(p1, T) + mean_evib_host(p2, T) - Ex;
        if (g < 0.0) lo = T; else hi = T;
    }
    const double Tc = 0.5 * (lo + hi);
    const double xi2 = p2.n_modes ? 2.0 * mean_evib_host(p2, Tc) / (KB * Tc) : 0.0;
    return (xi_tr + xi2) / 2.0 - 1.0;
}

// Tables of the reactions with the collision-temperature split: the
// products' K5 tables at exponent 1/2 (a product's exponent falls below the
// context's 3/2 - omega after an exchange or a recombination; not needed
// when that exponent is 1/2 already), and in FP32 mode each dissociation's
// and exchange's b1 over E_x = 2^(TCB_L0 + i / TCB_PER_OCTAVE) J.
hcao_status build_split_tables(hcao_ctx* ctx) {
    Consts& C = ctx->hc;
    dfree(ctx, ctx->d_H64h);
    dfree(ctx, ctx->d_k5eh);
    dfree(ctx, ctx->d_aeh);
    dfree(ctx, ctx->d_tcb);
    for (int i = 0; i < ctx->n_species; ++i) C.sp[i].tab_off_h = -1;
    bool any = false;
    for (int r = 0; r < C.n_reactions; ++r)
        if (C.rx[r].prod_split == HCAO_SPLIT_TCOLL) any = true;
    if (!any) return HCAO_OK;
    const bool fp32 = ctx->cfg.precision == HCAO_FP32;
    std::vector<double> H64;
    std::vector<K5Ent> k5e;
    std::vector<AliasEnt> ae;
    std::vector<float> tcb;
    for (int r = 0; r < C.n_reactions; ++r) {
        DevReaction& R = C.rx[r];
        if (R.prod_split != HCAO_SPLIT_TCOLL) continue;
        for (int k = 0; k < 2 && C.amode != 2; ++k) {
            const int p = k ? R.P1 : R.P0;
            if (p < 0) continue;
            DevSpecies& D = C.sp[p];
            const HostSpecies& s = ctx->sp[p];
            const int nm = s.n_modes;
            if (nm == 0 || D.tab_off_h >= 0) continue;
            if (!fp32) {
                std::vector<double> L[MAXM];
                for (int j = 0; j < nm; ++j) L[j] = s.lev[j];
                std::vector<double> t;
                build_tables<double>(2, nm, L, D.base, D.cq, D.MT, t);
                D.tab_off_h = (int)H64.size();
                H64.insert(H64.end(), t.begin(), t.end());
            } else {
                std::vector<float> L[MAXM];
                for (int j = 0; j < nm; ++j) {
                    L[j].resize(s.lev[j].size());
                    for (size_t l = 0; l < s.lev[j].size(); ++l) L[j][l] = (float)s.lev[j][l];
                }
                std::vector<float> t;
                build_tables_f32(2, nm, L, D.base_f, D.gshift, D.gj0, D.MT, t);
                D.tab_off_h = (int)k5e.size();
                build_alias_f32(2, nm, L, D.base_f, D.gshift, D.gj0, D.MT, t, k5e, ae);
            }
        }
        if (fp32 && R.type != HCAO_RECOMB) {
            R.tcb_off = (int)tcb.size();
            const double xi_tr = R.type == HCAO_DISS ? 6.0 : 3.0;
            for (int i = 0; i < TCB_N; ++i) {
                const double Ex = std::exp2(TCB_L0 + (double)i / TCB_PER_OCTAVE);
                tcb.push_back((float)b1_host(ctx->sp[R.P0], ctx->sp[R.P1], xi_tr, Ex));
            }
        }
    }
    if (!H64.empty()) {
        CU(dalloc(ctx, &ctx->d_H64h, H64.size()));
        CU(cudaMemcpyAsync(ctx->d_H64h, H64.data(), sizeof(double) * H64.size(), cudaMemcpyHostToDevice,
                           ctx->stream));
    }
    if (!k5e.empty()) {
        CU(dalloc(ctx, &ctx->d_k5eh, k5e.size()));
        CU(cudaMemcpyAsync(ctx->d_k5eh, k5e.data(), sizeof(K5Ent) * k5e.size(), cudaMemcpyHostToDevice,
                           ctx->stream));
        CU(dalloc(ctx, &ctx->d_aeh, std::max<size_t>(ae.size(), 1)));
        if (!ae.empty())
            CU(cudaMemcpyAsync(ctx->d_aeh, ae.data(), sizeof(AliasEnt) * ae.size(), cudaMemcpyHostToDevice,
                               ctx->stream));
    }
    if (!tcb.empty()) {
        CU(dalloc(ctx, &ctx->d_tcb, tcb.size()));
        CU(cudaMemcpyAsync(ctx->d_tcb, tcb.data(), sizeof(float) * tcb.size(), cudaMemcpyHostToDevice,
                           ctx->stream));
    }
    return HCAO_OK;
}

hcao_status hcao_set_reactions(hcao_ctx* ctx, const hcao_reaction* rx, int n) {
    DeviceScope ds_(ctx);
    if (!ctx || n < 0 || n > MAXR || (n > 0 && !rx)) return fail(ctx, HCAO_EINVAL, "set_reactions: bad arguments");
    if (ctx->n_species == 0) return fail(ctx, HCAO_EINVAL, "set_reactions: species first");
    for (auto& r : ctx->res)
        if (r.live) return fail(ctx, HCAO_EINVAL, "set_reactions: before any reservoir");
    Consts& C = ctx->hc;
    const int S = ctx->n_species;
    int creates = 0, n_rec = 0;
    for (int i = 0; i < MAXS * MAXS; ++i) C.rec_pair[i] = -1;
    for (int i = 0; i < n; ++i) {
        const hcao_reaction& r = rx[i];
        DevReaction& D = C.rx[i];
        std::memset(&D, 0, sizeof D);
        D.type = r.type;
        ctx->rx_host[i] = r;
        ctx->rx_host[i].alpha = nullptr;  // not kept: copied into D.alpha below
        if (r.model != 0 && r.model != 1)
            return fail(ctx, HCAO_EINVAL, "set_reactions: bad model");
        if (r.prod_split != HCAO_SPLIT_RELAX && r.prod_split != HCAO_SPLIT_TCOLL)
            return fail(ctx, HCAO_EINVAL, "set_reactions: bad prod_split");
        if (r.type != HCAO_DISS && r.type != HCAO_EXCH && r.type != HCAO_RECOMB)
            return fail(ctx, HCAO_EINVAL, "set_reactions: bad type");
        if (r.type == HCAO_RECOMB) {
            // B + C + M -> A + M: stored as A := B, B := C, P0 := A
            D.A = r.reactants[0];
            D.B = r.reactants[1];
            D.P0 = r.products[0];
            D.P1 = -1;
            if (D.A < 0 || D.A >= S || D.B < 0 || D.B >= S || D.P0 < 0 || D.P0 >= S)
                return fail(ctx, HCAO_EINVAL, "set_reactions: species index out of range");
            const HostSpecies& P = ctx->sp[D.P0];
            if (P.d.n_stretch == 0 || r.diss_mode_mask == 0u || (r.diss_mode_mask >> P.d.n_stretch) != 0)
                return fail(ctx, HCAO_EINVAL, "set_reactions: recombination mask outside the product's stretches");
            for (int o = 0; o < 2; ++o) {
                const int a = o ? D.B : D.A, b = o ? D.A : D.B;
                if (C.rec_pair[a * MAXS + b] >= 0)
                    return fail(ctx, HCAO_EINVAL, "set_reactions: two recombinations of one species pair");
            }
            D.mask = r.diss_mode_mask;
            D.prod_split = r.prod_split;
            // the reverse dissociation's threshold terms (Eq. Ecoll-diss) and the released energy
            D.zpesum = P.zpe + ctx->sp[D.A].zpe + ctx->sp[D.B].zpe;
            D.dEf = P.d.E_form - (ctx->sp[D.A].d.E_form + ctx->sp[D.B].d.E_form);
            D.dEf_fix = to_fix(D.dEf);
            D.rslot = n_rec++;
            C.rec_pair[D.A * MAXS + D.B] = i;               // side 0: P is B
            if (D.B != D.A) C.rec_pair[D.B * MAXS + D.A] = i | (1 << 3);
            creates = 1;  // removed positions use the per-pair scratch slots
            continue;
        }
        D.A = r.reactants[0];
        D.B = r.type == HCAO_EXCH ? r.reactants[1] : -1;
        D.P0 = r.products[0];
        D.P1 = r.products[1];
        if (D.A < 0 || D.A >= S || D.P0 < 0 || D.P0 >= S || D.P1 < 0 || D.P1 >= S ||
            (r.type == HCAO_EXCH && (D.B < 0 || D.B >= S)))
            return fail(ctx, HCAO_EINVAL, "set_reactions: species index out of range");
        const HostSpecies& A = ctx->sp[D.A];
        D.mask = r.diss_mode_mask;
        D.Ea = r.Ea;
        D.steric = r.steric;
        D.alpha_mode = r.alpha_mode;
        D.model = r.model;
        if (!(r.gamma >= 0.0 && r.gamma <= 1.0)) return fail(ctx, HCAO_EINVAL, "set_reactions: gamma outside [0, 1]");
        D.gamma = r.gamma;
        D.gamma_f = (float)r.gamma;
        D.prod_split = r.prod_split;
        if (r.model == HCAO_MODEL_TCE) {
            const double b = r.arrhenius[1], z = r.tce_zeta;
            if (!(r.arrhenius[0] >= 0.0) || !(r.arrhenius[2] >= 0.0) || !(z >= 0.0) || !(z + b + 1.5 > 0.0))
                return fail(ctx, HCAO_EINVAL, "set_reactions: TCE needs A >= 0, E_a >= 0, zeta >= 0 and "
                                              "zeta + b + 3/2 > 0");
            D.tce_Ea = r.arrhenius[2];
            D.tce_zeta_on = z > 0.0 ? 1 : 0;
            int mode = 0;
            while (mode < 31 && !((r.diss_mode_mask >> mode) & 1u)) mode++;
            D.tce_mode = r.type == HCAO_DISS ? mode : 0;
        }
        if (r.type == HCAO_DISS) {
            if (A.d.n_stretch == 0 || (r.diss_mode_mask >> A.d.n_stretch) != 0)
                return fail(ctx, HCAO_EINVAL, "set_reactions: dissociation mask outside the stretches");
            // Eq. Ecoll-diss subtracts the ZPEs of A, B and C
            D.zpesum = A.zpe + ctx->sp[D.P0].zpe + ctx->sp[D.P1].zpe;
            D.dEf = (ctx->sp[D.P0].d.E_form + ctx->sp[D.P1].d.E_form) - A.d.E_form;
            D.zpesum_fix = C.sp[D.A].zpe_fix + C.sp[D.P0].zpe_fix + C.sp[D.P1].zpe_fix;
            creates = 1;
        } else {
            if (r.alpha_mode == HCAO_ALPHA_ONE_RANDOM_STRETCH && A.d.n_stretch == 0)
                return fail(ctx, HCAO_EINVAL, "set_reactions: exchange coupling needs a stretch");
            if (r.alpha_mode == HCAO_ALPHA_PER_MODE && r.alpha)
                for (int j = 0; j < A.n_modes; ++j) D.alpha[j] = r.alpha[j];
            D.dEf = (ctx->sp[D.P0].d.E_form + ctx->sp[D.P1].d.E_form) -
                    (A.d.E_form + ctx->sp[D.B].d.E_form);
        }
        D.dEf_fix = to_fix(D.dEf);
        D.Ea_fix = to_fix(D.Ea);
    }
    // species pairs that some QK dissociation or exchange can take (the
    // FP32 relaxation kernel skips the QK test for all others)
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
            uint32_t qk = 0u;
            for (int i = 0; i < n; ++i) {
                const DevReaction& D = C.rx[i];
                if (D.model == HCAO_MODEL_TCE) continue;
                if (D.type == HCAO_DISS && (D.A == a || D.A == b)) qk = 1u;
                if (D.type == HCAO_EXCH && ((D.A == a && D.B == b) || (D.A == b && D.B == a))) qk = 1u;
            }
            C.pair[a * MAXS + b].qk = qk;
        }
    C.n_reactions = n;
    C.creates = creates;
    C.has_recomb = n_rec > 0 ? 1 : 0;
    ctx->n_reactions = n;
    ctx->n_recomb = n_rec;
    if (n_rec > 0) {
        hcao_status st = build_recomb_tables(ctx);
        if (st != HCAO_OK) return st;
    }
    {
        hcao_status st = build_tce_tables(ctx);
        if (st != HCAO_OK) return st;
    }
    {
        hcao_status st = build_split_tables(ctx);
        if (st != HCAO_OK) return st;
    }
    return upload_consts(ctx);
}

hcao_status hcao_add_reservoir(hcao_ctx* ctx, int n_cells, double cell_volume, double weight, double dt,
                               uint64_t seed, double T_sgmax, int* id) {
    DeviceScope ds_(ctx);
    SERVE_GUARD(ctx);
    if (!ctx || n_cells < 1 || !(cell_volume > 0) || !(weight > 0) || !(dt > 0) || !(T_sgmax > 0) || !id)
        return fail(ctx, HCAO_EINVAL, "add_reservoir: bad arguments");
    if (ctx->n_species == 0) return fail(ctx, HCAO_EINVAL, "add_reservoir: species first");
    Reservoir r;
    r.live = true;
    r.n_cells = n_cells;
    r.Vc = cell_volume;
    r.w = weight;
    r.dt = dt;
    r.seed = seed;
    r.T_sgmax = T_sgmax;
    ctx->res.push_back(r);
    *id = (int)ctx->res.size() - 1;
    return HCAO_OK;
}

hcao_status hcao_set_cell_base(hcao_ctx* ctx, int id, uint32_t base) {
    DeviceScope ds_(ctx);
    SERVE_GUARD(ctx);
    if (!ctx) return HCAO_EINVAL;
    Reservoir* r = get_res(ctx, id);
    if (!r) return fail(ctx, HCAO_ENOTFOUND, "set_cell_base: no such reservoir");
    if (r->loaded) return fail(ctx, HCAO_EINVAL, "set_cell_base: before the reservoir is loaded");
    if ((uint64_t)base + (uint64_t)r->n_cells > 0x100000000ull)
        return fail(ctx, HCAO_EINVAL, "set_cell_base: cell indices beyond 32 bits");
    r->cell_base = base;
    return HCAO_OK;
}

hcao_status hcao_remove_reservoir(hcao_ctx* ctx, int id) {
    DeviceScope ds_(ctx);
    SERVE_GUARD(ctx);
    if (!ctx) return HCAO_EINVAL;
    Reservoir* r = get_res(ctx, id);
    if (!r) return fail(ctx, HCAO_ENOTFOUND, "remove_reservoir: no such reservoir");
    CU(cudaStreamSynchronize(ctx->stream));
    if (r->recs) cudaFreeAsync(r->recs, ctx->stream);
    r->recs = nullptr;
    const bool was_loaded = r->loaded;
    r->live = false;
    r->loaded = false;
    if (ctx->d_res && id < ctx->d_res_cap) {
        DevRes dr{};
        dr.active = 0;
        CU(cudaMemcpyAsync(ctx->d_res + id, &dr, sizeof dr, cudaMemcpyHostToDevice, ctx->stream));
    }
    if (was_loaded) return relayout(ctx, -1, nullptr);
    return HCAO_OK;
}

hcao_status hcao_cell_sort(hcao_ctx* ctx, const uint32_t* keys, int64_t n, uint32_t n_cells, uint32_t* perm,
                           uint32_t* offsets) {
    DeviceScope ds_(ctx);
    if (!ctx || n < 0 || n > 0xFFFFFFFFll || n_cells < 1 || (n > 0 && (!keys || !perm)) || !offsets)
        return fail(ctx, HCAO_EINVAL, "cell_sort: bad arguments");
    hcao_status st = ensure_scratch(ctx, sort_scratch_words(n, n_cells));
    if (st != HCAO_OK) return st;
    CU(cell_sort(keys, n, n_cells, perm, offsets, ctx->d_scratch, ctx->stream, &ctx->launches));
    return HCAO_OK;
}

// One load path for FP64 (v) or FP32 (vf) host velocities, exactly one given.
static hcao_status load_impl(hcao_ctx* ctx, int id, int64_t n, const double* v, const float* vf,
                             const uint8_t* qn, const int32_t* species, const int32_t* cell) {
    DeviceScope ds_(ctx);
    SERVE_GUARD(ctx);
    if (!ctx) return HCAO_EINVAL;
    Reservoir* r = get_res(ctx, id);
    if (!r) return fail(ctx, HCAO_ENOTFOUND, "load_particles: no such reservoir");
    if (n < 0 || n > 0x7FFFFFFFll || (n > 0 && ((!v && !vf) || !qn || !species || !cell)))
        return fail(ctx, HCAO_EINVAL, "load_particles: bad arguments");
    CU(cudaStreamSynchronize(ctx->stream));
    // stage the host arrays; validate and count on the device (a sort by cell
    // gives the per-cell counts); host work stays O(cells)
    double* dv = nullptr;
    float* dvf = nullptr;
    uint8_t* dq = nullptr;
    int32_t* ds = nullptr;
    uint32_t *dk = nullptr, *dperm = nullptr, *doff = nullptr, *dflags = nullptr;
    uint64_t* dslot = nullptr;
    auto release = [&]() {
        dfree(ctx, dv); dfree(ctx, dvf); dfree(ctx, dq); dfree(ctx, ds); dfree(ctx, dk);
        dfree(ctx, dperm); dfree(ctx, doff); dfree(ctx, dslot); dfree(ctx, dflags);
    };
    std::vector<uint32_t> off((size_t)r->n_cells + 1, 0u);
    uint32_t flags[2] = {0u, 0u};
    if (n > 0) {
        if (vf) CU(dalloc(ctx, &dvf, (size_t)n * 3));
        else CU(dalloc(ctx, &dv, (size_t)n * 3));
        CU(dalloc(ctx, &dq, (size_t)n * 16));
        CU(dalloc(ctx, &ds, (size_t)n));
        CU(dalloc(ctx, &dk, (size_t)n));
        CU(dalloc(ctx, &dperm, (size_t)n));
        CU(dalloc(ctx, &doff, (size_t)r->n_cells + 1));
        CU(dalloc(ctx, &dslot, (size_t)r->n_cells));
        CU(dalloc(ctx, &dflags, 2));
        CU(cudaMemsetAsync(dflags, 0, 2 * sizeof(uint32_t), ctx->stream));
        // The cell keys first, and their sort (safe for any key: a key out of
        // range is only misplaced, and the input is rejected below) on the
        // context's stream, while the other arrays copy on a second stream.
        if (!ctx->aux_stream) {
            CU(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
            CU(cudaEventCreateWithFlags(&ctx->ev_aux0, cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&ctx->ev_aux1, cudaEventDisableTiming));
        }
        CU(cudaEventRecord(ctx->ev_aux0, ctx->stream));  // the staging buffers exist
        CU(cudaStreamWaitEvent(ctx->aux_stream, ctx->ev_aux0, 0));
        // on any early return below, the second stream's copies finish first:
        // they read the caller's host arrays, which the caller may release
        struct AuxDrain {
            cudaStream_t s;
            ~AuxDrain() { cudaStreamSynchronize(s); }
        } aux_drain{ctx->aux_stream};
        CU(cudaMemcpyAsync(dk, cell, sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
        if (vf) CU(cudaMemcpyAsync(dvf, vf, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, ctx->aux_stream));
        else CU(cudaMemcpyAsync(dv, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->aux_stream));
        CU(cudaMemcpyAsync(dq, qn, (size_t)16 * n, cudaMemcpyHostToDevice, ctx->aux_stream));
        CU(cudaMemcpyAsync(ds, species, sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->aux_stream));
        CU(cudaEventRecord(ctx->ev_aux1, ctx->aux_stream));
        hcao_status st = hcao_cell_sort(ctx, dk, n, (uint32_t)r->n_cells, dperm, doff);
        CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_aux1, 0));  // every array is on the device
        if (st != HCAO_OK) {
            CU(cudaStreamSynchronize(ctx->stream));
            release();
            return st;
        }
        launch_validate_load(ctx->d_consts, r->n_cells, reinterpret_cast<const int32_t*>(dk), ds, dq, n, dflags,
                             ctx->stream);
        ctx->launches++;
        CU(cudaMemcpyAsync(flags, dflags, sizeof flags, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaMemcpyAsync(off.data(), doff, sizeof(uint32_t) * off.size(), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        if (flags[0] & (LOAD_BAD_CELL | LOAD_BAD_SPECIES)) {
            release();
            return fail(ctx, HCAO_EINVAL, (flags[0] & LOAD_BAD_CELL) ? "load_particles: cell out of range"
                                                                     : "load_particles: species out of range");
        }
        if (flags[0] & LOAD_BAD_LEVEL) {
            release();
            return fail(ctx, HCAO_ELEVEL_OVERFLOW, "load_particles: quantum number outside the level list");
        }
    }
    // capacities and slot bases
    const double f = ctx->cfg.capacity_factor;
    std::vector<DevCell> cells(r->n_cells);
    std::vector<uint64_t> slot0(r->n_cells);
    uint64_t tot = 0;
    double mx = 0.0;
    for (int a = 0; a < ctx->n_species; ++a)
        for (int b = 0; b < ctx->n_species; ++b)
            if (((flags[1] >> a) & 1u) && ((flags[1] >> b) & 1u)) {
                const double m = mean_sigma_g(ctx, a, b, r->T_sgmax);
                if (m > mx) mx = m;
            }
    // a context whose reactions neither create nor remove particles keeps
    // every cell's count for good: its cells need no spare slots
    const bool grows = ctx->hc.creates != 0;
    uint32_t max_cap = 0;
    for (int c = 0; c < r->n_cells; ++c) {
        const uint32_t count = off[c + 1] - off[c];
        uint64_t cap = grows ? (uint64_t)std::ceil(count * f) + (uint64_t)ctx->cfg.capacity_extra : (uint64_t)count;
        cap = (cap + 7) & ~(uint64_t)7;
        if (cap > max_cap) max_cap = (uint32_t)std::min<uint64_t>(cap, 0xFFFFFFFFull);
        slot0[c] = tot;
        tot += cap;
        DevCell& d = cells[c];
        std::memset(&d, 0, sizeof d);
        d.n = count;
        d.cap = (uint32_t)cap;
        d.res = (uint32_t)id;
        d.lcell = r->cell_base + (uint32_t)c;  // the cell's index in every random-number key
        d.sgmax = 2.0 * mx;  // reading A10: 2 <sigma_T g>(T_sgmax), largest pair present
    }
    const size_t rs = rec_size(ctx);
    r->total_cap = tot;
    r->max_cap = max_cap;
    r->rec_bytes = (size_t)tot * rs;
    // the old records go only now, once the new input has passed its checks;
    // until relayout completes, the cell table may point at freed records
    if (r->recs) {
        ctx->layout_ok = false;
        cudaFreeAsync(r->recs, ctx->stream);
        r->recs = nullptr;
    }
    CU(cudaMallocFromPoolAsync(&r->recs, std::max<size_t>(r->rec_bytes, 64), ctx->pool, ctx->stream));
    CU(cudaMemsetAsync(r->recs, 0, std::max<size_t>(r->rec_bytes, 64), ctx->stream));
    for (int c = 0; c < r->n_cells; ++c)
        cells[c].rec = static_cast<char*>(r->recs) + slot0[c] * rs;
    if (n > 0) {
        // scatter the staged particles into their cells' slots in sorted order
        CU(cudaMemcpyAsync(dslot, slot0.data(), sizeof(uint64_t) * r->n_cells, cudaMemcpyHostToDevice, ctx->stream));
        if (ctx->cfg.precision == HCAO_FP64)
            launch_scatter_load<double>(r->recs, dperm, doff, dslot, r->n_cells, dv, dvf, dq, ds, n, ctx->stream);
        else
            launch_scatter_load<float>(r->recs, dperm, doff, dslot, r->n_cells, dv, dvf, dq, ds, n, ctx->stream);
        ctx->launches++;
        CU(cudaGetLastError());
        release();
    }
    r->loaded = true;
    hcao_status st = relayout(ctx, id, &cells);
    if (st != HCAO_OK) return st;
    DevRes dr{};
    dr.seed = r->seed;
    dr.step = 0;
    dr.active = 1;
    dr.w = r->w;
    dr.dt = r->dt;
    dr.Vc = r->Vc;
    CU(cudaMemcpyAsync(ctx->d_res + id, &dr, sizeof dr, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return HCAO_OK;
}

hcao_status hcao_load_particles(hcao_ctx* ctx, int id, int64_t n, const double* v, const uint8_t* qn,
                                const int32_t* species, const int32_t* cell) {
    return load_impl(ctx, id, n, v, nullptr, qn, species, cell);
}

hcao_status hcao_load_particles_f32(hcao_ctx* ctx, int id, int64_t n, const float* v, const uint8_t* qn,
                                    const int32_t* species, const int32_t* cell) {
    return load_impl(ctx, id, n, nullptr, v, qn, species, cell);
}

hcao_status hcao_init_vibration(hcao_ctx* ctx, int id, double T) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    SERVE_GUARD(ctx);
    if (!ctx) return HCAO_EINVAL;
    Reservoir* r = get_res(ctx, id);
    if (!r || !r->loaded) return fail(ctx, HCAO_ENOTFOUND, "init_vibration: no loaded reservoir");
    if (!(T > 0)) return fail(ctx, HCAO_EINVAL, "init_vibration: T_vib must be > 0");
    // bends: thresholds exp(-k Theta / T), k = 1..L (i >= k <=> u <= threshold);
    // stretches: acceptance exp(-(E_i - E_0)/(k T)) per level (Eq. accept-quant)
    std::vector<double> bt, sa;
    std::vector<int> off(MAXS * MAXM, 0);
    for (int s = 0; s < ctx->n_species; ++s) {
        const HostSpecies& S = ctx->sp[s];
        for (int j = 0; j < S.n_modes; ++j) {
            if (S.bend[j]) {
                off[s * MAXM + j] = (int)bt.size();
                const double th = S.theta[j - S.d.n_stretch];
                for (size_t k = 1; k <= S.lev[j].size(); ++k) bt.push_back(std::exp(-(double)k * th / T));
            } else {
                off[s * MAXM + j] = (int)sa.size();
                for (double Ei : S.lev[j]) sa.push_back(std::exp(-(Ei - S.lev[j][0]) / (KB * T)));
            }
        }
    }
    DevTemp<double> dbt(ctx), dsa(ctx);
    DevTemp<int> doff(ctx);
    DevTemp<uint64_t> dpo(ctx);
    CU(dalloc(ctx, &dbt.p, bt.size()));
    CU(dalloc(ctx, &dsa.p, sa.size()));
    CU(dalloc(ctx, &doff.p, off.size()));
    if (!bt.empty()) CU(cudaMemcpyAsync(dbt.p, bt.data(), sizeof(double) * bt.size(), cudaMemcpyHostToDevice, ctx->stream));
    if (!sa.empty()) CU(cudaMemcpyAsync(dsa.p, sa.data(), sizeof(double) * sa.size(), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(doff.p, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, ctx->stream));
    uint64_t total = 0;
    hcao_status pst = particle_prefix(ctx, *r, &dpo.p, &total);
    if (pst != HCAO_OK) return pst;
    if (ctx->cfg.precision == HCAO_FP64)
        launch_init_vib<double>(ctx->d_cells, r->cell0, r->n_cells, dpo.p, total, ctx->d_res, id, ctx->d_consts,
                                dbt.p, dsa.p, doff.p, ctx->cfg.reject_cap, ctx->d_err, ctx->stream);
    else
        launch_init_vib<float>(ctx->d_cells, r->cell0, r->n_cells, dpo.p, total, ctx->d_res, id, ctx->d_consts,
                               dbt.p, dsa.p, doff.p, ctx->cfg.reject_cap, ctx->d_err, ctx->stream);
    ctx->launches++;
    CU(cudaGetLastError());
    return map_err(ctx);
}

hcao_status hcao_sample_lb(hcao_ctx* ctx, int sp, double Ec, uint64_t seed, int64_t n, uint8_t* host_qn,
                           uint64_t* host_trials) {
    DeviceScope ds_(ctx);
    if (!ctx || n < 0 || (n > 0 && !host_qn)) return HCAO_EINVAL;
    if (sp < 0 || sp >= ctx->n_species || ctx->sp[sp].n_modes == 0)
        return fail(ctx, HCAO_EINVAL, "sample_lb: species without vibrational modes");
    uint8_t* dq = nullptr;
    unsigned long long* dt = nullptr;
    int* dst = nullptr;
    CU(dalloc(ctx, &dq, (size_t)std::max<int64_t>(n, 1) * 16));
    CU(dalloc(ctx, &dt, 1));
    CU(dalloc(ctx, &dst, 1));
    CU(cudaMemsetAsync(dt, 0, sizeof(unsigned long long), ctx->stream));
    CU(cudaMemsetAsync(dst, 0, sizeof(int), ctx->stream));
    StepArgs a = make_args(ctx);
    if (ctx->cfg.precision == HCAO_FP64)
        launch_sample_diag<double>(a, sp, Ec, seed, n, dq, dt, dst, ctx->stream);
    else
        launch_sample_diag<float>(a, sp, Ec, seed, n, dq, dt, dst, ctx->stream);
    ctx->launches++;
    CU(cudaGetLastError());
    unsigned long long tr = 0;
    int status = 0;
    if (n > 0) CU(cudaMemcpyAsync(host_qn, dq, (size_t)n * 16, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(&tr, dt, sizeof tr, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(&status, dst, sizeof status, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, dq);
    dfree(ctx, dt);
    dfree(ctx, dst);
    if (host_trials) *host_trials = tr;
    if (status != 0) return fail(ctx, HCAO_EINVAL, "sample_lb: collision energy outside the tables");
    return map_err(ctx);
}

hcao_status hcao_set_log(hcao_ctx* ctx, int enable) {
    DeviceScope ds_(ctx);
    if (!ctx) return HCAO_EINVAL;
    ctx->log_on = enable != 0;
    if (ctx->log_on && !ctx->d_log && ctx->pair_cap > 0) CU(dalloc(ctx, &ctx->d_log, (size_t)ctx->pair_cap));
    return HCAO_OK;
}

hcao_status hcao_step(hcao_ctx* ctx, int n_steps) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    SERVE_GUARD(ctx);
    if (!ctx || n_steps < 0) return fail(ctx, HCAO_EINVAL, "step: bad arguments");
    if (ctx->n_cells_total == 0 || n_steps == 0) return HCAO_OK;
    int smem_recs = 0;
    const bool fused = use_fused(ctx, &smem_recs);
    if (ctx->step_path == HCAO_PATH_FUSED && !fused)
        return fail(ctx, HCAO_EINVAL, "step: the fused path needs FP32, no reaction that creates or removes "
                                      "particles, no per-pair log and cells of at most 4096 slots");
    if (!fused) {
        const hcao_status st = ensure_pair_buffers(ctx);
        if (st != HCAO_OK) return st;
    } else if (ctx->fused_smem_set != smem_recs) {
        CU(fused_prepare(smem_recs));
        ctx->fused_smem_set = smem_recs;
    }
    StepArgs a = make_args(ctx);
    const int block = 128;
    const int grid = ctx->sm_count * 8;
    const bool f64 = ctx->cfg.precision == HCAO_FP64;
    if (fused) {
        // the whole collision phase of a step as one kernel (one CTA per cell)
        a.fused_recs = smem_recs;  // part of the graph's key: a new shared-memory size re-captures
        if (!ctx->prof_on && ctx->use_graph) {
            if (!ctx->graph || std::memcmp(&a, &ctx->graph_args, sizeof a) != 0) {
                if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
                ctx->graph = nullptr;
                if (!ctx->cap_stream) CU(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
                cudaGraph_t g = nullptr;
                CU(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
                launch_fused(a, smem_recs, ctx->cap_stream);
                CU(cudaStreamEndCapture(ctx->cap_stream, &g));
                cudaError_t e = cudaGraphInstantiate(&ctx->graph, g, 0);
                cudaGraphDestroy(g);
                CU(e);
                ctx->graph_args = a;
            }
            for (int s = 0; s < n_steps; ++s) {
                CU(cudaGraphLaunch(ctx->graph, ctx->stream));
                ctx->launches += 1;
            }
            return HCAO_OK;
        }
        for (int s = 0; s < n_steps; ++s) {
            std::pair<cudaEvent_t, cudaEvent_t>* ev = nullptr;
            if (ctx->prof_on) {
                auto& pool = ctx->prof_ev[5];
                if (ctx->prof_used[5] == pool.size()) {
                    cudaEvent_t e0, e1;
                    CU(cudaEventCreate(&e0));
                    CU(cudaEventCreate(&e1));
                    pool.emplace_back(e0, e1);
                }
                ev = &pool[ctx->prof_used[5]++];
                CU(cudaEventRecord(ev->first, ctx->stream));
            }
            launch_fused(a, smem_recs, ctx->stream);
            ctx->launches += 1;
            if (ev) CU(cudaEventRecord(ev->second, ctx->stream));
        }
        CU(cudaGetLastError());
        return HCAO_OK;
    }
    if (!ctx->prof_on && ctx->use_graph) {
        // one step as a CUDA graph, launched n_steps times on the caller's stream
        if (!ctx->graph || std::memcmp(&a, &ctx->graph_args, sizeof a) != 0) {
            if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
            ctx->graph = nullptr;
            if (!ctx->cap_stream) CU(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            CU(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
            uint64_t in_graph = 0;
            if (f64) launch_step<double>(a, grid, block, ctx->cap_stream, &in_graph);
            else launch_step<float>(a, grid, block, ctx->cap_stream, &in_graph);
            CU(cudaStreamEndCapture(ctx->cap_stream, &g));
            ctx->graph_launches = in_graph;
            cudaError_t e = cudaGraphInstantiate(&ctx->graph, g, 0);
            cudaGraphDestroy(g);
            CU(e);
            ctx->graph_args = a;
        }
        for (int s = 0; s < n_steps; ++s) {
            CU(cudaGraphLaunch(ctx->graph, ctx->stream));
            ctx->launches += ctx->graph_launches;  // the kernels captured in the graph
        }
        return HCAO_OK;
    }
    for (int s = 0; s < n_steps; ++s) {
        if (!ctx->prof_on) {
            if (f64) launch_step<double>(a, grid, block, ctx->stream, &ctx->launches);
            else launch_step<float>(a, grid, block, ctx->stream, &ctx->launches);
            continue;
        }
        // setup, then per round select / relax / react, then finish
        int seq[2 + 3 * MAX_ROUNDS][2];
        int ns = 0;
        seq[ns][0] = 0; seq[ns++][1] = 0;
        for (int r = 0; r < a.max_rounds; ++r)
            for (int ph = 0; ph < 3; ++ph) {
                if (ph == 2 && !a.has_reactions) continue;
                seq[ns][0] = 1 + ph; seq[ns++][1] = r;
            }
        seq[ns][0] = 4; seq[ns++][1] = 0;
        for (int q = 0; q < ns; ++q) {
            const int k = seq[q][0], r = seq[q][1];
            auto& pool = ctx->prof_ev[k];
            if (ctx->prof_used[k] == pool.size()) {
                cudaEvent_t e0, e1;
                CU(cudaEventCreate(&e0));
                CU(cudaEventCreate(&e1));
                pool.emplace_back(e0, e1);
            }
            auto& ev = pool[ctx->prof_used[k]++];
            CU(cudaEventRecord(ev.first, ctx->stream));
            if (k == 0) {
                ctx->launches += launch_setup(a, ctx->stream) - 1;
                if (a.has_recomb) {
                    if (f64) launch_cellstats<double>(a, ctx->stream);
                    else launch_cellstats<float>(a, ctx->stream);
                    ctx->launches++;
                }
            } else if (k == 4) {
                if (f64) launch_finish<double>(a, ctx->stream);
                else launch_finish<float>(a, ctx->stream);
                ctx->launches += ctx->hc.creates ? 2 : 1;
                if (a.has_recomb) {
                    if (f64) launch_compact<double>(a, ctx->stream);
                    else launch_compact<float>(a, ctx->stream);
                    ctx->launches++;
                }
            } else {
                if (f64) launch_phase<double>(a, r, k - 1, grid, ctx->stream);
                else launch_phase<float>(a, r, k - 1, grid, ctx->stream);
                if (k == 1 && !f64 && a.qorder) ctx->launches++;  // the FP32 queue placement after the selection
            }
            CU(cudaEventRecord(ev.second, ctx->stream));
            ctx->launches++;
        }
    }
    CU(cudaGetLastError());
    return HCAO_OK;
}

hcao_status hcao_set_step_path(hcao_ctx* ctx, int path) {
    DeviceScope ds_(ctx);
    if (!ctx || path < HCAO_PATH_AUTO || path > HCAO_PATH_FUSED) return fail(ctx, HCAO_EINVAL, "set_step_path: bad path");
    SERVE_GUARD(ctx);
    ctx->step_path = path;
    return HCAO_OK;
}

hcao_status hcao_get_step_path(const hcao_ctx* ctx, int* path) {
    if (!ctx || !path) return HCAO_EINVAL;
    *path = use_fused(ctx, nullptr) ? HCAO_PATH_FUSED : HCAO_PATH_QUEUE;
    return HCAO_OK;
}

hcao_status hcao_set_profiling(hcao_ctx* ctx, int enable) {
    DeviceScope ds_(ctx);
    if (!ctx) return HCAO_EINVAL;
    ctx->prof_on = enable != 0;
    for (int k = 0; k < hcao_ctx::NPROF; ++k) {
        ctx->prof_used[k] = 0;
        ctx->prof_ms[k] = 0.0;
        ctx->prof_n[k] = 0;
    }
    return HCAO_OK;
}

hcao_status hcao_read_profile(hcao_ctx* ctx, double* ms, uint64_t* launches, int max, int* n_out) {
    DeviceScope ds_(ctx);
    if (!ctx || !ms || !launches || max < 1) return HCAO_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < hcao_ctx::NPROF; ++k) {
        for (size_t i = 0; i < ctx->prof_used[k]; ++i) {
            float t = 0.0f;
            CU(cudaEventElapsedTime(&t, ctx->prof_ev[k][i].first, ctx->prof_ev[k][i].second));
            ctx->prof_ms[k] += t;
            ctx->prof_n[k]++;
        }
        ctx->prof_used[k] = 0;
    }
    const int n = std::min(max, hcao_ctx::NPROF);
    for (int k = 0; k < n; ++k) {
        ms[k] = ctx->prof_ms[k];
        launches[k] = ctx->prof_n[k];
    }
    if (n_out) *n_out = n;
    return HCAO_OK;
}

hcao_status hcao_autotune(hcao_ctx* ctx, int steps_per_candidate, int* chosen) {
    DeviceScope ds_(ctx);
    if (!ctx || steps_per_candidate < 1) return HCAO_EINVAL;
    if (ctx->n_cells_total == 0) return HCAO_OK;
    const int sm = ctx->sm_count;
    const int sel_cand[4] = {2 * sm, 4 * sm, 8 * sm, 16 * sm};
    const int rel_cand[3] = {4 * sm, 5 * sm, 8 * sm};
    const bool was_prof = ctx->prof_on;
    ctx->prof_on = true;
    // ms of profile classes k (and k2, when >= 0) over one candidate's steps
    auto time_phase = [&](int k, int k2 = -1) -> double {
        for (int j = 0; j < hcao_ctx::NPROF; ++j) { ctx->prof_used[j] = 0; ctx->prof_ms[j] = 0; ctx->prof_n[j] = 0; }
        if (hcao_step(ctx, steps_per_candidate) != HCAO_OK) return 1e30;
        double ms[hcao_ctx::NPROF];
        uint64_t n[hcao_ctx::NPROF];
        int got = 0;
        if (hcao_read_profile(ctx, ms, n, hcao_ctx::NPROF, &got) != HCAO_OK) return 1e30;
        return ms[k] + (k2 >= 0 ? ms[k2] : 0.0);
    };
    double best = 1e30;
    int bs = ctx->grid_select, br = ctx->grid_relax;
    for (int c : sel_cand) {
        ctx->grid_select = c;
        const double t = time_phase(1);
        if (t < best) { best = t; bs = c; }
    }
    ctx->grid_select = bs;
    best = 1e30;
    for (int c : rel_cand) {
        ctx->grid_relax = c;
        const double t = time_phase(2);
        if (t < best) { best = t; br = c; }
    }
    ctx->grid_relax = br;
    // the FP32 relaxation queue's placement by work class: kept where it pays
    // (selection with the placement + relaxation, against both without it)
    if (ctx->cfg.precision == HCAO_FP32 && ctx->hc.n_cls > 1 && !use_fused(ctx, nullptr)) {
        ctx->qorder_off = false;
        const double t_on = time_phase(1, 2);
        ctx->qorder_off = true;
        const double t_off = time_phase(1, 2);
        ctx->qorder_off = t_off < t_on;
    }
    ctx->prof_on = was_prof;
    for (int j = 0; j < hcao_ctx::NPROF; ++j) { ctx->prof_used[j] = 0; ctx->prof_ms[j] = 0; ctx->prof_n[j] = 0; }
    if (chosen) {
        chosen[0] = bs;
        chosen[1] = br;
        chosen[2] = (ctx->hc.n_cls > 1 && !ctx->qorder_off) ? 1 : 0;
    }
    return map_err(ctx);
}

hcao_status hcao_read_work(hcao_ctx* ctx, uint64_t* out, int max, int* n_out) {
    DeviceScope ds_(ctx);
    if (!ctx || !out || max < 1) return HCAO_EINVAL;
    unsigned long long w[4];
    CU(cudaMemcpyAsync(w, ctx->d_work, sizeof w, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const int n = std::min(max, 4);
    for (int i = 0; i < n; ++i) out[i] = w[i];
    if (n_out) *n_out = n;
    return HCAO_OK;
}

hcao_status hcao_sync(hcao_ctx* ctx) {
    DeviceScope ds_(ctx);
    if (!ctx) return HCAO_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream));
    return map_err(ctx);
}

hcao_status hcao_count(hcao_ctx* ctx, int id, int64_t* n) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    if (!ctx || !n) return HCAO_EINVAL;
    Reservoir* r = get_res(ctx, id);
    if (!r) return fail(ctx, HCAO_ENOTFOUND, "count: no such reservoir");
    *n = 0;
    if (!r->loaded) return HCAO_OK;
    DevTemp<uint64_t> dpo(ctx);
    uint64_t total = 0;
    hcao_status st = particle_prefix(ctx, *r, &dpo.p, &total);
    if (st != HCAO_OK) return st;
    *n = (int64_t)total;
    return map_err(ctx);
}

hcao_status hcao_read_particles(hcao_ctx* ctx, int id, double* v, uint8_t* qn, int32_t* species, int32_t* cell) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    if (!ctx) return HCAO_EINVAL;
    Reservoir* r = get_res(ctx, id);
    if (!r || !r->loaded) return fail(ctx, HCAO_ENOTFOUND, "read_particles: no loaded reservoir");
    DevTemp<uint64_t> doff(ctx);
    uint64_t n = 0;
    hcao_status st = particle_prefix(ctx, *r, &doff.p, &n);
    if (st != HCAO_OK) return st;
    if (n == 0) return map_err(ctx);
    DevTemp<double> dv(ctx);
    DevTemp<uint8_t> dq(ctx);
    DevTemp<int32_t> ds(ctx), dc(ctx);
    CU(dalloc(ctx, &dv.p, (size_t)n * 3));
    CU(dalloc(ctx, &dq.p, (size_t)n * 16));
    CU(dalloc(ctx, &ds.p, (size_t)n));
    CU(dalloc(ctx, &dc.p, (size_t)n));
    if (ctx->cfg.precision == HCAO_FP64)
        launch_pack<double>(ctx->d_cells, r->cell0, r->n_cells, doff.p, n, ctx->d_consts, dv.p, dq.p, ds.p, dc.p, ctx->stream);
    else
        launch_pack<float>(ctx->d_cells, r->cell0, r->n_cells, doff.p, n, ctx->d_consts, dv.p, dq.p, ds.p, dc.p, ctx->stream);
    ctx->launches++;
    CU(cudaGetLastError());
    if (v) CU(cudaMemcpyAsync(v, dv.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (qn) CU(cudaMemcpyAsync(qn, dq.p, (size_t)16 * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (species) CU(cudaMemcpyAsync(species, ds.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (cell) CU(cudaMemcpyAsync(cell, dc.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return map_err(ctx);
}

hcao_status hcao_read_moments(hcao_ctx* ctx, int id, hcao_moments* out) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    if (!ctx || !out) return HCAO_EINVAL;
    Reservoir* r = get_res(ctx, id);
    if (!r || !r->loaded) return fail(ctx, HCAO_ENOTFOUND, "read_moments: no loaded reservoir");
    DevTemp<double> dacc(ctx);
    DevTemp<unsigned long long> dcnt(ctx);
    DevTemp<uint64_t> dpo(ctx);
    CU(dalloc(ctx, &dacc.p, 5 + 2 * MAXS));
    CU(dalloc(ctx, &dcnt.p, MAXS));
    CU(cudaMemsetAsync(dacc.p, 0, sizeof(double) * (5 + 2 * MAXS), ctx->stream));
    CU(cudaMemsetAsync(dcnt.p, 0, sizeof(unsigned long long) * MAXS, ctx->stream));
    // the particle prefix on the device: no copy of the cell table, and the
    // total stays there too (the kernel reads it; the grid is the full one)
    CU(dalloc(ctx, &dpo.p, (size_t)r->n_cells + 1));
    launch_cell_prefix(ctx->d_cells, r->cell0, r->n_cells, dpo.p, ctx->stream);
    ctx->launches++;
    const uint64_t total = ~0ull;
    if (ctx->cfg.precision == HCAO_FP64)
        launch_moments<double>(ctx->d_cells, r->cell0, r->n_cells, dpo.p, total, ctx->d_consts, ctx->d_lev64,
                               ctx->d_levfix, dacc.p, dcnt.p, ctx->stream);
    else
        launch_moments<float>(ctx->d_cells, r->cell0, r->n_cells, dpo.p, total, ctx->d_consts, ctx->d_lev64,
                              ctx->d_levfix, dacc.p, dcnt.p, ctx->stream);
    ctx->launches++;
    CU(cudaGetLastError());
    double acc[5 + 2 * MAXS];
    unsigned long long cnt[MAXS];
    CU(cudaMemcpyAsync(acc, dacc.p, sizeof acc, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(cnt, dcnt.p, sizeof cnt, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    std::memset(out, 0, sizeof *out);
    double M = 0.0;
    int64_t N = 0;
    for (int s = 0; s < MAXS; ++s) {
        out->n[s] = (int64_t)cnt[s];
        N += out->n[s];
        if (s < ctx->n_species) M += ctx->sp[s].d.mass * (double)cnt[s];
    }
    for (int d = 0; d < 3; ++d) out->momentum[d] = acc[d];
    out->E_tr = acc[3];
    out->E_form = acc[4];
    for (int s = 0; s < MAXS; ++s) out->E_vib[s] = acc[5 + s];
    if (N > 0 && M > 0) {
        const double p2 = acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2];
        out->T_tr = 2.0 / 3.0 * (acc[3] - 0.5 * p2 / M) / ((double)N * KB);
    }
    for (int s = 0; s < ctx->n_species; ++s)
        if (cnt[s] > 0 && ctx->sp[s].n_modes > 0)
            out->T_vib[s] = tvib_host(ctx->sp[s], acc[5 + s] / (double)cnt[s] - ctx->sp[s].zpe);
    for (int s = 0; s < MAXS; ++s) out->E_rot[s] = acc[5 + MAXS + s];
    for (int s = 0; s < ctx->n_species; ++s)
        if (cnt[s] > 0 && ctx->sp[s].d.rot_dof > 0)
            out->T_rot[s] = 2.0 * (acc[5 + MAXS + s] / (double)cnt[s]) / ((double)ctx->sp[s].d.rot_dof * KB);
    return map_err(ctx);
}

// rotational energies in canonical order: out of the records (to_records 0)
// or into them (1)
hcao_status erot_copy(hcao_ctx* ctx, int id, double* host, int to_records) {
    Reservoir* r = get_res(ctx, id);
    if (!r || !r->loaded) return fail(ctx, HCAO_ENOTFOUND, "rotation: no loaded reservoir");
    DevTemp<uint64_t> dpo(ctx);
    DevTemp<double> de(ctx);
    uint64_t total = 0;
    hcao_status pst = particle_prefix(ctx, *r, &dpo.p, &total);
    if (pst != HCAO_OK) return pst;
    if (total == 0) return map_err(ctx);
    CU(dalloc(ctx, &de.p, (size_t)total));
    if (to_records) CU(cudaMemcpyAsync(de.p, host, sizeof(double) * total, cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->cfg.precision == HCAO_FP64)
        launch_erot<double>(ctx->d_cells, r->cell0, r->n_cells, dpo.p, total, ctx->d_consts, de.p, to_records,
                            ctx->stream);
    else
        launch_erot<float>(ctx->d_cells, r->cell0, r->n_cells, dpo.p, total, ctx->d_consts, de.p, to_records,
                           ctx->stream);
    ctx->launches++;
    CU(cudaGetLastError());
    if (!to_records) CU(cudaMemcpyAsync(host, de.p, sizeof(double) * total, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return map_err(ctx);
}

hcao_status hcao_read_erot(hcao_ctx* ctx, int id, double* host_erot) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    if (!ctx || !host_erot) return HCAO_EINVAL;
    return erot_copy(ctx, id, host_erot, 0);
}

hcao_status hcao_load_erot(hcao_ctx* ctx, int id, const double* host_erot) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    SERVE_GUARD(ctx);
    if (!ctx || !host_erot) return HCAO_EINVAL;
    return erot_copy(ctx, id, const_cast<double*>(host_erot), 1);
}

hcao_status hcao_init_rotation(hcao_ctx* ctx, int id, double T_rot) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    SERVE_GUARD(ctx);
    if (!ctx || !(T_rot >= 0.0)) return fail(ctx, HCAO_EINVAL, "init_rotation: bad arguments");
    Reservoir* r = get_res(ctx, id);
    if (!r || !r->loaded) return fail(ctx, HCAO_ENOTFOUND, "init_rotation: no loaded reservoir");
    DevTemp<uint64_t> dpo(ctx);
    uint64_t total = 0;
    hcao_status pst = particle_prefix(ctx, *r, &dpo.p, &total);
    if (pst != HCAO_OK) return pst;
    if (ctx->cfg.precision == HCAO_FP64)
        launch_init_rot<double>(ctx->d_cells, r->cell0, r->n_cells, dpo.p, total, ctx->d_res, id, ctx->d_consts,
                                T_rot, ctx->stream);
    else
        launch_init_rot<float>(ctx->d_cells, r->cell0, r->n_cells, dpo.p, total, ctx->d_res, id, ctx->d_consts,
                               T_rot, ctx->stream);
    ctx->launches++;
    CU(cudaGetLastError());
    return map_err(ctx);
}

hcao_status hcao_read_level_populations(hcao_ctx* ctx, int id, int sp, int mode, uint64_t* counts, int max_levels) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    if (!ctx || !counts || max_levels < 1) return HCAO_EINVAL;
    Reservoir* r = get_res(ctx, id);
    if (!r || !r->loaded) return fail(ctx, HCAO_ENOTFOUND, "read_level_populations: no loaded reservoir");
    if (sp < 0 || sp >= ctx->n_species || mode < 0 || mode >= ctx->sp[sp].n_modes)
        return fail(ctx, HCAO_EINVAL, "read_level_populations: bad species or mode");
    DevTemp<unsigned long long> dh(ctx);
    DevTemp<uint64_t> dpo(ctx);
    CU(dalloc(ctx, &dh.p, MAXL));
    CU(cudaMemsetAsync(dh.p, 0, sizeof(unsigned long long) * MAXL, ctx->stream));
    uint64_t total = 0;
    hcao_status pst = particle_prefix(ctx, *r, &dpo.p, &total);
    if (pst != HCAO_OK) return pst;
    if (ctx->cfg.precision == HCAO_FP64)
        launch_levelpop<double>(ctx->d_cells, r->cell0, r->n_cells, dpo.p, total, sp, mode, dh.p, ctx->stream);
    else
        launch_levelpop<float>(ctx->d_cells, r->cell0, r->n_cells, dpo.p, total, sp, mode, dh.p, ctx->stream);
    ctx->launches++;
    CU(cudaGetLastError());
    unsigned long long h[MAXL];
    CU(cudaMemcpyAsync(h, dh.p, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < max_levels; ++i) counts[i] = i < MAXL ? (uint64_t)h[i] : 0;
    return map_err(ctx);
}

hcao_status hcao_read_counters(hcao_ctx* ctx, int id, uint64_t* out, int max, int* n_out) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    if (!ctx || !out || max < 1) return HCAO_EINVAL;
    Reservoir* r = get_res(ctx, id);
    if (!r || !r->loaded) return fail(ctx, HCAO_ENOTFOUND, "read_counters: no loaded reservoir");
    // summed over the reservoir's cells on the device; NCNT words come back
    DevTemp<unsigned long long> dsum(ctx);
    CU(dalloc(ctx, &dsum.p, NCNT));
    CU(cudaMemsetAsync(dsum.p, 0, sizeof(unsigned long long) * NCNT, ctx->stream));
    launch_sum_counters(ctx->d_cellcnt, r->cell0, r->n_cells, NCNT,
                        dsum.p, ctx->stream);
    ctx->launches++;
    unsigned long long h[NCNT];
    CU(cudaMemcpyAsync(h, dsum.p, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    DevRes dr{};
    CU(cudaMemcpyAsync(&dr, ctx->d_res + id, sizeof dr, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const int n = std::min(max, 8 + ctx->n_reactions);
    for (int i = 0; i < n; ++i) out[i] = h[i];
    if (n > CNT_STEPS) out[CNT_STEPS] = dr.step;
    if (n_out) *n_out = n;
    return map_err(ctx);
}

hcao_status hcao_read_reaction_counts(hcao_ctx* ctx, int id, uint64_t* out, int n) {
    DeviceScope ds_(ctx);
    if (!ctx || !out || n < 0) return HCAO_EINVAL;
    uint64_t buf[8 + MAXR];
    int got = 0;
    hcao_status st = hcao_read_counters(ctx, id, buf, 8 + MAXR, &got);
    if (st != HCAO_OK) return st;
    for (int i = 0; i < n; ++i) out[i] = (8 + i < got) ? buf[8 + i] : 0;
    return HCAO_OK;
}

hcao_status hcao_read_cell_sgmax(hcao_ctx* ctx, int id, double* out) {
    DeviceScope ds_(ctx);
    LAYOUT_GUARD(ctx);
    if (!ctx || !out) return HCAO_EINVAL;
    Reservoir* r = get_res(ctx, id);
    if (!r || !r->loaded) return fail(ctx, HCAO_ENOTFOUND, "read_cell_sgmax: no loaded reservoir");
    std::vector<DevCell> cells;
    hcao_status st = read_cells(ctx, *r, cells);
    if (st != HCAO_OK) return st;
    for (int c = 0; c < r->n_cells; ++c) out[c] = cells[c].sgmax;
    return map_err(ctx);
}

hcao_status hcao_read_log(hcao_ctx* ctx, hcao_log_rec* out, int64_t max, int64_t* n_out) {
    DeviceScope ds_(ctx);
    if (!ctx || !n_out) return HCAO_EINVAL;
    *n_out = 0;
    if (!ctx->log_on) return fail(ctx, HCAO_EINVAL, "read_log: logging is off");
    if (!ctx->d_log) return HCAO_OK;  // no step since logging was switched on
    uint32_t tot[MAX_ROUNDS + 2];
    CU(cudaMemcpyAsync(tot, ctx->d_totals, sizeof tot, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const int64_t n = out ? std::min<int64_t>(max, tot[MAX_ROUNDS]) : (int64_t)tot[MAX_ROUNDS];
    if (n > 0 && out)
        CU(cudaMemcpyAsync(out, ctx->d_log, sizeof(hcao_log_rec) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *n_out = n;
    return map_err(ctx);
}

hcao_status hcao_level_energy(const hcao_ctx* ctx, int sp, int mode, int level, double* out) {
    if (!ctx || !out || sp < 0 || sp >= ctx->n_species || mode < 0 || mode >= ctx->sp[sp].n_modes ||
        level < 0 || level >= (int)ctx->sp[sp].lev[mode].size())
        return HCAO_EINVAL;
    *out = ctx->sp[sp].lev[mode][level];
    return HCAO_OK;
}

hcao_status hcao_n_levels(const hcao_ctx* ctx, int sp, int mode, int* out) {
    if (!ctx || !out || sp < 0 || sp >= ctx->n_species || mode < 0 || mode >= ctx->sp[sp].n_modes)
        return HCAO_EINVAL;
    *out = (int)ctx->sp[sp].lev[mode].size();
    return HCAO_OK;
}


}  // extern "C"

// ===================================================================== serving
// Continuous batching: queued jobs are admitted between engine iterations as
// the HBM budget and the resident-job limit allow; every iteration advances
// all resident jobs together by K steps (one graph launch per step), K the
// fewest steps any resident job still needs (capped); finished jobs are read
// back and their reservoirs freed.

static int64_t job_bytes(const hcao_ctx* ctx, const hcao_job& j) {
    const double f = ctx->cfg.capacity_factor;
    const int64_t cap = (int64_t)std::ceil((double)j.n * f) + (int64_t)ctx->cfg.capacity_extra * j.n_cells +
                        8 * (int64_t)j.n_cells;
    const int64_t rec = ctx->cfg.precision == HCAO_FP64 ? 64 : 32;
    // per pair slot: event word, relaxation queue (two entries: its FP32 regions), reaction queue, scratch record
    const int64_t pair = (int64_t)ctx->cfg.max_rounds * (cap / 2 + j.n_cells) * (4 + 2 * 16 + 16 + rec);
    return cap * rec + pair + (int64_t)j.n_cells * (int64_t)(sizeof(DevCell) + 8 * NCNT) +
           j.n * 48;  // staging of the host arrays during the load
}

static void serve_fail(hcao_ctx* ctx, const std::shared_ptr<Job>& jb, int status) {
    std::lock_guard<std::mutex> lock(ctx->serve_mu);
    jb->state = 3;
    jb->result.status = status;
    jb->result.t_done = now_s();
}

static void serve_loop(hcao_ctx* ctx) {
    tl_serve_engine = true;
    cudaSetDevice(ctx->cfg.device);  // the engine's own thread: the context's device throughout
    for (;;) {
        // ---- admission
        std::vector<std::shared_ptr<Job>> admit;
        double t0 = now_s();
        {
            std::unique_lock<std::mutex> lock(ctx->serve_mu);
            if (ctx->serve_active.empty() && ctx->serve_queue.empty()) {
                if (ctx->serve_stop) return;
                ctx->serve_cv.wait_for(lock, std::chrono::milliseconds(20));
                ctx->serve_t[3] += now_s() - t0;
                continue;
            }
            while (!ctx->serve_queue.empty() && (int)ctx->serve_active.size() + (int)admit.size() < ctx->serve_max_active) {
                auto& jb = ctx->serve_queue.front();
                if (ctx->serve_used + jb->est_bytes > ctx->serve_budget && !(ctx->serve_active.empty() && admit.empty()))
                    break;  // wait for memory (a job larger than the budget runs alone)
                ctx->serve_used += jb->est_bytes;
                admit.push_back(jb);
                ctx->serve_queue.pop_front();
            }
        }
        for (auto& jb : admit) {
            const hcao_job& j = jb->spec;
            int rid = -1;
            hcao_status st = hcao_add_reservoir(ctx, j.n_cells, j.cell_volume, j.weight, j.dt, j.seed, j.T_sgmax, &rid);
            if (st == HCAO_OK)
                st = hcao_load_particles(ctx, rid, j.n, jb->v.data(), jb->qn.data(), jb->sp.data(), jb->cell.data());
            if (st == HCAO_OK && j.T_vib > 0) st = hcao_init_vibration(ctx, rid, j.T_vib);
            if (st != HCAO_OK) {
                if (rid >= 0) hcao_remove_reservoir(ctx, rid);
                {
                    std::lock_guard<std::mutex> lock(ctx->serve_mu);
                    ctx->serve_used -= jb->est_bytes;
                }
                serve_fail(ctx, jb, st);
                continue;
            }
            jb->v.clear(); jb->v.shrink_to_fit();
            jb->qn.clear(); jb->qn.shrink_to_fit();
            jb->sp.clear(); jb->sp.shrink_to_fit();
            jb->cell.clear(); jb->cell.shrink_to_fit();
            jb->res = rid;
            jb->steps_left = j.n_steps;
            std::lock_guard<std::mutex> lock(ctx->serve_mu);
            jb->state = 1;
            jb->result.t_admit = now_s();
            ctx->serve_active.push_back(jb);
        }
        {
            const double t1 = now_s();
            ctx->serve_t[0] += t1 - t0;
            t0 = t1;
        }
        if (ctx->serve_active.empty()) continue;
        // ---- one engine iteration: every resident job advances K steps
        int K = ctx->serve_max_batch_steps;
        for (auto& jb : ctx->serve_active) K = std::min(K, jb->steps_left);
        if (K > 0) {
            hcao_status st = hcao_step(ctx, K);
            if (st == HCAO_OK) st = hcao_sync(ctx);
            if (st != HCAO_OK) {  // a device error fails every resident job
                for (auto& jb : ctx->serve_active) {
                    hcao_remove_reservoir(ctx, jb->res);
                    serve_fail(ctx, jb, st);
                }
                // the error word is sticky: clear it for the jobs that follow
                cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream);
                cudaStreamSynchronize(ctx->stream);
                std::lock_guard<std::mutex> lock(ctx->serve_mu);
                for (auto& jb : ctx->serve_active) ctx->serve_used -= jb->est_bytes;
                ctx->serve_active.clear();
                continue;
            }
            for (auto& jb : ctx->serve_active) jb->steps_left -= K;
            ctx->serve_iterations++;
        }
        {
            const double t1 = now_s();
            ctx->serve_t[1] += t1 - t0;
            t0 = t1;
        }
        // ---- retirement
        std::vector<std::shared_ptr<Job>> keep;
        for (auto& jb : ctx->serve_active) {
            bool cancelled;
            {
                std::lock_guard<std::mutex> lock(ctx->serve_mu);
                cancelled = jb->cancel;
            }
            if (cancelled) {
                hcao_remove_reservoir(ctx, jb->res);
                std::lock_guard<std::mutex> lock(ctx->serve_mu);
                ctx->serve_used -= jb->est_bytes;
                jb->result.status = HCAO_ECANCELLED;
                jb->result.t_done = now_s();
                jb->state = 3;
                continue;
            }
            if (jb->steps_left > 0) { keep.push_back(jb); continue; }
            hcao_job_result r = jb->result;
            hcao_status st = hcao_read_moments(ctx, jb->res, &r.moments);
            int got = 0;
            if (st == HCAO_OK) st = hcao_read_counters(ctx, jb->res, r.counters, 8 + MAXR, &got);
            if (st == HCAO_OK) st = hcao_count(ctx, jb->res, &r.n_particles);
            hcao_remove_reservoir(ctx, jb->res);
            std::lock_guard<std::mutex> lock(ctx->serve_mu);
            ctx->serve_used -= jb->est_bytes;
            r.status = st;
            r.steps = jb->spec.n_steps;
            r.t_done = now_s();
            jb->result = r;
            jb->state = st == HCAO_OK ? 2 : 3;
        }
        ctx->serve_active.swap(keep);
        ctx->serve_t[2] += now_s() - t0;
    }
}

extern "C" {

hcao_status hcao_serve_start(hcao_ctx* ctx, int64_t hbm_budget_bytes, int max_active, int max_batch_steps) {
    DeviceScope ds_(ctx);
    if (!ctx || max_active < 0 || max_batch_steps < 0) return HCAO_EINVAL;
    if (ctx->n_species == 0) return fail(ctx, HCAO_EINVAL, "serve_start: species first");
    if (ctx->serve_running) return fail(ctx, HCAO_EBUSY, "serve_start: already serving");
    for (auto& r : ctx->res)
        if (r.live) return fail(ctx, HCAO_EINVAL, "serve_start: the context must hold no reservoir");
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    ctx->serve_budget = hbm_budget_bytes > 0 ? hbm_budget_bytes : (int64_t)(0.8 * (double)free_b);
    ctx->serve_max_active = max_active > 0 ? max_active : 256;
    ctx->serve_max_batch_steps = max_batch_steps > 0 ? max_batch_steps : 8;
    ctx->serve_used = 0;
    for (double& t : ctx->serve_t) t = 0.0;
    ctx->serve_stop = false;
    ctx->serve_running = true;
    ctx->serve_thread = std::thread(serve_loop, ctx);
    return HCAO_OK;
}

hcao_status hcao_serve_submit(hcao_ctx* ctx, const hcao_job* job, uint64_t* job_id) {
    DeviceScope ds_(ctx);
    if (!ctx || !job || !job_id || job->n < 0 || job->n_cells < 1 || job->n_steps < 0 ||
        (job->n > 0 && (!job->v || !job->species || !job->cell)))
        return HCAO_EINVAL;
    if (!ctx->serve_running) return HCAO_EINVAL;
    auto jb = std::make_shared<Job>();
    jb->result.t_submit = now_s();
    jb->spec = *job;
    const size_t n = (size_t)job->n;
    jb->v.assign(job->v, job->v + 3 * n);
    if (job->qn) jb->qn.assign(job->qn, job->qn + 16 * n);
    else jb->qn.assign(16 * n, 0);
    jb->sp.assign(job->species, job->species + n);
    jb->cell.assign(job->cell, job->cell + n);
    jb->spec.v = nullptr; jb->spec.qn = nullptr; jb->spec.species = nullptr; jb->spec.cell = nullptr;
    jb->est_bytes = job_bytes(ctx, *job);
    std::lock_guard<std::mutex> lock(ctx->serve_mu);
    jb->id = ctx->serve_next_id++;
    ctx->serve_jobs[jb->id] = jb;
    ctx->serve_queue.push_back(jb);
    ctx->serve_cv.notify_one();
    *job_id = jb->id;
    return HCAO_OK;
}

hcao_status hcao_serve_poll(hcao_ctx* ctx, uint64_t job_id, hcao_job_result* out) {
    DeviceScope ds_(ctx);
    if (!ctx || !out) return HCAO_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->serve_mu);
    auto it = ctx->serve_jobs.find(job_id);
    if (it == ctx->serve_jobs.end()) return HCAO_ENOTFOUND;
    const auto& jb = it->second;
    if (jb->state < 2) return HCAO_EBUSY;
    *out = jb->result;
    const hcao_status st = (hcao_status)jb->result.status;
    ctx->serve_jobs.erase(it);
    return st;
}

hcao_status hcao_serve_stop(hcao_ctx* ctx) {
    DeviceScope ds_(ctx);
    if (!ctx) return HCAO_EINVAL;
    if (!ctx->serve_running) return HCAO_OK;
    {
        std::lock_guard<std::mutex> lock(ctx->serve_mu);
        ctx->serve_stop = true;
        ctx->serve_cv.notify_all();
    }
    ctx->serve_thread.join();
    ctx->serve_running = false;
    return HCAO_OK;
}

hcao_status hcao_serve_stats(hcao_ctx* ctx, int64_t* queued, int64_t* active, int64_t* used_bytes,
                             uint64_t* iterations) {
    DeviceScope ds_(ctx);
    if (!ctx) return HCAO_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->serve_mu);
    if (queued) *queued = (int64_t)ctx->serve_queue.size();
    if (active) *active = (int64_t)ctx->serve_active.size();
    if (used_bytes) *used_bytes = ctx->serve_used;
    if (iterations) *iterations = ctx->serve_iterations;
    return HCAO_OK;
}

hcao_status hcao_serve_cancel(hcao_ctx* ctx, uint64_t job_id) {
    if (!ctx) return HCAO_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->serve_mu);
    auto it = ctx->serve_jobs.find(job_id);
    if (it == ctx->serve_jobs.end()) return HCAO_ENOTFOUND;
    const std::shared_ptr<Job>& jb = it->second;
    if (jb->state == 0) {
        for (auto q = ctx->serve_queue.begin(); q != ctx->serve_queue.end(); ++q)
            if ((*q)->id == job_id) {
                ctx->serve_queue.erase(q);
                jb->state = 3;
                jb->result.status = HCAO_ECANCELLED;
                jb->result.t_done = now_s();
                return HCAO_OK;
            }
    }
    if (jb->state <= 1) {  // resident, or being admitted by the engine right now
        jb->cancel = true;
        return HCAO_OK;
    }
    return HCAO_ENOTFOUND;  // finished or failed
}

hcao_status hcao_clear_error(hcao_ctx* ctx) {
    DeviceScope ds_(ctx);
    SERVE_GUARD(ctx);
    if (!ctx) return HCAO_EINVAL;
    CU(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return HCAO_OK;
}

hcao_status hcao_debug_fail_allocs(hcao_ctx* ctx, int n) {
    if (!ctx) return HCAO_EINVAL;
    ctx->fail_allocs.store(n > 0 ? n : 0);
    return HCAO_OK;
}

hcao_status hcao_serve_timing(hcao_ctx* ctx, double* seconds4) {
    if (!ctx || !seconds4) return HCAO_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->serve_mu);
    for (int i = 0; i < 4; ++i) seconds4[i] = ctx->serve_t[i];
    return HCAO_OK;
}

}  // extern "C"

