// hcao_sort.cu -- stable counting sort of particles by cell key (sm_103a).
//
// LSD radix sort on 8-bit digits of the cell key, each pass a stable counting
// sort: per-tile digit histograms built with warp-aggregated shared-memory
// atomics (__match_any_sync: one atomic per group of lanes holding the same
// digit), one exclusive scan over the digit-major histogram matrix, and a
// stable scatter in which a particle's rank inside its tile is
//   (count of its digit in earlier rounds of the tile)
// + (count in earlier warps of this round) + (lanes below it with the same digit).
// Equal keys keep input order, so the particles of a cell stay in load order.
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/hcao.h"
#include "hcao_sort.h"

namespace hcao {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
static_assert(SORT_TILE == SORT_THREADS * SORT_ITEMS, "tile size");

static __global__ void __launch_bounds__(SORT_THREADS)
k_digit_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, uint32_t* hist, int nblocks) {
    __shared__ uint32_t cnt[256];
    const int tid = threadIdx.x, lane = tid & 31;
    cnt[tid] = 0u;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * SORT_TILE;
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const int64_t j = t0 + it * SORT_THREADS + tid;
        const bool valid = j < n;
        const uint32_t d = valid ? (keys[j] >> shift) & 255u : 256u;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&cnt[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    hist[(int64_t)tid * nblocks + blockIdx.x] = cnt[tid];
}

// exclusive scan of a[0..n) in place, one CTA of 1024 threads
static __global__ void __launch_bounds__(1024) k_scan_excl(uint32_t* a, int64_t n) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t i = base + tid;
        const uint32_t x = i < n ? a[i] : 0u;
        uint32_t v = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) wsum[wid] = v;
        __syncthreads();
        if (wid == 0) {
            uint32_t w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, w, o);
                if (lane >= o) w += t;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const uint32_t pre = carry + (wid > 0 ? wsum[wid - 1] : 0u);
        if (i < n) a[i] = pre + v - x;
        __syncthreads();
        if (tid == 0) carry += wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
}

// Exclusive scan of a long array in three steps: per-chunk sums, one CTA's
// scan of the sums, and per-chunk scans offset by them (the result equals the
// single-CTA scan: integer sums in any grouping).  SCAN_CHUNK elements per CTA,
// four per thread.
constexpr int SCAN_CHUNK = 4096;
constexpr int64_t SCAN_SINGLE_MAX = 65536;  // shorter arrays: the single-CTA scan

static __global__ void __launch_bounds__(1024) k_chunk_sums(const uint32_t* __restrict__ a, int64_t n,
                                                            uint32_t* sums) {
    __shared__ uint32_t ws[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    uint32_t v = 0u;
    for (int i = tid; i < SCAN_CHUNK; i += 1024) {
        const int64_t j = base + i;
        if (j < n) v += a[j];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = ws[lane];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xFFFFFFFFu, w, o);
        if (lane == 0) sums[blockIdx.x] = w;
    }
}

static __global__ void __launch_bounds__(1024) k_chunk_scan(uint32_t* a, int64_t n,
                                                            const uint32_t* __restrict__ sums_excl) {
    __shared__ uint32_t ws[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t j0 = (int64_t)blockIdx.x * SCAN_CHUNK + 4 * tid;
    uint32_t x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = j0 + i < n ? a[j0 + i] : 0u;
    const uint32_t t = x[0] + x[1] + x[2] + x[3];
    uint32_t v = t;  // inclusive scan of the threads' totals
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) ws[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    uint32_t run = sums_excl[blockIdx.x] + (wid > 0 ? ws[wid - 1] : 0u) + v - t;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (j0 + i < n) {
            a[j0 + i] = run;
            run += x[i];
        }
}

// a[0..n) exclusive scan in place on stream s; tmp holds scan_tmp_words(n)
static int64_t scan_tmp_words(int64_t n) { return n > SCAN_SINGLE_MAX ? (n + SCAN_CHUNK - 1) / SCAN_CHUNK : 0; }
static int scan_excl(uint32_t* a, int64_t n, uint32_t* tmp, cudaStream_t s) {
    if (n <= SCAN_SINGLE_MAX) {
        k_scan_excl<<<1, 1024, 0, s>>>(a, n);
        return 1;
    }
    const int64_t nc = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    k_chunk_sums<<<(unsigned)nc, 1024, 0, s>>>(a, n, tmp);
    k_scan_excl<<<1, 1024, 0, s>>>(tmp, nc);
    k_chunk_scan<<<(unsigned)nc, 1024, 0, s>>>(a, n, tmp);
    return 3;
}

static __global__ void __launch_bounds__(SORT_THREADS)
k_digit_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ iin, int64_t n,
                int shift, const uint32_t* __restrict__ hist, int nblocks, uint32_t* kout,
                uint32_t* iout) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[SORT_THREADS / 32][257];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    run[tid] = hist[(int64_t)tid * nblocks + blockIdx.x];
    const int64_t t0 = (int64_t)blockIdx.x * SORT_TILE;
    for (int it = 0; it < SORT_ITEMS; ++it) {
        for (int w = 0; w < SORT_THREADS / 32; ++w) wcnt[w][tid] = 0u;
        if (tid == 0)
            for (int w = 0; w < SORT_THREADS / 32; ++w) wcnt[w][256] = 0u;
        __syncthreads();
        const int64_t j = t0 + it * SORT_THREADS + tid;
        const bool valid = j < n;
        const uint32_t key = valid ? kin[j] : 0u;
        const uint32_t d = valid ? (key >> shift) & 255u : 256u;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t below = (uint32_t)__popc(peers & ((1u << lane) - 1u));
        if (lane == __ffs(peers) - 1) wcnt[wid][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = run[d] + below;
            for (int w = 0; w < wid; ++w) pos += wcnt[w][d];
            kout[pos] = key;
            iout[pos] = iin ? iin[j] : (uint32_t)j;
        }
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < SORT_THREADS / 32; ++w) add += wcnt[w][tid];
        run[tid] += add;
        __syncthreads();
    }
}

// per-cell counts with warp-aggregated atomics
static __global__ void k_cell_count(const uint32_t* __restrict__ keys, int64_t n, uint32_t n_cells,
                             uint32_t* cnt) {
    const int lane = threadIdx.x & 31;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < n; j0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = j0 + threadIdx.x;
        const bool valid = j < n;
        const uint32_t k = valid ? keys[j] : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, k);
        if (valid && k < n_cells && lane == __ffs(peers) - 1) atomicAdd(&cnt[k], (uint32_t)__popc(peers));
    }
}

static __global__ void k_zero(uint32_t* a, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = 0u;
}

int64_t sort_scratch_words(int64_t n, uint32_t n_cells) {
    const int64_t nblocks = (n + SORT_TILE - 1) / SORT_TILE;
    const int64_t nh = 256 * (nblocks > 0 ? nblocks : 1);
    (void)n_cells;
    return 4 * n + nh + scan_tmp_words(nh) + 1;
}

int sort_passes(uint32_t n_cells) {
    int bits = 1;
    while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)n_cells) bits++;
    return (bits + 7) / 8;
}

cudaError_t cell_sort(const uint32_t* keys, int64_t n, uint32_t n_cells, uint32_t* perm,
                      uint32_t* offsets, uint32_t* scratch, cudaStream_t s, uint64_t* launches) {
    if (n < 0) return cudaErrorInvalidValue;
    const int64_t nblocks = (n + SORT_TILE - 1) / SORT_TILE;
    uint32_t* kA = scratch;
    uint32_t* iA = scratch + n;
    uint32_t* kB = scratch + 2 * n;
    uint32_t* iB = scratch + 3 * n;
    uint32_t* hist = scratch + 4 * n;
    uint32_t* stmp = hist + 256 * (nblocks > 0 ? nblocks : 1);  // chunk sums of the long scans
    uint64_t L = 0;
    // offsets[c] = count of cell c, then one exclusive scan over n_cells + 1
    // entries: offsets[c] = start of cell c, offsets[n_cells] = n
    k_zero<<<64, 256, 0, s>>>(offsets, (int64_t)n_cells + 1);
    ++L;
    if (n > 0) {
        int g = (int)((n + 255) / 256);
        if (g > 4096) g = 4096;
        k_cell_count<<<g, 256, 0, s>>>(keys, n, n_cells, offsets);
        ++L;
    }
    k_scan_excl<<<1, 1024, 0, s>>>(offsets, (int64_t)n_cells + 1);
    ++L;
    if (n == 0) {
        if (launches) *launches += L;
        return cudaGetLastError();
    }
    const int passes = sort_passes(n_cells);
    const uint32_t* kin = keys;
    const uint32_t* iin = nullptr;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        uint32_t* kout = (p % 2 == 0) ? kA : kB;
        uint32_t* iout = (p == passes - 1) ? perm : ((p % 2 == 0) ? iA : iB);
        k_digit_hist<<<(unsigned)nblocks, SORT_THREADS, 0, s>>>(kin, n, shift, hist, (int)nblocks);
        L += (uint64_t)scan_excl(hist, 256 * nblocks, stmp, s);
        k_digit_scatter<<<(unsigned)nblocks, SORT_THREADS, 0, s>>>(kin, iin, n, shift, hist,
                                                                   (int)nblocks, kout, iout);
        L += 2;
        kin = kout;
        iin = iout;
    }
    if (launches) *launches += L;
    return cudaGetLastError();
}

}  // namespace hcao

// ---------------------------------------------------------------------------
// The same sort for callers that cannot allocate device memory.  Its scratch
// (radix ping-pong buffers and per-tile digit histograms) lives in one
// file-scope device array sized for HCAO_NOALLOC_SORT_MAX_KEYS keys; every
// GPU that loads this library holds that array until the process exits.
namespace {
constexpr int64_t kNoAllocTiles = (HCAO_NOALLOC_SORT_MAX_KEYS + hcao::SORT_TILE - 1) / hcao::SORT_TILE;
constexpr int64_t kNoAllocWords = 4 * (int64_t)HCAO_NOALLOC_SORT_MAX_KEYS + 256 * kNoAllocTiles +
                                  (256 * kNoAllocTiles + 4095) / 4096 + 1;
__device__ __align__(256) uint32_t g_noalloc_sort_scratch[kNoAllocWords];

// The array's device address on the current device.  In host code the
// array's name is only a stand-in, so the address is looked up on every call,
// with the calling thread's device current: a cached address would outlive a
// cudaDeviceReset or a re-created primary context, which load the module (and
// the array) again, possibly elsewhere.  The lookup is a host-side query, not
// a stream operation.
cudaError_t noalloc_scratch(uint32_t** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_sort_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<uint32_t*>(p);
    return cudaSuccess;
}
}  // namespace

extern "C" hcao_status hcao_cell_sort_noalloc(const uint32_t* keys, int64_t n, uint32_t n_cells,
                                              uint32_t* perm, uint32_t* offsets, void* cuda_stream) {
    if (n < 0 || n > HCAO_NOALLOC_SORT_MAX_KEYS || n_cells < 1 || (n > 0 && (!keys || !perm)) || !offsets)
        return HCAO_EINVAL;
    uint32_t* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return HCAO_ECUDA;
    // every buffer the kernels read is written earlier in the same call (the
    // offsets are zeroed first, each histogram is written before its scan), so
    // what an earlier call left in the array does not matter
    const cudaError_t e = hcao::cell_sort(keys, n, n_cells, perm, offsets, scratch,
                                          static_cast<cudaStream_t>(cuda_stream), nullptr);
    return e == cudaSuccess ? HCAO_OK : HCAO_ECUDA;
}

