// sort_prims.cuh -- device primitives of the binning stage (included by binning.cu only):
// an exclusive scan with a device-side length, compaction of visible splats, and a stable
// LSD radix sort of (key, value) pairs.
//
// Radix passes are block-chunked: each block owns a contiguous chunk, ranks 2048-element tiles
// of it with warp ballots, reorders each tile by digit in shared memory, and writes runs of
// equal digits with coalesced stores. No spin-waits anywhere; every result is deterministic.
#include "lobe_internal.cuh"

namespace lobe {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_MAX_BLOCKS = 1024;
constexpr int RS_WARPS = 8;
constexpr int RS_THREADS = RS_WARPS * 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // elements ranked and staged per step
constexpr int RS_MAX_BLOCKS = 1184;             // 8 per SM on 148 SMs
constexpr int BIN_THREADS = 256;

// ------------------------------------------------------------------ block scan helper

// Exclusive scan of one value per thread across the block; returns the block total.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t &excl, uint32_t *sm_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sm_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < THREADS / 32 ? sm_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < THREADS / 32) sm_warp[lane] = wi - w;
        if (lane == THREADS / 32 - 1) sm_warp[THREADS / 32] = wi;
    }
    __syncthreads();
    excl = sm_warp[warp] + inc - x;
    uint32_t total = sm_warp[THREADS / 32];
    __syncthreads();
    return total;
}

// ------------------------------------------------------------------ generic exclusive scan
//
// out[i] = sum_{j<i} in(j) for i < n, with n read from device memory when n_dev is given (the
// launch shape then depends only on an upper bound, so the call is graph-capturable). Three
// kernels: per-block totals, scan of the totals (one block), per-block scan with its offset.
// In-place use (out == the loaded array) is safe: each element is read and then written by
// the same thread.

struct LoadVisible {  // 1 where a projected entry touches at least one tile
    const int *tiles;
    __device__ uint32_t operator()(long long i) const { return tiles[i] > 0 ? 1u : 0u; }
};
struct LoadPlain {
    const uint32_t *src;
    __device__ uint32_t operator()(long long i) const { return src[i]; }
};

__device__ __forceinline__ void chunk_of(long long n, int b, int nb, long long &lo, long long &hi)
{
    long long chunk = (n + nb - 1) / nb;
    lo = (long long)b * chunk;
    hi = lo + chunk < n ? lo + chunk : n;
    if (lo > n) lo = n;
}

template <class L>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(L load, const uint32_t *n_dev, long long n_host,
                                                              uint32_t *block_sums)
{
    __shared__ uint32_t red[SCAN_THREADS / 32];
    const long long n = n_dev ? (long long)*n_dev : n_host;
    long long lo, hi;
    chunk_of(n, blockIdx.x, gridDim.x, lo, hi);
    uint32_t s = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += SCAN_THREADS) s += load(i);
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += red[w];
        block_sums[blockIdx.x] = t;
    }
}

// Scans block_sums[0..nb) in place (exclusive), writes the grand total to total32/total64
// (nullable), and the count the next stage may use: the total, or 0 with a latched
// capacity error when it exceeds `capacity` (capacity < 0: unlimited).
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *block_sums, int nb, uint32_t *total32, long long *total64,
                                                   uint32_t *n_use, long long capacity, int *status)
{
    __shared__ uint32_t sm[33];
    uint32_t x = threadIdx.x < nb ? block_sums[threadIdx.x] : 0u, ex;
    uint32_t total = block_exclusive_scan<1024>(x, ex, sm);
    if (threadIdx.x < nb) block_sums[threadIdx.x] = ex;
    if (threadIdx.x == 0) {
        if (total32) *total32 = total;
        if (total64) *total64 = (long long)total;
        if (n_use) {
            bool over = capacity >= 0 && (long long)total > capacity;
            *n_use = over ? 0u : total;
            if (over) set_status(status, STATUS_CAPACITY);
        }
    }
}

template <class L>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(L load, const uint32_t *n_dev, long long n_host,
                                                            const uint32_t *block_sums, uint32_t *out)
{
    __shared__ uint32_t sm[SCAN_THREADS / 32 + 1];
    const long long n = n_dev ? (long long)*n_dev : n_host;
    long long lo, hi;
    chunk_of(n, blockIdx.x, gridDim.x, lo, hi);
    uint32_t carry = block_sums[blockIdx.x];
    for (long long base = lo; base < hi; base += SCAN_THREADS) {
        long long i = base + threadIdx.x;
        uint32_t x = i < hi ? load(i) : 0u, ex;
        uint32_t tot = block_exclusive_scan<SCAN_THREADS>(x, ex, sm);
        if (i < hi) out[i] = carry + ex;
        carry += tot;
    }
}

template <class L>
static void scan(L load, const uint32_t *n_dev, long long n_max, uint32_t *out, uint32_t *block_sums,
                 uint32_t *total32, long long *total64, uint32_t *n_use, long long capacity, int *status,
                 cudaStream_t st)
{
    int nb = (int)((n_max + 4 * SCAN_THREADS - 1) / (4 * SCAN_THREADS));
    nb = nb < 1 ? 1 : (nb > SCAN_MAX_BLOCKS ? SCAN_MAX_BLOCKS : nb);
    long long n_host = n_dev ? 0 : n_max;
    count_launch(3);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, st>>>(load, n_dev, n_host, block_sums);
    k_scan_top<<<1, 1024, 0, st>>>(block_sums, nb, total32, total64, n_use, capacity, status);
    k_scan_down<<<nb, SCAN_THREADS, 0, st>>>(load, n_dev, n_host, block_sums, out);
}

// ------------------------------------------------------------------ compaction of visible splats

// keys = fp32 depth bits (positive depths order like unsigned ints), values = entry id
__global__ void __launch_bounds__(256) k_compact(long long n_entries, const int *__restrict__ tiles,
                                                 const float *__restrict__ splat, const uint32_t *__restrict__ pos,
                                                 uint32_t *__restrict__ dkeys, uint32_t *__restrict__ dvals)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_entries || tiles[e] <= 0) return;
    uint32_t p = pos[e];
    dkeys[p] = __float_as_uint(splat[12 * e + 9]);
    dvals[p] = (uint32_t)e;
}

// ------------------------------------------------------------------ radix sort (LSD, <= 8 bits/pass)

// Lanes of the warp holding the same digit as this lane (restricted to `valid`).
__device__ __forceinline__ unsigned warp_peers(uint32_t d, int nbits, unsigned valid)
{
    unsigned peers = valid;
    for (int b = 0; b < nbits; ++b) {
        unsigned bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bal : ~bal;
    }
    return peers;
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_count(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                                                            int shift, int nbits, uint32_t *__restrict__ counts)
{
    __shared__ uint32_t h[RS_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) h[warp][d] = 0;
    __syncwarp();
    long long lo, hi;
    chunk_of(*n_dev, blockIdx.x, gridDim.x, lo, hi);
    const uint32_t mask = (1u << nbits) - 1u;
    for (long long base = lo + warp * 32; base < hi; base += RS_THREADS * 4) {
        uint32_t k[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            long long i = base + j * RS_THREADS + lane;
            k[j] = i < hi ? keys[i] : 0u;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            long long i = base + j * RS_THREADS + lane;
            unsigned valid = __ballot_sync(0xffffffffu, i < hi);
            uint32_t d = (k[j] >> shift) & mask;
            unsigned peers = warp_peers(d, nbits, valid);
            if (i < hi && lane == __ffs(peers) - 1) h[warp][d] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
        uint32_t s = 0;
        for (int w = 0; w < RS_WARPS; ++w) s += h[w][d];
        counts[(long long)d * gridDim.x + blockIdx.x] = s;
    }
}

// One pass: block b scatters its chunk [lo, hi) to offsets[d * nb + b] + (running count).
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                              const uint32_t *__restrict__ vin,
                                                              uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                              const uint32_t *n_dev, int shift, int nbits,
                                                              const uint32_t *__restrict__ offsets)
{
    __shared__ uint32_t s_k[RS_TILE];
    __shared__ uint32_t s_v[RS_TILE];
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t local_off[256], tile_cnt[256], grun[256];
    __shared__ uint32_t scan_sm[RS_THREADS / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const unsigned lt = lanemask_lt();
    const uint32_t mask = (1u << nbits) - 1u;
    long long lo, hi;
    chunk_of(*n_dev, blockIdx.x, gridDim.x, lo, hi);
    grun[tid] = offsets[(long long)tid * gridDim.x + blockIdx.x];  // RS_THREADS == 256 digits
    for (long long tb = lo; tb < hi; tb += RS_TILE) {
        for (int d = lane; d < 256; d += 32) wcnt[warp][d] = 0;
        __syncwarp();
        uint32_t k[RS_ITEMS], v[RS_ITEMS], dg[RS_ITEMS], rk[RS_ITEMS];
        bool ok[RS_ITEMS];
#pragma unroll
        for (int j = 0; j < RS_ITEMS; ++j) {
            const long long i = tb + warp * (32 * RS_ITEMS) + j * 32 + lane;
            ok[j] = i < hi;
            k[j] = ok[j] ? kin[i] : 0u;
            v[j] = ok[j] ? vin[i] : 0u;
        }
        // rank within the warp's 256 consecutive elements, in order
#pragma unroll
        for (int j = 0; j < RS_ITEMS; ++j) {
            dg[j] = (k[j] >> shift) & mask;
            const unsigned valid = __ballot_sync(0xffffffffu, ok[j]);
            const unsigned peers = warp_peers(dg[j], nbits, valid);
            const int leader = ok[j] ? __ffs(peers) - 1 : lane;
            uint32_t base = (ok[j] && lane == leader) ? wcnt[warp][dg[j]] : 0u;
            base = __shfl_sync(0xffffffffu, base, leader);
            rk[j] = base + __popc(peers & lt);
            __syncwarp();
            if (ok[j] && lane == leader) wcnt[warp][dg[j]] = base + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {  // per digit: exclusive prefix over warps and the tile's digit totals
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
            tile_cnt[tid] = run;
            uint32_t ex;
            block_exclusive_scan<RS_THREADS>(run, ex, scan_sm);
            local_off[tid] = ex;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < RS_ITEMS; ++j) {
            if (ok[j]) {
                const uint32_t pos = local_off[dg[j]] + wcnt[warp][dg[j]] + rk[j];
                s_k[pos] = k[j];
                s_v[pos] = v[j];
            }
        }
        __syncthreads();
        const int n_tile = (int)(hi - tb < RS_TILE ? hi - tb : RS_TILE);
        for (int i = tid; i < n_tile; i += RS_THREADS) {
            const uint32_t key = s_k[i];
            const uint32_t d = (key >> shift) & mask;
            const uint32_t g = grun[d] + (uint32_t)i - local_off[d];
            kout[g] = key;
            vout[g] = s_v[i];
        }
        __syncthreads();
        grun[tid] += tile_cnt[tid];
        __syncthreads();
    }
}

// one 2048-element tile per block up to 8 blocks per SM, then several tiles per block
static int radix_blocks(long long n_max)
{
    long long nb = (n_max + RS_TILE - 1) / RS_TILE;
    return (int)(nb < 1 ? 1 : (nb > RS_MAX_BLOCKS ? RS_MAX_BLOCKS : nb));
}

// Stable LSD sort of (k0, v0) by key bits [shift0, shift0 + nbits); ping-pongs through
// (k1, v1); the final pass writes to (kf, vf), which must not alias the last pass's source.
// Digits of a pass are ceil(nbits / passes) wide. Keys move with their values, so bits
// outside the sorted range travel along untouched.
static void radix_sort(const uint32_t *n_dev, long long n_max, int shift0, int nbits, uint32_t *k0, uint32_t *v0,
                       uint32_t *k1, uint32_t *v1, uint32_t *kf, uint32_t *vf, uint32_t *counts,
                       uint32_t *block_sums, cudaStream_t st)
{
    if (nbits < 1) nbits = 1;
    const int passes = (nbits + 7) / 8;
    const int width = (nbits + passes - 1) / passes;
    const int nb = radix_blocks(n_max);
    const long long ncounts = 256LL * nb;
    for (int p = 0; p < passes; ++p) {
        const int lo = width * p, bits = nbits - lo < width ? nbits - lo : width;
        uint32_t *ks = (p & 1) ? k1 : k0, *vs = (p & 1) ? v1 : v0;
        uint32_t *kd = (p & 1) ? k0 : k1, *vd = (p & 1) ? v0 : v1;
        if (p == passes - 1) {
            kd = kf;
            vd = vf;
        }
        count_launch(2);
        k_radix_count<<<nb, RS_THREADS, 0, st>>>(ks, n_dev, shift0 + lo, bits, counts);
        scan(LoadPlain{counts}, nullptr, ncounts, counts, block_sums, nullptr, nullptr, nullptr, -1, nullptr, st);
        k_radix_scatter<<<nb, RS_THREADS, 0, st>>>(ks, vs, kd, vd, n_dev, shift0 + lo, bits, counts);
    }
}

}  // namespace lobe
