// sort.cu -- tile binning: every (splat, tile) pair, grouped by tile, in (depth, entry) order.
//
// The 3DGS rasterizer obtains this order by radix-sorting 64-bit (tile << 32 | depth) keys of
// all duplicated pairs. Wide splats make that list long (tens of millions of pairs for a
// 200k-splat view) while each pixel uses only its first few hundred entries, so the sort
// dominates. Here the same order is reached without sorting the pairs at all:
//
//   1. compact the visible splats and sort them by depth (a few hundred thousand keys);
//   2. duplicate them per SUPER-tile (S x S tiles, 64 px) in depth order and stably sort those
//      few million pairs by super-tile id: each super-tile now holds its splats in depth order;
//   3. one CTA per super-tile walks its list in chunks of 256 and, for each of its S*S tiles,
//      compacts the splats covering that tile with warp ballots: first counting (tile sizes ->
//      tile_start by a scan), then emitting ids to each tile's range with coalesced stores.
//
// A tile's list is its super-tile's list filtered by "tile in the splat's tile rectangle",
// which preserves (depth, entry) order, so the output equals the global pair sort bit for bit.
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

static int radix_blocks(long long n_max)
{
    long long nb = (n_max + 2LL * RS_TILE - 1) / (2LL * RS_TILE);
    return (int)(nb < 1 ? 1 : (nb > RS_MAX_BLOCKS ? RS_MAX_BLOCKS : nb));
}

// Stable LSD sort of (k0, v0) by key bits [0, nbits); ping-pongs through (k1, v1); the final
// pass writes to (kf, vf), which must not alias the last pass's source. Digits of a pass are
// ceil(nbits / passes) wide.
static void radix_sort(const uint32_t *n_dev, long long n_max, int nbits, uint32_t *k0, uint32_t *v0, uint32_t *k1,
                       uint32_t *v1, uint32_t *kf, uint32_t *vf, uint32_t *counts, uint32_t *block_sums,
                       cudaStream_t st)
{
    if (nbits < 1) nbits = 1;
    const int passes = (nbits + 7) / 8;
    const int width = (nbits + passes - 1) / passes;
    const int nb = radix_blocks(n_max);
    const long long ncounts = 256LL * nb;
    for (int p = 0; p < passes; ++p) {
        const int shift = width * p, bits = nbits - shift < width ? nbits - shift : width;
        uint32_t *ks = (p & 1) ? k1 : k0, *vs = (p & 1) ? v1 : v0;
        uint32_t *kd = (p & 1) ? k0 : k1, *vd = (p & 1) ? v0 : v1;
        if (p == passes - 1) {
            kd = kf;
            vd = vf;
        }
        count_launch(2);
        k_radix_count<<<nb, RS_THREADS, 0, st>>>(ks, n_dev, shift, bits, counts);
        scan(LoadPlain{counts}, nullptr, ncounts, counts, block_sums, nullptr, nullptr, nullptr, -1, nullptr, st);
        k_radix_scatter<<<nb, RS_THREADS, 0, st>>>(ks, vs, kd, vd, n_dev, shift, bits, counts);
    }
}

// ------------------------------------------------------------------ super-tile pairs

__device__ __forceinline__ void splat_rect(const BatchParams &P, const ItemParams &I, const float *splat,
                                           const int *radius, uint32_t e, int &x0, int &y0, int &x1, int &y1)
{
    const float2 uv = *reinterpret_cast<const float2 *>(splat + 12LL * e);
    tile_rect(uv.x, uv.y, radius[e], P.tw, P.th, I.gx, I.gy, x0, y0, x1, y1);
}

// super-rectangle area of the k-th depth-ordered visible splat
__global__ void __launch_bounds__(256) k_super_area(const __grid_constant__ BatchParams P, const uint32_t *V_dev,
                                                    const uint32_t *__restrict__ order, const float *__restrict__ splat,
                                                    const int *__restrict__ radius, uint32_t *__restrict__ area)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *V_dev) return;
    const uint32_t e = order[k];
    const ItemParams &I = P.item[item_of_entry(P, e)];
    int x0, y0, x1, y1;
    splat_rect(P, I, splat, radius, e, x0, y0, x1, y1);
    const int S = P.S;
    area[k] = (uint32_t)(((x1 + S - 1) / S - x0 / S) * ((y1 + S - 1) / S - y0 / S));
}

// Each warp takes 32 consecutive depth-ordered splats; their super pairs occupy one contiguous
// output range, written lane-strided (coalesced); a lane finds its splat by binary search
// over the warp's 32 offsets.
__global__ void __launch_bounds__(256) k_super_dup(const __grid_constant__ BatchParams P, const uint32_t *V_dev,
                                                   const uint32_t *__restrict__ order, const uint32_t *__restrict__ offs,
                                                   const float *__restrict__ splat, const int *__restrict__ radius,
                                                   const uint32_t *n_sp_use, uint32_t *__restrict__ skeys,
                                                   uint32_t *__restrict__ svals)
{
    const int lane = threadIdx.x & 31;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t V = *V_dev;
    if ((long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31) >= V) return;
    if (*n_sp_use == 0) return;  // nothing to emit (no pairs, or scratch capacity exceeded)
    const bool valid = k < V;
    const int S = P.S;
    uint32_t off = 0xffffffffu, cnt = 0, base = 0, w = 1, sg = 1, e = 0;
    if (valid) {
        e = order[k];
        off = offs[k];
        const ItemParams &I = P.item[item_of_entry(P, e)];
        int x0, y0, x1, y1;
        splat_rect(P, I, splat, radius, e, x0, y0, x1, y1);
        const int sx0 = x0 / S, sy0 = y0 / S, sx1 = (x1 + S - 1) / S, sy1 = (y1 + S - 1) / S;
        base = (uint32_t)(I.super_off + sy0 * I.sgx + sx0);
        w = (uint32_t)(sx1 - sx0);
        sg = (uint32_t)I.sgx;
        cnt = (uint32_t)((sx1 - sx0) * (sy1 - sy0));
    }
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    const int last = 31 - __clz(vmask);
    const uint32_t p0 = __shfl_sync(0xffffffffu, off, 0);
    const uint32_t p1 = __shfl_sync(0xffffffffu, off + cnt, last);
    for (uint32_t p = p0 + lane; p - lane < p1; p += 32) {
        int j = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1) {
            uint32_t o = __shfl_sync(0xffffffffu, off, j + step);
            if (o <= p) j += step;
        }
        const uint32_t oj = __shfl_sync(0xffffffffu, off, j);
        const uint32_t wj = __shfl_sync(0xffffffffu, w, j);
        const uint32_t bj = __shfl_sync(0xffffffffu, base, j);
        const uint32_t gj = __shfl_sync(0xffffffffu, sg, j);
        const uint32_t ej = __shfl_sync(0xffffffffu, e, j);
        if (p < p1) {
            const uint32_t local = p - oj;
            const uint32_t sy = local / wj, sx = local - sy * wj;
            skeys[p] = bj + sy * gj + sx;
            svals[p] = ej;
        }
    }
}

// range starts of sorted keys: start[t] = first k with keys[k] >= t, t in [0, n_keys]
__global__ void __launch_bounds__(256) k_key_ranges(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                                                    long long n_max, int n_keys, uint32_t *__restrict__ start)
{
    const long long n = *n_dev < n_max ? (long long)*n_dev : n_max;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += (long long)gridDim.x * blockDim.x) {
        const long long prev = k > 0 ? (long long)keys[k - 1] : -1;
        const long long cur = k < n ? (long long)keys[k] : (long long)n_keys;
        for (long long t = prev + 1; t <= cur && t <= n_keys; ++t) start[t] = (uint32_t)k;
    }
}

// ------------------------------------------------------------------ per-tile lists

// Local tile rectangle (relative to the super-tile origin) of the splat at position i of the
// super-tile's list, or an empty one.
template <int S>
__device__ __forceinline__ void local_rect(const BatchParams &P, const ItemParams &I, const uint32_t *sp_ids,
                                           const float *splat, const int *radius, long long i, long long end, int tx0,
                                           int ty0, int &lx0, int &ly0, int &lx1, int &ly1, uint32_t &e)
{
    lx0 = ly0 = lx1 = ly1 = 0;
    e = 0;
    if (i < end) {
        e = sp_ids[i];
        int x0, y0, x1, y1;
        splat_rect(P, I, splat, radius, e, x0, y0, x1, y1);
        lx0 = x0 - tx0; lx1 = x1 - tx0; ly0 = y0 - ty0; ly1 = y1 - ty0;
    }
}

// Pass 1: number of splats covering each tile (written into tile_count[global tile]).
template <int S>
__global__ void __launch_bounds__(BIN_THREADS) k_tile_count(const __grid_constant__ BatchParams P,
                                                            const uint32_t *__restrict__ sp_ids,
                                                            const uint32_t *__restrict__ super_start,
                                                            const float *__restrict__ splat,
                                                            const int *__restrict__ radius, uint32_t *__restrict__ tile_count)
{
    constexpr int NT = S * S, NL = (NT + 31) / 32;
    __shared__ uint32_t red[BIN_THREADS / 32][NT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = blockIdx.x;
    const ItemParams &I = P.item[item_of_super(P, s)];
    const int ls = s - I.super_off, tx0 = (ls % I.sgx) * S, ty0 = (ls / I.sgx) * S;
    const long long start = super_start[s], end = super_start[s + 1];
    uint32_t cnt[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) cnt[q] = 0;
    for (long long base = start; base < end; base += BIN_THREADS) {
        int lx0, ly0, lx1, ly1;
        uint32_t e;
        local_rect<S>(P, I, sp_ids, splat, radius, base + threadIdx.x, end, tx0, ty0, lx0, ly0, lx1, ly1, e);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int tx = t % S, ty = t / S;
            const unsigned m = __ballot_sync(0xffffffffu, tx >= lx0 && tx < lx1 && ty >= ly0 && ty < ly1);
            if (lane == (t & 31)) cnt[t >> 5] += __popc(m);
        }
    }
#pragma unroll
    for (int q = 0; q < NL; ++q)
        if (q * 32 + lane < NT) red[warp][q * 32 + lane] = cnt[q];
    __syncthreads();
    if (threadIdx.x < NT) {
        const int tx = tx0 + (int)threadIdx.x % S, ty = ty0 + (int)threadIdx.x / S;
        if (tx < I.gx && ty < I.gy) {
            uint32_t c = 0;
            for (int w = 0; w < BIN_THREADS / 32; ++w) c += red[w][threadIdx.x];
            tile_count[I.tile_off + ty * I.gx + tx] = c;
        }
    }
}

// Pass 2: each tile's splats, in list order, to [tile_start[t], tile_start[t+1]).
template <int S>
__global__ void __launch_bounds__(BIN_THREADS) k_tile_emit(const __grid_constant__ BatchParams P,
                                                           const uint32_t *__restrict__ sp_ids,
                                                           const uint32_t *__restrict__ super_start,
                                                           const float *__restrict__ splat, const int *__restrict__ radius,
                                                           const int *__restrict__ tile_start, const uint32_t *n_use,
                                                           int *__restrict__ gauss_ids)
{
    constexpr int NT = S * S;
    __shared__ uint32_t wc[BIN_THREADS / 32][NT];
    __shared__ uint32_t run[NT], tot[NT];
    if (*n_use == 0) return;  // no pairs, or more than the bins hold
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int s = blockIdx.x;
    const ItemParams &I = P.item[item_of_super(P, s)];
    const int ls = s - I.super_off, tx0 = (ls % I.sgx) * S, ty0 = (ls / I.sgx) * S;
    const long long start = super_start[s], end = super_start[s + 1];
    if (threadIdx.x < NT) {
        const int tx = tx0 + (int)threadIdx.x % S, ty = ty0 + (int)threadIdx.x / S;
        run[threadIdx.x] = (tx < I.gx && ty < I.gy) ? (uint32_t)tile_start[I.tile_off + ty * I.gx + tx] : 0u;
    }
    for (long long base = start; base < end; base += BIN_THREADS) {
        int lx0, ly0, lx1, ly1;
        uint32_t e;
        local_rect<S>(P, I, sp_ids, splat, radius, base + threadIdx.x, end, tx0, ty0, lx0, ly0, lx1, ly1, e);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int tx = t % S, ty = t / S;
            const unsigned m = __ballot_sync(0xffffffffu, tx >= lx0 && tx < lx1 && ty >= ly0 && ty < ly1);
            if (lane == (t & 31)) wc[warp][t] = __popc(m);
        }
        __syncthreads();
        if (threadIdx.x < NT) {
            uint32_t r = 0;
#pragma unroll
            for (int w = 0; w < BIN_THREADS / 32; ++w) {
                const uint32_t c = wc[w][threadIdx.x];
                wc[w][threadIdx.x] = r;
                r += c;
            }
            tot[threadIdx.x] = r;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int tx = t % S, ty = t / S;
            const bool cov = tx >= lx0 && tx < lx1 && ty >= ly0 && ty < ly1;
            const unsigned m = __ballot_sync(0xffffffffu, cov);
            if (cov) gauss_ids[run[t] + wc[warp][t] + __popc(m & lt)] = (int)e;
        }
        __syncthreads();
        if (threadIdx.x < NT) run[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
}

// after an overflow the bins describe empty tiles
__global__ void __launch_bounds__(256) k_clear_on_overflow(const uint32_t *n_use, const long long *total, int n_tiles,
                                                           int *__restrict__ tile_start)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= n_tiles && *n_use == 0 && *total != 0) tile_start[t] = 0;
}

// ------------------------------------------------------------------ orchestration

// Steps 1 and the super-pair count: visible splats in depth order (vis_pos), per-splat super
// pair offsets (offs), the super pair total (scalars[4]) and its usable count (scalars[1]: the
// total, or 0 with a latched error when it exceeds pair_capacity; < 0 = unchecked).
cudaError_t bin_super_count(const BatchParams &P, const float *splat, const int *radius, const int *tiles,
                            BinScratch &b, long long pair_capacity, cudaStream_t st)
{
    const long long n = P.n_entries;
    uint32_t *V = b.scalars, *n_sp = b.scalars + 1, *sp_total = b.scalars + 4;
    // 1. visible entries -> (depth key, entry), sorted by depth; the order ends in vis_pos
    scan(LoadVisible{tiles}, nullptr, n, b.vis_pos, b.block_sums, V, nullptr, nullptr, -1, nullptr, st);
    if (n > 0) {
        count_launch();
        k_compact<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, tiles, splat, b.vis_pos, b.dkA, b.dvA);
    }
    radix_sort(V, n, 32, b.dkA, b.dvA, b.dkB, b.dvB, b.dkA, b.vis_pos, b.counts, b.block_sums, st);
    // 2. super-tile pairs in depth order, stably sorted by super-tile id
    if (n > 0) {
        count_launch();
        k_super_area<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, V, b.vis_pos, splat, radius, b.offs);
    }
    scan(LoadPlain{b.offs}, V, n, b.offs, b.block_sums, sp_total, nullptr, n_sp, pair_capacity, b.status, st);
    return cudaGetLastError();
}

// Super pairs -> sorted super-tile lists -> tile sizes -> tile_start (in place), the pair
// count (n_isect) and its usable count (scalars[2], 0 when above isect_capacity).
cudaError_t bin_tile_count(const BatchParams &P, const float *splat, const int *radius, BinScratch &b,
                           long long pair_capacity, long long *n_isect_dev, int *tile_start, long long isect_capacity,
                           cudaStream_t st)
{
    const long long n = P.n_entries;
    uint32_t *V = b.scalars, *n_sp = b.scalars + 1, *n_use = b.scalars + 2;
    if (n > 0) {
        count_launch();
        k_super_dup<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, V, b.vis_pos, b.offs, splat, radius, n_sp, b.skA,
                                                                 b.svA);
    }
    int nbits = 0;
    while ((1LL << nbits) < (long long)P.n_super) ++nbits;
    const int passes = nbits < 1 ? 1 : (nbits + 7) / 8;
    uint32_t *kfinal = (passes & 1) ? b.skB : b.skA;  // not the last pass's source
    uint32_t *vfinal = (passes & 1) ? b.svB : b.svA;
    radix_sort(n_sp, pair_capacity, nbits, b.skA, b.svA, b.skB, b.svB, kfinal, vfinal, b.counts, b.block_sums, st);
    b.sp_ids = vfinal;
    count_launch();
    const long long rblocks = (pair_capacity + 1 + 255) / 256;
    k_key_ranges<<<(unsigned)(rblocks < 2368 ? rblocks : 2368), 256, 0, st>>>(kfinal, n_sp, pair_capacity, P.n_super,
                                                                                b.super_start);
    // 3. tile sizes -> tile_start (in place), pair count, capacity check
    uint32_t *ts = reinterpret_cast<uint32_t *>(tile_start);
    if (P.n_super > 0) {
        count_launch();
        if (P.S == 8)
            k_tile_count<8><<<P.n_super, BIN_THREADS, 0, st>>>(P, b.sp_ids, b.super_start, splat, radius, ts);
        else
            k_tile_count<4><<<P.n_super, BIN_THREADS, 0, st>>>(P, b.sp_ids, b.super_start, splat, radius, ts);
    }
    // the scan's grand total lands in tile_start[n_tiles] and in the caller's n_isect
    scan(LoadPlain{ts}, nullptr, P.n_tiles, ts, b.block_sums, ts + P.n_tiles, n_isect_dev, n_use, isect_capacity,
         b.status, st);
    return cudaGetLastError();
}

cudaError_t bin_sort_emit(const BatchParams &P, const float *splat, const int *radius, BinScratch &b,
                          const long long *n_isect_dev, int *gauss_ids, int *tile_start, cudaStream_t st)
{
    const uint32_t *n_use = b.scalars + 2;
    if (P.n_super > 0) {
        count_launch();
        if (P.S == 8)
            k_tile_emit<8><<<P.n_super, BIN_THREADS, 0, st>>>(P, b.sp_ids, b.super_start, splat, radius, tile_start,
                                                              n_use, gauss_ids);
        else
            k_tile_emit<4><<<P.n_super, BIN_THREADS, 0, st>>>(P, b.sp_ids, b.super_start, splat, radius, tile_start,
                                                              n_use, gauss_ids);
    }
    count_launch();
    k_clear_on_overflow<<<(P.n_tiles + 1 + 255) / 256, 256, 0, st>>>(n_use, n_isect_dev, P.n_tiles, tile_start);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ scratch layout
//
// entry part: 6 arrays of max_entries words + radix digit counts + scan block sums + scalars
// pair part:  4 arrays of max_pairs words (super-tile pairs, ping-pong)
// super part: max_super + 1 words (super-tile list starts)

static size_t words_rounded(size_t words) { return ((words * 4 + 255) / 256) * 256; }

size_t entry_scratch_bytes(long long max_entries)
{
    size_t e = (size_t)(max_entries > 0 ? max_entries : 1);
    return 6 * words_rounded(e) + words_rounded(256ull * RS_MAX_BLOCKS) + words_rounded(SCAN_MAX_BLOCKS) +
           words_rounded(16);
}

size_t pair_scratch_bytes(long long max_pairs)
{
    size_t i = (size_t)(max_pairs > 0 ? max_pairs : 1);
    return 4 * words_rounded(i);
}

size_t super_scratch_bytes(long long max_super) { return words_rounded((size_t)(max_super > 0 ? max_super : 1) + 1); }

struct Carver {
    char *p;
    uint32_t *take(size_t words)
    {
        uint32_t *r = reinterpret_cast<uint32_t *>(p);
        p += words_rounded(words);
        return r;
    }
};

void entry_scratch_carve(void *mem, long long max_entries, int *status, BinScratch &b)
{
    size_t e = (size_t)(max_entries > 0 ? max_entries : 1);
    Carver c{static_cast<char *>(mem)};
    b.vis_pos = c.take(e); b.dkA = c.take(e); b.dvA = c.take(e); b.dkB = c.take(e); b.dvB = c.take(e);
    b.offs = c.take(e);
    b.counts = c.take(256ull * RS_MAX_BLOCKS);
    b.block_sums = c.take(SCAN_MAX_BLOCKS);
    b.scalars = c.take(16);
    b.status = status;
}

void pair_scratch_carve(void *mem, long long max_pairs, BinScratch &b)
{
    size_t i = (size_t)(max_pairs > 0 ? max_pairs : 1);
    Carver c{static_cast<char *>(mem)};
    b.skA = c.take(i); b.svA = c.take(i); b.skB = c.take(i); b.svB = c.take(i);
}

void super_scratch_carve(void *mem, BinScratch &b) { b.super_start = static_cast<uint32_t *>(mem); }

}  // namespace lobe
