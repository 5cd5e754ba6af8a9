// sort.cu -- tile binning: visible-splat compaction, depth sort, key duplication, stable
// tile sort, tile ranges.
//
// Result: every (splat, tile) pair ordered by (global tile, fp32 depth bits, entry id), the
// order the 3DGS rasterizer obtains by radix-sorting 64-bit (tile << 32 | depth) keys. Here
// it is reached in two cheaper steps: the visible splats (a few hundred thousand) are sorted
// by depth once, then the duplicated pairs -- emitted in depth order -- are stably sorted by
// tile id on only ceil(log2(n_tiles)) bits (2 passes of 8 bits for up to 65536 tiles).
// A stable LSD sort of a depth-ordered sequence by tile gives exactly the (tile, depth,
// entry) order, with 4-byte keys instead of 8-byte ones and 2 passes instead of ~6.
//
// Radix passes are "segment per warp": each warp owns a contiguous segment of the input,
// counts its digits (pass 1), all segment counts are scanned digit-major (pass 2), and each
// warp scatters its segment in order using warp ballots to rank equal digits (pass 3). No
// block-wide barriers in the hot loops, no spin-waits, fully deterministic and stable.
#include "lobe_internal.cuh"

namespace lobe {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_MAX_BLOCKS = 1024;
constexpr int RS_WARPS = 8;
constexpr int RS_THREADS = RS_WARPS * 32;
constexpr int RS_UNROLL = 4;
constexpr int RS_MAX_BLOCKS = 592;  // 4 per SM on 148 SMs

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
// out[i] = sum_{j<i} in(j) for i < n, with n read from device memory (so the launch shape
// depends only on an upper bound and the call is graph-capturable). Three kernels:
// per-block totals, scan of the totals (one block), per-block scan with the block offset.

struct LoadVisible {  // 1 where a projected entry touches at least one tile
    const int *tiles;
    __device__ uint32_t operator()(long long i) const { return tiles[i] > 0 ? 1u : 0u; }
};
struct LoadGatherTiles {  // tiles touched by the k-th splat in depth order
    const int *tiles;
    const uint32_t *order;
    __device__ uint32_t operator()(long long i) const { return (uint32_t)tiles[order[i]]; }
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

__device__ __forceinline__ void segment_of(uint32_t n, long long seg, long long nseg, long long &lo, long long &hi)
{
    long long len = ((long long)n + nseg - 1) / nseg;
    lo = seg * len;
    hi = lo + len < (long long)n ? lo + len : (long long)n;
    if (lo > (long long)n) lo = n;
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_count(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                                                            int shift, int nbits, uint32_t *__restrict__ counts)
{
    __shared__ uint32_t h[RS_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) h[warp][d] = 0;
    __syncwarp();
    const long long nseg = (long long)gridDim.x * RS_WARPS, seg = (long long)blockIdx.x * RS_WARPS + warp;
    long long lo, hi;
    segment_of(*n_dev, seg, nseg, lo, hi);
    const uint32_t mask = (1u << nbits) - 1u;
    for (long long base = lo; base < hi; base += 32 * RS_UNROLL) {
        uint32_t k[RS_UNROLL];
#pragma unroll
        for (int j = 0; j < RS_UNROLL; ++j) {
            long long i = base + j * 32 + lane;
            k[j] = i < hi ? keys[i] : 0u;
        }
#pragma unroll
        for (int j = 0; j < RS_UNROLL; ++j) {
            long long i = base + j * 32 + lane;
            unsigned valid = __ballot_sync(0xffffffffu, i < hi);
            uint32_t d = (k[j] >> shift) & mask;
            unsigned peers = warp_peers(d, nbits, valid);
            if (i < hi && lane == __ffs(peers) - 1) h[warp][d] += __popc(peers);
            __syncwarp();
        }
    }
    __syncwarp();
    for (int d = lane; d < 256; d += 32) counts[(long long)d * nseg + seg] = h[warp][d];
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                              const uint32_t *__restrict__ vin,
                                                              uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                              const uint32_t *n_dev, int shift, int nbits,
                                                              const uint32_t *__restrict__ offsets)
{
    __shared__ uint32_t run[RS_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long nseg = (long long)gridDim.x * RS_WARPS, seg = (long long)blockIdx.x * RS_WARPS + warp;
    for (int d = lane; d < 256; d += 32) run[warp][d] = offsets[(long long)d * nseg + seg];
    __syncwarp();
    long long lo, hi;
    segment_of(*n_dev, seg, nseg, lo, hi);
    const uint32_t mask = (1u << nbits) - 1u;
    const unsigned lt = lanemask_lt();
    for (long long base = lo; base < hi; base += 32 * RS_UNROLL) {
        uint32_t k[RS_UNROLL], v[RS_UNROLL];
#pragma unroll
        for (int j = 0; j < RS_UNROLL; ++j) {
            long long i = base + j * 32 + lane;
            k[j] = i < hi ? kin[i] : 0u;
            v[j] = i < hi ? vin[i] : 0u;
        }
#pragma unroll
        for (int j = 0; j < RS_UNROLL; ++j) {
            long long i = base + j * 32 + lane;
            const bool ok = i < hi;
            unsigned valid = __ballot_sync(0xffffffffu, ok);
            uint32_t d = (k[j] >> shift) & mask;
            unsigned peers = warp_peers(d, nbits, valid);
            int leader = ok ? __ffs(peers) - 1 : lane;
            uint32_t p0 = (ok && lane == leader) ? run[warp][d] : 0u;
            p0 = __shfl_sync(0xffffffffu, p0, leader);
            if (ok) {
                uint32_t pos = p0 + __popc(peers & lt);
                kout[pos] = k[j];
                vout[pos] = v[j];
            }
            __syncwarp();
            if (ok && lane == leader) run[warp][d] = p0 + __popc(peers);
            __syncwarp();
        }
    }
}

static int radix_blocks(long long n_max)
{
    long long nb = (n_max + RS_WARPS * 1024 - 1) / (RS_WARPS * 1024);
    return (int)(nb < 1 ? 1 : (nb > RS_MAX_BLOCKS ? RS_MAX_BLOCKS : nb));
}

// Stable LSD sort of (k0, v0) by key bits [0, nbits); ping-pongs through (k1, v1); the final
// pass writes to (kf, vf), which must not alias the last pass's source.
static void radix_sort(const uint32_t *n_dev, long long n_max, int nbits, uint32_t *k0, uint32_t *v0, uint32_t *k1,
                        uint32_t *v1, uint32_t *kf, uint32_t *vf, const SortScratch &s, cudaStream_t st)
{
    if (nbits < 1) nbits = 1;
    const int passes = (nbits + 7) / 8;
    const int nb = radix_blocks(n_max);
    const long long ncounts = 256LL * nb * RS_WARPS;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p, bits = nbits - shift < 8 ? nbits - shift : 8;
        uint32_t *ks = (p & 1) ? k1 : k0, *vs = (p & 1) ? v1 : v0;
        uint32_t *kd = (p & 1) ? k0 : k1, *vd = (p & 1) ? v0 : v1;
        if (p == passes - 1) {
            kd = kf;
            vd = vf;
        }
        count_launch(2);
        k_radix_count<<<nb, RS_THREADS, 0, st>>>(ks, n_dev, shift, bits, s.counts);
        scan(LoadPlain{s.counts}, nullptr, ncounts, s.counts, s.block_sums, nullptr, nullptr, nullptr, -1, nullptr, st);
        k_radix_scatter<<<nb, RS_THREADS, 0, st>>>(ks, vs, kd, vd, n_dev, shift, bits, s.counts);
    }
}

// ------------------------------------------------------------------ key duplication

// Each warp takes 32 consecutive depth-ordered splats; their pairs occupy one contiguous
// range of the output, which the warp writes cooperatively (lane-strided, coalesced), each
// lane finding its splat by a 5-step binary search over the warp's offsets.
__global__ void __launch_bounds__(256) k_duplicate(const __grid_constant__ BatchParams P, const uint32_t *V_dev,
                                                   const uint32_t *__restrict__ order, const uint32_t *__restrict__ offs,
                                                   const float *__restrict__ splat, const int *__restrict__ radius,
                                                   const int *__restrict__ tiles, const uint32_t *n_use,
                                                   uint32_t *__restrict__ tkeys, uint32_t *__restrict__ tvals)
{
    const int lane = threadIdx.x & 31;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t V = *V_dev;
    if ((long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31) >= V) return;
    if (*n_use == 0) return;  // nothing to emit (no pairs, or capacity exceeded)
    const bool valid = k < V;
    uint32_t off = 0xffffffffu, cnt = 0, base = 0, w = 1, gx = 1, e = 0;
    if (valid) {
        e = order[k];
        off = offs[k];
        cnt = (uint32_t)tiles[e];
        const ItemParams &I = P.item[item_of_entry(P, e)];
        int x0, y0, x1, y1;
        tile_rect(splat[12 * e + 0], splat[12 * e + 1], radius[e], P.tw, P.th, I.gx, I.gy, x0, y0, x1, y1);
        base = (uint32_t)(I.tile_off + y0 * I.gx + x0);
        w = (uint32_t)(x1 - x0);
        gx = (uint32_t)I.gx;
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
        const uint32_t gj = __shfl_sync(0xffffffffu, gx, j);
        const uint32_t ej = __shfl_sync(0xffffffffu, e, j);
        if (p < p1) {
            const uint32_t local = p - oj;
            const uint32_t ty = local / wj, tx = local - ty * wj;
            tkeys[p] = bj + ty * gj + tx;
            tvals[p] = ej;
        }
    }
}

// ------------------------------------------------------------------ tile ranges

__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                                                     long long n_max, int n_tiles, int *__restrict__ tile_start)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = *n_dev;
    if (k > n || k > n_max) return;
    const long long prev = k > 0 ? (long long)keys[k - 1] : -1;
    const long long cur = k < n ? (long long)keys[k] : (long long)n_tiles;
    for (long long t = prev + 1; t <= cur && t <= n_tiles; ++t) tile_start[t] = (int)k;
}

// ------------------------------------------------------------------ orchestration

cudaError_t bin_sort_count(const BatchParams &P, const float *splat, const int *tiles, BinScratch &b,
                           long long *n_isect_dev, long long capacity, cudaStream_t st)
{
    const long long n = P.n_entries;
    uint32_t *V = b.scalars, *n_use = b.scalars + 1;
    // 1. visible entries -> compact (depth key, entry)
    scan(LoadVisible{tiles}, nullptr, n, b.vis_pos, b.sort.block_sums, V, nullptr, nullptr, -1, nullptr, st);
    if (n > 0) count_launch();
    if (n > 0) k_compact<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, tiles, splat, b.vis_pos, b.dkA, b.dvA);
    // 2. sort visible splats by depth (32 key bits); result (keys unused) ends in dvB
    radix_sort(V, n, 32, b.dkA, b.dvA, b.dkB, b.dvB, b.dkA /*final keys*/, b.vis_pos /*final order*/, b.sort, st);
    // 3. pair offsets in depth order; total -> n_isect; usable count (0 on overflow)
    scan(LoadGatherTiles{tiles, b.vis_pos}, V, n, b.offs, b.sort.block_sums, nullptr, n_isect_dev, n_use, capacity,
         b.status, st);
    return cudaGetLastError();
}

cudaError_t bin_sort_emit(const BatchParams &P, const float *splat, const int *radius, const int *tiles,
                          BinScratch &b, long long isect_max, int *gauss_ids, int *tile_start, cudaStream_t st)
{
    const long long n = P.n_entries;
    uint32_t *V = b.scalars, *n_use = b.scalars + 1;
    if (n > 0) count_launch();
    if (n > 0)
        k_duplicate<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, V, b.vis_pos, b.offs, splat, radius, tiles, n_use,
                                                                 b.tkA, b.tvA);
    int nbits = 0;
    while ((1LL << nbits) < (long long)P.n_tiles) ++nbits;
    const int passes = nbits < 1 ? 1 : (nbits + 7) / 8;
    // the last pass reads from A when the pass count is odd, from B when even
    uint32_t *kfinal = (passes & 1) ? b.tkB : b.tkA;
    radix_sort(n_use, isect_max, nbits, b.tkA, b.tvA, b.tkB, b.tvB, kfinal, reinterpret_cast<uint32_t *>(gauss_ids),
               b.sort, st);
    const long long nr = isect_max + 1;
    count_launch();
    k_tile_ranges<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(kfinal, n_use, isect_max, P.n_tiles, tile_start);
    return cudaGetLastError();
}

static size_t words_rounded(size_t words) { return ((words * 4 + 255) / 256) * 256; }

size_t entry_scratch_bytes(long long max_entries)
{
    size_t e = (size_t)(max_entries > 0 ? max_entries : 1);
    return 6 * words_rounded(e) + words_rounded(256ull * RS_MAX_BLOCKS * RS_WARPS) + words_rounded(SCAN_MAX_BLOCKS) +
           words_rounded(16);
}

size_t isect_scratch_bytes(long long max_isect)
{
    size_t i = (size_t)(max_isect > 0 ? max_isect : 1);
    return 4 * words_rounded(i);
}

void entry_scratch_carve(void *mem, long long max_entries, int *status, BinScratch &b)
{
    size_t e = (size_t)(max_entries > 0 ? max_entries : 1);
    char *p = static_cast<char *>(mem);
    auto take = [&](size_t words) {
        uint32_t *r = reinterpret_cast<uint32_t *>(p);
        p += words_rounded(words);
        return r;
    };
    b.vis_pos = take(e); b.dkA = take(e); b.dvA = take(e); b.dkB = take(e); b.dvB = take(e); b.offs = take(e);
    b.sort.counts = take(256ull * RS_MAX_BLOCKS * RS_WARPS);
    b.sort.block_sums = take(SCAN_MAX_BLOCKS);
    b.scalars = take(16);
    b.status = status;
}

void isect_scratch_carve(void *mem, long long max_isect, BinScratch &b)
{
    size_t i = (size_t)(max_isect > 0 ? max_isect : 1);
    char *p = static_cast<char *>(mem);
    auto take = [&](size_t words) {
        uint32_t *r = reinterpret_cast<uint32_t *>(p);
        p += words_rounded(words);
        return r;
    };
    b.tkA = take(i); b.tvA = take(i); b.tkB = take(i); b.tvB = take(i);
}

}  // namespace lobe
