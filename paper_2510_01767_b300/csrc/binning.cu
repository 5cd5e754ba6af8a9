// binning.cu -- tile binning: every (splat, tile) pair, grouped by tile, in (depth, entry) order.
//
// The 3DGS rasterizer obtains this order by radix-sorting 64-bit (tile << 32 | depth) keys of
// all duplicated pairs. Wide splats make that list long (tens of millions of pairs for a
// 200k-splat view) while each pixel uses only its first few hundred entries, so the sort
// dominates. Here the same order is reached without sorting the pairs at all:
//
//   1. compact the visible splats and sort them by depth (a few hundred thousand keys; four
//      one-launch radix passes);
//   2. duplicate them per SUPER-tile (S x S tiles, 64 px) in depth order -- the key carries the
//      super-tile id (bits 16..31) and the splat's tile rectangle relative to that super-tile
//      (4 x 4 bits) -- and stably sort those few million pairs by super-tile id: each
//      super-tile then holds its splats in depth order;
//   3. cut every super-tile's list into chunks of 256 (one CTA each); per chunk and tile, warp
//      ballots count the splats covering the tile; per (super-tile, tile) a prefix over its
//      chunks gives each chunk's offset and the tile's size; a scan of the sizes gives
//      tile_start; the chunks then write their splats' ids to each tile's range, in order,
//      with coalesced stores.
//
// A tile's list is its super-tile's list filtered by "tile in the splat's tile rectangle",
// which preserves (depth, entry) order, so the output equals the global pair sort bit for bit.
#include <type_traits>

#include "sort_prims.cuh"

namespace lobe {

constexpr int CHUNK = 256;    // splats per work item (BIN_THREADS)
constexpr int NT_MAX = 64;    // tiles per super-tile (S <= 8)
constexpr int KEY_SHIFT = 16; // super-tile id above, packed local rectangle below
constexpr long long MAX_SUPER = 1LL << 16;
constexpr long long MAX_SCAN_TILES = 1LL << 22;  // tiles per call (the tile scan's length)

// Per depth-ordered visible splat k: its super-rectangle area (area[k]) and what the pair
// expansion needs, in three words: info0 = super-tile id of the rectangle's origin | super
// grid width << 16, info1 = (x0, x1) and info2 = (y0, y1) of its tile rectangle relative to
// that origin (16 bits each). The rectangle comes from rect[e], stored by the compaction.
__global__ void __launch_bounds__(256) k_super_area(const __grid_constant__ BatchParams P, const uint32_t *V_dev,
                                                    const uint32_t *__restrict__ order, const uint2 *__restrict__ rect,
                                                    uint32_t *__restrict__ area, uint32_t *__restrict__ info0,
                                                    uint32_t *__restrict__ info1, uint32_t *__restrict__ info2)
{
    // the items' entry offsets and super-tile grids, in shared memory: the splats of a warp
    // belong to different items, and a search over the kernel parameters would serialise
    static_assert(LOBE_MAX_ITEMS <= 256, "one thread of the block per item");
    __shared__ int s_eoff[LOBE_MAX_ITEMS], s_soff[LOBE_MAX_ITEMS], s_sgx[LOBE_MAX_ITEMS];
    pdl_wait();
    const int n_items = P.n_items;
    if (threadIdx.x < n_items) {
        const ItemParams &I = P.item[threadIdx.x];
        s_eoff[threadIdx.x] = (int)I.entry_off;
        s_soff[threadIdx.x] = I.super_off;
        s_sgx[threadIdx.x] = I.sgx;
    }
    __syncthreads();
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *V_dev) return;
    const uint32_t e = order[k];
    const uint2 r = rect[e];
    int lo = 0, hi = n_items - 1;  // item of entry e: the last whose entries start at or before e
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((uint32_t)s_eoff[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const int x0 = (int)(r.x & 0xffffu), y0 = (int)(r.x >> 16), x1 = (int)(r.y & 0xffffu), y1 = (int)(r.y >> 16);
    const int S = P.S, sgx = s_sgx[lo];
    const int sx0 = x0 / S, sy0 = y0 / S;
    area[k] = (uint32_t)(((x1 + S - 1) / S - sx0) * ((y1 + S - 1) / S - sy0));
    info0[k] = (uint32_t)(s_soff[lo] + sy0 * sgx + sx0) | ((uint32_t)sgx << 16);
    info1[k] = (uint32_t)(x0 - sx0 * S) | ((uint32_t)(x1 - sx0 * S) << 16);
    info2[k] = (uint32_t)(y0 - sy0 * S) | ((uint32_t)(y1 - sy0 * S) << 16);
}

// Largest k in [0, n) with a[k] <= x, for non-decreasing a with a[0] <= x; called by a full
// warp (32-way search: about log32(n) rounds of one load per lane).
__device__ __forceinline__ uint32_t warp_upper_index(const uint32_t *a, uint32_t n, uint32_t x)
{
    const int lane = threadIdx.x & 31;
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t idx = lo + (uint32_t)lane * step;
        const bool ok = idx < hi && a[idx] <= x;
        const int c = __popc(__ballot_sync(0xffffffffu, ok));  // lanes 0..c-1 (a is sorted)
        lo += (uint32_t)(c - 1) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Expands the depth-ordered splats into super pairs, DUP_PAIRS output pairs per block (the
// work is even whatever the splat sizes): the block finds the splats overlapping its output
// range, marks each one's first pair, and a max-scan gives every pair its splat. Output p of
// splat k (local index l = p - offs[k] over its super-rectangle, row-major) gets key
// super-tile id << 16 | the splat's tile rectangle relative to that super-tile (x0, x1, y0, y1,
// clipped to [0, S], 4 bits each), value = entry id.
constexpr int DUP_PAIRS = 4096;
constexpr int DUP_PER = DUP_PAIRS / 256;  // scan positions per thread

__global__ void __launch_bounds__(256) k_super_dup(int S, const uint32_t *V_dev, const uint32_t *__restrict__ order,
                                                   const uint32_t *__restrict__ offs,
                                                   const uint32_t *__restrict__ info0,
                                                   const uint32_t *__restrict__ info1,
                                                   const uint32_t *__restrict__ info2, const uint32_t *n_sp_use,
                                                   uint32_t *__restrict__ skeys, uint32_t *__restrict__ svals)
{
    pdl_wait();
    __shared__ int s_idx[DUP_PAIRS + DUP_PAIRS / 32];  // padded: position j lives at j + j / 32
    __shared__ uint32_t s_k[2];
    __shared__ int s_wmax[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n = *n_sp_use;  // 0: no pairs, or more than the scratch holds
    const uint32_t P0 = blockIdx.x * DUP_PAIRS;
    if (P0 >= n) return;
    const uint32_t P1 = min(P0 + DUP_PAIRS, n);
    const uint32_t V = *V_dev;
    if (warp < 2) {
        const uint32_t k = warp_upper_index(offs, V, warp == 0 ? P0 : P1 - 1);
        if (lane == 0) s_k[warp] = k;
    }
    for (int j = threadIdx.x; j < DUP_PAIRS + DUP_PAIRS / 32; j += 256) s_idx[j] = -1;
    __syncthreads();
    const uint32_t k0 = s_k[0], m = s_k[1] - k0 + 1;  // m <= DUP_PAIRS (every splat has a pair)
    for (uint32_t i = threadIdx.x; i < m; i += 256) {
        const uint32_t o = offs[k0 + i];
        const uint32_t j = o > P0 ? o - P0 : 0u;
        s_idx[j + j / 32] = (int)i;
    }
    __syncthreads();
    // inclusive max-scan of s_idx: each thread owns DUP_PER consecutive positions
    int v[DUP_PER], run = -1;
#pragma unroll
    for (int r = 0; r < DUP_PER; ++r) {
        const int j = DUP_PER * threadIdx.x + r;
        run = max(run, s_idx[j + j / 32]);
        v[r] = run;
    }
    int inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = max(inc, y);
    }
    if (lane == 31) s_wmax[warp] = inc;
    __syncthreads();
    int before = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) before = -1;
    for (int w = 0; w < warp; ++w) before = max(before, s_wmax[w]);
#pragma unroll
    for (int r = 0; r < DUP_PER; ++r) {
        const int j = DUP_PER * threadIdx.x + r;
        s_idx[j + j / 32] = max(before, v[r]);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < (int)(P1 - P0); j += 256) {
        const uint32_t k = k0 + (uint32_t)s_idx[j + j / 32];
        const uint32_t p = P0 + (uint32_t)j;
        const uint32_t i0 = info0[k], i1 = info1[k], i2 = info2[k];
        const int rx0 = (int)(i1 & 0xffffu), rx1 = (int)(i1 >> 16), ry0 = (int)(i2 & 0xffffu), ry1 = (int)(i2 >> 16);
        const uint32_t w = (uint32_t)((rx1 + S - 1) / S);
        const uint32_t local = p - offs[k];
        const int sy = (int)(local / w), sx = (int)(local - (uint32_t)sy * w);
        const int lx0 = max(rx0 - sx * S, 0), lx1 = min(rx1 - sx * S, S);
        const int ly0 = max(ry0 - sy * S, 0), ly1 = min(ry1 - sy * S, S);
        skeys[p] = (((i0 & 0xffffu) + (uint32_t)sy * (i0 >> 16) + (uint32_t)sx) << KEY_SHIFT) |
                   (uint32_t)(lx0 | (lx1 << 4) | (ly0 << 8) | (ly1 << 12));
        svals[p] = order[k];
    }
}

// start[t] = first k with (keys[k] >> shift) >= t, for t in [0, n_keys]
__global__ void __launch_bounds__(256) k_key_ranges(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                                                    long long n_max, int shift, int n_keys, uint32_t *__restrict__ start)
{
    pdl_wait();
    const long long n = *n_dev < n_max ? (long long)*n_dev : n_max;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += (long long)gridDim.x * blockDim.x) {
        const long long prev = k > 0 ? (long long)(keys[k - 1] >> shift) : -1;
        const long long cur = k < n ? (long long)(keys[k] >> shift) : (long long)n_keys;
        for (long long t = prev + 1; t <= cur && t <= n_keys; ++t) start[t] = (uint32_t)k;
    }
}

// ------------------------------------------------------------------ chunk work items

struct LoadChunks {  // work items (chunks of CHUNK splats) of super-tile s
    const uint32_t *super_start;
    __device__ uint32_t operator()(long long s) const
    {
        return (super_start[s + 1] - super_start[s] + CHUNK - 1) / CHUNK;
    }
};

// Work item table: work[w] = (super-tile, first pair, end pair) of chunk w, so that the chunk
// kernels find their range with one load. One thread per super-tile writes its chunks.
__global__ void __launch_bounds__(256) k_chunk_map(const uint32_t *__restrict__ super_start,
                                                   const uint32_t *__restrict__ chunk_base, int n_super,
                                                   uint4 *__restrict__ work)
{
    pdl_wait();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_super) return;
    const uint32_t b0 = chunk_base[s], b1 = chunk_base[s + 1], p0 = super_start[s], p1 = super_start[s + 1];
    for (uint32_t w = b0; w < b1; ++w) {
        const uint32_t lo = p0 + (w - b0) * CHUNK;
        work[w] = make_uint4((uint32_t)s, lo, min(lo + CHUNK, p1), 0u);
    }
}

// Local tiles of the super-tile that a super pair's key covers, as a bit mask (bit ty * S + tx):
// the row's bits [x0, x1) repeated on rows [y0, y1). The row spreads as a multiplication by a
// word with bit S * y set for every covered row, so no carries cross rows (the row is S bits
// wide). An empty rectangle (the key 0 of a missing pair) gives 0.
template <int S>
struct CoverMask {
    using T = typename std::conditional<S == 8, unsigned long long, uint32_t>::type;
    static constexpr T ROWS = S == 8 ? (T)0x0101010101010101ull : (T)0x1111u;  // bit S * y for y < S
    __device__ static __forceinline__ T of(uint32_t key)
    {
        const uint32_t x0 = key & 15u, x1 = (key >> 4) & 15u, y0 = (key >> 8) & 15u, y1 = (key >> 12) & 15u;
        const uint32_t row = ((1u << x1) - 1u) & ~((1u << x0) - 1u);
        const T below1 = y1 >= (uint32_t)S ? ROWS : (T)(ROWS & (((T)1 << (S * y1)) - 1));
        const T below0 = y0 >= (uint32_t)S ? ROWS : (T)(ROWS & (((T)1 << (S * y0)) - 1));
        return (T)row * (below1 & ~below0);
    }
};

// Per local tile, how many of the warp's 32 keys cover it, four tiles a word: byte j of
// word q counts tile 4q + j (at most 32, so the bytes never carry). Each lane spreads four
// mask bits into the low bits of four bytes (the multiplication places bit j at bit 8j, the
// mask drops the other copies) and one integer warp reduction adds the words of all lanes.
template <int S>
__device__ __forceinline__ void warp_tile_counts(typename CoverMask<S>::T mask, uint32_t (&c)[S * S / 4])
{
#pragma unroll
    for (int q = 0; q < S * S / 4; ++q) {
        const uint32_t nib = (uint32_t)(mask >> (4 * q)) & 15u;
        c[q] = __reduce_add_sync(0xffffffffu, (nib * 0x00204081u) & 0x01010101u);
    }
}

// Pass 1: cnt[w * S*S + t] = splats of chunk w covering local tile t.
template <int S>
__global__ void __launch_bounds__(BIN_THREADS) k_chunk_count(const uint32_t *__restrict__ keys,
                                                             const uint4 *__restrict__ work,
                                                             const uint32_t *__restrict__ chunk_base, int n_super,
                                                             uint32_t *__restrict__ cnt)
{
    pdl_wait();
    constexpr int NT = S * S;
    __shared__ uint32_t wc[BIN_THREADS / 32][NT / 4];  // packed per-warp counts
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n_work = chunk_base[n_super];
    uint32_t w = blockIdx.x;
    uint4 wk = w < n_work ? work[w] : make_uint4(0u, 0u, 0u, 0u);
    while (w < n_work) {
        const uint32_t i = wk.y + threadIdx.x;
        const auto mask = CoverMask<S>::of(i < wk.z ? keys[i] : 0u);  // 0 = empty rectangle
        const uint32_t wn = w + gridDim.x;
        const uint4 wkn = wn < n_work ? work[wn] : make_uint4(0u, 0u, 0u, 0u);  // next item, in flight
        uint32_t c4[NT / 4];
        warp_tile_counts<S>(mask, c4);
#pragma unroll
        for (int q = 0; q < NT / 4; ++q)
            if (lane == q) wc[warp][q] = c4[q];
        __syncthreads();
        if (threadIdx.x < NT) {
            uint32_t c = 0;
#pragma unroll
            for (int q = 0; q < BIN_THREADS / 32; ++q) c += (wc[q][threadIdx.x >> 2] >> (8 * (threadIdx.x & 3))) & 255u;
            cnt[(size_t)w * NT + threadIdx.x] = c;
        }
        __syncthreads();
        w = wn;
        wk = wkn;
    }
}

// Pass 2, one block per super-tile: per local tile, the chunk counts become each chunk's offset
// within the tile (in place) and their sum the tile's size -> tile_count[global tile]. The
// block's 256 threads are NT tiles x G groups; group g scans a contiguous run of the chunks.
template <int S>
__global__ void __launch_bounds__(256) k_chunk_prefix(const __grid_constant__ BatchParams P,
                                                      const uint32_t *__restrict__ chunk_base, uint32_t *__restrict__ cnt,
                                                      uint32_t *__restrict__ tile_count)
{
    pdl_wait();
    constexpr int NT = S * S, G = 256 / NT;
    __shared__ uint32_t part[G][NT];
    const int s = blockIdx.x, t = threadIdx.x % NT, g = threadIdx.x / NT;
    const uint32_t c0 = chunk_base[s], c1 = chunk_base[s + 1];
    const uint32_t per = (c1 - c0 + G - 1) / G;
    const uint32_t w0 = min(c0 + g * per, c1), w1 = min(w0 + per, c1);
    uint32_t sum = 0;
    for (uint32_t w = w0; w < w1; ++w) sum += cnt[(size_t)w * NT + t];
    part[g][t] = sum;
    __syncthreads();
    uint32_t run = 0, total = 0;
#pragma unroll
    for (int q = 0; q < G; ++q) {
        const uint32_t v = part[q][t];
        run += q < g ? v : 0u;
        total += v;
    }
    for (uint32_t w = w0; w < w1; ++w) {
        const uint32_t c = cnt[(size_t)w * NT + t];
        cnt[(size_t)w * NT + t] = run;
        run += c;
    }
    if (g == 0) {
        const ItemParams &I = P.item[item_of_super(P, s)];
        const int ls = s - I.super_off, tx = (ls % I.sgx) * S + t % S, ty = (ls / I.sgx) * S + t / S;
        if (tx < I.gx && ty < I.gy) tile_count[I.tile_off + ty * I.gx + tx] = total;
    }
}

// Pass 3: each chunk's splats, in list order, to their tiles' ranges. Per tile, warp w's
// splats start at (tile's range start) + (chunk's offset in the tile) + (splats of warps < w):
// that sum is formed once per (warp, tile) in shared memory; a splat's rank among its warp's
// splats of the tile is the count of lower lanes in the tile's ballot.
template <int S>
__global__ void __launch_bounds__(BIN_THREADS) k_chunk_emit(const __grid_constant__ BatchParams P,
                                                            const uint32_t *__restrict__ keys,
                                                            const uint32_t *__restrict__ vals,
                                                            const uint4 *__restrict__ work,
                                                            const uint32_t *__restrict__ chunk_base,
                                                            const uint32_t *__restrict__ cnt,
                                                            const int *__restrict__ tile_start, const uint32_t *n_use,
                                                            int *__restrict__ gauss_ids)
{
    pdl_wait();
    constexpr int NT = S * S;
    __shared__ uint32_t wc[BIN_THREADS / 32][NT];
    __shared__ uint32_t wcp[BIN_THREADS / 32][NT / 4];  // packed per-warp counts
    if (*n_use == 0) return;  // no pairs, or more than the bins hold
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int n_super = P.n_super;
    const uint32_t n_work = chunk_base[n_super];
    uint32_t w = blockIdx.x;
    uint4 wk = w < n_work ? work[w] : make_uint4(0u, 0u, 0u, 0u);
    while (w < n_work) {
        // this chunk's splats, its tiles' bases and the next work item, loaded together
        const int s = (int)wk.x;
        const uint32_t i = wk.y + threadIdx.x;
        const auto mask = CoverMask<S>::of(i < wk.z ? keys[i] : 0u);
        const int id = i < wk.z ? (int)vals[i] : 0;
        uint32_t tbase = 0;
        if (threadIdx.x < NT) {
            const ItemParams &I = P.item[item_of_super(P, s)];
            const int ls = s - I.super_off;
            const int tx = (ls % I.sgx) * S + (int)threadIdx.x % S, ty = (ls / I.sgx) * S + (int)threadIdx.x / S;
            const uint32_t ts = (tx < I.gx && ty < I.gy) ? (uint32_t)tile_start[I.tile_off + ty * I.gx + tx] : 0u;
            tbase = ts + cnt[(size_t)w * NT + threadIdx.x];
        }
        const uint32_t wn = w + gridDim.x;
        const uint4 wkn = wn < n_work ? work[wn] : make_uint4(0u, 0u, 0u, 0u);
        uint32_t c4[NT / 4];
        warp_tile_counts<S>(mask, c4);
#pragma unroll
        for (int q = 0; q < NT / 4; ++q)
            if (lane == q) wcp[warp][q] = c4[q];
        __syncthreads();
        if (threadIdx.x < NT) {
            uint32_t r = tbase;
#pragma unroll
            for (int q = 0; q < BIN_THREADS / 32; ++q) {
                wc[q][threadIdx.x] = r;
                r += (wcp[q][threadIdx.x >> 2] >> (8 * (threadIdx.x & 3))) & 255u;
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const bool cov = (mask >> t) & 1u;
            const unsigned m = __ballot_sync(0xffffffffu, cov);
            if (cov) gauss_ids[wc[warp][t] + __popc(m & lt)] = id;
        }
        __syncthreads();
        w = wn;
        wk = wkn;
    }
}

// after an overflow the bins describe empty tiles
__global__ void __launch_bounds__(256) k_clear_on_overflow(const uint32_t *n_use, const long long *total, int n_tiles,
                                                           int *__restrict__ tile_start)
{
    pdl_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= n_tiles && *n_use == 0 && *total != 0) tile_start[t] = 0;
}

// ------------------------------------------------------------------ orchestration

// Grid of the persistent chunk kernels: 16 blocks for every SM of the current device (two
// rounds of the 8 resident 256-thread blocks an SM holds), or fewer for fewer work items.
static unsigned persistent_grid(long long work_max)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    const long long cap = (long long)sms * 16;
    return (unsigned)(work_max < 1 ? 1 : (work_max < cap ? work_max : cap));
}

static LB lb_of(const BinScratch &b, int stage) { return LB{b.scan_slots, b.ctl, stage}; }

// Step 1 and the super-pair count: visible splats in depth order (vis_pos), per-splat super
// pair offsets (offs), the super pair total (scalars[4]) and its usable count (scalars[1]: the
// total, or 0 with a latched error when it exceeds pair_capacity; < 0 = unchecked). The first
// kernel opens the call's look-back generation.
cudaError_t bin_super_count(const BatchParams &P, const float *splat, const int *radius, const int *tiles,
                            BinScratch &b, long long pair_capacity, cudaStream_t st)
{
    const long long n = P.n_entries;
    uint32_t *V = b.scalars, *n_sp = b.scalars + 1, *sp_total = b.scalars + 4;
    {
        const long long nt = (n + CH_SPAN - 1) / CH_SPAN;
        count_launch();
        launch_pdl(k_compact, dim3((unsigned)(nt < 1 ? 1 : nt)), dim3(CH_THREADS), 0, st, P, tiles, splat, radius, b.dkA,
                   b.dvA, b.rect, b.os_hist, V, lb_of(b, ST_SCAN_VISIBLE));
    }
    onesweep_sort32(V, n, b.dkA, b.dvA, b.dkB, b.dvB, b.dkA, b.vis_pos, b.os_hist, b.os_slots, lb_of(b, ST_DEPTH_PASS),
                    st);
    if (n > 0) {
        count_launch();
        launch_pdl(k_super_area, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, P, V, b.vis_pos, b.rect, b.offs, b.dkA,
                   b.dvA, b.dkB);  // free after the depth sort
    }
    scan(LoadPlain{b.offs}, V, n, b.offs, sp_total, nullptr, n_sp, pair_capacity, lb_of(b, ST_SCAN_OFFS), st);
    return cudaGetLastError();
}

// Super pairs -> sorted super-tile lists -> per-chunk tile counts -> tile_start (in place), the
// pair count (n_isect) and its usable count (scalars[2], 0 when above isect_capacity).
cudaError_t bin_tile_count(const BatchParams &P, const float *splat, const int *radius, BinScratch &b,
                           long long pair_capacity, long long *n_isect_dev, int *tile_start, long long isect_capacity,
                           cudaStream_t st)
{
    const long long n = P.n_entries;
    uint32_t *V = b.scalars, *n_sp = b.scalars + 1, *n_use = b.scalars + 2;
    {
        count_launch();
        const long long nb = (pair_capacity + DUP_PAIRS - 1) / DUP_PAIRS;
        launch_pdl(k_super_dup, dim3((unsigned)(nb < 1 ? 1 : nb)), dim3(256), 0, st, P.S, V, b.vis_pos, b.offs, b.dkA, b.dvA, b.dkB, n_sp,
                                                                 b.skA, b.svA);
    }
    int nbits = 0;
    while ((1LL << nbits) < (long long)P.n_super) ++nbits;
    const int passes = nbits < 1 ? 1 : (nbits + 8) / 9;  // as radix_sort
    uint32_t *kfinal = (passes & 1) ? b.skB : b.skA;  // not the last pass's source
    uint32_t *vfinal = (passes & 1) ? b.svB : b.svA;
    radix_sort(n_sp, pair_capacity, KEY_SHIFT, nbits, b.skA, b.svA, b.skB, b.svB, kfinal, vfinal, b.counts,
               lb_of(b, ST_SUPER_PASS), st);
    b.sp_keys = kfinal;
    b.sp_ids = vfinal;
    count_launch();
    const long long rblocks = (pair_capacity + 1 + 255) / 256;
    launch_pdl(k_key_ranges, dim3((unsigned)(rblocks < 2368 ? rblocks : 2368)), dim3(256), 0, st, kfinal, n_sp, pair_capacity, KEY_SHIFT,
                                                                                P.n_super, b.super_start);
    // chunk work items: chunk_base[s] = first work item of super-tile s, chunk_base[n_super] = total
    scan(LoadChunks{b.super_start}, nullptr, P.n_super, b.chunk_base, b.chunk_base + P.n_super, nullptr, nullptr, -1,
         lb_of(b, ST_SCAN_CHUNKS), st);
    const long long work_max = pair_capacity / CHUNK + P.n_super + 1;
    uint32_t *ts = reinterpret_cast<uint32_t *>(tile_start);
    if (P.n_super > 0) {
        count_launch(3);
        launch_pdl(k_chunk_map, dim3((P.n_super + 255) / 256), dim3(256), 0, st, b.super_start, b.chunk_base, P.n_super, b.work);
        if (P.S == 8) {
            launch_pdl(k_chunk_count<8>, dim3(persistent_grid(work_max)), dim3(BIN_THREADS), 0, st, b.sp_keys, b.work, b.chunk_base,
                                                                                P.n_super, b.chunk_cnt);
            launch_pdl(k_chunk_prefix<8>, dim3(P.n_super), dim3(256), 0, st, P, b.chunk_base, b.chunk_cnt, ts);
        } else {
            launch_pdl(k_chunk_count<4>, dim3(persistent_grid(work_max)), dim3(BIN_THREADS), 0, st, b.sp_keys, b.work, b.chunk_base,
                                                                                P.n_super, b.chunk_cnt);
            launch_pdl(k_chunk_prefix<4>, dim3(P.n_super), dim3(256), 0, st, P, b.chunk_base, b.chunk_cnt, ts);
        }
    }
    // the scan's grand total lands in tile_start[n_tiles] and in the caller's n_isect
    scan(LoadPlain{ts}, nullptr, P.n_tiles, ts, ts + P.n_tiles, n_isect_dev, n_use, isect_capacity,
         lb_of(b, ST_SCAN_TILES), st);
    b.work_max = work_max;
    return cudaGetLastError();
}

cudaError_t bin_sort_emit(const BatchParams &P, const float *splat, const int *radius, BinScratch &b,
                          const long long *n_isect_dev, int *gauss_ids, int *tile_start, cudaStream_t st)
{
    (void)splat;
    (void)radius;
    const uint32_t *n_use = b.scalars + 2;
    if (P.n_super > 0) {
        count_launch();
        const unsigned grid = persistent_grid(b.work_max);
        if (P.S == 8)
            launch_pdl(k_chunk_emit<8>, dim3(grid), dim3(BIN_THREADS), 0, st, P, b.sp_keys, b.sp_ids, b.work, b.chunk_base,
                                                          b.chunk_cnt, tile_start, n_use, gauss_ids);
        else
            launch_pdl(k_chunk_emit<4>, dim3(grid), dim3(BIN_THREADS), 0, st, P, b.sp_keys, b.sp_ids, b.work, b.chunk_base,
                                                          b.chunk_cnt, tile_start, n_use, gauss_ids);
    }
    count_launch();
    launch_pdl(k_clear_on_overflow, dim3((P.n_tiles + 1 + 255) / 256), dim3(256), 0, st, n_use, n_isect_dev, P.n_tiles, tile_start);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ scratch layout
//
// entry part: 6 arrays of max_entries words, the radix digit counts (sized for the larger of
//             the counts and 2 words per entry: the same words hold the tile rectangles from
//             the compaction to the pass over the depth-ordered splats, before the super-tile
//             sort counts), scalars, the look-back words of the scans and the compaction (one
//             per tile of the longest of them), the depth keys' four digit histograms, the depth sort's look-back
//             words (256 per OS_TILE entries)
// pair part:  4 arrays of max_pairs words (super-tile pairs, ping-pong), the chunk work table
//             (16 B per chunk), per-chunk tile counts
// super part: super-tile list starts and chunk bases (max_super + 1 words each)
// Look-back slots must be zero (or hold words of earlier calls) before first use.

static size_t words_rounded(size_t words) { return ((words * 4 + 255) / 256) * 256; }
// look-back words of the scans and of the compaction (one per tile of the longest of them)
static long long lookback_slots(long long max_entries)
{
    const long long a = scan_slots(max_scan_length(max_entries));
    const long long c = ((max_entries > 0 ? max_entries : 1) + CH_SPAN - 1) / CH_SPAN;
    return a > c ? a : c;
}
static size_t count_words(size_t e)
{
    const size_t c = (size_t)RS_MAX_DIGITS * RS_MAX_BLOCKS;
    return c > 2 * e ? c : 2 * e;
}
static size_t slots_rounded(long long slots) { return (((size_t)slots * 8 + 255) / 256) * 256; }

size_t entry_scratch_bytes(long long max_entries)
{
    size_t e = (size_t)(max_entries > 0 ? max_entries : 1);
    return 6 * words_rounded(e) + words_rounded(count_words(e)) + words_rounded(16) +
           slots_rounded(lookback_slots(max_entries)) + words_rounded(4 * 256) +
           slots_rounded(onesweep_slots(max_entries));
}

size_t pair_scratch_bytes(long long max_pairs, long long max_super)
{
    size_t i = (size_t)(max_pairs > 0 ? max_pairs : 1);
    size_t chunks = (size_t)(max_pairs / CHUNK + (max_super > 0 ? max_super : 1) + 1);
    return 4 * words_rounded(i) + words_rounded(chunks * 4) + words_rounded(chunks * NT_MAX);
}

size_t super_scratch_bytes(long long max_super)
{
    return 2 * words_rounded((size_t)(max_super > 0 ? max_super : 1) + 1);
}

long long max_super_tiles() { return MAX_SUPER; }
long long max_scan_length(long long max_entries)
{
    return max_entries > MAX_SCAN_TILES ? max_entries : MAX_SCAN_TILES;
}

struct Carver {
    char *p;
    uint32_t *take(size_t words)
    {
        uint32_t *r = reinterpret_cast<uint32_t *>(p);
        p += words_rounded(words);
        return r;
    }
    unsigned long long *take_slots(long long slots)
    {
        unsigned long long *r = reinterpret_cast<unsigned long long *>(p);
        p += slots_rounded(slots);
        return r;
    }
};

void entry_scratch_carve(void *mem, long long max_entries, int *ctl, BinScratch &b)
{
    size_t e = (size_t)(max_entries > 0 ? max_entries : 1);
    Carver c{static_cast<char *>(mem)};
    b.vis_pos = c.take(e); b.dkA = c.take(e); b.dvA = c.take(e); b.dkB = c.take(e); b.dvB = c.take(e);
    b.offs = c.take(e);
    b.counts = c.take(count_words(e));
    b.rect = reinterpret_cast<uint2 *>(b.counts);
    b.scalars = c.take(16);
    b.scan_slots = c.take_slots(lookback_slots(max_entries));
    b.os_hist = c.take(4 * 256);
    b.os_slots = c.take_slots(onesweep_slots(max_entries));
    b.ctl = ctl;
    b.status = ctl;
}

void pair_scratch_carve(void *mem, long long max_pairs, long long max_super, BinScratch &b)
{
    size_t i = (size_t)(max_pairs > 0 ? max_pairs : 1);
    Carver c{static_cast<char *>(mem)};
    b.skA = c.take(i); b.svA = c.take(i); b.skB = c.take(i); b.svB = c.take(i);
    const size_t chunks = (size_t)(max_pairs / CHUNK) + (size_t)(max_super > 0 ? max_super : 1) + 1;
    b.work = reinterpret_cast<uint4 *>(c.take(chunks * 4));
    b.chunk_cnt = c.take(1);  // the per-chunk counts run to the end of the region
}

void super_scratch_carve(void *mem, long long max_super, BinScratch &b)
{
    Carver c{static_cast<char *>(mem)};
    const size_t w = (size_t)(max_super > 0 ? max_super : 1) + 1;
    b.super_start = c.take(w);
    b.chunk_base = c.take(w);
}

}  // namespace lobe
