// sort_prims.cuh -- device primitives of the binning stage (included by binning.cu only):
// a single-pass exclusive scan with a device-side length (decoupled look-back, lookback.cuh),
// compaction of visible splats with the digit histograms of their depth keys, and two stable
// LSD radix sorts of (key, value) pairs:
//   - radix_sort: per pass, digit counts per block, their scan, a block-chunked scatter (three
//     launches a pass; any digit width up to 9 bits);
//   - onesweep_sort32: all 32 bits in four 8-bit passes of one launch each, the digit offsets
//     of earlier tiles found by per-digit look-back (Adinets & Merrill, "Onesweep: A Faster
//     Least Significant Digit Radix Sort for GPUs", 2022).
// Both rank tiles of keys with warp ballots, reorder each tile by digit in shared memory
// and write runs of equal digits with coalesced stores. Every result is deterministic.
#include "lookback.cuh"

namespace lobe {

constexpr int RS_WARPS = 8;
constexpr int RS_THREADS = RS_WARPS * 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // elements ranked and staged per tile
constexpr int RS_MAX_BLOCKS = 1184;             // 8 per SM on 148 SMs
constexpr int BIN_THREADS = 256;

// ------------------------------------------------------------------ compaction of visible splats

// One pass over the projected entries, in ticket order with decoupled look-back: the visible
// ones (touching at least one tile) are compacted in entry order to (dkeys, dvals) = (fp32
// depth bits, entry id) -- positive depths order like unsigned ints -- and their count goes to
// *V. Each block also adds its keys' digit counts to the four 8-bit digit histograms of the
// depth sort, hist[p * 256 + d] = visible keys with (key >> 8p) & 255 == d, and stores each
// visible entry's tile rectangle, rect[e] = (x0 | y0 << 16, x1 | y1 << 16): the pass over the
// depth-ordered splats then gathers these 8 bytes instead of the splat's position and radius.
// The block of tile 0 zeroes hist before it publishes its prefix; every other block adds to
// hist only after its look-back has seen a published prefix, which orders the additions after
// the zeroing. Warp w of a block owns CH_ITEMS rounds of 32 consecutive entries.
constexpr int CH_THREADS = 256;
constexpr int CH_ITEMS = 8;
constexpr int CH_SPAN = CH_THREADS * CH_ITEMS;

__global__ void __launch_bounds__(CH_THREADS) k_compact(const __grid_constant__ BatchParams P,
                                                        const int *__restrict__ tiles, const float *__restrict__ splat,
                                                        const int *__restrict__ radius, uint32_t *__restrict__ dkeys,
                                                        uint32_t *__restrict__ dvals, uint2 *__restrict__ rect,
                                                        uint32_t *__restrict__ hist, uint32_t *__restrict__ V, LB lb)
{
    pdl_wait();
    __shared__ uint32_t h[4 * 256];
    __shared__ int s_tile;
    __shared__ uint32_t s_gen, s_prefix;
    __shared__ uint32_t s_warp[CH_THREADS / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        int t;
        uint32_t g;
        lb_take(lb.ctl, lb.stage, true, t, g);  // opens this call's look-back generation
        s_tile = t;
        s_gen = g;
    }
    for (int i = threadIdx.x; i < 4 * 256; i += CH_THREADS) h[i] = 0;
    __syncthreads();
    const int tile = s_tile;
    const long long n = P.n_entries;
    const long long ntiles = (n + CH_SPAN - 1) / CH_SPAN;
    if (tile >= (ntiles > 0 ? ntiles : 1)) return;
    const uint32_t tag = lb_tag(s_gen, lb.stage);
    const long long w0 = (long long)tile * CH_SPAN + (long long)warp * (32 * CH_ITEMS);
    const unsigned lt = lanemask_lt();
    bool vis[CH_ITEMS];
    uint32_t rank[CH_ITEMS], key[CH_ITEMS], carry = 0;
#pragma unroll
    for (int r = 0; r < CH_ITEMS; ++r) {
        const long long e = w0 + r * 32 + lane;
        vis[r] = e < n && tiles[e] > 0;
        const unsigned m = __ballot_sync(0xffffffffu, vis[r]);
        rank[r] = carry + __popc(m & lt);
        carry += __popc(m);
    }
#pragma unroll
    for (int r = 0; r < CH_ITEMS; ++r) {
        key[r] = 0u;
        if (!vis[r]) continue;
        const long long e = w0 + r * 32 + lane;
        key[r] = __float_as_uint(splat[12 * e + 9]);
        const ItemParams &I = P.item[item_of_entry(P, e)];
        const float2 uv = *reinterpret_cast<const float2 *>(splat + 12 * e);
        int x0, y0, x1, y1;
        tile_rect(uv.x, uv.y, radius[e], P.tw, P.th, I.gx, I.gy, x0, y0, x1, y1);
        rect[e] = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
        atomicAdd(&h[key[r] & 255u], 1u);
        atomicAdd(&h[256 + ((key[r] >> 8) & 255u)], 1u);
        atomicAdd(&h[512 + ((key[r] >> 16) & 255u)], 1u);
        atomicAdd(&h[768 + (key[r] >> 24)], 1u);
    }
    uint32_t wex;
    const uint32_t agg = block_exclusive_scan<CH_THREADS>(lane == 0 ? carry : 0u, wex, s_warp);
    wex = __shfl_sync(0xffffffffu, wex, 0);
    if (warp == 0) {
        unsigned long long *slot = lb.slots + tile;
        uint32_t prefix = 0;
        if (tile == 0) {
            for (int i = lane; i < 4 * 256; i += 32) hist[i] = 0u;
            __threadfence();
            if (lane == 0) lb_publish(slot, tag, LB_INC, agg);
        } else {
            if (lane == 0) lb_publish(slot, tag, LB_AGG, agg);
            prefix = lb_exclusive_warp(lb.slots, tile, tag, lb.ctl);
            __threadfence();  // the zeroing of hist is visible from here on
            if (lane == 0) lb_publish(slot, tag, LB_INC, prefix + agg);
        }
        if (lane == 0) {
            s_prefix = prefix;
            if (tile == (ntiles > 0 ? ntiles - 1 : 0)) *V = prefix + agg;
        }
    }
    __syncthreads();
    const uint32_t base = s_prefix + wex;
#pragma unroll
    for (int r = 0; r < CH_ITEMS; ++r) {
        if (!vis[r]) continue;
        dkeys[base + rank[r]] = key[r];
        dvals[base + rank[r]] = (uint32_t)(w0 + r * 32 + lane);
    }
    for (int i = threadIdx.x; i < 4 * 256; i += CH_THREADS)
        if (h[i]) atomicAdd(hist + i, h[i]);
}

// ------------------------------------------------------------------ radix sort (LSD, <= 9 bits/pass)

__device__ __forceinline__ void chunk_of(long long n, int b, int nb, long long &lo, long long &hi)
{
    long long chunk = (n + nb - 1) / nb;
    lo = (long long)b * chunk;
    hi = lo + chunk < n ? lo + chunk : n;
    if (lo > n) lo = n;
}

// Lanes of the warp holding the same digit as this lane (restricted to `valid`): one ballot a
// digit bit (measured faster here than __match_any_sync).
__device__ __forceinline__ unsigned warp_peers(uint32_t d, int nbits, unsigned valid)
{
    unsigned peers = valid;
    for (int b = 0; b < nbits; ++b) {
        unsigned bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bal : ~bal;
    }
    return peers;
}

// Radix passes take digits of up to 9 bits: DIG = 256 or 512 digit slots per pass.
constexpr int RS_MAX_DIGITS = 512;

// counts[d * nb + b] = keys of block b's chunk with digit d
template <int DIG>
__global__ void __launch_bounds__(RS_THREADS) k_radix_count(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                                                            int shift, int nbits, uint32_t *__restrict__ counts)
{
    pdl_wait();
    __shared__ uint32_t h[RS_WARPS][DIG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < DIG; d += 32) h[warp][d] = 0;
    __syncwarp();
    long long lo, hi;
    chunk_of(*n_dev, blockIdx.x, gridDim.x, lo, hi);
    const uint32_t mask = (1u << nbits) - 1u;
    // counts only (no ranks): one shared-memory atomic a key into the warp's own histogram,
    // eight independent loads a thread in flight
    for (long long base = lo + warp * 32; base < hi; base += RS_THREADS * 8) {
        uint32_t k[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const long long i = base + j * RS_THREADS + lane;
            k[j] = i < hi ? keys[i] : 0u;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (base + j * RS_THREADS + lane < hi) atomicAdd(&h[warp][(k[j] >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < DIG; d += RS_THREADS) {
        uint32_t s = 0;
        for (int w = 0; w < RS_WARPS; ++w) s += h[w][d];
        counts[(long long)d * gridDim.x + blockIdx.x] = s;
    }
}

// One pass: block b scatters its chunk [lo, hi) to offsets[d * nb + b] + (running count).
// Thread t handles digits t * DPT .. t * DPT + DPT - 1 (DPT = DIG / 256) in the per-digit steps.
template <int DIG>
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                              const uint32_t *__restrict__ vin,
                                                              uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                              const uint32_t *n_dev, int shift, int nbits,
                                                              const uint32_t *__restrict__ offsets)
{
    pdl_wait();
    constexpr int DPT = DIG / RS_THREADS;
    __shared__ uint32_t s_k[RS_TILE];
    __shared__ uint32_t s_v[RS_TILE];
    __shared__ uint32_t wcnt[RS_WARPS][DIG];
    __shared__ uint32_t local_off[DIG], tile_cnt[DIG], grun[DIG];
    __shared__ uint32_t scan_sm[RS_THREADS / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    const unsigned lt = lanemask_lt();
    const uint32_t mask = (1u << nbits) - 1u;
    long long lo, hi;
    chunk_of(*n_dev, blockIdx.x, gridDim.x, lo, hi);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        grun[d] = offsets[(long long)d * gridDim.x + blockIdx.x];
    }
    for (long long tb = lo; tb < hi; tb += RS_TILE) {
        for (int d = lane; d < DIG; d += 32) wcnt[warp][d] = 0;
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
            uint32_t run[DPT], sum = 0;
#pragma unroll
            for (int q = 0; q < DPT; ++q) {
                const int d = tid * DPT + q;
                uint32_t r = 0;
#pragma unroll
                for (int w = 0; w < RS_WARPS; ++w) {
                    uint32_t c = wcnt[w][d];
                    wcnt[w][d] = r;
                    r += c;
                }
                tile_cnt[d] = r;
                run[q] = r;
                sum += r;
            }
            uint32_t ex;
            block_exclusive_scan<RS_THREADS>(sum, ex, scan_sm);
#pragma unroll
            for (int q = 0; q < DPT; ++q) {
                local_off[tid * DPT + q] = ex;
                ex += run[q];
            }
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
#pragma unroll
        for (int q = 0; q < DPT; ++q) grun[tid * DPT + q] += tile_cnt[tid * DPT + q];
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
// Passes = ceil(nbits / 9) with digits ceil(nbits / passes) wide. Keys move with their values,
// so bits outside the sorted range travel along untouched. Pass p's count scan is stage
// lb.stage + p.
static void radix_sort(const uint32_t *n_dev, long long n_max, int shift0, int nbits, uint32_t *k0, uint32_t *v0,
                       uint32_t *k1, uint32_t *v1, uint32_t *kf, uint32_t *vf, uint32_t *counts, LB lb,
                       cudaStream_t st)
{
    if (nbits < 1) nbits = 1;
    const int passes = (nbits + 8) / 9;
    const int width = (nbits + passes - 1) / passes;
    const int nb = radix_blocks(n_max);
    const int stage0 = lb.stage;
    for (int p = 0; p < passes; ++p) {
        const int lo = width * p, bits = nbits - lo < width ? nbits - lo : width;
        uint32_t *ks = (p & 1) ? k1 : k0, *vs = (p & 1) ? v1 : v0;
        uint32_t *kd = (p & 1) ? k0 : k1, *vd = (p & 1) ? v0 : v1;
        if (p == passes - 1) {
            kd = kf;
            vd = vf;
        }
        lb.stage = stage0 + p;
        count_launch(2);
        if (bits <= 8) {
            launch_pdl(k_radix_count<256>, dim3(nb), dim3(RS_THREADS), 0, st, ks, n_dev, shift0 + lo, bits, counts);
            scan(LoadPlain{counts}, nullptr, 256LL * nb, counts, nullptr, nullptr, nullptr, -1, lb, st);
            launch_pdl(k_radix_scatter<256>, dim3(nb), dim3(RS_THREADS), 0, st, ks, vs, kd, vd, n_dev, shift0 + lo, bits, counts);
        } else {
            launch_pdl(k_radix_count<512>, dim3(nb), dim3(RS_THREADS), 0, st, ks, n_dev, shift0 + lo, bits, counts);
            scan(LoadPlain{counts}, nullptr, 512LL * nb, counts, nullptr, nullptr, nullptr, -1, lb, st);
            launch_pdl(k_radix_scatter<512>, dim3(nb), dim3(RS_THREADS), 0, st, ks, vs, kd, vd, n_dev, shift0 + lo, bits, counts);
        }
    }
}

// ------------------------------------------------------------------ onesweep (one launch a pass)

// Tile of a onesweep pass (OS_ITEMS keys a thread) and the look-back window (predecessor
// words a digit's thread reads at once). The ranking (eight ballots a key) keeps the pass near
// half of the issue slots; 4096-key tiles halve the tiles (look-back, block scans, barriers)
// and measured 0.1 ms faster on the 16-view batch than 2048, a 16-word window no faster.
#ifndef LOBE_OS_ITEMS
#define LOBE_OS_ITEMS 16
#endif
#ifndef LOBE_OS_W
#define LOBE_OS_W 8
#endif
constexpr int OS_ITEMS = LOBE_OS_ITEMS;
constexpr int OS_TILE = RS_THREADS * OS_ITEMS;
constexpr int OS_W = LOBE_OS_W;

// The sum of one digit's counts over tiles [0, tile), for the calling thread alone: the words
// slots[j * 256 + d] of tiles j = tile - 1, tile - 2, ... are read eight at a time (independent
// loads) and summed down to the nearest inclusive word; a word not yet published ends the
// window and is polled again (at most LB_SPIN_LIMIT times, then STATUS_TIMEOUT is latched).
// A timed-out sum only undercounts, so the scatter that uses it stays in bounds.
__device__ __forceinline__ uint32_t lb_exclusive_digit(const unsigned long long *slots, int tile, int d, uint32_t tag,
                                                       int *status)
{
    constexpr int W = OS_W;
    uint32_t sum = 0;
    int j = tile - 1, spins = 0;
    while (j >= 0) {
        unsigned long long w[W];
#pragma unroll
        for (int q = 0; q < W; ++q) w[q] = j - q >= 0 ? lb_load(slots + (long long)(j - q) * 256 + d) : 0ull;
        int used = 0;
        bool stop = false, blocked = false;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (stop || blocked || j - q < 0) continue;
            if ((uint32_t)(w[q] >> 34) != tag) {
                blocked = true;
                continue;
            }
            sum += (uint32_t)w[q];
            ++used;
            stop = ((uint32_t)(w[q] >> 32) & 3u) == LB_INC;
        }
        if (stop) break;
        j -= used;
        if (blocked) {
            if (++spins > LB_SPIN_LIMIT) {
                set_status(status, STATUS_TIMEOUT);
                break;
            }
            __nanosleep(40);
        }
    }
    return sum;
}

// One pass of the stable LSD sort by the 8-bit digit at `shift`. The block with ticket t ranks
// tile t (keys [t * OS_TILE, (t + 1) * OS_TILE)) by digit as k_radix_scatter does, publishes its 256
// digit counts (slots[t * 256 + d], aggregate first, inclusive once known), gets per digit the
// keys of earlier tiles by look-back, and scatters: a key of digit d goes to start(d) + (digit-d
// keys of earlier tiles) + (its rank among the tile's digit-d keys), start being the exclusive
// scan of the whole key set's digit histogram `hist`. Tiles go in ticket order, so every wait
// is on a block that is already running.
__global__ void __launch_bounds__(RS_THREADS) k_onesweep(const uint32_t *__restrict__ kin,
                                                         const uint32_t *__restrict__ vin,
                                                         uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                         const uint32_t *n_dev, int shift,
                                                         const uint32_t *__restrict__ hist,
                                                         unsigned long long *slots, LB lb)
{
    pdl_wait();
    __shared__ uint32_t s_k[OS_TILE];
    __shared__ uint32_t s_v[OS_TILE];
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t local_off[256], grun[256];
    __shared__ uint32_t scan_sm[RS_THREADS / 32 + 1];
    __shared__ int s_tile;
    __shared__ uint32_t s_gen;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    if (tid == 0) {
        int t;
        uint32_t g;
        lb_take(lb.ctl, lb.stage, false, t, g);
        s_tile = t;
        s_gen = g;
    }
    for (int d = lane; d < 256; d += 32) wcnt[warp][d] = 0;
    __syncthreads();
    const int tile = s_tile;
    const long long n = *n_dev;
    const long long tb = (long long)tile * OS_TILE;
    if (tb >= n) return;
    const long long hi = n - tb < OS_TILE ? n : tb + OS_TILE;
    const uint32_t tag = lb_tag(s_gen, lb.stage);
    const unsigned lt = lanemask_lt();
    const uint32_t hcount = hist[tid];
    uint32_t k[OS_ITEMS], v[OS_ITEMS], dg[OS_ITEMS], rk[OS_ITEMS];
    bool ok[OS_ITEMS];
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        const long long i = tb + warp * (32 * OS_ITEMS) + j * 32 + lane;
        ok[j] = i < hi;
        k[j] = ok[j] ? kin[i] : 0u;
        v[j] = ok[j] ? vin[i] : 0u;
    }
    // rank within the warp's 256 consecutive elements, in order
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        dg[j] = (k[j] >> shift) & 255u;
        const unsigned valid = __ballot_sync(0xffffffffu, ok[j]);
        const unsigned peers = warp_peers(dg[j], 8, valid);
        const int leader = ok[j] ? __ffs(peers) - 1 : lane;
        uint32_t base = (ok[j] && lane == leader) ? wcnt[warp][dg[j]] : 0u;
        base = __shfl_sync(0xffffffffu, base, leader);
        rk[j] = base + __popc(peers & lt);
        __syncwarp();
        if (ok[j] && lane == leader) wcnt[warp][dg[j]] = base + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread tid = digit: exclusive prefix over warps, the tile's count, its look-back
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
        const uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = cnt;
        cnt += c;
    }
    unsigned long long *slot = slots + (long long)tile * 256 + tid;
    lb_publish(slot, tag, tile == 0 ? LB_INC : LB_AGG, cnt);
    uint32_t before = 0;
    if (tile > 0) {
        before = lb_exclusive_digit(slots, tile, tid, tag, lb.ctl);
        lb_publish(slot, tag, LB_INC, before + cnt);
    }
    uint32_t ex, start;
    block_exclusive_scan<RS_THREADS>(cnt, ex, scan_sm);
    local_off[tid] = ex;
    block_exclusive_scan<RS_THREADS>(hcount, start, scan_sm);
    grun[tid] = start + before;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
        if (ok[j]) {
            const uint32_t p = local_off[dg[j]] + wcnt[warp][dg[j]] + rk[j];
            s_k[p] = k[j];
            s_v[p] = v[j];
        }
    }
    __syncthreads();
    const int n_tile = (int)(hi - tb);
    for (int i = tid; i < n_tile; i += RS_THREADS) {
        const uint32_t key = s_k[i];
        const uint32_t d = (key >> shift) & 255u;
        const uint32_t g = grun[d] + (uint32_t)i - local_off[d];
        if ((long long)g < n) {
            kout[g] = key;
            vout[g] = s_v[i];
        }
    }
}

// Look-back words of the onesweep passes for up to n keys (256 per tile).
static inline long long onesweep_slots(long long n) { return ((n > 0 ? n : 1) + OS_TILE - 1) / OS_TILE * 256; }

// Stable sort of the first *n_dev (<= n_max) pairs (kA, vA) by all 32 key bits: four onesweep
// passes A -> B -> A -> B -> (kf, vf); (kf, vf) must not alias (kB, vB). hist holds the four
// digit histograms of the keys; pass p takes its tickets and tags from stage lb.stage + p.
static void onesweep_sort32(const uint32_t *n_dev, long long n_max, uint32_t *kA, uint32_t *vA, uint32_t *kB,
                            uint32_t *vB, uint32_t *kf, uint32_t *vf, const uint32_t *hist,
                            unsigned long long *slots, LB lb, cudaStream_t st)
{
    const long long tiles = (n_max + OS_TILE - 1) / OS_TILE;
    const unsigned grid = (unsigned)(tiles < 1 ? 1 : tiles);
    const int stage0 = lb.stage;
    for (int p = 0; p < 4; ++p) {
        const uint32_t *ks = (p & 1) ? kB : kA, *vs = (p & 1) ? vB : vA;
        uint32_t *kd = (p & 1) ? kA : kB, *vd = (p & 1) ? vA : vB;
        if (p == 3) {
            kd = kf;
            vd = vf;
        }
        lb.stage = stage0 + p;
        count_launch();
        launch_pdl(k_onesweep, dim3(grid), dim3(RS_THREADS), 0, st, ks, vs, kd, vd, n_dev, 8 * p, hist + 256 * p,
                   slots, lb);
    }
}

// Look-back words a scan of up to n elements needs (one per tile).
static inline long long scan_slots(long long n) { return ((n > 0 ? n : 1) + SCAN_TILE - 1) / SCAN_TILE; }

}  // namespace lobe
