// lookback.cuh -- decoupled look-back state shared by the single-pass scans of the binning
// stage and the visible-Gaussian compaction of the projection adjoint (Merrill & Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016).
//
// A block takes a tile in ticket order, publishes the tile's aggregate, then one warp reads the
// words of the 32 tiles before it at a time and adds their values back to the nearest tile that
// already carries its inclusive prefix; the block then publishes its own inclusive prefix. A
// tile only waits on tiles with smaller tickets, held by blocks that are already running, so
// every wait ends; each wait is also bounded (LB_SPIN_LIMIT polls, then STATUS_TIMEOUT is
// latched and the block carries on).
//
// A published word is (tag << 34 | flag << 32 | value). The tag combines a generation number,
// advanced by the first kernel of every binning call and of every projection adjoint, with the
// stage (which scan), so words left by earlier launches never match and nothing has to be
// cleared between calls. The generation, the per-stage ticket counters and the status word live
// in one small control block that is zeroed once when it is allocated.
#pragma once
#include "lobe_internal.cuh"

namespace lobe {

// ------------------------------------------------------------------ look-back control

constexpr int LB_STAGES = 16;
constexpr int LB_SPIN_LIMIT = 1 << 22;
enum : uint32_t { LB_AGG = 1u, LB_INC = 2u };
// control block (int words): [0] status, [1] generation, [2 + stage] ticket counter
constexpr int CTL_WORDS = 2 + LB_STAGES;

enum : int {  // look-back stages (each scan has its own ticket counter and tag)
    ST_SCAN_VISIBLE = 0,  // compaction of the visible entries (opens a binning call)
    ST_DEPTH_PASS = 1,  // .. 4: the depth sort's onesweep passes
    ST_SCAN_OFFS = 5,
    ST_SUPER_PASS = 6,  // .. 7: digit-count scans of the super-tile sort
    ST_SCAN_CHUNKS = 8,
    ST_SCAN_TILES = 9,
    ST_PBWD_LIST = 10,  // projection adjoint: list of the Gaussians some item sees
    ST_DENSIFY = 11,    // densification: output offsets
};

struct LB {
    unsigned long long *slots;
    int *ctl;
    int stage;
};

__device__ __forceinline__ uint32_t lb_tag(uint32_t gen, int stage)
{
    return (((gen % ((1u << 26) - 1u)) + 1u) << 4) | (uint32_t)stage;  // never 0, 30 bits
}

__device__ __forceinline__ void lb_publish(unsigned long long *slot, uint32_t tag, uint32_t flag, uint32_t v)
{
    const unsigned long long w = ((unsigned long long)tag << 34) | ((unsigned long long)flag << 32) | v;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(slot), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long *slot)
{
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(slot) : "memory");
    return w;
}

// Called by one full warp: the sum of the values of tiles [0, tile) (the tile's exclusive
// prefix), in every lane. Lane l reads tile j - l of the current window of 32; the window's
// values up to the nearest inclusive word are summed; without one the window moves down 32.
__device__ __forceinline__ uint32_t lb_exclusive_warp(const unsigned long long *slots, int tile, uint32_t tag,
                                                      int *status)
{
    const int lane = threadIdx.x & 31;
    uint32_t sum = 0;
    int j = tile - 1, spins = 0;
    while (j >= 0) {
        const int k = j - lane;
        bool ready = true, inc = false;
        uint32_t v = 0;
        if (k >= 0) {
            const unsigned long long w = lb_load(slots + k);
            ready = (uint32_t)(w >> 34) == tag;
            inc = ready && (((uint32_t)(w >> 32) & 3u) == LB_INC);
            v = ready ? (uint32_t)w : 0u;
        }
        const unsigned incm = __ballot_sync(0xffffffffu, inc);
        const unsigned waitm = __ballot_sync(0xffffffffu, !ready);
        const int first = incm ? __ffs(incm) - 1 : 31;  // nearest inclusive word (or the whole window)
        const unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
        if (waitm & need) {
            if (++spins > LB_SPIN_LIMIT) {
                if (lane == 0) set_status(status, STATUS_TIMEOUT);
                break;
            }
            __nanosleep(40);
            continue;
        }
        uint32_t part = lane <= first ? v : 0u;
#pragma unroll
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        sum += part;
        if (incm) break;
        j -= 32;
    }
    return sum;
}

// Thread 0: the block's ticket and the generation of this call. With bump, this launch opens
// the call: it uses generation + 1 and its last ticket holder stores it (every block read the
// old value before taking its ticket). The last ticket holder also re-arms the counter.
__device__ __forceinline__ void lb_take(int *ctl, int stage, bool bump, int &ticket, uint32_t &gen)
{
    // an acquire load: the ticket below cannot be taken before the generation is read
    uint32_t g;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(ctl + 1) : "memory");
    ticket = atomicAdd(ctl + 2 + stage, 1);
    gen = bump ? g + 1u : g;
    if (ticket == (int)gridDim.x - 1) {
        atomicExch(ctl + 2 + stage, 0);
        if (bump) atomicExch(ctl + 1, (int)(g + 1u));
    }
}

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

constexpr int SCAN_THREADS = 256;
#ifndef LOBE_SCAN_ITEMS
#define LOBE_SCAN_ITEMS 16
#endif
constexpr int SCAN_ITEMS = LOBE_SCAN_ITEMS;          // per lane, warp-striped
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // elements per tile

// ------------------------------------------------------------------ single-pass exclusive scan
//
// out[i] = sum_{j<i} in(j) for i < n, n read from device memory when n_dev is given (the launch
// shape then depends only on an upper bound, so the call is graph-capturable). Each block scans
// one SCAN_TILE-element tile (warp-striped, coalesced) and gets the tile's offset by look-back. The
// block of the last tile writes the grand total to total32/total64 (nullable) and the count the
// next stage may use to n_use: the total, or 0 with a latched capacity error when it exceeds
// `capacity` (< 0: unlimited). In-place use (out == the loaded array) is safe: each element is
// read and later written by the same thread. The block with ticket 0 zeroes zero_words words at
// zero_buf (accumulators of later kernels).

struct LoadPlain {
    const uint32_t *src;
    __device__ uint32_t operator()(long long i) const { return src[i]; }
};

template <class L>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan(L load, const uint32_t *n_dev, long long n_host, uint32_t *out,
                                                       uint32_t *total32, long long *total64, uint32_t *n_use,
                                                       long long capacity, LB lb, int bump, uint32_t *zero_buf,
                                                       int zero_words)
{
    pdl_wait();
    __shared__ int s_tile;
    __shared__ uint32_t s_gen, s_prefix;
    __shared__ uint32_t s_warp[SCAN_THREADS / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        int t;
        uint32_t g;
        lb_take(lb.ctl, lb.stage, bump != 0, t, g);
        s_tile = t;
        s_gen = g;
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile == 0)
        for (int i = threadIdx.x; i < zero_words; i += SCAN_THREADS) zero_buf[i] = 0u;
    const long long n = n_dev ? (long long)*n_dev : n_host;
    const long long ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tile >= (ntiles > 0 ? ntiles : 1)) return;
    const uint32_t tag = lb_tag(s_gen, lb.stage);
    // warp w owns elements [t0 + w * 32 * SCAN_ITEMS, t0 + (w + 1) * 32 * SCAN_ITEMS), lane-striped
    const long long w0 = (long long)tile * SCAN_TILE + (long long)warp * (32 * SCAN_ITEMS);
    uint32_t x[SCAN_ITEMS];
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; ++r) {
        const long long i = w0 + r * 32 + lane;
        x[r] = i < n ? load(i) : 0u;
    }
    uint32_t carry = 0;  // warp-exclusive running sum
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; ++r) {
        uint32_t inc = x[r];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
        x[r] = carry + inc - x[r];
        carry += tot;
    }
    uint32_t wex;
    const uint32_t agg = block_exclusive_scan<SCAN_THREADS>(lane == 0 ? carry : 0u, wex, s_warp);
    wex = __shfl_sync(0xffffffffu, wex, 0);
    if (warp == 0) {
        unsigned long long *slot = lb.slots + tile;
        uint32_t prefix = 0;
        if (tile == 0) {
            if (lane == 0) lb_publish(slot, tag, LB_INC, agg);
        } else {
            if (lane == 0) lb_publish(slot, tag, LB_AGG, agg);
            prefix = lb_exclusive_warp(lb.slots, tile, tag, lb.ctl);
            if (lane == 0) lb_publish(slot, tag, LB_INC, prefix + agg);
        }
        if (lane == 0) s_prefix = prefix;
        if (lane == 0 && tile == (ntiles > 0 ? ntiles - 1 : 0)) {
            const uint32_t total = prefix + agg;
            if (total32) *total32 = total;
            if (total64) *total64 = (long long)total;
            if (n_use) {
                const bool over = capacity >= 0 && (long long)total > capacity;
                *n_use = over ? 0u : total;
                if (over) set_status(lb.ctl, STATUS_CAPACITY);
            }
        }
    }
    __syncthreads();
    const uint32_t base = s_prefix + wex;
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; ++r) {
        const long long i = w0 + r * 32 + lane;
        if (i < n) out[i] = base + x[r];
    }
}

template <class L>
static void scan(L load, const uint32_t *n_dev, long long n_max, uint32_t *out, uint32_t *total32, long long *total64,
                 uint32_t *n_use, long long capacity, LB lb, cudaStream_t st, bool bump = false,
                 uint32_t *zero_buf = nullptr, int zero_words = 0)
{
    long long nb = (n_max + SCAN_TILE - 1) / SCAN_TILE;
    if (nb < 1) nb = 1;
    const long long n_host = n_dev ? 0 : n_max;
    count_launch();
    launch_pdl(k_scan<L>, dim3((unsigned)nb), dim3(SCAN_THREADS), 0, st, load, n_dev, n_host, out, total32, total64, n_use, capacity, lb,
                                                  bump ? 1 : 0, zero_buf, zero_words);
}

}  // namespace lobe
