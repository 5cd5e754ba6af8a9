// bin_small.cu -- tile binning of a small batch in one launch of one CTA.
//
// The general binning (binning.cu) is a chain of about twenty kernels whose fixed cost (launch,
// ramp-up, drain: ~0.1 ms) dominates when a batch holds a few thousand projected entries. For
// such batches one CTA does all of it in shared memory, with the same result bit for bit:
//   1. the visible entries' keys (float32 depth bits << 32 | entry id), padded to a power of two;
//   2. a bitonic sort of the keys: (depth, entry) order, which is the order the general path's
//      stable depth sort of the entry-ordered visible splats produces;
//   3. every sorted splat's tile rectangle (the same integer rectangle as the general path);
//   4. per tile (one warp each): ballots over the sorted splats count those covering it;
//   5. an exclusive scan of the counts gives tile_start and the pair count;
//   6. per tile again, the covering splats' ids are written in order (ranks from the ballots).
// A pair count above the bins' capacity latches the capacity status, stores the count and
// leaves every tile empty, as the general path does.
#include <atomic>
#include "lookback.cuh"

namespace lobe {

constexpr int BS_THREADS = 1024;
constexpr int BS_MAX_ENTRIES = 4096;
constexpr int BS_MAX_TILES = 4096;
constexpr long long BS_MAX_WORK = 1LL << 20;  // tiles x entries: bounds the per-tile ballot passes

struct BinSmallSmem {
    unsigned long long key[BS_MAX_ENTRIES];  // (depth bits << 32 | entry), sorted in place
    uint32_t rx[BS_MAX_ENTRIES];             // x0 | x1 << 16 of the sorted splat's tile rectangle
    uint32_t ry[BS_MAX_ENTRIES];             // y0 | y1 << 16
    uint8_t item[BS_MAX_ENTRIES];            // the splat's item
    uint32_t start[BS_MAX_TILES];            // per tile: count, then first pair
    uint32_t scan[BS_THREADS / 32 + 1];
    uint32_t visible;
};

__global__ void __launch_bounds__(BS_THREADS, 1)
    k_bin_small(const __grid_constant__ BatchParams P, const float *__restrict__ splat, const int *__restrict__ radius,
                const int *__restrict__ tiles, int *__restrict__ gauss_ids, int *__restrict__ tile_start,
                long long *__restrict__ n_isect, long long capacity, int *status)
{
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BinSmallSmem &S = *reinterpret_cast<BinSmallSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = lanemask_lt();
    const int n = (int)P.n_entries, n_tiles = P.n_tiles;
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    if (tid == 0) S.visible = 0;
    __syncthreads();
    // 1. keys of the visible entries; the others sort to the end
    uint32_t vis = 0;
    for (int i = tid; i < n2; i += BS_THREADS) {
        unsigned long long k = ~0ull;
        if (i < n && tiles[i] > 0) {
            k = ((unsigned long long)__float_as_uint(splat[12LL * i + 9]) << 32) | (uint32_t)i;
            ++vis;
        }
        S.key[i] = k;
    }
    vis = __reduce_add_sync(0xffffffffu, vis);
    if (lane == 0 && vis) atomicAdd(&S.visible, vis);
    // 2. bitonic sort, ascending
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = tid; i < (n2 >> 1); i += BS_THREADS) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const unsigned long long a = S.key[lo], b = S.key[hi];
                if ((a > b) == ((lo & size) == 0)) {
                    S.key[lo] = b;
                    S.key[hi] = a;
                }
            }
        }
    }
    __syncthreads();
    const int V = (int)S.visible;
    // 3. tile rectangles of the sorted splats
    for (int k = tid; k < V; k += BS_THREADS) {
        const uint32_t e = (uint32_t)S.key[k];
        const int it = item_of_entry(P, e);
        const ItemParams &I = P.item[it];
        int x0, y0, x1, y1;
        tile_rect(splat[12LL * e], splat[12LL * e + 1], radius[e], P.tw, P.th, I.gx, I.gy, x0, y0, x1, y1);
        S.rx[k] = (uint32_t)x0 | ((uint32_t)x1 << 16);
        S.ry[k] = (uint32_t)y0 | ((uint32_t)y1 << 16);
        S.item[k] = (uint8_t)it;
    }
    __syncthreads();
    // 4. per tile: splats covering it (one warp a tile)
    for (int t = warp; t < n_tiles; t += BS_THREADS / 32) {
        const int it = item_of_tile(P, t);
        const ItemParams &I = P.item[it];
        const int lt_ = t - I.tile_off, tx = lt_ % I.gx, ty = lt_ / I.gx;
        uint32_t c = 0;
        for (int k0 = 0; k0 < V; k0 += 32) {
            const int k = k0 + lane;
            bool cov = false;
            if (k < V) {
                const uint32_t rx = S.rx[k], ry = S.ry[k];
                cov = S.item[k] == it && tx >= (int)(rx & 0xffffu) && tx < (int)(rx >> 16) &&
                      ty >= (int)(ry & 0xffffu) && ty < (int)(ry >> 16);
            }
            c += __popc(__ballot_sync(0xffffffffu, cov));
        }
        if (lane == 0) S.start[t] = c;
    }
    __syncthreads();
    // 5. exclusive scan of the counts: four tiles a thread
    uint32_t v[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int t = 4 * tid + q;
        v[q] = t < n_tiles ? S.start[t] : 0u;
        sum += v[q];
    }
    uint32_t ex;
    const uint32_t total = block_exclusive_scan<BS_THREADS>(sum, ex, S.scan);
    const bool over = (long long)total > capacity;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int t = 4 * tid + q;
        if (t < n_tiles) {
            S.start[t] = ex;
            tile_start[t] = over ? 0 : (int)ex;
        }
        ex += v[q];
    }
    if (tid == 0) {
        tile_start[n_tiles] = over ? 0 : (int)total;
        *n_isect = (long long)total;
        if (over) set_status(status, STATUS_CAPACITY);
    }
    if (over) return;
    __syncthreads();
    // 6. ids, per tile in (depth, entry) order
    for (int t = warp; t < n_tiles; t += BS_THREADS / 32) {
        const int it = item_of_tile(P, t);
        const ItemParams &I = P.item[it];
        const int lt_ = t - I.tile_off, tx = lt_ % I.gx, ty = lt_ / I.gx;
        uint32_t pos = S.start[t];
        for (int k0 = 0; k0 < V; k0 += 32) {
            const int k = k0 + lane;
            bool cov = false;
            if (k < V) {
                const uint32_t rx = S.rx[k], ry = S.ry[k];
                cov = S.item[k] == it && tx >= (int)(rx & 0xffffu) && tx < (int)(rx >> 16) &&
                      ty >= (int)(ry & 0xffffu) && ty < (int)(ry >> 16);
            }
            const unsigned m = __ballot_sync(0xffffffffu, cov);
            if (cov) gauss_ids[pos + __popc(m & lt)] = (int)(uint32_t)S.key[k];
            pos += __popc(m);
        }
    }
}

bool bin_small_fits(const BatchParams &P)
{
    return P.n_entries <= BS_MAX_ENTRIES && P.n_tiles <= BS_MAX_TILES && P.n_items <= 256 &&
           (long long)P.n_tiles * P.n_entries <= BS_MAX_WORK;
}

cudaError_t launch_bin_small(const BatchParams &P, const float *splat, const int *radius, const int *tiles,
                             int *gauss_ids, int *tile_start, long long *n_isect, long long capacity, int *status,
                             cudaStream_t st)
{
    // the kernel's shared-memory limit, raised once per process (idempotent: host threads with
    // their own contexts may both get here first)
    static std::atomic<bool> configured{false};
    if (!configured.load(std::memory_order_acquire)) {
        const cudaError_t e = cudaFuncSetAttribute(k_bin_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sizeof(BinSmallSmem));
        if (e != cudaSuccess) return e;
        configured.store(true, std::memory_order_release);
    }
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(BS_THREADS);
    cfg.dynamicSmemBytes = sizeof(BinSmallSmem);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_bin_small, P, splat, radius, tiles, gauss_ids, tile_start, n_isect, capacity,
                              status);
}

}  // namespace lobe
