// noalloc.cu -- lobe_bin_sort_noalloc: the binning stage with its scratch in a file-scope
// device array instead of context-owned cudaMalloc memory, for callers that may not
// allocate device memory (see include/lobe.h). It runs the same kernels as lobe_bin_sort.
#include <mutex>

#include "lobe_internal.cuh"

using namespace lobe;

lobe_status lobe_internal_build_params(const lobe_config *cfg, const lobe_batch *b, BatchParams &P);

namespace {

constexpr long long kMaxEntries = LOBE_NOALLOC_MAX_ENTRIES;
constexpr long long kMaxTiles = LOBE_NOALLOC_MAX_TILES;
constexpr long long kMaxPairs = LOBE_NOALLOC_MAX_PAIRS;
constexpr long long kMaxSuper = 8192;  // 64x64-pixel blocks; 65536 tiles make about 4100
constexpr size_t kScratchBytes = size_t(20) << 20;
constexpr size_t kStatusBytes = CTL_BYTES;  // status word + look-back control block
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void *g_addr[kMaxDevices];  // device address of the array, per device, set on first use

}  // namespace

// The scratch itself: one copy per device, alive until the process exits. In host code its
// name only stands in for the symbol; kernels get the address looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Once per device, with that device current: the array's device address.
static lobe_status scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LOBE_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LOBE_ERR_STATE;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return LOBE_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return LOBE_OK;
}

extern "C" lobe_status lobe_bin_sort_noalloc(const lobe_config *cfg, void *stream, const lobe_batch *batch,
                                             const lobe_projected *proj, const lobe_bins *bins, int64_t *n_isect_host)
{
    // the parameter block (~15 KB) lives in per-thread static storage, not on the heap
    static thread_local BatchParams P;
    lobe_status s = lobe_internal_build_params(cfg, batch, P);
    if (s != LOBE_OK) return s;
    if (!proj || (P.n_entries > 0 && (!proj->splat || !proj->radius || !proj->tiles_touched))) return LOBE_ERR_ARG;
    if (!bins || !bins->gauss_ids || !bins->tile_start || !bins->n_isect || bins->capacity < 0) return LOBE_ERR_ARG;
    if (P.n_entries > kMaxEntries || P.n_tiles > kMaxTiles || P.n_super > kMaxSuper) return LOBE_ERR_CAPACITY;
    static_assert(kMaxTiles <= (1LL << 22), "the tile scan serves at most 2^22 tiles");
    if (entry_scratch_bytes(kMaxEntries) + pair_scratch_bytes(kMaxPairs, kMaxSuper) + super_scratch_bytes(kMaxSuper) +
            kStatusBytes > kScratchBytes)
        return LOBE_ERR_STATE;

    void *base = nullptr;
    s = scratch_address(&base);
    if (s != LOBE_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // carve: status word, entry part, pair part, super-tile part
    char *p = static_cast<char *>(base);
    int *status = reinterpret_cast<int *>(p);
    p += kStatusBytes;
    BinScratch b{};
    entry_scratch_carve(p, kMaxEntries, status, b);
    p += entry_scratch_bytes(kMaxEntries);
    pair_scratch_carve(p, kMaxPairs, kMaxSuper, b);
    p += pair_scratch_bytes(kMaxPairs, kMaxSuper);
    super_scratch_carve(p, kMaxSuper, b);

    // the array keeps the previous call's contents: only the status word must start at zero
    // (the look-back generation and ticket counters after it carry over between calls; every
    // other scratch value is written before it is read, or is a look-back word of an earlier
    // call, which matches no later one)
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return LOBE_ERR_CUDA;
    if (bin_super_count(P, proj->splat, proj->radius, proj->tiles_touched, b, kMaxPairs, st) != cudaSuccess)
        return LOBE_ERR_CUDA;
    uint32_t n_sp = 0;
    if (cudaMemcpyAsync(&n_sp, b.scalars + 4, sizeof n_sp, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LOBE_ERR_CUDA;
    if ((long long)n_sp > kMaxPairs) return LOBE_ERR_CAPACITY;

    long long *n_isect = reinterpret_cast<long long *>(bins->n_isect);
    if (bin_tile_count(P, proj->splat, proj->radius, b, kMaxPairs, n_isect, bins->tile_start, bins->capacity, st) !=
            cudaSuccess ||
        bin_sort_emit(P, proj->splat, proj->radius, b, n_isect, bins->gauss_ids, bins->tile_start, st) != cudaSuccess)
        return LOBE_ERR_CUDA;
    long long total = 0;
    if (cudaMemcpyAsync(&total, n_isect, sizeof total, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LOBE_ERR_CUDA;
    if (n_isect_host) *n_isect_host = total;
    return total > bins->capacity ? LOBE_ERR_CAPACITY : LOBE_OK;
}
