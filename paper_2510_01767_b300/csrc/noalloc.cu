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

struct DeviceSlot {
    unsigned long long ctx_id;  // driver context the address belongs to (0: not looked up yet)
    void *addr;                 // device address of the array in that context
};
std::mutex g_mu;
DeviceSlot g_slot[kMaxDevices];

}  // namespace

// The scratch itself: one copy per device, alive until the process exits. In host code its
// name only stands in for the symbol; kernels get the address looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Unique id of the calling thread's current driver context (driver entry points fetched
// through the runtime, so the library needs no link against the driver library). 0 when the
// driver cannot tell, in which case the address is looked up on every call.
static unsigned long long current_context_id()
{
    typedef int (*GetCurrent)(void **);
    typedef int (*GetId)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || ctx == nullptr || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Set-up, once per device (again only if that device's context was destroyed and created
// anew, e.g. after cudaDeviceReset, since the array may then sit elsewhere), with the device
// current: the array's device address.
static lobe_status scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LOBE_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LOBE_ERR_STATE;
    const unsigned long long id = current_context_id();  // 0 before the runtime made a context current
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSlot &s = g_slot[dev];
    if (s.addr == nullptr || id == 0 || s.ctx_id != id) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return LOBE_ERR_CUDA;
        s.addr = p;
        s.ctx_id = current_context_id();  // the lookup has made the device's context current
    }
    *out = s.addr;
    return LOBE_OK;
}

// Status latched by the kernels in the array's control block -> the call's return code.
static lobe_status device_status(int code)
{
    return code == STATUS_TIMEOUT ? LOBE_ERR_TIMEOUT : (code == STATUS_CAPACITY ? LOBE_ERR_CAPACITY : LOBE_OK);
}

extern "C" lobe_status lobe_bin_sort_noalloc(const lobe_config *cfg, void *stream, const lobe_batch *batch,
                                             const lobe_projected *proj, const lobe_bins *bins, int64_t *n_isect_host)
{
    // the parameter block (~15 KB) is host memory: per-thread storage, set up once per host
    // thread on its first call (no device memory is allocated, here or anywhere in this call)
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
    int code = STATUS_OK;
    if (cudaMemcpyAsync(&n_sp, b.scalars + 4, sizeof n_sp, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&code, status, sizeof code, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LOBE_ERR_CUDA;
    // a bounded wait that gave up leaves the counts undefined: report it, bins not written
    if (device_status(code) != LOBE_OK) return device_status(code);
    if ((long long)n_sp > kMaxPairs) return LOBE_ERR_CAPACITY;

    long long *n_isect = reinterpret_cast<long long *>(bins->n_isect);
    if (bin_tile_count(P, proj->splat, proj->radius, b, kMaxPairs, n_isect, bins->tile_start, bins->capacity, st) !=
            cudaSuccess ||
        bin_sort_emit(P, proj->splat, proj->radius, b, n_isect, bins->gauss_ids, bins->tile_start, st) != cudaSuccess)
        return LOBE_ERR_CUDA;
    long long total = 0;
    if (cudaMemcpyAsync(&total, n_isect, sizeof total, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&code, status, sizeof code, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LOBE_ERR_CUDA;
    if (n_isect_host) *n_isect_host = total;
    // the device's own verdict first: a timed-out wait (LOBE_ERR_TIMEOUT) or a latched overflow
    if (device_status(code) != LOBE_OK) return device_status(code);
    return total > bins->capacity ? LOBE_ERR_CAPACITY : LOBE_OK;
}
