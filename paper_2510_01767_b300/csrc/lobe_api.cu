// lobe_api.cu -- the extern "C" entry points declared in include/lobe.h.
//
// The host side only validates arguments, packs the batch into one parameter block and
// enqueues kernels on the context's stream; every step of the rasterizer runs on the GPU.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "lookback.cuh"


#include <atomic>

static std::atomic<long long> g_launches{0};

void lobe::count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

using namespace lobe;

struct lobe_ctx {
    cudaStream_t stream = nullptr;
    lobe_config cfg{};
    int device = 0;
    int *status = nullptr;
    void *entry_mem = nullptr, *pair_mem = nullptr, *super_mem = nullptr;
    long long max_entries = 0, max_pairs = 0, max_super = 0;
    int *order = nullptr;       // persistent compositing: tile order [max_order]
    unsigned *order_ctl = nullptr;  // and its counters [ORDER_CTL]
    long long max_order = 0;
    size_t pair_bytes = 0;
    BinScratch bins{};
    char err[512] = {0};
};

static lobe_status fail(lobe_ctx *ctx, lobe_status code, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

static lobe_status cuda_fail(lobe_ctx *ctx, cudaError_t e, const char *where)
{
    return fail(ctx, LOBE_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CUDA_TRY(expr, where)                              \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, where); \
    } while (0)

static bool valid_tile(int tw, int th)
{
    return (tw == 16 && th == 16) || (tw == 16 && th == 8) || (tw == 8 && th == 8) || (tw == 32 && th == 16);
}

static lobe_status check_config(lobe_ctx *ctx, const lobe_config *cfg)
{
    if (!cfg) return fail(ctx, LOBE_ERR_ARG, "config is NULL");
    if (!valid_tile(cfg->tile_w, cfg->tile_h))
        return fail(ctx, LOBE_ERR_ARG, "tile %dx%d not one of 8x8, 16x8, 16x16, 32x16", cfg->tile_w, cfg->tile_h);
    if (cfg->sh_degree < 0 || cfg->sh_degree > 3) return fail(ctx, LOBE_ERR_ARG, "sh_degree %d not in 0..3", cfg->sh_degree);
    if (!valid_px(cfg->tile_w, cfg->tile_h, cfg->px_fwd) || !valid_px(cfg->tile_w, cfg->tile_h, cfg->px_bwd))
        return fail(ctx, LOBE_ERR_ARG, "pixels per lane %d/%d not supported with %dx%d tiles", cfg->px_fwd, cfg->px_bwd,
                    cfg->tile_w, cfg->tile_h);
    const int pf = cfg->px_fwd ? cfg->px_fwd : default_px(cfg->tile_w, cfg->tile_h, false);
    const int pb = cfg->px_bwd ? cfg->px_bwd : default_px(cfg->tile_w, cfg->tile_h, true);
    const auto batch_ok = [](int b) { return b == 0 || b == 32 || b == 64; };
    if (!batch_ok(cfg->batch_fwd) || !batch_ok(cfg->batch_bwd) || (cfg->batch_fwd == 64 && pf < 2) ||
        (cfg->batch_bwd == 64 && pb % 2 != 0))
        return fail(ctx, LOBE_ERR_ARG, "staging batch %d/%d not supported with %d/%d pixels a lane", cfg->batch_fwd,
                    cfg->batch_bwd, pf, pb);
    return LOBE_OK;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Packs a host batch description into the kernel parameter block.
static lobe_status build_params(lobe_ctx *ctx, const lobe_config &cfg, const lobe_batch *b, BatchParams &P)
{
    if (!b) return fail(ctx, LOBE_ERR_ARG, "batch is NULL");
    if (b->n_sets < 1 || b->n_sets > LOBE_MAX_SETS) return fail(ctx, LOBE_ERR_ARG, "n_sets %d not in 1..%d", b->n_sets, LOBE_MAX_SETS);
    if (b->n_items < 1 || b->n_items > LOBE_MAX_ITEMS)
        return fail(ctx, LOBE_ERR_ARG, "n_items %d not in 1..%d", b->n_items, LOBE_MAX_ITEMS);
    if (!b->sets || !b->items || !b->cameras || b->n_cameras < 1) return fail(ctx, LOBE_ERR_ARG, "batch arrays missing");
    if (b->n_blocks > 0 && !b->blocks) return fail(ctx, LOBE_ERR_ARG, "blocks is NULL with n_blocks > 0");
    memset(&P, 0, sizeof P);
    P.n_sets = b->n_sets;
    P.n_items = b->n_items;
    P.tw = cfg.tile_w;
    P.th = cfg.tile_h;
    P.px_fwd = cfg.px_fwd;
    P.px_bwd = cfg.px_bwd;
    P.nb_fwd = cfg.batch_fwd == 64 ? 2 : 1;
    P.nb_bwd = cfg.batch_bwd == 64 ? 2 : 1;
    P.sh_degree = cfg.sh_degree;
    for (int c = 0; c < 3; ++c) P.bg[c] = cfg.bg[c];
    long long goff = 0;
    for (int s = 0; s < b->n_sets; ++s) {
        const lobe_gaussians &G = b->sets[s];
        if (G.n < 0) return fail(ctx, LOBE_ERR_ARG, "set %d: n < 0", s);
        if (G.n > 0 && (!G.means || !G.log_scales || !G.quats || !G.opacity_logits || !G.sh))
            return fail(ctx, LOBE_ERR_ARG, "set %d: parameter pointer is NULL", s);
        if (!aligned16(G.quats) || !aligned16(G.sh)) return fail(ctx, LOBE_ERR_ARG, "set %d: quats/sh not 16-byte aligned", s);
        SetParams &S = P.set[s];
        S.means = G.means;
        S.log_scales = G.log_scales;
        S.quats = G.quats;
        S.logits = G.opacity_logits;
        S.sh = G.sh;
        S.crop = G.crop_mask;
        S.n = G.n;
        S.gauss_off = goff;
        goff += G.n;
    }
    P.n_gauss = goff;
    // items grouped by set (stable), for the set-major projection kernels
    int k = 0;
    for (int s = 0; s < b->n_sets; ++s) {
        P.set[s].item_begin = k;
        for (int i = 0; i < b->n_items; ++i)
            if (b->items[i].set == s) P.set_items[k++] = i;
        P.set[s].item_count = k - P.set[s].item_begin;
    }
    long long eoff = 0, poff = 0, toff = 0, soff = 0;
    P.S = super_edge(cfg.tile_w);
    for (int i = 0; i < b->n_items; ++i) {
        const lobe_item &it = b->items[i];
        if (it.set < 0 || it.set >= b->n_sets) return fail(ctx, LOBE_ERR_ARG, "item %d: set %d out of range", i, it.set);
        if (it.camera < 0 || it.camera >= b->n_cameras)
            return fail(ctx, LOBE_ERR_ARG, "item %d: camera %d out of range", i, it.camera);
        if (it.block >= b->n_blocks || it.block < -1)
            return fail(ctx, LOBE_ERR_ARG, "item %d: block %d out of range", i, it.block);
        const lobe_camera &c = b->cameras[it.camera];
        if (c.width <= 0 || c.height <= 0 || !(c.fx > 0.f) || !(c.fy > 0.f))
            return fail(ctx, LOBE_ERR_ARG, "camera %d: bad intrinsics", it.camera);
        ItemParams &I = P.item[i];
        for (int r = 0; r < 12; ++r) I.V[r] = c.viewmat[r];
        for (int r = 0; r < 4; ++r) I.Vz[r] = (double)c.viewmat[8 + r];
        I.fx = c.fx; I.fy = c.fy; I.cx = c.cx; I.cy = c.cy;
        I.near_plane = (double)c.near_plane;
        I.far_plane = (double)c.far_plane;
        // camera centre of the rigid transform [R|t]: -R^T t
        for (int a = 0; a < 3; ++a) {
            double v = 0.0;
            for (int r = 0; r < 3; ++r) v -= (double)c.viewmat[4 * r + a] * (double)c.viewmat[4 * r + 3];
            I.campos[a] = (float)v;
        }
        I.limx = (float)(1.3 * (0.5 * c.width) / (double)c.fx);
        I.limy = (float)(1.3 * (0.5 * c.height) / (double)c.fy);
        for (int a = 0; a < 3; ++a) {
            I.lo[a] = it.block >= 0 ? b->blocks[it.block].lo[a] : -INFINITY;
            I.hi[a] = it.block >= 0 ? b->blocks[it.block].hi[a] : INFINITY;
        }
        I.W = c.width;
        I.H = c.height;
        I.gx = (c.width + cfg.tile_w - 1) / cfg.tile_w;
        I.gy = (c.height + cfg.tile_h - 1) / cfg.tile_h;
        if (I.gx > 65535 || I.gy > 65535)  // tile rectangles are packed in 16-bit fields
            return fail(ctx, LOBE_ERR_ARG, "camera %d: more than 65535 tiles in a row or column", it.camera);
        I.tile_off = (int)toff;
        I.sgx = (I.gx + P.S - 1) / P.S;
        I.sgy = (I.gy + P.S - 1) / P.S;
        I.super_off = (int)soff;
        soff += (long long)I.sgx * I.sgy;
        I.set = it.set;
        I.entry_off = eoff;
        I.pix_off = poff;
        eoff += b->sets[it.set].n;
        poff += (long long)c.width * c.height;
        toff += (long long)I.gx * I.gy;
    }
    if (eoff >= (1LL << 31)) return fail(ctx, LOBE_ERR_ARG, "%lld projected entries exceed 2^31", eoff);
    if (toff >= (1LL << 30)) return fail(ctx, LOBE_ERR_ARG, "%lld tiles exceed 2^30", toff);
    P.n_entries = eoff;
    P.n_pixels = poff;
    P.n_tiles = (int)toff;
    P.n_super = (int)soff;
    return LOBE_OK;
}

// Argument validation and parameter packing for entry points without a context (noalloc.cu).
lobe_status lobe_internal_build_params(const lobe_config *cfg, const lobe_batch *b, BatchParams &P)
{
    lobe_status s = check_config(nullptr, cfg);
    return s != LOBE_OK ? s : build_params(nullptr, *cfg, b, P);
}

extern "C" {

int32_t lobe_abi_version(void) { return LOBE_ABI_VERSION; }

int64_t lobe_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

lobe_status lobe_batch_sizes(const lobe_config *cfg, const lobe_batch *batch, int64_t out[3])
{
    if (!out) return LOBE_ERR_ARG;
    lobe_status s = check_config(nullptr, cfg);
    if (s != LOBE_OK) return s;
    BatchParams *P = new (std::nothrow) BatchParams;
    if (!P) return LOBE_ERR_OOM;
    s = build_params(nullptr, *cfg, batch, *P);
    if (s == LOBE_OK) {
        out[0] = P->n_entries;
        out[1] = P->n_tiles;
        out[2] = P->n_pixels;
    }
    delete P;
    return s;
}

lobe_status lobe_ctx_create(lobe_ctx **out, void *stream, const lobe_config *cfg)
{
    if (!out) return LOBE_ERR_ARG;
    *out = nullptr;
    lobe_status s = check_config(nullptr, cfg);
    if (s != LOBE_OK) return s;
    lobe_ctx *ctx = new (std::nothrow) lobe_ctx;
    if (!ctx) return LOBE_ERR_OOM;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&ctx->device);
    // status word + look-back control block of the binning scratch, zeroed once
    if (e == cudaSuccess) e = cudaMalloc(&ctx->status, CTL_BYTES);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status, 0, CTL_BYTES, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        delete ctx;
        return LOBE_ERR_CUDA;
    }
    *out = ctx;
    return LOBE_OK;
}

lobe_status lobe_ctx_destroy(lobe_ctx *ctx)
{
    if (!ctx) return LOBE_ERR_ARG;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    cudaFree(ctx->entry_mem);
    cudaFree(ctx->pair_mem);
    cudaFree(ctx->super_mem);
    cudaFree(ctx->order);
    cudaFree(ctx->order_ctl);
    cudaFree(ctx->status);
    delete ctx;
    return LOBE_OK;
}

lobe_status lobe_ctx_set_stream(lobe_ctx *ctx, void *stream)
{
    if (!ctx) return LOBE_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return LOBE_OK;
}

lobe_status lobe_ctx_set_config(lobe_ctx *ctx, const lobe_config *cfg)
{
    if (!ctx) return LOBE_ERR_ARG;
    lobe_status s = check_config(ctx, cfg);
    if (s != LOBE_OK) return s;
    ctx->cfg = *cfg;
    return LOBE_OK;
}

const char *lobe_last_error(const lobe_ctx *ctx) { return ctx ? ctx->err : "no context"; }

static lobe_status grow_region(lobe_ctx *ctx, void *&mem, long long &have, long long need, long long floor_n,
                               size_t (*bytes)(long long), const char *what)
{
    if (need <= have && mem) return LOBE_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    cudaFree(mem);
    mem = nullptr;
    have = 0;
    long long n = need < floor_n ? floor_n : need;
    cudaError_t e = cudaMalloc(&mem, bytes(n));
    if (e != cudaSuccess) return fail(ctx, LOBE_ERR_OOM, "%s scratch (%lld): %s", what, n, cudaGetErrorString(e));
    e = cudaMemsetAsync(mem, 0, bytes(n), ctx->stream);  // look-back words start out matching no call
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(ctx, LOBE_ERR_CUDA, "%s scratch clear: %s", what, cudaGetErrorString(e));
    have = n;
    return LOBE_OK;
}

static lobe_status grow_entries(lobe_ctx *ctx, long long need)
{
    lobe_status s = grow_region(ctx, ctx->entry_mem, ctx->max_entries, need, 1024, entry_scratch_bytes, "entry");
    if (s == LOBE_OK) entry_scratch_carve(ctx->entry_mem, ctx->max_entries, ctx->status, ctx->bins);
    return s;
}

// The pair region also holds per-chunk counts, so its size depends on max_super as well.
static lobe_status grow_pairs(lobe_ctx *ctx, long long need)
{
    long long n = need < 4096 ? 4096 : need;
    if (n < ctx->max_pairs) n = ctx->max_pairs;
    const size_t bytes = pair_scratch_bytes(n, ctx->max_super);
    if (ctx->pair_mem && bytes <= ctx->pair_bytes && n <= ctx->max_pairs) return LOBE_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->pair_mem);
    ctx->pair_mem = nullptr;
    ctx->max_pairs = 0;
    ctx->pair_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->pair_mem, bytes);
    if (e != cudaSuccess) return fail(ctx, LOBE_ERR_OOM, "pair scratch (%lld): %s", n, cudaGetErrorString(e));
    e = cudaMemsetAsync(ctx->pair_mem, 0, bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(ctx, LOBE_ERR_CUDA, "pair scratch clear: %s", cudaGetErrorString(e));
    ctx->max_pairs = n;
    ctx->pair_bytes = bytes;
    pair_scratch_carve(ctx->pair_mem, n, ctx->max_super, ctx->bins);
    return LOBE_OK;
}

static lobe_status grow_super(lobe_ctx *ctx, long long need)
{
    lobe_status s = grow_region(ctx, ctx->super_mem, ctx->max_super, need, 1024, super_scratch_bytes, "super-tile");
    if (s == LOBE_OK) super_scratch_carve(ctx->super_mem, ctx->max_super, ctx->bins);
    if (s == LOBE_OK && ctx->pair_mem) s = grow_pairs(ctx, ctx->max_pairs);  // chunk counts follow max_super
    return s;
}

// Scratch of the persistent compositing (the tile order and its counters) for n_tiles tiles;
// grows only outside a stream capture.
static lobe_status grow_order(lobe_ctx *ctx, long long n_tiles)
{
    if (ctx->order_ctl && n_tiles <= ctx->max_order) return LOBE_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (ctx->stream) CUDA_TRY(cudaStreamIsCapturing(ctx->stream, &cs), "capture query");
    if (cs != cudaStreamCaptureStatusNone)
        return fail(ctx, LOBE_ERR_STATE, "persistent compositing of %lld tiles needs lobe_ctx_reserve before capture",
                    n_tiles);
    if (!ctx->order_ctl) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(unsigned) * ORDER_CTL) != cudaSuccess) return fail(ctx, LOBE_ERR_OOM, "order counters");
        ctx->order_ctl = static_cast<unsigned *>(p);
    }
    if (n_tiles > ctx->max_order) {
        const long long cap = n_tiles + n_tiles / 4 + 1024;
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(int) * cap) != cudaSuccess) return fail(ctx, LOBE_ERR_OOM, "tile order of %lld", cap);
        cudaFree(ctx->order);
        ctx->order = static_cast<int *>(p);
        ctx->max_order = cap;
    }
    return LOBE_OK;
}

lobe_status lobe_ctx_reserve(lobe_ctx *ctx, int64_t max_entries, int64_t max_isect, int64_t max_tiles)
{
    if (!ctx || max_entries < 0 || max_isect < 0 || max_tiles < 0) return fail(ctx, LOBE_ERR_ARG, "bad reserve arguments");
    if (max_tiles > max_super_tiles() * 64) return fail(ctx, LOBE_ERR_ARG, "max_tiles above the supported maximum");
    lobe_status s = grow_entries(ctx, max_entries);
    if (s == LOBE_OK) s = grow_super(ctx, max_tiles);
    if (s == LOBE_OK) s = grow_pairs(ctx, max_isect);
    if (s == LOBE_OK) s = grow_order(ctx, max_tiles);
    return s;
}

lobe_status lobe_get_status(lobe_ctx *ctx)
{
    if (!ctx) return LOBE_ERR_ARG;
    int st = 0;
    CUDA_TRY(cudaMemcpyAsync(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "status read");
    CUDA_TRY(cudaStreamSynchronize(ctx->stream), "status sync");
    CUDA_TRY(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "status clear");
    if (st == STATUS_CAPACITY) return fail(ctx, LOBE_ERR_CAPACITY, "pair count exceeded the bins' capacity");
    if (st == STATUS_TIMEOUT) return fail(ctx, LOBE_ERR_TIMEOUT, "device wait expired");
    return LOBE_OK;
}

lobe_status lobe_sync_status(lobe_ctx *ctx) { return lobe_get_status(ctx); }

lobe_status lobe_fcs_select(const uint32_t *counts, const uint32_t *n_points, int32_t n_items, int32_t n_blocks,
                            double tau, double *V, uint8_t *assign)
{
    if (n_items < 0 || n_blocks < 0 || (n_items > 0 && n_blocks > 0 && (!counts || !n_points || !V || !assign)))
        return LOBE_ERR_ARG;
    for (int32_t c = 0; c < n_items; ++c)
        for (int32_t b = 0; b < n_blocks; ++b) {
            const int64_t k = (int64_t)c * n_blocks + b;
            const double np = n_points[c] > 0 ? (double)n_points[c] : 1.0;
            V[k] = (double)counts[k] / np;
            assign[k] = V[k] >= tau ? 1 : 0;
        }
    return LOBE_OK;
}

lobe_status lobe_selftest_wait(lobe_ctx *ctx)
{
    if (!ctx) return LOBE_ERR_ARG;
    CUDA_TRY(launch_selftest_wait(ctx->status, ctx->stream), "wait self-test");
    return LOBE_OK;
}

// Parameter blocks are ~13 KB: keep them off the host stack of the caller's thread.
struct ParamHolder {
    BatchParams *p;
    ParamHolder() : p(new (std::nothrow) BatchParams) {}
    ~ParamHolder() { delete p; }
};

#define BUILD_PARAMS(H)                                                       \
    if (!ctx) return LOBE_ERR_ARG;                                            \
    ParamHolder H;                                                            \
    if (!H.p) return fail(ctx, LOBE_ERR_OOM, "host parameter block");         \
    {                                                                         \
        lobe_status _s = build_params(ctx, ctx->cfg, batch, *H.p);            \
        if (_s != LOBE_OK) return _s;                                         \
    }

lobe_status lobe_project(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *out)
{
    BUILD_PARAMS(H);
    if (!out || (H.p->n_entries > 0 && (!out->splat || !out->radius || !out->tiles_touched)))
        return fail(ctx, LOBE_ERR_ARG, "projected buffers missing");
    if (!aligned16(out->splat)) return fail(ctx, LOBE_ERR_ARG, "splat not 16-byte aligned");
    CUDA_TRY(launch_project_fwd(*H.p, out->splat, out->radius, out->tiles_touched, ctx->stream), "project");
    return LOBE_OK;
}

lobe_status lobe_bin_sort(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj, const lobe_bins *bins,
                          int64_t *n_isect_host)
{
    BUILD_PARAMS(H);
    const BatchParams &P = *H.p;
    const bool sync = n_isect_host != nullptr;
    if (!proj || (P.n_entries > 0 && (!proj->splat || !proj->radius || !proj->tiles_touched)))
        return fail(ctx, LOBE_ERR_ARG, "projected buffers missing");
    if (!bins || !bins->gauss_ids || !bins->tile_start || !bins->n_isect || bins->capacity < 0)
        return fail(ctx, LOBE_ERR_ARG, "bins missing");
    if (!ctx->cfg.bin_general && bin_small_fits(P)) {  // one CTA, no scratch
        long long *n_isect = reinterpret_cast<long long *>(bins->n_isect);
        CUDA_TRY(launch_bin_small(P, proj->splat, proj->radius, proj->tiles_touched, bins->gauss_ids,
                                  bins->tile_start, n_isect, bins->capacity, ctx->status, ctx->stream),
                 "bin small");
        if (sync) {
            long long total = 0;
            CUDA_TRY(cudaMemcpyAsync(&total, n_isect, sizeof total, cudaMemcpyDeviceToHost, ctx->stream), "n_isect read");
            CUDA_TRY(cudaStreamSynchronize(ctx->stream), "n_isect sync");
            *n_isect_host = total;
            if (total > bins->capacity) {  // the caller is told synchronously instead
                CUDA_TRY(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "status clear");
                return fail(ctx, LOBE_ERR_CAPACITY, "%lld pairs exceed capacity %lld", total, (long long)bins->capacity);
            }
        }
        return LOBE_OK;
    }
    if (P.n_super > max_super_tiles())
        return fail(ctx, LOBE_ERR_ARG, "%d super-tiles (64x64-pixel blocks) exceed %lld", P.n_super, max_super_tiles());
    if (P.n_tiles > max_scan_length(0))
        return fail(ctx, LOBE_ERR_ARG, "%d tiles exceed %lld", P.n_tiles, max_scan_length(0));
    if (P.n_entries > ctx->max_entries || !ctx->entry_mem || P.n_super > ctx->max_super || !ctx->super_mem ||
        !ctx->pair_mem) {
        if (!sync)
            return fail(ctx, LOBE_ERR_STATE,
                        "scratch holds %lld entries / %lld tiles, batch needs %lld / %d: call lobe_ctx_reserve",
                        ctx->max_entries, ctx->max_super, P.n_entries, P.n_tiles);
        lobe_status s = grow_entries(ctx, P.n_entries);
        if (s == LOBE_OK) s = grow_super(ctx, P.n_super);
        if (s == LOBE_OK) s = grow_pairs(ctx, 4096);
        if (s != LOBE_OK) return s;
    }
    long long *n_isect = reinterpret_cast<long long *>(bins->n_isect);
    long long cap = bins->capacity;
    if (!sync && cap > ctx->max_pairs) cap = ctx->max_pairs;
    if (sync) {
        // size the super-tile pair scratch from the exact count before emitting pairs
        long long n_sp = 0;
        CUDA_TRY(bin_super_count(P, proj->splat, proj->radius, proj->tiles_touched, ctx->bins, -1, ctx->stream),
                 "bin count");
        CUDA_TRY(cudaMemcpyAsync(&n_sp, ctx->bins.scalars + 4, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream),
                 "pair count read");
        CUDA_TRY(cudaStreamSynchronize(ctx->stream), "pair count sync");
        n_sp &= 0xffffffffLL;
        if (n_sp > ctx->max_pairs) {
            lobe_status s = grow_pairs(ctx, n_sp + n_sp / 4);
            if (s != LOBE_OK) return s;
        }
    } else {
        CUDA_TRY(bin_super_count(P, proj->splat, proj->radius, proj->tiles_touched, ctx->bins, ctx->max_pairs,
                                 ctx->stream),
                 "bin count");
    }
    CUDA_TRY(bin_tile_count(P, proj->splat, proj->radius, ctx->bins, ctx->max_pairs, n_isect, bins->tile_start, cap,
                            ctx->stream),
             "tile count");
    if (sync) {
        long long total = 0;
        CUDA_TRY(cudaMemcpyAsync(&total, n_isect, sizeof total, cudaMemcpyDeviceToHost, ctx->stream), "n_isect read");
        CUDA_TRY(cudaStreamSynchronize(ctx->stream), "n_isect sync");
        *n_isect_host = total;
        if (total > bins->capacity) {
            // the device latched the overflow too; the caller is told synchronously instead
            CUDA_TRY(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "status clear");
            CUDA_TRY(bin_sort_emit(P, proj->splat, proj->radius, ctx->bins, n_isect, bins->gauss_ids, bins->tile_start,
                                   ctx->stream),
                     "bin emit");
            return fail(ctx, LOBE_ERR_CAPACITY, "%lld pairs exceed capacity %lld", total, (long long)bins->capacity);
        }
    }
    CUDA_TRY(bin_sort_emit(P, proj->splat, proj->radius, ctx->bins, n_isect, bins->gauss_ids, bins->tile_start,
                           ctx->stream),
             "bin emit");
    return LOBE_OK;
}

lobe_status lobe_render_fwd(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj, const lobe_bins *bins,
                            const lobe_image *image)
{
    BUILD_PARAMS(H);
    if (!proj || (H.p->n_entries > 0 && !proj->splat) || !bins || !bins->gauss_ids || !bins->tile_start)
        return fail(ctx, LOBE_ERR_ARG, "inputs missing");
    if (!image || !image->rgb || !image->T_final || !image->n_contrib) return fail(ctx, LOBE_ERR_ARG, "image buffers missing");
    if (ctx->cfg.persistent) {
        lobe_status s = grow_order(ctx, H.p->n_tiles);
        if (s != LOBE_OK) return s;
    }
    CUDA_TRY(launch_render_fwd(*H.p, proj->splat, bins->tile_start, bins->gauss_ids, image->rgb, image->T_final,
                               image->n_contrib, nullptr, ctx->cfg.persistent ? ctx->order : nullptr, ctx->order_ctl,
                               ctx->stream),
             "render fwd");
    return LOBE_OK;
}

lobe_status lobe_render_depth(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj,
                              const lobe_bins *bins, const lobe_image *image, float *depth)
{
    BUILD_PARAMS(H);
    if (!proj || (H.p->n_entries > 0 && !proj->splat) || !bins || !bins->gauss_ids || !bins->tile_start)
        return fail(ctx, LOBE_ERR_ARG, "inputs missing");
    if (!image || !image->rgb || !image->T_final || !image->n_contrib) return fail(ctx, LOBE_ERR_ARG, "image buffers missing");
    if (!depth && H.p->n_pixels > 0) return fail(ctx, LOBE_ERR_ARG, "depth is NULL");
    if (ctx->cfg.persistent) {
        lobe_status s = grow_order(ctx, H.p->n_tiles);
        if (s != LOBE_OK) return s;
    }
    CUDA_TRY(launch_render_fwd(*H.p, proj->splat, bins->tile_start, bins->gauss_ids, image->rgb, image->T_final,
                               image->n_contrib, depth, ctx->cfg.persistent ? ctx->order : nullptr, ctx->order_ctl,
                               ctx->stream),
             "render depth");
    return LOBE_OK;
}

lobe_status lobe_fcs_coverage(lobe_ctx *ctx, const lobe_batch *batch, const lobe_image *image, const float *depth,
                              const lobe_aabb *blocks, int32_t n_blocks, int32_t normalize, uint32_t *counts,
                              uint32_t *n_points)
{
    BUILD_PARAMS(H);
    if (n_blocks < 0 || n_blocks > FCS_MAX_BLOCKS)
        return fail(ctx, LOBE_ERR_ARG, "n_blocks %d outside [0, %d]", n_blocks, FCS_MAX_BLOCKS);
    if (n_blocks > 0 && !blocks) return fail(ctx, LOBE_ERR_ARG, "blocks is NULL");
    if (!counts || !n_points) return fail(ctx, LOBE_ERR_ARG, "outputs missing");
    if (H.p->n_pixels > 0 && (!image || !image->T_final || !depth)) return fail(ctx, LOBE_ERR_ARG, "inputs missing");
    FcsBlocks B{};
    B.n = n_blocks;
    for (int b = 0; b < n_blocks; ++b)
        for (int k = 0; k < 3; ++k) {
            B.lo[b][k] = blocks[b].lo[k];
            B.hi[b][k] = blocks[b].hi[k];
        }
    CUDA_TRY(launch_fcs_coverage(*H.p, B, depth, image ? image->T_final : nullptr, normalize ? 1 : 0, counts, n_points,
                                 ctx->stream),
             "fcs coverage");
    return LOBE_OK;
}

lobe_status lobe_render_bwd(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj, const lobe_bins *bins,
                            const lobe_image *image, const float *dL_drgb, float *grad2d)
{
    BUILD_PARAMS(H);
    const bool rec = ctx->cfg.recompute_T != 0;
    const bool has_e = H.p->n_entries > 0;
    if (!proj || (has_e && !proj->splat) || !bins || !bins->gauss_ids || !bins->tile_start)
        return fail(ctx, LOBE_ERR_ARG, "inputs missing");
    if (!dL_drgb || (has_e && (!grad2d || !aligned16(grad2d))))
        return fail(ctx, LOBE_ERR_ARG, "dL_drgb/grad2d missing or misaligned");
    if (!rec && (!image || !image->T_final || !image->n_contrib))
        return fail(ctx, LOBE_ERR_ARG, "saved forward state missing (recompute_T = 0)");
    if (ctx->cfg.persistent) {
        lobe_status s = grow_order(ctx, H.p->n_tiles);
        if (s != LOBE_OK) return s;
    }
    CUDA_TRY(launch_render_bwd(*H.p, rec, proj->splat, bins->tile_start, bins->gauss_ids, rec ? nullptr : image->T_final,
                               rec ? nullptr : image->n_contrib, dL_drgb, grad2d,
                               ctx->cfg.persistent ? ctx->order : nullptr, ctx->order_ctl, ctx->stream),
             "render bwd");
    return LOBE_OK;
}

lobe_status lobe_project_bwd(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj, const float *grad2d,
                             const lobe_grads *grads, int32_t accumulate)
{
    BUILD_PARAMS(H);
    BatchParams &P = *H.p;
    if (!grads || (P.n_entries > 0 && (!proj || !proj->splat || !proj->radius || !grad2d)))
        return fail(ctx, LOBE_ERR_ARG, "inputs missing");
    for (int s = 0; s < P.n_sets; ++s) {
        const lobe_grads &g = grads[s];
        if (P.set[s].n > 0 && (!g.means || !g.log_scales || !g.quats || !g.opacity_logits || !g.sh))
            return fail(ctx, LOBE_ERR_ARG, "set %d: gradient pointer is NULL", s);
        if (!aligned16(g.quats) || !aligned16(g.sh)) return fail(ctx, LOBE_ERR_ARG, "set %d: quats/sh grads misaligned", s);
        if ((g.sd_acc == nullptr) != (g.sd_cnt == nullptr)) return fail(ctx, LOBE_ERR_ARG, "set %d: sd_acc/sd_cnt mismatch", s);
        P.set[s].g_means = g.means;
        P.set[s].g_log_scales = g.log_scales;
        P.set[s].g_quats = g.quats;
        P.set[s].g_logits = g.opacity_logits;
        P.set[s].g_sh = g.sh;
        P.set[s].sd_acc = g.sd_acc;
        P.set[s].sd_cnt = g.sd_cnt;
    }
    // the list of Gaussians some item sees goes to the binning scratch (free once bin_sort has
    // returned), its length to scalars[8]; at most n_entries Gaussians can be seen
    // (the compaction's look-back words, one per 4096 Gaussians, come from the same scratch)
    if (!ctx->entry_mem || ctx->max_entries < P.n_entries || max_scan_length(ctx->max_entries) < P.n_gauss) {
        lobe_status s = grow_entries(ctx, P.n_entries > P.n_gauss ? P.n_entries : P.n_gauss);
        if (s != LOBE_OK) return s;
    }
    CUDA_TRY(launch_project_bwd(P, proj->splat, proj->radius, grad2d, accumulate ? 1 : 0, ctx->bins.dkB,
                                ctx->bins.scalars + 8, ctx->bins.scan_slots, ctx->bins.ctl, ctx->stream),
             "project bwd");
    return LOBE_OK;
}

// ------------------------------------------------------------------ Adam

static bool adam_arrays_ok(const lobe_param_arrays &a)
{
    return a.means && a.log_scales && a.quats && a.opacity_logits && a.sh && aligned16(a.means) &&
           aligned16(a.log_scales) && aligned16(a.quats) && aligned16(a.opacity_logits) && aligned16(a.sh);
}

static void adam_set(const lobe_adam_state &st, AdamSet &z)
{
    const lobe_param_arrays *arr[3] = {&st.param, &st.exp_avg, &st.exp_avg_sq};
    float **dst[3] = {z.p, z.m, z.v};
    for (int i = 0; i < 3; ++i) {
        dst[i][0] = arr[i]->means;
        dst[i][1] = arr[i]->log_scales;
        dst[i][2] = arr[i]->quats;
        dst[i][3] = arr[i]->opacity_logits;
        dst[i][4] = arr[i]->sh;
    }
}

static lobe_status adam_constants(lobe_ctx *ctx, const lobe_adam_params *prm, AdamK &k)
{
    if (!prm) return fail(ctx, LOBE_ERR_ARG, "adam parameters missing");
    if (prm->step < 1) return fail(ctx, LOBE_ERR_ARG, "adam step %lld < 1", (long long)prm->step);
    if (!(prm->beta1 >= 0.0 && prm->beta1 < 1.0 && prm->beta2 >= 0.0 && prm->beta2 < 1.0) || !(prm->eps >= 0.f))
        return fail(ctx, LOBE_ERR_ARG, "adam betas outside [0, 1) or eps negative");
    const double t = (double)prm->step;
    const double bc1 = 1.0 - std::pow(prm->beta1, t), bc2 = 1.0 - std::pow(prm->beta2, t);
    if (!(bc1 > 0.0 && bc2 > 0.0)) return fail(ctx, LOBE_ERR_ARG, "adam bias correction is zero");
    k.b1 = (float)prm->beta1;
    k.b2 = (float)prm->beta2;
    k.omb1 = (float)(1.0 - prm->beta1);
    k.omb2 = (float)(1.0 - prm->beta2);
    k.eps = prm->eps;
    k.rsb2 = (float)(1.0 / std::sqrt(bc2));
    const float lr[AG_COUNT] = {prm->lr_means, prm->lr_log_scales, prm->lr_quats,
                                prm->lr_opacity, prm->lr_sh_dc, prm->lr_sh_rest};
    for (int i = 0; i < AG_COUNT; ++i) k.ss[i] = (float)((double)lr[i] / bc1);
    return LOBE_OK;
}

lobe_status lobe_adam(lobe_ctx *ctx, int64_t n, const lobe_adam_state *state, const lobe_param_arrays *grad,
                      const uint8_t *rows, const lobe_adam_params *prm)
{
    if (!ctx) return LOBE_ERR_ARG;
    if (n < 0) return fail(ctx, LOBE_ERR_ARG, "negative size");
    AdamK k;
    lobe_status st = adam_constants(ctx, prm, k);
    if (st != LOBE_OK) return st;
    if (n == 0) return LOBE_OK;
    if (12 * n > (1ll << 32) - (1ll << 22)) return fail(ctx, LOBE_ERR_ARG, "adam: more than 357M Gaussians in one set");
    if (!state || !grad) return fail(ctx, LOBE_ERR_ARG, "state or gradients missing");
    if (!adam_arrays_ok(state->param) || !adam_arrays_ok(state->exp_avg) || !adam_arrays_ok(state->exp_avg_sq) ||
        !adam_arrays_ok(*grad))
        return fail(ctx, LOBE_ERR_ARG, "adam arrays missing or not 16-byte aligned");
    AdamSet z;
    adam_set(*state, z);
    const float *g[5] = {grad->means, grad->log_scales, grad->quats, grad->opacity_logits, grad->sh};
    CUDA_TRY(launch_adam(n, z, g, rows, rows ? 1 : 0, k, ctx->stream), "adam");
    return LOBE_OK;
}

lobe_status lobe_project_bwd_adam(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj,
                                  const float *grad2d, const lobe_grads *sd, const lobe_adam_state *states,
                                  const lobe_adam_params *prm, int32_t sparse)
{
    BUILD_PARAMS(H);
    BatchParams &P = *H.p;
    AdamBatch *A = new (std::nothrow) AdamBatch;
    if (!A) return fail(ctx, LOBE_ERR_OOM, "host parameter block");
    struct Free {
        AdamBatch *a;
        ~Free() { delete a; }
    } free_a{A};
    memset(A, 0, sizeof *A);
    if (!prm) return fail(ctx, LOBE_ERR_ARG, "adam parameters missing");
    for (int s = 0; s < P.n_sets; ++s) {
        lobe_status st = adam_constants(ctx, prm + s, A->k[s]);
        if (st != LOBE_OK) return st;
    }
    if (!states || (P.n_entries > 0 && (!proj || !proj->splat || !proj->radius || !grad2d)))
        return fail(ctx, LOBE_ERR_ARG, "inputs missing");
    for (int s = 0; s < P.n_sets; ++s) {
        const lobe_adam_state &z = states[s];
        const lobe_gaussians &G = batch->sets[s];
        if (12 * P.set[s].n > (1ll << 32) - (1ll << 22))
            return fail(ctx, LOBE_ERR_ARG, "set %d: adam takes at most 357M Gaussians a set", s);
        if (P.set[s].n > 0) {
            if (!adam_arrays_ok(z.param) || !adam_arrays_ok(z.exp_avg) || !adam_arrays_ok(z.exp_avg_sq))
                return fail(ctx, LOBE_ERR_ARG, "set %d: adam arrays missing or not 16-byte aligned", s);
            if (z.param.means != G.means || z.param.log_scales != G.log_scales || z.param.quats != G.quats ||
                z.param.opacity_logits != G.opacity_logits || z.param.sh != G.sh)
                return fail(ctx, LOBE_ERR_ARG, "set %d: adam parameters are not the batch's set", s);
        }
        adam_set(z, A->set[s]);
        if (sd) {
            if ((sd[s].sd_acc == nullptr) != (sd[s].sd_cnt == nullptr))
                return fail(ctx, LOBE_ERR_ARG, "set %d: sd_acc/sd_cnt mismatch", s);
            P.set[s].sd_acc = sd[s].sd_acc;
            P.set[s].sd_cnt = sd[s].sd_cnt;
        }
    }
    if (!ctx->entry_mem || ctx->max_entries < P.n_entries || max_scan_length(ctx->max_entries) < P.n_gauss) {
        lobe_status s = grow_entries(ctx, P.n_entries > P.n_gauss ? P.n_entries : P.n_gauss);
        if (s != LOBE_OK) return s;
    }
    // standard Adam: the list kernel records who is seen (one byte per Gaussian, in the
    // binning scratch) for the zero-gradient pass over the others
    uint8_t *seen = reinterpret_cast<uint8_t *>(ctx->bins.offs);
    if (!sparse)
        for (int s = 0; s < P.n_sets; ++s) P.set[s].vis_mask = seen + P.set[s].gauss_off;
    CUDA_TRY(launch_project_bwd(P, proj->splat, proj->radius, grad2d, 1, ctx->bins.dkB, ctx->bins.scalars + 8,
                                ctx->bins.scan_slots, ctx->bins.ctl, ctx->stream, A),
             "project bwd + adam");
    if (!sparse)
        for (int s = 0; s < P.n_sets; ++s)
            CUDA_TRY(launch_adam(P.set[s].n, A->set[s], nullptr, seen + P.set[s].gauss_off, 2, A->k[s], ctx->stream),
                     "adam (unseen Gaussians)");
    return LOBE_OK;
}

lobe_status lobe_densify(lobe_ctx *ctx, const lobe_gaussians *set, const float *sd_acc, const int32_t *sd_cnt,
                         const float *normals, const lobe_densify_params *prm, const lobe_params_out *out,
                         int32_t *source, int64_t *n_out_host)
{
    if (!ctx) return LOBE_ERR_ARG;
    if (!set || !prm || !out || !n_out_host) return fail(ctx, LOBE_ERR_ARG, "arguments missing");
    const long long n = set->n;
    if (n < 0 || out->capacity < 0) return fail(ctx, LOBE_ERR_ARG, "negative size");
    if (n > 0 && (!set->means || !set->log_scales || !set->quats || !set->opacity_logits || !set->sh || !sd_acc ||
                  !sd_cnt || !normals))
        return fail(ctx, LOBE_ERR_ARG, "input pointers missing");
    if (out->capacity > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh))
        return fail(ctx, LOBE_ERR_ARG, "output pointers missing");
    if (prm->n_split < 1 || prm->n_split > 4) return fail(ctx, LOBE_ERR_ARG, "n_split %d outside [1, 4]", prm->n_split);
    if (!aligned16(set->quats) || !aligned16(set->sh) || !aligned16(out->quats) || !aligned16(out->sh))
        return fail(ctx, LOBE_ERR_ARG, "quats/sh misaligned");
    if (n > (long long)UINT32_MAX / 4) return fail(ctx, LOBE_ERR_ARG, "too many Gaussians");
    // per-Gaussian action (1 byte) and output count/offset (4 bytes) live in the entry scratch
    if (!ctx->entry_mem || ctx->max_entries < n) {
        lobe_status s = grow_entries(ctx, n);
        if (s != LOBE_OK) return s;
    }
    uint8_t *action = reinterpret_cast<uint8_t *>(ctx->bins.offs);
    uint32_t *offs = ctx->bins.vis_pos, *total = ctx->bins.scalars + 9;
    CUDA_TRY(launch_densify_count(n, *set, sd_acc, sd_cnt, *prm, action, offs, total,
                                  LB{ctx->bins.scan_slots, ctx->bins.ctl, ST_DENSIFY}, ctx->stream),
             "densify count");
    uint32_t n_out = 0;
    CUDA_TRY(cudaMemcpyAsync(&n_out, total, sizeof n_out, cudaMemcpyDeviceToHost, ctx->stream), "densify count read");
    CUDA_TRY(cudaStreamSynchronize(ctx->stream), "densify sync");
    *n_out_host = (int64_t)n_out;
    if ((long long)n_out > out->capacity)
        return fail(ctx, LOBE_ERR_CAPACITY, "%u outputs exceed capacity %lld", n_out, (long long)out->capacity);
    CUDA_TRY(launch_densify_emit(n, *set, action, offs, total, normals, *prm, *out, source, ctx->stream), "densify emit");
    return LOBE_OK;
}

lobe_status lobe_visibility_crop(lobe_ctx *ctx, const lobe_batch *batch, uint8_t *const *masks)
{
    BUILD_PARAMS(H);
    BatchParams &P = *H.p;
    if (!masks) return fail(ctx, LOBE_ERR_ARG, "masks is NULL");
    for (int s = 0; s < P.n_sets; ++s) {
        if (P.set[s].n > 0 && !masks[s]) return fail(ctx, LOBE_ERR_ARG, "set %d: mask is NULL", s);
        P.set[s].vis_mask = masks[s];
    }
    CUDA_TRY(launch_visibility(P, ctx->stream), "visibility crop");
    return LOBE_OK;
}

}  // extern "C"
