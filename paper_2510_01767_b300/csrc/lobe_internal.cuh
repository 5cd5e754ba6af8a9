// lobe_internal.cuh -- device-side parameter blocks and helpers shared by the kernels.
//
// Every kernel receives the whole batch description by value (a __grid_constant__
// parameter block of ~13 KB), so a launch carries no host->device copy and a captured
// CUDA graph replays with the parameters baked in.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <utility>

#include "lobe.h"

namespace lobe {

// ------------------------------------------------------------------ parameter blocks

struct SetParams {
    const float *means, *log_scales, *quats, *logits, *sh;
    const uint8_t *crop;
    // projection backward outputs (only read by the backward kernel)
    float *g_means, *g_log_scales, *g_quats, *g_logits, *g_sh;
    float *sd_acc;
    int32_t *sd_cnt;
    uint8_t *vis_mask;
    long long n;
    long long gauss_off;  // first thread index of this set in set-major kernels
    int item_begin;       // into BatchParams::set_items
    int item_count;
};

struct ItemParams {
    float V[12];          // rows 0..2 of the row-major world->camera matrix
    double Vz[4];         // row 2 widened to double (exact), for the depth key
    float fx, fy, cx, cy;
    double near_plane, far_plane;
    float campos[3];
    float limx, limy;     // 1.3 * tan(fov/2) per axis
    float lo[3], hi[3];   // block box
    int W, H;
    int gx, gy;           // tiles per row / column
    int tile_off;         // first global tile id
    int sgx, sgy;         // super-tiles per row / column (super-tile = S x S tiles)
    int super_off;        // first global super-tile id
    int set;
    long long entry_off;  // first projected entry
    long long pix_off;    // first pixel
};

struct BatchParams {
    SetParams set[LOBE_MAX_SETS];
    ItemParams item[LOBE_MAX_ITEMS];
    int set_items[LOBE_MAX_ITEMS];  // item indices grouped by set
    int n_sets, n_items;
    long long n_gauss;    // sum of set sizes
    long long n_entries;  // sum over items of the set size
    int n_tiles;
    int n_super;          // super-tiles over all items
    int S;                // super-tile edge in tiles
    long long n_pixels;
    int tw, th;
    int px_fwd, px_bwd;   // pixels per lane of the render kernels (0 = default)
    int nb_fwd, nb_bwd;   // 32-splat staging rounds a warp fetches at once in the render kernels (1 or 2)
    int sh_degree;
    float bg[3];
};

int default_px(int tw, int th, bool backward);
bool valid_px(int tw, int th, int px);

// Super-tile edge (in tiles) of the two-level binning: 64 px for 8x8 and 16x16 tiles.
__host__ __device__ inline int super_edge(int tw) { return tw == 8 ? 8 : 4; }

__device__ __forceinline__ int item_of_super(const BatchParams &P, int s)
{
    int lo = 0, hi = P.n_items - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.item[mid].super_off <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------ device status

enum : int { STATUS_OK = 0, STATUS_CAPACITY = 1, STATUS_TIMEOUT = 2 };

__device__ __forceinline__ void set_status(int *status, int code)
{
    atomicCAS(status, STATUS_OK, code);
}

// ------------------------------------------------------------------ lookups

__device__ __forceinline__ int item_of_tile(const BatchParams &P, int t)
{
    int lo = 0, hi = P.n_items - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.item[mid].tile_off <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int item_of_entry(const BatchParams &P, long long e)
{
    int lo = 0, hi = P.n_items - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.item[mid].entry_off <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int set_of_gauss(const BatchParams &P, long long t)
{
    int s = 0;
    while (s + 1 < P.n_sets && t >= P.set[s + 1].gauss_off) ++s;
    return s;
}

// Tile rectangle of a splat: [floor((u-r)/tw), ceil((u+r)/tw)) x [floor((v-r)/th), ceil((v+r)/th))
// clamped to the grid, evaluated exactly in integers: for integer r and t > 0,
// floor((u-r)/t) = floor((floor(u)-r)/t) and ceil((u+r)/t) = ceil((ceil(u)+r)/t); t is a
// power of two, so the divisions are arithmetic shifts. Every kernel that needs the
// rectangle gets the same answer, equal to the real-number definition.
__device__ __forceinline__ int floor_div_pow2(int a, int t) { return a >> (31 - __clz(t)); }
__device__ __forceinline__ int ceil_div_pow2(int a, int t) { return -((-a) >> (31 - __clz(t))); }

__device__ __forceinline__ void tile_rect(float u, float v, int r, int tw, int th, int gx, int gy,
                                          int &x0, int &y0, int &x1, int &y1)
{
    // |u|, |v| are bounded by the 1.3x field-of-view guard, far inside the int range
    const int fu = (int)floorf(u), cu = (int)ceilf(u), fv = (int)floorf(v), cv = (int)ceilf(v);
    x0 = min(max(floor_div_pow2(fu - r, tw), 0), gx);
    y0 = min(max(floor_div_pow2(fv - r, th), 0), gy);
    x1 = min(max(ceil_div_pow2(cu + r, tw), 0), gx);
    y1 = min(max(ceil_div_pow2(cv + r, th), 0), gy);
}

// ------------------------------------------------------------------ PTX helpers

// hardware base-2 exponential (PTX ex2.approx.ftz.f32)
__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// vector reduction-add of four floats into global memory (sm_90+)
__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

__device__ __forceinline__ void red_add_f32(float *addr, float a)
{
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(a) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------------------------ compositing step
//
// Constants of the compositing step (render.cu). The staged splat holds the conic pre-scaled
// into the base-2 exponent domain:
//   A = -0.5 a log2(e), B = -b log2(e), C = -0.5 c log2(e)  =>  G = exp(-sigma) = 2^(A dx^2 + B dx dy + C dy^2)

constexpr float LOG2E = 1.4426950408889634f;
constexpr float LN2 = 0.6931471805599453f;
constexpr float ALPHA_MIN = 1.0f / 255.0f;
constexpr float ALPHA_MAX = 0.99f;
constexpr float T_MIN = 1e-4f;

// T after a contributor; the stop rule is `next_T(T, alpha) < T_MIN` (checked before adding)
__device__ __forceinline__ float next_T(float T, float alpha) { return __fmul_rn(T, __fsub_rn(1.0f, alpha)); }

// ------------------------------------------------------------------ Adam
//
// One Adam update (Kingma and Ba) per element, in float32: with 1 - b1, 1 - b2,
// ss = lr / (1 - b1^t) and rsb2 = 1 / sqrt(1 - b2^t) formed on the host in double (from
// double betas: 1 - 0.999f would be off by 1.3e-5),
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,  p <- p - ss m / (sqrt(v) rsb2 + eps),
// which is p - lr m_hat / (sqrt(v_hat) + eps) with the bias-corrected moments. The fused
// projection adjoint and the standalone kernel share this step.

// learning-rate groups of a Gaussian set (the SH split into its degree-0 and other bands)
enum AdamGroup { AG_MEANS = 0, AG_LOG_SCALES, AG_QUATS, AG_OPACITY, AG_SH_DC, AG_SH_REST, AG_COUNT };

struct AdamK {
    float b1, b2, omb1, omb2, eps, rsb2;
    float ss[AG_COUNT];
};

// The square root and the division take the PTX approximations (sqrt.approx.f32: relative
// error at most 2^-23; div.approx.f32: at most 2 ulp for a denominator in [2^-126, 2^126],
// which eps >= 1e-15 and any finite moment keep): one instruction each instead of the
// correctly rounded sequences, which would triple the update's instruction count.
__device__ __forceinline__ float adam_sqrt(float x)
{
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void adam_step(const AdamK &k, float ss, float g, float &p, float &m, float &v)
{
    m = fmaf(k.b1, m, k.omb1 * g);
    v = fmaf(k.b2, v, k.omb2 * (g * g));
    p = p - ss * __fdividef(m, fmaf(adam_sqrt(v), k.rsb2, k.eps));
}

// zero gradient (a Gaussian no item sees, under standard Adam)
__device__ __forceinline__ void adam_decay(const AdamK &k, float ss, float &p, float &m, float &v)
{
    m = k.b1 * m;
    v = k.b2 * v;
    p = p - ss * __fdividef(m, fmaf(adam_sqrt(v), k.rsb2, k.eps));
}

// the parameters and moments of one set, in the order means, log_scales, quats, opacity, sh
struct AdamSet {
    float *p[5], *m[5], *v[5];
};

// fused adjoint + Adam: per set of the batch
struct AdamBatch {
    AdamSet set[LOBE_MAX_SETS];
    AdamK k[LOBE_MAX_SETS];
};

// ------------------------------------------------------------------ scratch and launchers

// Scratch of the binning stage (context-owned, or carved from any device buffer). The
// "entry" part scales with the projected entries, the "pair" part with the super-tile pairs
// (at most the (splat, tile) pairs), the "super" part with the super-tiles; each can grow
// independently.
struct BinScratch {
    uint32_t *vis_pos, *dkA, *dvA, *dkB, *dvB, *offs;  // [max_entries]
    uint32_t *counts;   // radix digit counts per block [256][blocks], scanned in place
    uint2 *rect;        // [max_entries] tile rectangles of the visible entries (aliases counts)
    uint32_t *scalars;  // [0] visible splats, [1] usable super pairs, [2] usable pairs, [4] super pairs
    unsigned long long *scan_slots;                    // decoupled look-back words of the scans
    uint32_t *os_hist;                                 // [4][256] digit histograms of the depth keys
    unsigned long long *os_slots;                      // depth sort look-back words [tiles][256]
    uint32_t *skA, *svA, *skB, *svB;                   // [max_pairs]
    uint32_t *sp_keys, *sp_ids;                        // sorted super pairs (one of the A/B arrays)
    uint4 *work;                                       // per chunk: (super-tile, first pair, end pair)
    uint32_t *chunk_cnt;                               // per (chunk, tile) counts, then offsets
    uint32_t *super_start, *chunk_base;                // [max_super + 1] each
    long long work_max;                                // bound on chunk work items of the last call
    int *ctl;     // control block: [0] status, [1] look-back generation, [2..17] ticket counters
    int *status;  // == ctl
};

// Programmatic dependent launch: a kernel launched with launch_pdl may be scheduled while its
// predecessor on the stream is still finishing, which hides the launch latency of the chains
// of short kernels (binning runs ~20 in a row). Every kernel of this library begins with
// pdl_wait(), which returns once the predecessor grid has completed and its writes are
// visible (and at once when there is no programmatic predecessor), then lets its own
// dependents be scheduled (pdl_trigger).
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
}

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                     Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Counts kernel launches made by this library (process-wide, all contexts).
void count_launch(int n = 1);

cudaError_t launch_project_fwd(const BatchParams &, float *, int *, int *, cudaStream_t);
cudaError_t launch_visibility(const BatchParams &, cudaStream_t);
cudaError_t launch_project_bwd(const BatchParams &, const float *, const int *, const float *, int, uint32_t *list,
                               uint32_t *count, unsigned long long *lb_slots, int *ctl, cudaStream_t,
                               const AdamBatch *adam = nullptr);
// Binning of a small batch (<= 4096 entries and tiles, tiles x entries <= 2^20) in one CTA,
// bit-identical to the general path: tile_start, gauss_ids, n_isect; capacity overflow latched.
bool bin_small_fits(const BatchParams &P);
cudaError_t launch_bin_small(const BatchParams &P, const float *splat, const int *radius, const int *tiles,
                             int *gauss_ids, int *tile_start, long long *n_isect, long long capacity, int *status,
                             cudaStream_t st);
// One warp waits on a look-back word nothing publishes until its spin limit latches
// STATUS_TIMEOUT in ctl[0] (the bounded-wait self-test).
cudaError_t launch_selftest_wait(int *ctl, cudaStream_t st);
// Standalone Adam over one set: mode 0 every row, 1 rows with rows[r] != 0 (sparse), 2 rows
// with rows[r] == 0 and a zero gradient (grad unused: the Gaussians no item saw, after the
// fused adjoint has updated the others).
cudaError_t launch_adam(long long n, const AdamSet &s, const float *const grad[5], const uint8_t *rows, int mode,
                        const AdamK &k, cudaStream_t);
// Compositing and its adjoint. order/ctl non-null: persistent mode (tiles longest list first);
// order holds n_tiles ints, ctl ORDER_CTL words (both device scratch).
constexpr int ORDER_CTL = 67;
cudaError_t launch_render_fwd(const BatchParams &, const float *, const int *, const int *, float *, float *, int *,
                              float *depth, int *order, unsigned *ctl, cudaStream_t);

// Block boxes of fast camera selection (kernel parameter).
constexpr int FCS_MAX_BLOCKS = 64;
struct FcsBlocks {
    float lo[FCS_MAX_BLOCKS][3], hi[FCS_MAX_BLOCKS][3];
    int n;
};
struct LB;
cudaError_t launch_densify_count(long long n, const lobe_gaussians &in, const float *acc, const int *cnt,
                                 const lobe_densify_params &prm, uint8_t *action, uint32_t *n_out, uint32_t *total,
                                 LB lb, cudaStream_t st);
cudaError_t launch_densify_emit(long long n, const lobe_gaussians &in, const uint8_t *action, const uint32_t *off,
                                const uint32_t *total, const float *normals, const lobe_densify_params &prm,
                                const lobe_params_out &out, int *source, cudaStream_t st);
cudaError_t launch_fcs_coverage(const BatchParams &, const FcsBlocks &, const float *depth, const float *Tfin,
                                int normalize, uint32_t *counts, uint32_t *n_points, cudaStream_t);
cudaError_t launch_render_bwd(const BatchParams &, bool, const float *, const int *, const int *, const float *,
                              const int *, const float *, float *, int *order, unsigned *ctl, cudaStream_t);
cudaError_t bin_super_count(const BatchParams &P, const float *splat, const int *radius, const int *tiles,
                            BinScratch &b, long long pair_capacity, cudaStream_t st);
cudaError_t bin_tile_count(const BatchParams &P, const float *splat, const int *radius, BinScratch &b,
                           long long pair_capacity, long long *n_isect_dev, int *tile_start, long long isect_capacity,
                           cudaStream_t st);
cudaError_t bin_sort_emit(const BatchParams &P, const float *splat, const int *radius, BinScratch &b,
                          const long long *n_isect_dev, int *gauss_ids, int *tile_start, cudaStream_t st);
size_t entry_scratch_bytes(long long max_entries);
size_t pair_scratch_bytes(long long max_pairs, long long max_super);
size_t super_scratch_bytes(long long max_super);
long long max_super_tiles();  // super-tile ids must fit the 16 key bits that carry them
long long max_scan_length(long long max_entries);  // longest scan the entry scratch serves (>= 2^22 tiles)
constexpr size_t CTL_BYTES = 256;                  // control block of a binning scratch (zeroed once)
void entry_scratch_carve(void *mem, long long max_entries, int *ctl, BinScratch &b);
void pair_scratch_carve(void *mem, long long max_pairs, long long max_super, BinScratch &b);
void super_scratch_carve(void *mem, long long max_super, BinScratch &b);

}  // namespace lobe
