/*
 * lobe.h -- C ABI of the B300 (sm_103a) differentiable tile rasterizer used by the
 * per-block fine-training step of LoBE-GS (arXiv 2510.01767).
 *
 * The paper trains each KD-tree block with the vanilla 3DGS procedure (appendix,
 * "3DGS Training"): differentiable rasterization of 3D Gaussians (Sec. 2.1), frustum
 * culling during rasterization (Sec. 3.3), front-to-back alpha blending (the blending
 * equation of Sec. 3.2, with colour in place of depth), visibility cropping and
 * selective densification (Sec. 3.3). This library implements that rasterizer as four
 * stages plus their adjoints:
 *
 *   lobe_project      Gaussians -> 2D splats (mean, conic, colour, opacity, depth, radius)
 *   lobe_bin_sort     splats -> per-tile lists ordered by (tile, depth, index)
 *   lobe_render_fwd   per-tile front-to-back compositing
 *   lobe_render_bwd   adjoint of the composite -> per-splat 2D gradients
 *   lobe_project_bwd  adjoint of the projection -> parameter gradients + SD statistics
 *   lobe_render_depth, lobe_fcs_coverage   fast camera selection (Sec. 3.2)
 *   lobe_densify      selective densification (Sec. 3.3) with 3DGS density control
 *
 * A "batch" is a list of items (Gaussian set, camera, block); one call processes every
 * item of the batch in one launch per stage. The plain single-view path is a batch of one.
 *
 * Conventions (all calls):
 *  - Every pointer inside the structs below is a DEVICE pointer allocated and owned by the
 *    caller, except the struct arrays themselves (lobe_batch members), which are HOST
 *    memory read during the call only. The library never frees caller memory.
 *  - Every call is asynchronous on the context's CUDA stream and returns after enqueueing,
 *    except where a host output pointer is given (then it synchronises that stream).
 *  - Argument errors are reported synchronously (LOBE_ERR_ARG) and nothing is enqueued.
 *  - Errors found on the device (intersection count above capacity) are latched in a
 *    device status word; lobe_get_status() reads and clears it.
 *  - All floating-point data is float32, little-endian, C-contiguous.
 *  - The calls that take a context are safe to capture in a CUDA graph when no host
 *    output pointer is passed and lobe_ctx_reserve() was called beforehand.
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef LOBE_H
#define LOBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LOBE_ABI_VERSION 1
#define LOBE_MAX_SETS 16
#define LOBE_MAX_ITEMS 64
#define LOBE_SH_COEFFS 16

typedef enum {
    LOBE_OK = 0,
    LOBE_ERR_ARG = -1,      /* invalid argument; nothing was enqueued */
    LOBE_ERR_CAPACITY = -2, /* more (Gaussian, tile) pairs than the bins' capacity */
    LOBE_ERR_CUDA = -3,     /* a CUDA runtime call failed; see lobe_last_error() */
    LOBE_ERR_TIMEOUT = -4,  /* a bounded device-side wait expired */
    LOBE_ERR_OOM = -5,      /* device allocation of context scratch failed */
    LOBE_ERR_STATE = -6     /* call order violated (e.g. scratch not reserved) */
} lobe_status;

typedef struct lobe_ctx lobe_ctx;

/* One set of 3D Gaussians, structure of arrays (device memory, caller-owned, read only).
 * Parameterisation (Sec. 3.2 "opacity determined by covariance and opacity"): log-scales,
 * a quaternion (w,x,y,z) that need not be normalised, an opacity logit and real SH
 * coefficients (band-major, DC first, 16 x RGB). crop_mask (nullable) is the visibility
 * crop of Sec. 3.3: a Gaussian with crop_mask[g] == 0 is culled. Every value must be finite
 * and every quaternion nonzero; other inputs give unspecified splats for those Gaussians. */
typedef struct {
    const float *means;          /* [n][3] */
    const float *log_scales;     /* [n][3] */
    const float *quats;          /* [n][4], 16-byte aligned */
    const float *opacity_logits; /* [n]    */
    const float *sh;             /* [n][16][3], 16-byte aligned */
    const uint8_t *crop_mask;    /* [n] or NULL */
    int64_t n;
} lobe_gaussians;

/* Pinhole camera (host struct). viewmat is the row-major 4x4 world->camera rigid transform
 * in OpenCV axes (x right, y down, +z forward); pixel (i,j) has centre (i+0.5, j+0.5).
 * An image may span at most 65535 tiles in each direction (LOBE_ERR_ARG beyond). */
typedef struct {
    float viewmat[16];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_plane, far_plane;
} lobe_camera;

/* Block box B^(b) of the KD partition (Sec. 3.1). A mean is inside when lo <= mu < hi on
 * every axis; +-INFINITY bounds are allowed (the partition splits only x and y). */
typedef struct {
    float lo[3];
    float hi[3];
} lobe_aabb;

/* One render item: Gaussian set index, camera index, block index (-1: unbounded box). */
typedef struct {
    int32_t set;
    int32_t camera;
    int32_t block;
} lobe_item;

/* Host description of a batch. Items of the same set must share the set's parameters. */
typedef struct {
    const lobe_gaussians *sets;
    int32_t n_sets;
    const lobe_camera *cameras;
    int32_t n_cameras;
    const lobe_aabb *blocks; /* may be NULL when n_blocks == 0 */
    int32_t n_blocks;
    const lobe_item *items;
    int32_t n_items;
} lobe_batch;

/* Context configuration. tile_w x tile_h must be one of 8x8, 16x8, 16x16, 32x16. */
typedef struct {
    int32_t tile_w, tile_h;
    int32_t sh_degree;  /* active SH degree, 0..3 */
    float bg[3];        /* background colour */
    int32_t recompute_T; /* 1: render_bwd re-derives the per-pixel state (T_final, n_contrib)
                            with a forward sweep instead of reading the saved one */
    int32_t px_fwd;      /* pixels per lane in render_fwd: 0 = default; 2, 4, 8 (16x8 tiles: 1, 2, 4;
                            8x8 tiles: 1, 2) */
    int32_t px_bwd;      /* pixels per lane in render_bwd: same choices */
    int32_t bin_general; /* 1: lobe_bin_sort always takes the general multi-kernel path; 0: batches of
                            at most 4096 entries and 4096 tiles (tiles x entries <= 2^20) are binned
                            by one CTA in one launch (the same result bit for bit) */
    int32_t persistent;  /* 1: lobe_render_fwd / lobe_render_bwd run as persistent kernels (one wave of
                            resident blocks) whose warps take (tile, slab) work from a device counter,
                            tiles ordered longest list first; the images are identical, the adjoint's
                            float32 sums may add in another order. Uses context scratch of 4 B a tile
                            (sized by lobe_ctx_reserve's max_tiles, or grown by an uncaptured call) */
    int32_t batch_fwd;   /* splats each warp stages from its tile's list per round in render_fwd: 0 or 32
                            (default), or 64 (two per lane: twice the prefetch depth, half the rounds;
                            needs two or more pixels a lane; lobe_render_depth always stages 32).
                            The results do not depend on it */
    int32_t batch_bwd;   /* the same for render_bwd: 0, 32 or 64 (64 needs an even pixels-per-lane count) */
    int32_t reserved;
} lobe_config;

/* Sizes implied by a batch under a config: out[0] = projected entries (sum over items of
 * the set size), out[1] = tiles (sum over items of ceil(W/tw) ceil(H/th)), out[2] = pixels. */
lobe_status lobe_batch_sizes(const lobe_config *cfg, const lobe_batch *batch, int64_t out[3]);

/* Projected splats, one entry per (item, Gaussian): entry = item_entry_offset + g, where
 * item_entry_offset is the sum of the set sizes of the preceding items.
 *   splat[e][0..11] = u, v, conic_a, conic_b, conic_c, opacity, r, g, b, depth, 0, 0
 *     (conic = inverse 2D covariance [[a,b],[b,c]]; depth = camera-space z rounded to fp32;
 *     r, g, b = max(0, SH + 0.5), a clamped channel stored as -0.0 so that lobe_project_bwd
 *     can mask its gradient by the forward's own decision)
 *   radius[e]        = ceil(3 sqrt(lambda_max)), 0 when culled (splat then undefined)
 *   tiles_touched[e] = number of tiles in the splat's tile rectangle, 0 when culled
 * splat must be 16-byte aligned. */
typedef struct {
    float *splat;           /* [entries][12] */
    int32_t *radius;        /* [entries] */
    int32_t *tiles_touched; /* [entries] */
} lobe_projected;

/* Tile bins. gauss_ids[k] is the entry id of the k-th (Gaussian, tile) pair in
 * (global tile, fp32 depth bits, entry) order; tile_start[t] is the first pair of global
 * tile t (tile_start[n_tiles] = number of pairs). Global tile t of item i is
 * item_tile_offset(i) + ty * ceil(W/tw) + tx. n_isect receives the pair count. */
typedef struct {
    int32_t *gauss_ids;  /* [capacity] */
    int32_t *tile_start; /* [n_tiles + 1] */
    int64_t *n_isect;    /* [1] */
    int64_t capacity;
} lobe_bins;

/* Rendered images. Item i occupies pixels [pix_off(i), pix_off(i) + W*H) with pix_off the
 * prefix sum of W*H. rgb is planar per item: rgb[3*pix_off + c*W*H + y*W + x].
 * n_contrib = 1 + position (within the tile list) of the last Gaussian that contributed. */
typedef struct {
    float *rgb;         /* [3 * pixels] */
    float *T_final;     /* [pixels] */
    int32_t *n_contrib; /* [pixels] */
} lobe_image;

/* Parameter gradients of one set (device, caller-owned, same shapes as lobe_gaussians).
 * sd_acc/sd_cnt (nullable) receive the selective-densification statistic of Sec. 3.3:
 * per view in which the Gaussian is visible and its mean lies in the item's block box,
 * sd_acc += |(dL/du * W/2, dL/dv * H/2)| and sd_cnt += 1 (always accumulated). */
typedef struct {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logits;
    float *sh;
    float *sd_acc;   /* [n] or NULL */
    int32_t *sd_cnt; /* [n] or NULL */
} lobe_grads;

/* Adaptive density control of the 3DGS procedure (appendix "3DGS Training"), restricted to
 * the block by selective densification (Sec. 3.3): only Gaussians with a nonzero SD count
 * (seen with their mean inside the block) may clone or split. Defaults of 3DGS in brackets. */
typedef struct {
    float grad_threshold;      /* mean SD gradient norm acc/cnt at or above which a Gaussian densifies [2e-4] */
    float max_clone_log_scale; /* largest max(log-scale) that clones rather than splits [log(0.01 * extent)] */
    float prune_logit;         /* Gaussians whose opacity logit is below this are removed [logit(0.005)] */
    int32_t n_split;           /* children of a split Gaussian, 1..4 [2] */
    float split_log_shrink;    /* subtracted from the children's log-scales [log(0.8 * n_split)] */
} lobe_densify_params;

/* Output parameter arrays (device, caller-owned), room for `capacity` Gaussians. */
typedef struct {
    float *means;          /* [capacity][3] */
    float *log_scales;     /* [capacity][3] */
    float *quats;          /* [capacity][4], 16-byte aligned */
    float *opacity_logits; /* [capacity] */
    float *sh;             /* [capacity][16][3], 16-byte aligned */
    int64_t capacity;
} lobe_params_out;

int32_t lobe_abi_version(void);

/* Number of CUDA kernels this library has enqueued since it was loaded (all contexts,
 * all threads). Kernels replayed from a captured CUDA graph are not counted again. */
int64_t lobe_kernel_launches(void);

/* Creates a context bound to `stream` (a cudaStream_t, NULL = legacy default stream) on the
 * current device. Allocates only a small device status word. */
lobe_status lobe_ctx_create(lobe_ctx **out, void *stream, const lobe_config *cfg);
lobe_status lobe_ctx_destroy(lobe_ctx *ctx);
lobe_status lobe_ctx_set_stream(lobe_ctx *ctx, void *stream);
lobe_status lobe_ctx_set_config(lobe_ctx *ctx, const lobe_config *cfg);
/* Message of the last error on this context (static storage owned by the context). */
const char *lobe_last_error(const lobe_ctx *ctx);
/* Sizes the context-owned binning scratch for up to max_entries projected entries,
 * max_isect (splat, tile) pairs and max_tiles tiles per batch (grows only). Calls of
 * lobe_bin_sort without a host count pointer never allocate and need this first; those with
 * one grow the scratch themselves. Scratch: 25 B per entry + 18 B per pair + 8 B per
 * 64x64-pixel block + about 20 KB. */
lobe_status lobe_ctx_reserve(lobe_ctx *ctx, int64_t max_entries, int64_t max_isect, int64_t max_tiles);
/* Synchronises the stream, returns and clears the latched device status. */
lobe_status lobe_get_status(lobe_ctx *ctx);
/* The same call under the name of the scope table's boundary. */
lobe_status lobe_sync_status(lobe_ctx *ctx);

/* EWA projection + SH colour + culling (near/far, 1.3x fov guard, crop mask, empty
 * rectangle) of every (item, Gaussian). Writes `out` for all entries. Follows the
 * differentiable rasterization the paper builds on (Sec. 2.1; appendix "3DGS Training"),
 * frustum culling (Sec. 3.3) and the visibility crop (Sec. 3.3). */
lobe_status lobe_project(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *out);

/* Key duplication and sort of all (Gaussian, tile) pairs of the batch, tile ranges: the
 * depth order of the blending equation (Sec. 3.2: splats composited nearest first), per tile.
 * If n_isect_host is non-NULL the call synchronises, stores the pair count there and
 * returns LOBE_ERR_CAPACITY without sorting when it exceeds bins->capacity (the caller can
 * grow the bins and call again). Otherwise an overflow is latched on the device and the
 * bins describe empty tiles. */
lobe_status lobe_bin_sort(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj,
                          const lobe_bins *bins, int64_t *n_isect_host);

/* Binning without any device allocation. The paper has no counterpart: this exists for
 * callers that must not call cudaMalloc -- code embedded in a host application that owns
 * all device memory through its own pool or budget, and real-time loops where an
 * allocation (and the device synchronisation it can imply) is not acceptable. Creating a
 * lobe_ctx allocates, so this call takes the configuration and stream directly.
 *
 * Computes exactly what lobe_bin_sort computes (same kernels, same output), but its
 * scratch is one file-scope device array of 20 MiB that every GPU loading this library
 * holds until the process exits. Limits: at most LOBE_NOALLOC_MAX_ENTRIES projected entries,
 * LOBE_NOALLOC_MAX_TILES tiles (at most 8192 blocks of 64x64 pixels) and LOBE_NOALLOC_MAX_PAIRS
 * super-tile pairs (pairs of a splat
 * and a 64x64-pixel block it overlaps; 128x64 with 32x16 tiles) per call; larger batches
 * return LOBE_ERR_CAPACITY.
 * Entries and tiles are checked before anything is enqueued; the super-tile pair count is
 * data-dependent, so the call synchronises `stream` to read it (then the bins are not
 * written). The call synchronises again at the end and stores the (splat, tile) pair count
 * in *n_isect_host (nullable); more pairs than bins->capacity gives LOBE_ERR_CAPACITY and
 * bins describing empty tiles.
 * The first call on a device (and the first after that device's context was destroyed and
 * created again) looks up the array's device address (and may load the library's kernels).
 * All calls share the one array: calls
 * whose work overlaps on the GPU (other threads, other streams) race and must be serialised
 * by the caller. At each of its two synchronisations the call also reads the status word
 * that the kernels latch in the array (cleared at the start of every call):
 * LOBE_ERR_TIMEOUT when a bounded device-side wait gave up (the bins are then undefined),
 * LOBE_ERR_CAPACITY when an overflow was latched. Other errors: LOBE_ERR_ARG (bad
 * arguments), LOBE_ERR_CUDA (a CUDA call failed). */
#define LOBE_NOALLOC_MAX_ENTRIES 262144
#define LOBE_NOALLOC_MAX_TILES 65536
#define LOBE_NOALLOC_MAX_PAIRS 524288
lobe_status lobe_bin_sort_noalloc(const lobe_config *cfg, void *stream, const lobe_batch *batch,
                                  const lobe_projected *proj, const lobe_bins *bins, int64_t *n_isect_host);

/* Front-to-back compositing of every tile of every item: the blending equation of Sec. 3.2
 * with each splat's colour in place of its depth, C = sum_i c_i alpha_i prod_{j<i}(1 - alpha_j)
 * + T bg (skip alpha < 1/255, clamp 0.99, stop at T < 1e-4: the 3DGS rules of the appendix). */
lobe_status lobe_render_fwd(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj,
                            const lobe_bins *bins, const lobe_image *image);

/* lobe_render_fwd plus the depth channel of fast camera selection (Sec. 3.2): depth[p] =
 * sum_i d_i alpha_i T_i over the pixel's composite (d_i = the splat's camera-space depth; the
 * paper's unnormalised compositing), same layout as T_final. The image is written as by
 * lobe_render_fwd. depth must not be NULL when the batch has pixels. */
lobe_status lobe_render_depth(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj,
                              const lobe_bins *bins, const lobe_image *image, float *depth);

/* Fast camera selection (Sec. 3.2): back-projects every pixel that some splat reached
 * (T_final < 1) at depth D (depth[p], divided by 1 - T_final when normalize != 0) through its
 * item's pinhole, p_c = ((x + 0.5 - cx) D / fx, (y + 0.5 - cy) D / fy, D), p_w = R^T (p_c - t),
 * and counts the points inside each box (lo <= p_w < hi per axis): counts[item * n_blocks + b]
 * and n_points[item] (device, overwritten). The visibility ratio of the paper is
 * V(item, b) = counts / n_points; a camera is assigned to a block when V >= tau (0.1).
 * n_blocks <= 64. Items' own blocks are ignored; any Gaussian set may be referenced. */
lobe_status lobe_fcs_coverage(lobe_ctx *ctx, const lobe_batch *batch, const lobe_image *image, const float *depth,
                              const lobe_aabb *blocks, int32_t n_blocks, int32_t normalize, uint32_t *counts,
                              uint32_t *n_points);

/* Camera assignment of fast camera selection (Sec. 3.2, the visibility ratio and its threshold
 * tau): V[c][b] = counts[c][b] / n_points[c] (0 when the camera has no point) and assign[c][b]
 * = (V >= tau), for n_items cameras and n_blocks blocks; the paper uses tau = 0.1. HOST arrays
 * (the counts of lobe_fcs_coverage copied back), row-major [n_items][n_blocks]; plain host
 * code, no device work. LOBE_ERR_ARG on a null array or negative size. */
lobe_status lobe_fcs_select(const uint32_t *counts, const uint32_t *n_points, int32_t n_items, int32_t n_blocks,
                            double tau, double *V, uint8_t *assign);

/* Selective densification (Sec. 3.3) with 3DGS adaptive density control: classifies every
 * Gaussian of `set` (prune / clone / split / keep, see lobe_densify_params) from its SD
 * statistic sd_acc / sd_cnt and writes the resulting set to `out`, in source order (a kept
 * Gaussian once, a clone twice, a split one as n_split children), and source[o] = the index
 * of output o's source Gaussian (nullable). normals[g][k][3] (device) are the caller's
 * standard normal draws for child k of Gaussian g (read only for split Gaussians). Child k's
 * mean is mu + R(q) (exp(log_s) * normals[g][k]). Synchronises; the output count is stored in
 * *n_out_host (non-NULL); LOBE_ERR_CAPACITY (nothing written) when it exceeds out->capacity. */
lobe_status lobe_densify(lobe_ctx *ctx, const lobe_gaussians *set, const float *sd_acc, const int32_t *sd_cnt,
                         const float *normals, const lobe_densify_params *prm, const lobe_params_out *out,
                         int32_t *source, int64_t *n_out_host);

/* Adjoint of lobe_render_fwd (the reverse-order derivative of the blending equation of
 * Sec. 3.2, as the 3DGS training of the appendix back-propagates it). dL_drgb has the layout
 * of image->rgb. Reads image->T_final
 * and image->n_contrib unless the context has recompute_T set (then only dL_drgb).
 * Overwrites grad2d[entries][12] = dL/d(u, v, conic_a, conic_b, conic_c, opacity, r, g, b)
 * followed by three zeros. grad2d must be 16-byte aligned. */
lobe_status lobe_render_bwd(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj,
                            const lobe_bins *bins, const lobe_image *image, const float *dL_drgb,
                            float *grad2d);

/* Adjoint of lobe_project (chain rule of the projection of Sec. 2.1 / appendix "3DGS
 * Training"), with the SD statistic of Sec. 3.3: chain rule from grad2d to the raw parameters of every set,
 * summed over the set's items. proj must be the output of lobe_project for this batch (the
 * colour clamp is read from the sign of the stored colour). grads[s] belongs to batch->sets[s]. accumulate = 0
 * overwrites the parameter gradients, 1 adds to them; sd_acc/sd_cnt always accumulate. */
lobe_status lobe_project_bwd(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj,
                             const float *grad2d, const lobe_grads *grads, int32_t accumulate);

/* Self-test of the bounded device-side waits (failure detection without a GPU fault): one
 * warp waits, on the ctx stream, for a look-back word that nothing publishes; after the wait
 * limit (a few seconds of polling) it latches the timeout status and returns. The next
 * lobe_get_status returns LOBE_ERR_TIMEOUT (and clears it); the context stays usable. Returns
 * LOBE_OK once the kernel is enqueued. */
lobe_status lobe_selftest_wait(lobe_ctx *ctx);

/* Mutable SoA arrays of one Gaussian set (device, caller-owned), in the shapes of
 * lobe_gaussians: means [n][3], log_scales [n][3], quats [n][4], opacity_logits [n],
 * sh [n][16][3]. Every pointer 16-byte aligned. */
typedef struct {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logits;
    float *sh;
} lobe_param_arrays;

/* Adam (Kingma and Ba, Algorithm 1), the optimizer of the 3DGS procedure that the per-block
 * fine-training follows (appendix "3DGS Training"). Per element, with t = step:
 *   m <- beta1 m + (1 - beta1) g,  v <- beta2 v + (1 - beta2) g^2,
 *   p <- p - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps),
 * computed in float32 (the bias corrections in double on the host). Learning rates per
 * group; sh_dc is the degree-0 band sh[g][0][0..2], sh_rest the other 45 floats. 3DGS values
 * in brackets. */
typedef struct {
    float lr_means;       /* [1.6e-4 * scene extent, decayed] */
    float lr_log_scales;  /* [5e-3] */
    float lr_quats;       /* [1e-3] */
    float lr_opacity;     /* [5e-2] */
    float lr_sh_dc;       /* [2.5e-3] */
    float lr_sh_rest;     /* [2.5e-3 / 20] */
    double beta1, beta2;  /* [0.9, 0.999]; double, so that 1 - beta is exact to float32 rounding */
    float eps;            /* [1e-15] */
    int64_t step;         /* t >= 1: the index of this update (the caller counts) */
} lobe_adam_params;

/* Parameters (updated in place) and the two moment buffers of one set, all in the same
 * layout; moments start at zero. */
typedef struct {
    lobe_param_arrays param;
    lobe_param_arrays exp_avg;    /* m */
    lobe_param_arrays exp_avg_sq; /* v */
} lobe_adam_state;

/* One Adam update of a set of n Gaussians from the gradients `grad` (device, read only).
 * rows (device uint8 [n], nullable): when given, only Gaussians with rows[g] != 0 change,
 * parameters and moments alike (the sparse Adam of coarse training, appendix "3DGS
 * Training"); NULL updates every Gaussian (standard Adam). Asynchronous on the ctx stream.
 * n is at most 357,564,416 (LOBE_ERR_ARG beyond). */
lobe_status lobe_adam(lobe_ctx *ctx, int64_t n, const lobe_adam_state *state, const lobe_param_arrays *grad,
                      const uint8_t *rows, const lobe_adam_params *prm);

/* lobe_project_bwd fused with the Adam update: the adjoint of the batch (summed over each
 * set's items, as lobe_project_bwd with accumulate = 0) is applied to states[s] with the
 * hyper-parameters prm[s] (one of each per set; states[s].param must be the arrays of
 * batch->sets[s]) without being written out. sparse = 1
 * changes only the Gaussians some item of the batch sees (sparse Adam); sparse = 0 applies
 * standard Adam to every Gaussian of every set (zero gradient for the unseen ones). sd
 * (nullable; one per set, only sd_acc / sd_cnt read) receives the selective-densification
 * statistic as in lobe_project_bwd. Asynchronous on the ctx stream. */
lobe_status lobe_project_bwd_adam(lobe_ctx *ctx, const lobe_batch *batch, const lobe_projected *proj,
                                  const float *grad2d, const lobe_grads *sd, const lobe_adam_state *states,
                                  const lobe_adam_params *prm, int32_t sparse);

/* Visibility cropping (Sec. 3.3): for every set, mask[s][g] |= 1 when Gaussian g is visible
 * (passes the culling rules, crop mask ignored) from at least one item of that set.
 * masks[s] are device pointers (uint8 [n]); they are OR-ed into, not cleared. */
lobe_status lobe_visibility_crop(lobe_ctx *ctx, const lobe_batch *batch, uint8_t *const *masks);

/* Load-balanced KD-tree partition with cutline refinement (Alg. 1, Sec. 3.1). Host code, no
 * device work of its own. The tree grows best first on the workload L(B) = |C(B)|, the number
 * of cameras assigned to a box (largest first; the earliest created among equals); a node is
 * cut along the longer of the x / y extents of the coarse centres inside it (centers: HOST
 * [n][3], doubles), at the q-quantile of those centres' coordinates (linear interpolation
 * between order statistics at (n - 1) q), q starting at 0.5 and, for `steps` rounds, moved by
 * bisection toward the lighter child within [q_lo, q_hi]; the children of the last evaluated cut
 * are kept. A child's cameras are its parent's whose visibility ratio V (Sec. 3.2) for the
 * child box reaches tau. Boxes are half-open, lo <= p < hi, and may be infinite.
 * `ratios(user, boxes, n_boxes, V)` must write V[c * n_boxes + b] for every camera c < n_cams
 * and return 0 (nonzero aborts with LOBE_ERR_ARG); on the GPU it is one lobe_fcs_coverage pass
 * over the cameras' depth maps. Outputs (host): leaves[n_blocks] in creation order and
 * leaf_cams[n_blocks][n_cams] (1 = camera assigned). The paper's values: tau = 0.1, q in [0.1,
 * 0.9], 3 rounds. */
typedef struct {
    double lo[3];
    double hi[3];
} lobe_box_d;
typedef int32_t (*lobe_ratio_fn)(void *user, const lobe_box_d *boxes, int32_t n_boxes, double *V);
typedef struct {
    int32_t n_blocks;  /* leaves to grow, >= 1 */
    double tau;        /* camera assignment threshold on V [0.1] */
    double q_lo, q_hi; /* bounds of the cut percentile [0.1, 0.9] */
    int32_t steps;     /* refinement rounds, >= 1 [3] */
} lobe_kd_params;
lobe_status lobe_kd_partition(const double *centers, int64_t n, const lobe_box_d *root, int32_t n_cams,
                              lobe_ratio_fn ratios, void *user, const lobe_kd_params *prm, lobe_box_d *leaves,
                              uint8_t *leaf_cams);

/* Throughput probe of one instruction kind (a measurement helper, not part of the method):
 * `blocks` blocks of 256 threads, each thread running eight independent chains of `iters`
 * steps of kind 0 = scalar fma.rn.f32 (2 FLOP), 1 = packed fma.rn.f32x2 (4 FLOP), 2 =
 * ex2.approx.f32 (1 op), asynchronously on `stream`. Per launch: blocks * 256 * 8 * iters
 * steps. sink (device, >= 256 floats) is written only in an impossible case. The compositing
 * kernels' rooflines are taken against the rates these reach. */
lobe_status lobe_peak_probe(void *stream, int32_t kind, int32_t blocks, int32_t iters, float *sink);

#ifdef __cplusplus
}
#endif
#endif /* LOBE_H */
