// render.cu -- per-tile front-to-back compositing (forward) and its adjoint.
//
// Forward (the blending equation of Sec. 3.2 with colour c_i in place of depth d_i):
//   C = sum_i c_i alpha_i T_i + T_N bg,  T_i = prod_{j<i} (1 - alpha_j),
//   alpha_i = min(0.99, o_i exp(-sigma_i)), sigma = 0.5 (a dx^2 + c dy^2) + b dx dy;
//   a splat is skipped when sigma < 0 or alpha < 1/255; the walk stops, before adding, at the
//   first splat with T (1 - alpha) < 1e-4.
//
// Adjoint, walked back to front from each pixel's last contributor with the same alpha
// decisions as the forward: with B_i the colour seen behind splat i (B starts as the
// background) and T_i the transmittance in front of it (recovered as T_{i+1} / (1 - alpha_i)
// from T_final),
//   dL/dc_i     = alpha_i T_i dL/dC
//   dL/dalpha_i = T_i (c_i - B_i) . dL/dC,      B_{i-1} = alpha_i c_i + (1 - alpha_i) B_i.
// B is accumulated from the back, so it keeps relative precision even deep in a long list
// (a front-to-back form C - sum c_j w_j loses it to cancellation). The per-pixel state it
// needs, T_final and the stop position, is either read from the forward's outputs ("store")
// or re-derived by a forward sweep inside the kernel ("recompute").
//
// Work decomposition (B300): one warp walks one slab of a tile -- 32 lanes x PX pixels,
// each lane owning PX pixels of one column -- through the tile's list in batches of 32 (or
// 64) splats staged in warp-private shared memory (the next batch is prefetched into
// registers while the current one is composited). Per splat a lane loads the splat once and
// applies it to its PX pixels, sharing the column terms of the exponent. The adjoint sums
// each splat's 9 gradient values over the lane's pixels in registers, then over the warp --
// through rows of a shared-memory slot summed column by column (the paired kernel), or a
// reduce-scatter butterfly of shuffles (one pixel a lane) -- so that one update per splat and
// warp (up to 256 pixels) reaches global memory instead of one per pixel; splats that only a
// few lanes reach skip the warp sum and those lanes add their own values. Warps need no block
// barriers.
#include <map>
#include <mutex>

#include "lobe_internal.cuh"

namespace lobe {

template <int TW, int TH, int PX>
struct Slab {
    static constexpr int ROWG = 32 / TW;     // lane rows per warp
    static constexpr int WROWS = ROWG * PX;  // tile rows per warp
    static constexpr int WARPS = TH / WROWS;
    static_assert(32 % TW == 0 && WARPS * WROWS == TH, "tile shape / pixels per lane mismatch");
};

// Exponent of one (pixel, splat) pair in base 2, with the column terms shared across a lane's
// pixels: p2 = A dx^2 + dy (B dx + C dy) with A = -0.5 a log2e, B = -b log2e, C = -0.5 c log2e.
// Forward and both adjoint sweeps call exactly this code, so their alpha decisions match.
struct Column {
    float dx, a2, b1;
};

__device__ __forceinline__ Column column_terms(float u, float A, float B, float pxc)
{
    Column c;
    c.dx = __fsub_rn(u, pxc);
    c.a2 = __fmul_rn(__fmul_rn(A, c.dx), c.dx);
    c.b1 = __fmul_rn(B, c.dx);
    return c;
}

struct PairEval {
    float dy, G, alpha;
    bool use, clamped;
};

// The skip rules are tested on the exponent before it is exponentiated: sigma >= 0 is
// p2 <= 0, and alpha = min(0.99, o 2^p2) >= 1/255 is p2 >= pmin = -log2(255 o) (the clamp
// sits above 1/255), so a skipped pair costs no exponential.
__device__ __forceinline__ PairEval pair_eval(const Column &cl, float v, float C, float o, float pmin, float pyc)
{
    PairEval r;
    r.dy = __fsub_rn(v, pyc);
    const float p2 = __fmaf_rn(r.dy, __fmaf_rn(C, r.dy, cl.b1), cl.a2);
    r.use = (p2 <= 0.0f) && (p2 >= pmin);
    r.G = 0.0f;
    r.alpha = 0.0f;
    r.clamped = false;
    if (r.use) {
        r.G = ex2(p2);
        const float araw = __fmul_rn(o, r.G);
        r.clamped = araw >= ALPHA_MAX;
        r.alpha = fminf(ALPHA_MAX, araw);
    }
    return r;
}

// Staged splat: s0 = (u, v, A, B), s1 = (C, opacity, r, g), s2 = (b, pmin).
struct Staged {
    float4 s0, s1;
    float2 s2;
    float dep;  // camera-space depth (the depth channel of fast camera selection)
    int id;
};

// Pixel-centre extent of the slab a warp composites.
struct SlabBox {
    float xa, xb, ya, yb;
};

// Conservative reachability of the alpha >= 1/255 test from the slab: false only when every
// pixel centre of the slab fails it, so a splat for which this is false changes nothing there
// and the warp skips it as a whole. The largest base-2 exponent p2 = A dx^2 + B dx dy + C dy^2
// (a concave quadratic, A, C < 0) over the box is 0 when the mean is inside it, else it is
// attained on the edge(s) facing the mean, each a 1D concave maximum clamped to the edge. The
// margin covers float32 rounding of p2 at any pixel of the box (a few ulps of the largest
// term sum S there); the clamp at 0.99 sits above 1/255 and does not enter.
__device__ __forceinline__ bool slab_reachable(const SlabBox &bx, float u, float v, float A, float B, float C,
                                               float pmin)
{
    if (!(pmin <= 0.0f)) return false;  // opacity below 1/255: no pixel passes
    const float dxa = bx.xa - u, dxb = bx.xb - u, dya = bx.ya - v, dyb = bx.yb - v;
    const bool in_x = dxa <= 0.0f && dxb >= 0.0f, in_y = dya <= 0.0f && dyb >= 0.0f;
    if (in_x && in_y) return true;
    float best = -INFINITY;
    if (!in_x) {  // vertical edge facing the mean
        const float dx = dxa > 0.0f ? dxa : dxb;
        const float dy = fminf(fmaxf(__fdividef(-B * dx, 2.0f * C), dya), dyb);
        best = fmaxf(best, A * dx * dx + B * dx * dy + C * dy * dy);
    }
    if (!in_y) {  // horizontal edge facing the mean
        const float dy = dya > 0.0f ? dya : dyb;
        const float dx = fminf(fmaxf(__fdividef(-B * dy, 2.0f * A), dxa), dxb);
        best = fmaxf(best, A * dx * dx + B * dx * dy + C * dy * dy);
    }
    const float DX = fmaxf(fabsf(dxa), fabsf(dxb)), DY = fmaxf(fabsf(dya), fabsf(dyb));
    const float S = fabsf(A) * DX * DX + fabsf(B) * DX * DY + fabsf(C) * DY * DY;
    return best + (2e-6f * S + 1e-6f) >= pmin;
}

// Loads list position k (if k < end) into s and tests it against the warp's slab.
__device__ __forceinline__ void fetch(const float4 *__restrict__ splat, const int *__restrict__ ids, int k, int end,
                                      const SlabBox &bx, Staged &s, bool &hit)
{
    hit = false;
    if (k < end) {
        const int e = ids[k];
        const float4 a = splat[3 * e], b = splat[3 * e + 1];
        s.s0 = make_float4(a.x, a.y, -0.5f * LOG2E * a.z, -LOG2E * a.w);
        s.s1 = make_float4(-0.5f * LOG2E * b.x, b.y, b.z, b.w);
        const float4 c = splat[3 * e + 2];
        s.s2 = make_float2(c.x, -log2f(255.0f * b.y));
        s.dep = c.y;
        s.id = e;
        hit = slab_reachable(bx, s.s0.x, s.s0.y, s.s0.z, s.s0.w, s.s1.x, s.s2.y);
    }
}

// Packed float32x2 arithmetic (add/sub/mul/fma .f32x2: one instruction for two values, each
// half rounded exactly like the scalar operation).
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float sum2(f2 v)
{
    float a, b;
    upk(v, a, b);
    return a + b;
}

// A warp's staged batch: 32 NB splats of its tile's list (NB = 1 or 2: each lane fetches NB
// splats a round; 2 doubles the prefetch depth and halves the rounds of long sparse lists).
template <int NB = 1>
struct WarpStageN {
    float4 s0[32 * NB];
    float4 s1[32 * NB];
    float2 s2[32 * NB];
    int id[32 * NB];
    float dep[32 * NB];
};
using WarpStage = WarpStageN<1>;

// Front-to-back walk of [start, end) for a lane's PX pixels (forward, and the first sweep
// of the recompute adjoint). live[k] must be false for pixels outside the image. With DEPTH,
// D[k] also accumulates sum_i d_i alpha_i T_i (the depth compositing of fast camera selection,
// Sec. 3.2: the blending equation with each splat's camera-space depth in place of colour).
template <int PX, bool DEPTH = false, int NB = 1>
__device__ __forceinline__ void forward_sweep(const float4 *__restrict__ splat, const int *__restrict__ ids, int start,
                                              int end, const SlabBox &bx, float pxc, const float (&pyc)[PX],
                                              bool (&live)[PX], float (&T)[PX], float (&C0)[PX], float (&C1)[PX],
                                              float (&C2)[PX], int (&last)[PX], WarpStageN<NB> &st, float *D = nullptr)
{
    const int lane = threadIdx.x & 31;
    Staged nx[NB];
    bool nh[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) fetch(splat, ids, start + 32 * b + lane, end, bx, nx[b], nh[b]);
    for (int base = start; base < end; base += 32 * NB) {
        bool any = false;
#pragma unroll
        for (int k = 0; k < PX; ++k) any |= live[k];
        if (!__any_sync(0xffffffffu, any)) break;
        unsigned hitb[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            st.s0[32 * b + lane] = nx[b].s0;
            st.s1[32 * b + lane] = nx[b].s1;
            st.s2[32 * b + lane] = nx[b].s2;
            if (DEPTH) st.dep[32 * b + lane] = nx[b].dep;
            hitb[b] = __ballot_sync(0xffffffffu, nh[b]);  // splats of the batch that can reach the slab
        }
        __syncwarp();
#pragma unroll
        for (int b = 0; b < NB; ++b) fetch(splat, ids, base + 32 * (NB + b) + lane, end, bx, nx[b], nh[b]);
#pragma unroll
        for (int b = 0; b < NB; ++b)
        for (unsigned hits = hitb[b]; hits;) {
            const int j = 32 * b + __ffs(hits) - 1;  // stage slot = list position - base
            hits &= hits - 1;
            const float4 q0 = st.s0[j], q1 = st.s1[j];
            const float cb = st.s2[j].x, pmin = st.s2[j].y;
            const float dj = DEPTH ? st.dep[j] : 0.0f;
            const Column cl = column_terms(q0.x, q0.z, q0.w, pxc);
            // the exponent of every pixel: in pairs (packed) when PX is even -- the same rounding
            // as pair_eval and as the paired adjoint
            float pv[PX];
            if constexpr (PX % 2 == 0) {
                const f2 v2 = pk(q0.y, q0.y), Cq = pk(q1.x, q1.x), a2 = pk(cl.a2, cl.a2), b1 = pk(cl.b1, cl.b1);
#pragma unroll
                for (int i = 0; i < PX / 2; ++i) {
                    const f2 dy2 = sub2(v2, pk(pyc[2 * i], pyc[2 * i + 1]));
                    upk(fma2(dy2, fma2(Cq, dy2, b1), a2), pv[2 * i], pv[2 * i + 1]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < PX; ++k) {
                    const float dy = __fsub_rn(q0.y, pyc[k]);
                    pv[k] = __fmaf_rn(dy, __fmaf_rn(q1.x, dy, cl.b1), cl.a2);
                }
            }
#pragma unroll
            for (int k = 0; k < PX; ++k) {
                if constexpr (PX == 1) {
                    if (!live[k]) continue;
                    const float p2 = pv[k];
                    if (!(p2 <= 0.0f && p2 >= pmin)) continue;  // sigma < 0 or alpha < 1/255: skipped
                    const float alpha = fminf(ALPHA_MAX, __fmul_rn(q1.y, ex2(p2)));
                    const float Tn = next_T(T[k], alpha);
                    if (Tn < T_MIN) {
                        live[k] = false;
                        continue;
                    }
                    const float w = alpha * T[k];
                    C0[k] += q1.z * w;
                    C1[k] += q1.w * w;
                    C2[k] += cb * w;
                    if (DEPTH) D[k] += dj * w;
                    T[k] = Tn;
                    last[k] = base - start + j + 1;
                } else if constexpr (PX % 2 == 0) {
                    // several pixels a lane, in pairs: branch-free, so the pixels' chains
                    // interleave, with the transmittance, the weights and the sums in packed
                    // f32x2 arithmetic (each half rounded as the scalar step). A pixel that
                    // skips or stops gets weight 0 and keeps T and last exactly
                    if (k % 2) continue;
                    const float pa = pv[k], pb = pv[k + 1];
                    const bool ua = live[k] && pa <= 0.0f && pa >= pmin, ub = live[k + 1] && pb <= 0.0f && pb >= pmin;
                    float ra, rb;
                    upk(mul2(pk(q1.y, q1.y), pk(ua ? ex2(pa) : 0.0f, ub ? ex2(pb) : 0.0f)), ra, rb);
                    const float aa = fminf(ALPHA_MAX, ra), ab = fminf(ALPHA_MAX, rb);
                    const f2 T2 = pk(T[k], T[k + 1]);
                    float ta, tb;
                    upk(mul2(T2, sub2(pk(1.0f, 1.0f), pk(aa, ab))), ta, tb);  // next_T of both pixels
                    const bool sa = ua && ta < T_MIN, sb = ub && tb < T_MIN;
                    if (!__any_sync(0xffffffffu, sa || sb)) {
                        // no pixel of the warp stops here (the common case: a pixel stops once):
                        // an unused pixel has alpha 0, so T (1 - 0) = T and its weight is 0 exactly
                        const f2 w2 = mul2(pk(aa, ab), T2);
                        upk(fma2(pk(q1.z, q1.z), w2, pk(C0[k], C0[k + 1])), C0[k], C0[k + 1]);
                        upk(fma2(pk(q1.w, q1.w), w2, pk(C1[k], C1[k + 1])), C1[k], C1[k + 1]);
                        upk(fma2(pk(cb, cb), w2, pk(C2[k], C2[k + 1])), C2[k], C2[k + 1]);
                        if (DEPTH) upk(fma2(pk(dj, dj), w2, pk(D[k], D[k + 1])), D[k], D[k + 1]);
                        T[k] = ta;
                        T[k + 1] = tb;
                        last[k] = ua ? base - start + j + 1 : last[k];
                        last[k + 1] = ub ? base - start + j + 1 : last[k + 1];
                        continue;
                    }
                    const bool wa = ua && !sa, wb = ub && !sb;
                    live[k] = live[k] && !sa;
                    live[k + 1] = live[k + 1] && !sb;
                    const f2 w2 = mul2(pk(wa ? aa : 0.0f, wb ? ab : 0.0f), T2);
                    upk(fma2(pk(q1.z, q1.z), w2, pk(C0[k], C0[k + 1])), C0[k], C0[k + 1]);
                    upk(fma2(pk(q1.w, q1.w), w2, pk(C1[k], C1[k + 1])), C1[k], C1[k + 1]);
                    upk(fma2(pk(cb, cb), w2, pk(C2[k], C2[k + 1])), C2[k], C2[k + 1]);
                    if (DEPTH) upk(fma2(pk(dj, dj), w2, pk(D[k], D[k + 1])), D[k], D[k + 1]);
                    T[k] = wa ? ta : T[k];
                    T[k + 1] = wb ? tb : T[k + 1];
                    last[k] = wa ? base - start + j + 1 : last[k];
                    last[k + 1] = wb ? base - start + j + 1 : last[k + 1];
                } else {
                    // several pixels a lane: branch-free, so the pixels' chains interleave; a
                    // pixel that skips or stops gets weight 0 and keeps T and last exactly
                    const float p2 = pv[k];
                    const bool use = live[k] && p2 <= 0.0f && p2 >= pmin;
                    const float alpha = use ? fminf(ALPHA_MAX, __fmul_rn(q1.y, ex2(p2))) : 0.0f;
                    const float Tn = next_T(T[k], alpha);
                    const bool stop = use && Tn < T_MIN;
                    const bool upd = use && !stop;
                    live[k] = live[k] && !stop;
                    const float w = upd ? alpha * T[k] : 0.0f;
                    C0[k] += q1.z * w;
                    C1[k] += q1.w * w;
                    C2[k] += cb * w;
                    if (DEPTH) D[k] += dj * w;
                    T[k] = upd ? Tn : T[k];
                    last[k] = upd ? base - start + j + 1 : last[k];
                }
            }
        }
        __syncwarp();
    }
}

// Pixel-centre box of the slab of warp `warp` in tile (tx, ty).
template <int TW, int TH, int PX>
__device__ __forceinline__ SlabBox slab_box(int tx, int ty, int warp)
{
    using G = Slab<TW, TH, PX>;
    SlabBox b;
    b.xa = (float)(tx * TW) + 0.5f;
    b.xb = b.xa + (float)(TW - 1);
    b.ya = (float)(ty * TH + warp * G::WROWS) + 0.5f;
    b.yb = b.ya + (float)(G::WROWS - 1);
    return b;
}

// Work distribution of the compositing kernels. Plain: one block per tile, warp w of the block
// takes slab w. Persistent (order != nullptr): a grid of resident blocks whose warps pull
// (tile, slab) items from a device counter, tiles in the order given (longest list first), so
// the longest tiles start first and no block waits for a straggler of the last wave.
struct WorkCursor {
    const int *order;
    unsigned *work;
    unsigned n_work;
    int warps;
    bool first;
    __device__ __forceinline__ bool next(int &t, int &slab, int pw)
    {
        if (!order) {
            if (!first) return false;
            first = false;
            t = blockIdx.x;
            slab = pw;
            return true;
        }
        unsigned k = 0;
        if ((threadIdx.x & 31) == 0) k = atomicAdd(work, 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= n_work) return false;
        t = order[k / warps];
        slab = (int)(k % warps);
        return true;
    }
};

#ifndef LOBE_FWD_REGS
#define LOBE_FWD_REGS 0  // 0: no cap beyond the compiler's choice
#endif
// Resident blocks an SM must fit for a register cap of `regs` a thread (0: no cap), at most
// the 32 blocks an SM holds.
constexpr int min_blocks_for(int regs, int warps)
{
    return regs > 0 ? (65536 / (regs * 32 * warps) < 32 ? 65536 / (regs * 32 * warps) : 32) : 1;
}

#if LOBE_FWD_REGS > 0
#define LOBE_FWD_BOUNDS(W) __launch_bounds__(32 * (W), min_blocks_for(LOBE_FWD_REGS, (W)))
#else
#define LOBE_FWD_BOUNDS(W) __launch_bounds__(32 * (W))
#endif
template <int TW, int TH, int PX, bool DEPTH, bool PERSIST, int NB = 1>
__global__ void LOBE_FWD_BOUNDS((Slab<TW, TH, PX>::WARPS))
    k_render_fwd(const __grid_constant__ BatchParams P, const float4 *__restrict__ splat,
                 const int *__restrict__ tile_start, const int *__restrict__ ids, float *__restrict__ rgb,
                 float *__restrict__ Tout, int *__restrict__ ncout, float *__restrict__ depth,
                 const int *__restrict__ order, unsigned *__restrict__ work)
{
    pdl_wait();
    using G = Slab<TW, TH, PX>;
    __shared__ WarpStageN<NB> stage[G::WARPS];
    const int lane = threadIdx.x & 31, pw = threadIdx.x >> 5;
    WorkCursor wc{order, work, (unsigned)P.n_tiles * (unsigned)G::WARPS, G::WARPS, true};
    auto tile_body = [&](const int t, const int warp) {
        const ItemParams &I = P.item[item_of_tile(P, t)];
        const int lt = t - I.tile_off, tx = lt % I.gx, ty = lt / I.gx;
        const int px = tx * TW + lane % TW;
        const int py0 = ty * TH + warp * G::WROWS + (lane / TW) * PX;
        const float pxc = (float)px + 0.5f;
        float pyc[PX], T[PX], C0[PX], C1[PX], C2[PX], D[PX];
        int last[PX];
        bool live[PX], inside[PX];
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            pyc[k] = (float)(py0 + k) + 0.5f;
            inside[k] = px < I.W && py0 + k < I.H;
            live[k] = inside[k];
            T[k] = 1.0f;
            C0[k] = C1[k] = C2[k] = D[k] = 0.0f;
            last[k] = 0;
        }
        forward_sweep<PX, DEPTH, NB>(splat, ids, tile_start[t], tile_start[t + 1], slab_box<TW, TH, PX>(tx, ty, warp), pxc, pyc,
                                 live, T, C0, C1, C2, last, stage[pw], D);
        const long long HW = (long long)I.W * I.H;
        float *out = rgb + 3 * I.pix_off;
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            if (!inside[k]) continue;
            const long long p = (long long)(py0 + k) * I.W + px;
            out[p] = C0[k] + T[k] * P.bg[0];
            out[HW + p] = C1[k] + T[k] * P.bg[1];
            out[2 * HW + p] = C2[k] + T[k] * P.bg[2];
            Tout[I.pix_off + p] = T[k];
            ncout[I.pix_off + p] = last[k];
            if (DEPTH) depth[I.pix_off + p] = D[k];
        }
        __syncwarp();
    };
    if constexpr (PERSIST) {
        int t, warp;
        while (wc.next(t, warp, pw)) tile_body(t, warp);
    } else {
        tile_body((int)blockIdx.x, pw);
    }
}

// Sum over the warp of nine per-lane values, reduce-scattered (a butterfly that halves the set
// of values each lane carries at every step: 5 + 3 + 2 + 1 + 1 shuffles instead of 9 x 5).
// Returns the total of value `idx` in 18 lanes (idx in [0, 9), one writer per index: lanes with
// bit 0 set get idx = -1) and idx = -1 elsewhere. Lane bits 4, 3, 2, 1 pick, in turn, which
// half of the remaining values a lane keeps.
__device__ __forceinline__ float warp_reduce9(const float (&v)[9], int &idx)
{
    const int lane = threadIdx.x & 31;
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4, b2 = lane & 2;
    float w[5];  // values {0..4} (bit 4 clear) or {5..8} (bit 4 set)
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float lo = v[i], hi = i < 4 ? v[5 + i] : 0.0f;
        w[i] = (b16 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b16 ? lo : hi, 16);
    }
    float x[3];  // w{0,1,2} or w{3,4}
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float a = w[i], b = i < 2 ? w[3 + i] : 0.0f;
        x[i] = (b8 ? b : a) + __shfl_xor_sync(0xffffffffu, b8 ? a : b, 8);
    }
    float y[2];  // x{0,1} or x{2}
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float a = x[i], b = i < 1 ? x[2] : 0.0f;
        y[i] = (b4 ? b : a) + __shfl_xor_sync(0xffffffffu, b4 ? a : b, 4);
    }
    float z = (b2 ? y[1] : y[0]) + __shfl_xor_sync(0xffffffffu, b2 ? y[0] : y[1], 2);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    const int q = b4 ? (b2 ? -1 : 2) : (b2 ? 1 : 0);   // position in x
    const int p = q < 0 ? -1 : (b8 ? (q <= 1 ? 3 + q : -1) : q);  // position in w
    idx = (p < 0 || (lane & 1)) ? -1 : (b16 ? (p <= 3 ? 5 + p : -1) : p);
    return z;
}

template <int TW, int TH, int PX, bool RECOMPUTE, bool PERSIST>
__global__ void __launch_bounds__(32 * Slab<TW, TH, PX>::WARPS)
    k_render_bwd(const __grid_constant__ BatchParams P, const float4 *__restrict__ splat,
                 const int *__restrict__ tile_start, const int *__restrict__ ids, const float *__restrict__ Tfin,
                 const int *__restrict__ ncin, const float *__restrict__ dL, float *__restrict__ grad2d,
                 const int *__restrict__ order, unsigned *__restrict__ work)
{
    pdl_wait();
    using G = Slab<TW, TH, PX>;
    __shared__ WarpStage stage[G::WARPS];
    WarpStage &st = stage[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31, pw = threadIdx.x >> 5;
    WorkCursor wc{order, work, (unsigned)P.n_tiles * (unsigned)G::WARPS, G::WARPS, true};
    auto tile_body = [&](const int t, const int warp) {
        const ItemParams &I = P.item[item_of_tile(P, t)];
        const int lt = t - I.tile_off, tx = lt % I.gx, ty = lt / I.gx;
        const int px = tx * TW + lane % TW;
        const int py0 = ty * TH + warp * G::WROWS + (lane / TW) * PX;
        const float pxc = (float)px + 0.5f;
        const int start = tile_start[t], end = tile_start[t + 1];
        const SlabBox bx = slab_box<TW, TH, PX>(tx, ty, warp);
        const long long HW = (long long)I.W * I.H;
        // per pixel: dL/dC, the colour seen behind the current splat (B, background included),
        // the transmittance after it (T, starting from T_final) and the stop position
        float pyc[PX], g0[PX], g1[PX], g2[PX], B0[PX], B1[PX], B2[PX], T[PX];
        int nc[PX];
        bool inside[PX];
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            pyc[k] = (float)(py0 + k) + 0.5f;
            inside[k] = px < I.W && py0 + k < I.H;
            g0[k] = g1[k] = g2[k] = 0.0f;
            T[k] = 1.0f;
            nc[k] = 0;
            if (inside[k]) {
                const long long p = (long long)(py0 + k) * I.W + px;
                const float *d = dL + 3 * I.pix_off;
                g0[k] = d[p];
                g1[k] = d[HW + p];
                g2[k] = d[2 * HW + p];
                if (!RECOMPUTE) {
                    T[k] = Tfin[I.pix_off + p];
                    nc[k] = ncin[I.pix_off + p];
                }
            }
        }
        if (RECOMPUTE) {
            bool live[PX];
#pragma unroll
            for (int k = 0; k < PX; ++k) {
                live[k] = inside[k];
                B0[k] = B1[k] = B2[k] = 0.0f;  // colour accumulators of the sweep (unused after it)
            }
            forward_sweep<PX>(splat, ids, start, end, bx, pxc, pyc, live, T, B0, B1, B2, nc, st);
        }
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            B0[k] = P.bg[0];
            B1[k] = P.bg[1];
            B2[k] = P.bg[2];
        }
        int m = 0;
#pragma unroll
        for (int k = 0; k < PX; ++k) m = max(m, nc[k]);
        m = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
        const int stop = min(start + m, end);

        // walk the list back to front in batches of 32, prefetching the batch below
        int top = stop, base = max(start, stop - 32);
        Staged nx;
        bool nh;
        fetch(splat, ids, base + lane, top, bx, nx, nh);
        while (top > start) {
            st.s0[lane] = nx.s0;
            st.s1[lane] = nx.s1;
            st.s2[lane] = nx.s2;
            st.id[lane] = nx.id;
            unsigned hits = __ballot_sync(0xffffffffu, nh);
            __syncwarp();
            const int nbase = max(start, base - 32);
            fetch(splat, ids, nbase + lane, base, bx, nx, nh);
            while (hits) {  // back to front: highest position first
                const int j = 31 - __clz(hits);
                hits &= ~(1u << j);
                const float4 q0 = st.s0[j], q1 = st.s1[j];
                const float cb = st.s2[j].x, pmin = st.s2[j].y;
                const int pos = base - start + j;
                const Column cl = column_terms(q0.x, q0.z, q0.w, pxc);
                float du = 0.f, dv = 0.f, dA = 0.f, dB = 0.f, dC = 0.f, dop = 0.f, dr = 0.f, dg = 0.f, db = 0.f;
                bool any = false;
#pragma unroll
                for (int k = 0; k < PX; ++k) {
                    if (pos >= nc[k]) continue;
                    const PairEval r = pair_eval(cl, q0.y, q1.x, q1.y, pmin, pyc[k]);
                    if (!r.use) continue;
                    any = true;
                    const float Ti = __fdividef(T[k], 1.0f - r.alpha);  // transmittance in front of it
                    const float w = r.alpha * Ti;
                    dr += w * g0[k];
                    dg += w * g1[k];
                    db += w * g2[k];
                    const float dalpha = Ti * (g0[k] * (q1.z - B0[k]) + g1[k] * (q1.w - B1[k]) + g2[k] * (cb - B2[k]));
                    B0[k] = fmaf(r.alpha, q1.z - B0[k], B0[k]);
                    B1[k] = fmaf(r.alpha, q1.w - B1[k], B1[k]);
                    B2[k] = fmaf(r.alpha, cb - B2[k], B2[k]);
                    T[k] = Ti;
                    if (!r.clamped) {
                        dop += dalpha * r.G;
                        const float dp2 = dalpha * r.alpha * LN2;
                        const float dpy = dp2 * r.dy;
                        dA += dp2 * cl.dx * cl.dx;
                        dB += dpy * cl.dx;
                        dC += dpy * r.dy;
                        du += dp2 * (2.f * q0.z * cl.dx + q0.w * r.dy);
                        dv += dp2 * q0.w * cl.dx + 2.f * q1.x * dpy;
                    }
                }
                if (__any_sync(0xffffffffu, any)) {
                    const float vals[9] = {du, dv, dA, dB, dC, dop, dr, dg, db};
                    int idx;
                    const float tot = warp_reduce9(vals, idx);
                    if (idx >= 0) {
                        // back from the base-2 exponent domain: A = -0.5 log2e a, B = -log2e b, C = -0.5 log2e c
                        const float sc = (idx == 2 || idx == 4) ? -0.5f * LOG2E : (idx == 3 ? -LOG2E : 1.0f);
                        red_add_f32(grad2d + 12LL * st.id[j] + idx, sc * tot);
                    }
                }
            }
            __syncwarp();
            top = base;
            base = nbase;
        }
        __syncwarp();
    };
    if constexpr (PERSIST) {
        int t, warp;
        while (wc.next(t, warp, pw)) tile_body(t, warp);
    } else {
        tile_body((int)blockIdx.x, pw);
    }
}

// --------------------------------------------------------------------------- paired adjoint
//
// The same adjoint with a lane's pixels taken two at a time (pixel rows 2i and 2i+1 of its
// column) in packed float32x2 arithmetic (add/sub/mul/fma .f32x2: one instruction for both
// pixels, each half rounded exactly like the scalar operation). The kernels are issue-bound,
// so halving the floating-point instructions of a contributing pixel pair is what counts.
// Per-pixel decisions stay scalar and identical to the forward's (same dy, p2, ex2, o * G in
// the same rounding); a pixel of the pair that does not use the splat gets G = 0, hence
// alpha = 0, which leaves its T, B and every gradient term unchanged.

// Register cap of the paired adjoint per pixels a lane (occupancy: the kernel is latency- as
// much as issue-bound), and the lanes below which a splat skips the warp reduction. Measured on
// B300 (16 views of a 6.5M-Gaussian city): one pixel pair a lane at 64 registers runs faster
// than at the compiler's choice; two pairs ask for 104, which one-warp blocks (16x8 tiles) get
// as 96 at 5 warps a scheduler (8.52 -> 8.12 ms against 80 registers at 6 warps; 128 at 4:
// 8.87 ms); four pairs keep 128 (lower caps spill). The direct path for splats that few lanes
// use saves ~10% where splats are small, and costs where they are large (four pairs a lane are
// chosen for large ones): up to 4 lanes with two pairs (8.61 -> 8.53 ms against 8; 16 lanes:
// 12.4 ms), 8 with one. Together: the city batch's adjoint 11.1 -> 8.1 ms.
#ifdef LOBE_BWD_REGS
constexpr int bwd_regs_for(int, int = 1) { return LOBE_BWD_REGS; }
#else
// 64-splat staging rounds keep a second prefetched splat per lane: 16 more registers
constexpr int bwd_regs_for(int px, int nb = 1) { return (px >= 8 ? 128 : (px >= 4 ? 104 : 64)) + 16 * (nb - 1); }
#endif
#ifdef LOBE_BWD_DIRECT
__host__ __device__ constexpr int bwd_direct_for(int) { return LOBE_BWD_DIRECT; }
#else
__host__ __device__ constexpr int bwd_direct_for(int px) { return px >= 8 ? 0 : (px >= 4 ? 4 : 8); }
#endif
// Per-splat sums of the warp reduction, through shared memory (LOBE_BWD_SLOTS, default on):
// each lane writes its nine values for a splat into a row of the warp's next slot; after
// RED_SLOTS such splats (or at the end of the slab) lane q < 9 RED_SLOTS adds column q --
// value q % 9 of slot q / 9 over the 32 rows -- and issues one red. Rows are 12 words (16-byte
// stores of values 0-7 at 48-byte strides: no bank conflicts); value 8 of slot s sits in word
// 8 + s of the first slot's row; slots are 396 words apart, so the 27 columns of a flush fall
// in 27 distinct banks.
#ifndef LOBE_BWD_SLOTS
#define LOBE_BWD_SLOTS 1
#endif
constexpr int RED_SLOTS = 3, RED_ROW = 12, RED_SLOT = 32 * RED_ROW + 12, RED_WORDS = RED_SLOTS * RED_SLOT;
static_assert(RED_SLOT % 4 == 0 && RED_SLOT % 32 == 12, "slot stride: 16-byte aligned, 12 banks apart");

template <int TW, int TH, int PX, bool RECOMPUTE, bool PERSIST, int NB = 1>
__global__ void __launch_bounds__(32 * Slab<TW, TH, PX>::WARPS,
                                  min_blocks_for(bwd_regs_for(PX, NB), Slab<TW, TH, PX>::WARPS))
    k_render_bwd2(const __grid_constant__ BatchParams P, const float4 *__restrict__ splat,
                  const int *__restrict__ tile_start, const int *__restrict__ ids, const float *__restrict__ Tfin,
                  const int *__restrict__ ncin, const float *__restrict__ dL, float *__restrict__ grad2d,
                 const int *__restrict__ order, unsigned *__restrict__ work)
{
    pdl_wait();
    static_assert(PX % 2 == 0, "pixels are paired");
    constexpr int NP = PX / 2;
    using G = Slab<TW, TH, PX>;
    __shared__ WarpStageN<NB> stage[G::WARPS];
    WarpStageN<NB> &st = stage[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31, pw = threadIdx.x >> 5;
#if LOBE_BWD_SLOTS
    __shared__ __align__(16) float s_red[G::WARPS][RED_WORDS];
    __shared__ int s_rid[G::WARPS][RED_SLOTS];
    // this lane's column of a flush: value rv of the splat in slot rs (27 lanes), its word in a
    // row and the factor back from the base-2 exponent domain (A = -0.5 log2e a, B = -log2e b,
    // C = -0.5 log2e c)
    const int rs = lane / 9, rv = lane - 9 * (lane / 9);
    const int rcol = rv < 8 ? rs * RED_SLOT + rv : 8 + rs;
    const float rsc = (rv == 2 || rv == 4) ? -0.5f * LOG2E : (rv == 3 ? -LOG2E : 1.0f);
    int nslot = 0;  // slots filled (warp-uniform)
    // the per-splat sums of the filled slots, each over the warp's 32 rows, added to grad2d
    auto flush = [&](const int n) {
        __syncwarp();
        if (lane < 9 * n) {
            const float *c = s_red[pw] + rcol;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
            for (int r = 0; r < 32; r += 4) {
                a0 += c[RED_ROW * r];
                a1 += c[RED_ROW * (r + 1)];
                a2 += c[RED_ROW * (r + 2)];
                a3 += c[RED_ROW * (r + 3)];
            }
            red_add_f32(grad2d + 12LL * s_rid[pw][rs] + rv, rsc * ((a0 + a1) + (a2 + a3)));
        }
        __syncwarp();
    };
#endif
    WorkCursor wc{order, work, (unsigned)P.n_tiles * (unsigned)G::WARPS, G::WARPS, true};
    auto tile_body = [&](const int t, const int warp) {
        const ItemParams &I = P.item[item_of_tile(P, t)];
        const int lt = t - I.tile_off, tx = lt % I.gx, ty = lt / I.gx;
        const int px = tx * TW + lane % TW;
        const int py0 = ty * TH + warp * G::WROWS + (lane / TW) * PX;
        const float pxc = (float)px + 0.5f;
        const int start = tile_start[t], end = tile_start[t + 1];
        const SlabBox bx = slab_box<TW, TH, PX>(tx, ty, warp);
        const long long HW = (long long)I.W * I.H;
        float pyc[PX], g0[PX], g1[PX], g2[PX], T[PX];
        int nc[PX];
        bool inside[PX];
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            pyc[k] = (float)(py0 + k) + 0.5f;
            inside[k] = px < I.W && py0 + k < I.H;
            g0[k] = g1[k] = g2[k] = 0.0f;
            T[k] = 1.0f;
            nc[k] = 0;
            if (inside[k]) {
                const long long p = (long long)(py0 + k) * I.W + px;
                const float *d = dL + 3 * I.pix_off;
                g0[k] = d[p];
                g1[k] = d[HW + p];
                g2[k] = d[2 * HW + p];
                if (!RECOMPUTE) {
                    T[k] = Tfin[I.pix_off + p];
                    nc[k] = ncin[I.pix_off + p];
                }
            }
        }
        if (RECOMPUTE) {
            bool live[PX];
            float c0[PX], c1[PX], c2[PX];
#pragma unroll
            for (int k = 0; k < PX; ++k) {
                live[k] = inside[k];
                c0[k] = c1[k] = c2[k] = 0.0f;
            }
            forward_sweep<PX, false, NB>(splat, ids, start, end, bx, pxc, pyc, live, T, c0, c1, c2, nc, st);
        }
        // per pixel pair: packed row centres, dL/dC, colour behind (from the background), T
        f2 pyc2[NP], G0[NP], G1[NP], G2[NP], B0[NP], B1[NP], B2[NP], T2[NP];
        const f2 bg0 = pk(P.bg[0], P.bg[0]), bg1 = pk(P.bg[1], P.bg[1]), bg2 = pk(P.bg[2], P.bg[2]);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            pyc2[i] = pk(pyc[2 * i], pyc[2 * i + 1]);
            G0[i] = pk(g0[2 * i], g0[2 * i + 1]);
            G1[i] = pk(g1[2 * i], g1[2 * i + 1]);
            G2[i] = pk(g2[2 * i], g2[2 * i + 1]);
            B0[i] = bg0;
            B1[i] = bg1;
            B2[i] = bg2;
            T2[i] = pk(T[2 * i], T[2 * i + 1]);
        }
        int m = 0;
#pragma unroll
        for (int k = 0; k < PX; ++k) m = max(m, nc[k]);
        m = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
        const int stop = min(start + m, end);
        const f2 one2 = pk(1.0f, 1.0f);

        // rounds of 32 NB list positions [base, top), stage slot j = position - base
        int top = stop, base = max(start, stop - 32 * NB);
        Staged nx[NB];
        bool nh[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) fetch(splat, ids, base + 32 * b + lane, top, bx, nx[b], nh[b]);
        while (top > start) {
            unsigned hitb[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                st.s0[32 * b + lane] = nx[b].s0;
                st.s1[32 * b + lane] = nx[b].s1;
                st.s2[32 * b + lane] = nx[b].s2;
                st.id[32 * b + lane] = nx[b].id;
                hitb[b] = __ballot_sync(0xffffffffu, nh[b]);
            }
            __syncwarp();
            const int nbase = max(start, base - 32 * NB);
#pragma unroll
            for (int b = 0; b < NB; ++b) fetch(splat, ids, nbase + 32 * b + lane, base, bx, nx[b], nh[b]);
#pragma unroll
            for (int b = NB - 1; b >= 0; --b)
            for (unsigned hits = hitb[b]; hits;) {  // back to front: highest position first
                const int jb = 31 - __clz(hits);
                hits &= ~(1u << jb);
                const int j = 32 * b + jb;
                const float4 q0 = st.s0[j], q1 = st.s1[j];
                const float cb = st.s2[j].x, pmin = st.s2[j].y;
                const int pos = base - start + j;
                const Column cl = column_terms(q0.x, q0.z, q0.w, pxc);
                const f2 v2 = pk(q0.y, q0.y), C2 = pk(q1.x, q1.x), a2 = pk(cl.a2, cl.a2), b1 = pk(cl.b1, cl.b1);
                // per lane over its pixels: dop = sum t, S2 = sum t dy, S3 = sum t dy^2 with t = dL/dalpha G
                // below the clamp (0 past it); dL/dp2 = o ln2 t, so the exponent's gradients follow from
                // these and the lane's own dx after the loop, with the factor o ln2 applied once.
                // With several pairs the first pair's terms initialise the sums (no zeroing, no add)
                f2 S2, S3, dop, dr, dg, db;
                if constexpr (NP == 1) S2 = S3 = dop = dr = dg = db = 0;  // 0 = (+0, +0)
                bool any = false;
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    const bool ok0 = pos < nc[2 * i], ok1 = pos < nc[2 * i + 1];
                    if (NP == 1 && !(ok0 || ok1)) continue;  // several pairs: branch-free, so the pairs interleave
                    const f2 dy2 = sub2(v2, pyc2[i]);
                    const f2 p2 = fma2(dy2, fma2(C2, dy2, b1), a2);
                    float pa, pb;
                    upk(p2, pa, pb);
                    const bool u0 = ok0 && pa <= 0.0f && pa >= pmin, u1 = ok1 && pb <= 0.0f && pb >= pmin;
                    if (NP == 1 && !(u0 || u1)) continue;
                    any |= u0 || u1;  // a pair neither pixel uses has alpha = 0 and leaves everything unchanged
                    const float Ga = u0 ? ex2(pa) : 0.0f, Gb = u1 ? ex2(pb) : 0.0f;
                    float ra, rb;
                    upk(mul2(pk(q1.y, q1.y), pk(Ga, Gb)), ra, rb);  // o * G, as in the forward
                    const bool ka = ra >= ALPHA_MAX, kb = rb >= ALPHA_MAX;
                    const float aa = fminf(ALPHA_MAX, ra), ab = fminf(ALPHA_MAX, rb);
                    const f2 al = pk(aa, ab);
                    float oma, omb;
                    upk(sub2(one2, al), oma, omb);
                    const f2 Ti = mul2(T2[i], pk(__fdividef(1.0f, oma), __fdividef(1.0f, omb)));  // T in front
                    const f2 w = mul2(al, Ti);
                    const bool first = NP > 1 && i == 0;  // resolved at compile time (unrolled)
                    dr = first ? mul2(w, G0[i]) : fma2(w, G0[i], dr);
                    dg = first ? mul2(w, G1[i]) : fma2(w, G1[i], dg);
                    db = first ? mul2(w, G2[i]) : fma2(w, G2[i], db);
                    const f2 d0 = sub2(pk(q1.z, q1.z), B0[i]), d1 = sub2(pk(q1.w, q1.w), B1[i]),
                             d2 = sub2(pk(cb, cb), B2[i]);
                    const f2 da = mul2(Ti, fma2(G2[i], d2, fma2(G1[i], d1, mul2(G0[i], d0))));  // dL/dalpha
                    B0[i] = fma2(al, d0, B0[i]);
                    B1[i] = fma2(al, d1, B1[i]);
                    B2[i] = fma2(al, d2, B2[i]);
                    if (NP == 1) {
                        T2[i] = Ti;
                    } else {  // an unused pixel keeps its T exactly (the reciprocal of 1 - 0 is approximate)
                        float t0, t1, n0, n1;
                        upk(T2[i], t0, t1);
                        upk(Ti, n0, n1);
                        T2[i] = pk(u0 ? n0 : t0, u1 ? n1 : t1);
                    }
                    // past the clamp alpha no longer depends on o or the exponent: dL/do = da G and
                    // dL/dp2 = da o G ln2 (alpha = o G below the clamp)
                    const f2 t = mul2(da, pk(ka ? 0.0f : Ga, kb ? 0.0f : Gb));
                    dop = first ? t : add2(dop, t);
                    const f2 ty = mul2(t, dy2);
                    S2 = first ? ty : add2(S2, ty);
                    S3 = first ? mul2(ty, dy2) : fma2(ty, dy2, S3);
                }
                const unsigned used = __ballot_sync(0xffffffffu, any);
                if (used) {
                    // p2 = A dx^2 + B dx dy + C dy^2 with dx = u - x, dy = v - y; s1, s2, s3 = the lane's
                    // sums of dL/dp2, dL/dp2 dy, dL/dp2 dy^2
                    const float oln = q1.y * LN2, sdop = sum2(dop), dx = cl.dx;
                    const float s1 = oln * sdop, s2 = oln * sum2(S2);
                    const float vals[9] = {fmaf(q0.w, s2, 2.f * q0.z * dx * s1), fmaf(q0.w * dx, s1, 2.f * q1.x * s2),
                                           dx * dx * s1, dx * s2, oln * sum2(S3), sdop, sum2(dr), sum2(dg), sum2(db)};
                    if (__popc(used) <= bwd_direct_for(PX)) {
                        // few lanes reached the splat: each adds its own nine values (fewer issue slots than
                        // the warp reduction; the same sums in another order)
                        if (any) {
                            float *g = grad2d + 12LL * st.id[j];
#pragma unroll
                            for (int i = 0; i < 9; ++i)
                                red_add_f32(g + i, (i == 2 || i == 4) ? -0.5f * LOG2E * vals[i]
                                                                      : (i == 3 ? -LOG2E * vals[i] : vals[i]));
                        }
                    } else {
#if LOBE_BWD_SLOTS
                        // the lane's nine values into the next slot's row; a full set of slots is
                        // summed column by column (27 lanes, no shuffles)
                        float *row = s_red[pw] + nslot * RED_SLOT + RED_ROW * lane;
                        *reinterpret_cast<float4 *>(row) = make_float4(vals[0], vals[1], vals[2], vals[3]);
                        *reinterpret_cast<float4 *>(row + 4) = make_float4(vals[4], vals[5], vals[6], vals[7]);
                        s_red[pw][RED_ROW * lane + 8 + nslot] = vals[8];
                        if (lane == 0) s_rid[pw][nslot] = st.id[j];
                        if (++nslot == RED_SLOTS) {
                            flush(RED_SLOTS);
                            nslot = 0;
                        }
#else
                        int idx;
                        const float tot = warp_reduce9(vals, idx);
                        if (idx >= 0) {
                            // back from the base-2 exponent domain: A = -0.5 log2e a, B = -log2e b, C = -0.5 log2e c
                            const float sc = (idx == 2 || idx == 4) ? -0.5f * LOG2E : (idx == 3 ? -LOG2E : 1.0f);
                            red_add_f32(grad2d + 12LL * st.id[j] + idx, sc * tot);
                        }
#endif
                    }
                }
            }
            __syncwarp();
            top = base;
            base = nbase;
        }
#if LOBE_BWD_SLOTS
        if (nslot) {
            flush(nslot);
            nslot = 0;
        }
#endif
        __syncwarp();
    };
    if constexpr (PERSIST) {
        int t, warp;
        while (wc.next(t, warp, pw)) tile_body(t, warp);
    } else {
        tile_body((int)blockIdx.x, pw);
    }
}

// --------------------------------------------------------------------------- tile order
//
// Longest list first (a longest-processing-time order of the tiles of every item): a counting
// sort of the tiles by the bit length of their list, descending (tiles of equal bit length in
// no particular order; every tile's result is independent of the order). ctl (ORDER_CTL words,
// zeroed before the first kernel): [0, 33) bucket sizes, [33, 66) bucket cursors, [66] the
// persistent kernel's work counter.

constexpr int ORDER_BUCKETS = 33;

__device__ __forceinline__ int list_bucket(const int *ts, int t)
{
    const int len = ts[t + 1] - ts[t];
    return len <= 0 ? 0 : 32 - __clz(len);  // bit length, 1..32
}

__global__ void __launch_bounds__(256) k_order_count(const int *__restrict__ ts, int n_tiles, unsigned *__restrict__ ctl)
{
    pdl_wait();
    __shared__ unsigned h[ORDER_BUCKETS];
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x)
        atomicAdd(&h[list_bucket(ts, t)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x)
        if (h[i]) atomicAdd(&ctl[i], h[i]);
}

__global__ void __launch_bounds__(256) k_order_place(const int *__restrict__ ts, int n_tiles, unsigned *__restrict__ ctl,
                                                     int *__restrict__ order)
{
    pdl_wait();
    __shared__ unsigned base[ORDER_BUCKETS], cnt[ORDER_BUCKETS], off[ORDER_BUCKETS];
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = ORDER_BUCKETS - 1; b >= 0; --b) {  // longest lists first
            base[b] = acc;
            acc += ctl[b];
        }
    }
    for (int t0 = blockIdx.x * blockDim.x; t0 < n_tiles; t0 += gridDim.x * blockDim.x) {
        for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        const int t = t0 + (int)threadIdx.x;
        int b = -1;
        unsigned rank = 0;
        if (t < n_tiles) {
            b = list_bucket(ts, t);
            rank = atomicAdd(&cnt[b], 1u);  // rank within the block's share of the bucket
        }
        __syncthreads();
        // one global reservation per (block round, bucket) instead of one per tile
        for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x)
            off[i] = cnt[i] ? atomicAdd(&ctl[ORDER_BUCKETS + i], cnt[i]) : 0u;
        __syncthreads();
        if (b >= 0) order[base[b] + off[b] + rank] = t;
        __syncthreads();
    }
}

cudaError_t launch_tile_order(const int *ts, int n_tiles, int *order, unsigned *ctl, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(unsigned) * ORDER_CTL, st);
    if (e != cudaSuccess || n_tiles == 0) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    const unsigned cap = 2u * (unsigned)sms;  // two 256-thread blocks an SM: a grid-stride pass over the tiles
    const unsigned blocks = (unsigned)(n_tiles + 255) / 256 < cap ? (unsigned)(n_tiles + 255) / 256 : cap;
    count_launch(2);
    launch_pdl(k_order_count, dim3(blocks), dim3(256), 0, st, ts, n_tiles, ctl);
    launch_pdl(k_order_place, dim3(blocks), dim3(256), 0, st, ts, n_tiles, ctl, order);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- launchers

// Persistent grid of a compositing kernel: as many blocks as fit resident on the current device
// (resident blocks per SM from the occupancy calculator, cached per kernel and device).
template <typename K>
static unsigned persistent_blocks(K kernel, int threads, unsigned n_tiles)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;  // (kernel, device) -> blocks
    int dev = 0;
    cudaGetDevice(&dev);
    int g = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto key = std::make_pair(reinterpret_cast<const void *>(kernel), dev);
        auto it = cache.find(key);
        if (it == cache.end()) {
            int sms = 1, b = 1;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, 0) != cudaSuccess || b < 1) b = 1;
            it = cache.emplace(key, b * (sms > 0 ? sms : 1)).first;
        }
        g = it->second;
    }
    return (unsigned)g < n_tiles ? (unsigned)g : (n_tiles > 0 ? n_tiles : 1);
}

template <typename K, typename... Args>
static void launch_render(K kernel, const BatchParams &P, int threads, const int *order, cudaStream_t st, Args &&...args)
{
    const unsigned grid = order ? persistent_blocks(kernel, threads, (unsigned)P.n_tiles) : (unsigned)P.n_tiles;
    launch_pdl(kernel, dim3(grid), dim3(threads), 0, st, P, std::forward<Args>(args)...);
}

template <int TW, int TH, int PX>
static cudaError_t fwd_t(const BatchParams &P, const float *splat, const int *ts, const int *ids, float *rgb, float *T,
                         int *nc, float *depth, const int *order, unsigned *work, cudaStream_t st)
{
    count_launch();
    const float4 *sp = reinterpret_cast<const float4 *>(splat);
    const int threads = 32 * Slab<TW, TH, PX>::WARPS;
    if constexpr (PX > 1) {  // 64-splat rounds (the depth channel keeps 32)
        if (P.nb_fwd == 2 && !depth) {
            if (order)
                launch_render(k_render_fwd<TW, TH, PX, false, true, 2>, P, threads, order, st, sp, ts, ids, rgb, T, nc,
                              (float *)nullptr, order, work);
            else
                launch_render(k_render_fwd<TW, TH, PX, false, false, 2>, P, threads, order, st, sp, ts, ids, rgb, T, nc,
                              (float *)nullptr, order, work);
            return cudaGetLastError();
        }
    }
    if (depth && order)
        launch_render(k_render_fwd<TW, TH, PX, true, true>, P, threads, order, st, sp, ts, ids, rgb, T, nc, depth, order, work);
    else if (depth)
        launch_render(k_render_fwd<TW, TH, PX, true, false>, P, threads, order, st, sp, ts, ids, rgb, T, nc, depth, order,
                      work);
    else if (order)
        launch_render(k_render_fwd<TW, TH, PX, false, true>, P, threads, order, st, sp, ts, ids, rgb, T, nc,
                      (float *)nullptr, order, work);
    else
        launch_render(k_render_fwd<TW, TH, PX, false, false>, P, threads, order, st, sp, ts, ids, rgb, T, nc,
                      (float *)nullptr, order, work);
    return cudaGetLastError();
}

template <int TW, int TH, int PX>
static cudaError_t bwd_t(const BatchParams &P, bool recompute, const float *splat, const int *ts, const int *ids,
                         const float *rgb, const int *nc, const float *dL, float *g2d, const int *order, unsigned *work,
                         cudaStream_t st)
{
    count_launch();
    const int threads = 32 * Slab<TW, TH, PX>::WARPS;
    const float4 *sp = reinterpret_cast<const float4 *>(splat);
#define LOBE_BWD_LAUNCH(K, R, Q) \
    launch_render(K<TW, TH, PX, R, Q>, P, threads, order, st, sp, ts, ids, rgb, nc, dL, g2d, order, work)
#define LOBE_BWD2_LAUNCH(R, Q, N) \
    launch_render(k_render_bwd2<TW, TH, PX, R, Q, N>, P, threads, order, st, sp, ts, ids, rgb, nc, dL, g2d, order, work)
    if constexpr (PX % 2 == 0) {  // pixel pairs in packed arithmetic
        if (P.nb_bwd == 2) {  // 64-splat rounds
            if (recompute && order) LOBE_BWD2_LAUNCH(true, true, 2);
            else if (recompute) LOBE_BWD2_LAUNCH(true, false, 2);
            else if (order) LOBE_BWD2_LAUNCH(false, true, 2);
            else LOBE_BWD2_LAUNCH(false, false, 2);
        } else {
            if (recompute && order) LOBE_BWD2_LAUNCH(true, true, 1);
            else if (recompute) LOBE_BWD2_LAUNCH(true, false, 1);
            else if (order) LOBE_BWD2_LAUNCH(false, true, 1);
            else LOBE_BWD2_LAUNCH(false, false, 1);
        }
    } else {
        if (recompute && order) LOBE_BWD_LAUNCH(k_render_bwd, true, true);
        else if (recompute) LOBE_BWD_LAUNCH(k_render_bwd, true, false);
        else if (order) LOBE_BWD_LAUNCH(k_render_bwd, false, true);
        else LOBE_BWD_LAUNCH(k_render_bwd, false, false);
    }
#undef LOBE_BWD_LAUNCH
#undef LOBE_BWD2_LAUNCH
    return cudaGetLastError();
}

// Pixels per lane: a config knob (0 = default). 16x16 and 32x16 tiles take 2, 4 or 8; 16x8
// tiles 1, 2 or 4; 8x8 tiles 1 or 2. Fewer pixels per lane = more warps per tile (finer early
// termination in the forward); more = fewer splat loads and cross-lane reductions per pixel
// (the adjoint).
int default_px(int tw, int th, bool backward)
{
    (void)backward;  // measured on B300: 4 is best or within 1% for both passes at 16x16 and 32x16
    return tw == 8 ? 2 : (th == 8 ? 2 : 4);
}

bool valid_px(int tw, int th, int px)
{
    if (px == 0) return true;
    if (tw == 8) return px == 1 || px == 2;
    if (th == 8) return px == 1 || px == 2 || px == 4;
    return px == 2 || px == 4 || px == 8;
}

#define LOBE_PX_DISPATCH(FN, ...)                                                                  \
    do {                                                                                          \
        if (P.tw == 16 && P.th == 16) {                                                           \
            if (px == 2) return FN<16, 16, 2>(__VA_ARGS__);                                       \
            if (px == 4) return FN<16, 16, 4>(__VA_ARGS__);                                       \
            if (px == 8) return FN<16, 16, 8>(__VA_ARGS__);                                       \
        } else if (P.tw == 16 && P.th == 8) {                                                     \
            if (px == 1) return FN<16, 8, 1>(__VA_ARGS__);                                        \
            if (px == 2) return FN<16, 8, 2>(__VA_ARGS__);                                        \
            if (px == 4) return FN<16, 8, 4>(__VA_ARGS__);                                        \
        } else if (P.tw == 32) {                                                                  \
            if (px == 2) return FN<32, 16, 2>(__VA_ARGS__);                                       \
            if (px == 4) return FN<32, 16, 4>(__VA_ARGS__);                                       \
            if (px == 8) return FN<32, 16, 8>(__VA_ARGS__);                                       \
        } else if (P.tw == 8) {                                                                   \
            if (px == 1) return FN<8, 8, 1>(__VA_ARGS__);                                         \
            if (px == 2) return FN<8, 8, 2>(__VA_ARGS__);                                         \
        }                                                                                         \
        return cudaErrorInvalidValue;                                                             \
    } while (0)

cudaError_t launch_render_fwd(const BatchParams &P, const float *splat, const int *ts, const int *ids, float *rgb,
                              float *T, int *nc, float *depth, int *order, unsigned *ctl, cudaStream_t st)
{
    if (P.n_tiles == 0) return cudaSuccess;
    if (order) {  // persistent: tiles longest list first
        cudaError_t e = launch_tile_order(ts, P.n_tiles, order, ctl, st);
        if (e != cudaSuccess) return e;
    }
    unsigned *work = order ? ctl + ORDER_CTL - 1 : nullptr;
    const int px = P.px_fwd ? P.px_fwd : default_px(P.tw, P.th, false);
    LOBE_PX_DISPATCH(fwd_t, P, splat, ts, ids, rgb, T, nc, depth, order, work, st);
}

cudaError_t launch_render_bwd(const BatchParams &P, bool recompute, const float *splat, const int *ts, const int *ids,
                              const float *rgb, const int *nc, const float *dL, float *g2d, int *order, unsigned *ctl,
                              cudaStream_t st)
{
    cudaError_t err = P.n_entries > 0 ? cudaMemsetAsync(g2d, 0, sizeof(float) * 12 * (size_t)P.n_entries, st)
                                      : cudaSuccess;
    if (err != cudaSuccess || P.n_tiles == 0) return err;
    if (order) {
        err = launch_tile_order(ts, P.n_tiles, order, ctl, st);
        if (err != cudaSuccess) return err;
    }
    unsigned *work = order ? ctl + ORDER_CTL - 1 : nullptr;
    const int px = P.px_bwd ? P.px_bwd : default_px(P.tw, P.th, true);
    LOBE_PX_DISPATCH(bwd_t, P, recompute, splat, ts, ids, rgb, nc, dL, g2d, order, work, st);
}

}  // namespace lobe
