// render.cu -- per-tile front-to-back compositing (forward) and its adjoint.
//
// Forward (the blending equation of Sec. 3.2 with colour c_i in place of depth d_i):
//   C = sum_i c_i alpha_i T_i + T_N bg,  T_i = prod_{j<i} (1 - alpha_j),
//   alpha_i = min(0.99, o_i exp(-sigma_i)), sigma = 0.5 (a dx^2 + c dy^2) + b dx dy;
//   a splat is skipped when sigma < 0 or alpha < 1/255; the walk stops, before adding, at the
//   first splat with T (1 - alpha) < 1e-4.
//
// Adjoint, walked front to back (the same order and the same alpha decisions as the
// forward, so no per-pixel list has to be reversed): with R_i = C - sum_{j<=i} c_j alpha_j T_j
// the colour still to come after splat i (background included),
//   dL/dc_i     = alpha_i T_i dL/dC
//   dL/dalpha_i = T_i (c_i . dL/dC) - (R_i . dL/dC) / (1 - alpha_i)
// which equals the textbook reverse-order form T_i (c_i - B_i) . dL/dC with B_i the colour
// seen behind splat i, because T_i B_i = R_i / (1 - alpha_i). The per-pixel state it needs,
// C (the rendered colour) and the stop position, is either read from the forward's outputs
// ("store") or re-derived by a forward sweep inside the kernel ("recompute").
//
// Per splat the 32 pixels of a warp are summed with shuffles and one lane adds the result to
// global memory with vector reductions, so a tile of 256 pixels issues 8 (not 256) atomic
// updates per splat.
#include "lobe_internal.cuh"

namespace lobe {

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_render_fwd(const __grid_constant__ BatchParams P,
                                                       const float4 *__restrict__ splat, const int *__restrict__ tile_start,
                                                       const int *__restrict__ ids, float *__restrict__ rgb,
                                                       float *__restrict__ Tout, int *__restrict__ ncout)
{
    constexpr int N = TW * TH;
    __shared__ float4 s0[N];
    __shared__ float4 s1[N];
    __shared__ float s2[N];
    const int t = blockIdx.x;
    const ItemParams &I = P.item[item_of_tile(P, t)];
    const int lt = t - I.tile_off, tx = lt % I.gx, ty = lt / I.gx;
    const int px = tx * TW + (int)threadIdx.x % TW, py = ty * TH + (int)threadIdx.x / TW;
    const bool inside = px < I.W && py < I.H;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const int start = tile_start[t], end = tile_start[t + 1];
    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int last = 0;
    bool done = !inside;
    for (int base = start; base < end; base += N) {
        if (__syncthreads_and(done)) break;
        const int k = base + (int)threadIdx.x;
        if (k < end) {
            const int e = ids[k];
            const float4 a = splat[3 * e], b = splat[3 * e + 1];
            s0[threadIdx.x] = make_float4(a.x, a.y, -0.5f * LOG2E * a.z, -LOG2E * a.w);
            s1[threadIdx.x] = make_float4(-0.5f * LOG2E * b.x, b.y, b.z, b.w);
            s2[threadIdx.x] = splat[3 * e + 2].x;
        }
        __syncthreads();
        const int cnt = min(N, end - base);
        for (int j = 0; j < cnt && !done; ++j) {
            const float4 a = s0[j], b = s1[j];
            const Eval r = eval_pair(a.x, a.y, a.z, a.w, b.x, b.y, pxc, pyc);
            if (!r.use) continue;
            const float Tn = next_T(T, r.alpha);
            if (Tn < T_MIN) {
                done = true;
                break;
            }
            const float w = r.alpha * T;
            C0 += b.z * w;
            C1 += b.w * w;
            C2 += s2[j] * w;
            T = Tn;
            last = base - start + j + 1;
        }
    }
    if (inside) {
        const long long HW = (long long)I.W * I.H, p = (long long)py * I.W + px;
        float *out = rgb + 3 * I.pix_off;
        out[p] = C0 + T * P.bg[0];
        out[HW + p] = C1 + T * P.bg[1];
        out[2 * HW + p] = C2 + T * P.bg[2];
        Tout[I.pix_off + p] = T;
        ncout[I.pix_off + p] = last;
    }
}

template <int TW, int TH, bool RECOMPUTE>
__global__ void __launch_bounds__(TW *TH) k_render_bwd(const __grid_constant__ BatchParams P,
                                                       const float4 *__restrict__ splat, const int *__restrict__ tile_start,
                                                       const int *__restrict__ ids, const float *__restrict__ rgb,
                                                       const int *__restrict__ ncin, const float *__restrict__ dL,
                                                       float *__restrict__ grad2d)
{
    constexpr int N = TW * TH;
    __shared__ float4 s0[N];
    __shared__ float4 s1[N];
    __shared__ float s2[N];
    __shared__ int sid[N];
    __shared__ int s_max;
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x;
    const ItemParams &I = P.item[item_of_tile(P, t)];
    const int lt = t - I.tile_off, tx = lt % I.gx, ty = lt / I.gx;
    const int px = tx * TW + (int)threadIdx.x % TW, py = ty * TH + (int)threadIdx.x / TW;
    const bool inside = px < I.W && py < I.H;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const int start = tile_start[t], end = tile_start[t + 1];
    const long long HW = (long long)I.W * I.H, p = (long long)py * I.W + px;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, R0 = 0.f, R1 = 0.f, R2 = 0.f;
    int nc = 0;
    if (threadIdx.x == 0) s_max = 0;
    if (inside) {
        const float *d = dL + 3 * I.pix_off;
        g0 = d[p];
        g1 = d[HW + p];
        g2 = d[2 * HW + p];
        if (!RECOMPUTE) {
            const float *c = rgb + 3 * I.pix_off;
            R0 = c[p];
            R1 = c[HW + p];
            R2 = c[2 * HW + p];
            nc = ncin[I.pix_off + p];
        }
    }
    if (RECOMPUTE) {
        // forward sweep: stop position and rendered colour, bit-identical decisions
        float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        bool done = !inside;
        for (int base = start; base < end; base += N) {
            if (__syncthreads_and(done)) break;
            const int k = base + (int)threadIdx.x;
            if (k < end) {
                const int e = ids[k];
                const float4 a = splat[3 * e], b = splat[3 * e + 1];
                s0[threadIdx.x] = make_float4(a.x, a.y, -0.5f * LOG2E * a.z, -LOG2E * a.w);
                s1[threadIdx.x] = make_float4(-0.5f * LOG2E * b.x, b.y, b.z, b.w);
                s2[threadIdx.x] = splat[3 * e + 2].x;
            }
            __syncthreads();
            const int cnt = min(N, end - base);
            for (int j = 0; j < cnt && !done; ++j) {
                const float4 a = s0[j], b = s1[j];
                const Eval r = eval_pair(a.x, a.y, a.z, a.w, b.x, b.y, pxc, pyc);
                if (!r.use) continue;
                const float Tn = next_T(T, r.alpha);
                if (Tn < T_MIN) {
                    done = true;
                    break;
                }
                const float w = r.alpha * T;
                C0 += b.z * w;
                C1 += b.w * w;
                C2 += s2[j] * w;
                T = Tn;
                nc = base - start + j + 1;
            }
        }
        R0 = C0 + T * P.bg[0];
        R1 = C1 + T * P.bg[1];
        R2 = C2 + T * P.bg[2];
        __syncthreads();
    }
    __syncthreads();
    if (nc > 0) atomicMax(&s_max, nc);
    __syncthreads();
    const int stop = min(start + s_max, end);
    float T = 1.0f;
    for (int base = start; base < stop; base += N) {
        __syncthreads();
        const int k = base + (int)threadIdx.x;
        if (k < stop) {
            const int e = ids[k];
            const float4 a = splat[3 * e], b = splat[3 * e + 1];
            s0[threadIdx.x] = make_float4(a.x, a.y, -0.5f * LOG2E * a.z, -LOG2E * a.w);
            s1[threadIdx.x] = make_float4(-0.5f * LOG2E * b.x, b.y, b.z, b.w);
            s2[threadIdx.x] = splat[3 * e + 2].x;
            sid[threadIdx.x] = e;
        }
        __syncthreads();
        const int cnt = min(N, stop - base);
        for (int j = 0; j < cnt; ++j) {
            const int pos = base - start + j;
            float du = 0.f, dv = 0.f, dA = 0.f, dB = 0.f, dC = 0.f, dop = 0.f, dr = 0.f, dg = 0.f, db = 0.f;
            bool contrib = false;
            if (pos < nc) {
                const float4 a = s0[j], b = s1[j];
                const Eval r = eval_pair(a.x, a.y, a.z, a.w, b.x, b.y, pxc, pyc);
                if (r.use) {
                    contrib = true;
                    const float cb = s2[j];
                    const float w = r.alpha * T;
                    dr = w * g0;
                    dg = w * g1;
                    db = w * g2;
                    R0 -= b.z * w;
                    R1 -= b.w * w;
                    R2 -= cb * w;
                    const float gc = g0 * b.z + g1 * b.w + g2 * cb;
                    const float gR = g0 * R0 + g1 * R1 + g2 * R2;
                    const float dalpha = T * gc - gR / (1.0f - r.alpha);
                    T = next_T(T, r.alpha);
                    if (!r.clamped) {
                        dop = dalpha * r.G;
                        const float dp2 = dalpha * r.alpha * LN2;
                        dA = dp2 * r.dx * r.dx;
                        dB = dp2 * r.dx * r.dy;
                        dC = dp2 * r.dy * r.dy;
                        du = dp2 * (2.f * a.z * r.dx + a.w * r.dy);
                        dv = dp2 * (a.w * r.dx + 2.f * b.x * r.dy);
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    du += __shfl_xor_sync(0xffffffffu, du, o);
                    dv += __shfl_xor_sync(0xffffffffu, dv, o);
                    dA += __shfl_xor_sync(0xffffffffu, dA, o);
                    dB += __shfl_xor_sync(0xffffffffu, dB, o);
                    dC += __shfl_xor_sync(0xffffffffu, dC, o);
                    dop += __shfl_xor_sync(0xffffffffu, dop, o);
                    dr += __shfl_xor_sync(0xffffffffu, dr, o);
                    dg += __shfl_xor_sync(0xffffffffu, dg, o);
                    db += __shfl_xor_sync(0xffffffffu, db, o);
                }
                if (lane == 0) {
                    float *gp = grad2d + 12LL * sid[j];
                    // back from the base-2 exponent domain: A = -0.5 log2e a, B = -log2e b, C = -0.5 log2e c
                    red_add_v4(gp, du, dv, -0.5f * LOG2E * dA, -LOG2E * dB);
                    red_add_v4(gp + 4, -0.5f * LOG2E * dC, dop, dr, dg);
                    red_add_f32(gp + 8, db);
                }
            }
        }
    }
}

// --------------------------------------------------------------------------- launchers

template <int TW, int TH>
static cudaError_t fwd_t(const BatchParams &P, const float *splat, const int *ts, const int *ids, float *rgb, float *T,
                         int *nc, cudaStream_t st)
{
    count_launch();
    k_render_fwd<TW, TH><<<P.n_tiles, TW * TH, 0, st>>>(P, reinterpret_cast<const float4 *>(splat), ts, ids, rgb, T, nc);
    return cudaGetLastError();
}

template <int TW, int TH>
static cudaError_t bwd_t(const BatchParams &P, bool recompute, const float *splat, const int *ts, const int *ids,
                         const float *rgb, const int *nc, const float *dL, float *g2d, cudaStream_t st)
{
    count_launch();
    if (recompute)
        k_render_bwd<TW, TH, true><<<P.n_tiles, TW * TH, 0, st>>>(P, reinterpret_cast<const float4 *>(splat), ts, ids,
                                                                   rgb, nc, dL, g2d);
    else
        k_render_bwd<TW, TH, false><<<P.n_tiles, TW * TH, 0, st>>>(P, reinterpret_cast<const float4 *>(splat), ts, ids,
                                                                    rgb, nc, dL, g2d);
    return cudaGetLastError();
}

cudaError_t launch_render_fwd(const BatchParams &P, const float *splat, const int *ts, const int *ids, float *rgb,
                              float *T, int *nc, cudaStream_t st)
{
    if (P.n_tiles == 0) return cudaSuccess;
    if (P.tw == 16 && P.th == 16) return fwd_t<16, 16>(P, splat, ts, ids, rgb, T, nc, st);
    if (P.tw == 8 && P.th == 8) return fwd_t<8, 8>(P, splat, ts, ids, rgb, T, nc, st);
    if (P.tw == 32 && P.th == 16) return fwd_t<32, 16>(P, splat, ts, ids, rgb, T, nc, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_render_bwd(const BatchParams &P, bool recompute, const float *splat, const int *ts, const int *ids,
                              const float *rgb, const int *nc, const float *dL, float *g2d, cudaStream_t st)
{
    cudaError_t err = P.n_entries > 0 ? cudaMemsetAsync(g2d, 0, sizeof(float) * 12 * (size_t)P.n_entries, st)
                                      : cudaSuccess;
    if (err != cudaSuccess || P.n_tiles == 0) return err;
    if (P.tw == 16 && P.th == 16) return bwd_t<16, 16>(P, recompute, splat, ts, ids, rgb, nc, dL, g2d, st);
    if (P.tw == 8 && P.th == 8) return bwd_t<8, 8>(P, recompute, splat, ts, ids, rgb, nc, dL, g2d, st);
    if (P.tw == 32 && P.th == 16) return bwd_t<32, 16>(P, recompute, splat, ts, ids, rgb, nc, dL, g2d, st);
    return cudaErrorInvalidValue;
}

}  // namespace lobe
