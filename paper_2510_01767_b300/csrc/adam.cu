// Standalone Adam update of one Gaussian set (the optimizer of the 3DGS procedure the
// fine-training follows, appendix "3DGS Training"; Kingma and Ba, Algorithm 1).
//
// The set's five SoA arrays (means [n][3], log_scales [n][3], quats [n][4], opacity [n],
// sh [n][16][3]) are updated as flat float arrays: every thread takes float4 chunks of one
// array at a time in a grid-stride loop, so each of p, g, m, v is read and p, m, v written
// once, coalesced -- 7 x 4 B per element, 1652 B per Gaussian, the HBM bound of the update.
// The learning rate of an element follows its array (the SH by column: the first three
// floats of a Gaussian's 48 are its degree-0 band). In the sparse modes a chunk none of whose
// rows is selected is skipped without touching its parameters.

#include <atomic>
#include "lobe_internal.cuh"

namespace lobe {

constexpr int AD_THREADS = 256;

struct AdamArrays {
    float *p[5], *m[5], *v[5];
    const float *g[5];
    uint32_t n;  // rows; 12 n < 2^32 (checked by the caller), so chunk and row indices fit 32 bits
};

template <int MODE>
__device__ __forceinline__ bool adam_selected(const uint8_t *rows, uint32_t r)
{
    if (MODE == 0) return true;
    const uint8_t b = __ldg(rows + r);
    return MODE == 1 ? b != 0 : b == 0;
}

// One array of W floats a row: float4 chunks in a grid-stride loop, then the n W % 4 last
// elements. A = lr group of the array (the SH array's degree-0 columns take AG_SH_DC).
template <int MODE, int W, int A>
__device__ __forceinline__ void adam_array(float *__restrict__ P, float *__restrict__ M, float *__restrict__ V,
                                           const float *__restrict__ G, uint32_t n, const uint8_t *__restrict__ rows,
                                           const AdamK &k, uint32_t tid, uint32_t stride)
{
    const uint32_t nc = (uint32_t)(((unsigned long long)n * W) >> 2);
    float4 *P4 = reinterpret_cast<float4 *>(P);
    float4 *M4 = reinterpret_cast<float4 *>(M);
    float4 *V4 = reinterpret_cast<float4 *>(V);
    const float4 *G4 = reinterpret_cast<const float4 *>(G);
    for (uint32_t c = tid; c < nc; c += stride) {
        bool sel[4];
        bool any = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // row of element 4c + i (one row per chunk when W is a multiple of 4)
            const uint32_t r = W % 4 == 0 ? c / (W / 4) : (4 * c + i) / W;
            sel[i] = adam_selected<MODE>(rows, r);
            any |= sel[i];
        }
        if (!any) continue;
        float4 p = P4[c];
        float4 m = __ldcs(M4 + c);
        float4 v = __ldcs(V4 + c);
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        if (MODE != 2) g = __ldcs(G4 + c);
        float *pp = &p.x, *mm = &m.x, *vv = &v.x;
        const float *gg = &g.x;
        // the SH array's degree-0 band: the first three floats of a row's 48
        const bool dc_chunk = A == AG_SH_REST && c % 12 == 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (!sel[i]) continue;
            const float ss = (A == AG_SH_REST && dc_chunk && i < 3) ? k.ss[AG_SH_DC] : k.ss[A];
            if (MODE == 2)
                adam_decay(k, ss, pp[i], mm[i], vv[i]);
            else
                adam_step(k, ss, gg[i], pp[i], mm[i], vv[i]);
        }
        P4[c] = p;
        __stcs(M4 + c, m);
        __stcs(V4 + c, v);
    }
    if (W % 4 != 0) {
        const unsigned long long e = 4ull * nc + tid;
        if (e < (unsigned long long)n * W && adam_selected<MODE>(rows, (uint32_t)(e / W))) {
            float p = P[e], m = M[e], v = V[e];
            if (MODE == 2)
                adam_decay(k, k.ss[A], p, m, v);
            else
                adam_step(k, k.ss[A], G[e], p, m, v);
            P[e] = p;
            M[e] = m;
            V[e] = v;
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(AD_THREADS) k_adam(const __grid_constant__ AdamArrays X, const uint8_t *__restrict__ rows,
                                                     const __grid_constant__ AdamK k)
{
    pdl_wait();
    const uint32_t stride = gridDim.x * AD_THREADS;
    const uint32_t tid = blockIdx.x * AD_THREADS + threadIdx.x;
    adam_array<MODE, 48, AG_SH_REST>(X.p[4], X.m[4], X.v[4], X.g[4], X.n, rows, k, tid, stride);
    adam_array<MODE, 3, AG_MEANS>(X.p[0], X.m[0], X.v[0], X.g[0], X.n, rows, k, tid, stride);
    adam_array<MODE, 3, AG_LOG_SCALES>(X.p[1], X.m[1], X.v[1], X.g[1], X.n, rows, k, tid, stride);
    adam_array<MODE, 4, AG_QUATS>(X.p[2], X.m[2], X.v[2], X.g[2], X.n, rows, k, tid, stride);
    adam_array<MODE, 1, AG_OPACITY>(X.p[3], X.m[3], X.v[3], X.g[3], X.n, rows, k, tid, stride);
}

cudaError_t launch_adam(long long n, const AdamSet &s, const float *const grad[5], const uint8_t *rows, int mode,
                        const AdamK &k, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (12 * n > (1ll << 32) - (1ll << 22)) return cudaErrorInvalidValue;  // 32-bit chunk indices, stride included
    AdamArrays X;
    for (int a = 0; a < 5; ++a) {
        X.p[a] = s.p[a];
        X.m[a] = s.m[a];
        X.v[a] = s.v[a];
        X.g[a] = grad ? grad[a] : nullptr;
    }
    X.n = (uint32_t)n;
    void (*kern)(AdamArrays, const uint8_t *, AdamK) = mode == 0 ? k_adam<0> : mode == 1 ? k_adam<1> : k_adam<2>;
    // one wave of resident blocks (grid-stride), or fewer when the set is small; the
    // largest array (SH, 12 chunks a row) sets the size
    // (the occupancy is a property of the kernel, looked up once; host threads with their own
    // contexts may get here at the same time, hence the atomic)
    static std::atomic<int> resident[3] = {0, 0, 0};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    int res = resident[mode].load(std::memory_order_relaxed);
    if (res == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, kern, AD_THREADS, 0) != cudaSuccess || res <= 0) res = 1;
        resident[mode].store(res, std::memory_order_relaxed);
    }
    long long blocks = (12 * n + AD_THREADS - 1) / AD_THREADS;
    const long long cap = (long long)sms * res;
    if (blocks > cap) blocks = cap;
    count_launch(1);
    launch_pdl(kern, dim3((unsigned)blocks), dim3(AD_THREADS), 0, st, X, rows, k);
    return cudaGetLastError();
}

}  // namespace lobe
