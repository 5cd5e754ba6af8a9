// fcs.cu -- fast camera selection (Sec. 3.2): the per-pixel composite depth of every camera is
// back-projected to a 3D point and counted against each block's box.
//
// A pixel yields a point when some splat contributed to it (T_final < 1). Its depth is the
// composite D = sum_i d_i alpha_i T_i of the paper's equation, optionally divided by the
// accumulated opacity 1 - T_final. With the pinhole of the item's camera, the point is
//   p_c = ((px + 0.5 - cx) / fx * D, (py + 0.5 - cy) / fy * D, D)   (camera space, z = D)
//   p_w = R^T (p_c - t)                                                (world, viewmat = [R | t])
// and it counts for block b when lo_b <= p_w < hi_b on every axis. Per (item, block) the
// counts, and per item the number of points, are added with warp-aggregated atomics.
#include "lobe_internal.cuh"

namespace lobe {

__device__ __forceinline__ int item_of_pixel(const BatchParams &P, long long p)
{
    int lo = 0, hi = P.n_items - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.item[mid].pix_off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_fcs_coverage(const __grid_constant__ BatchParams P,
                                                      const __grid_constant__ FcsBlocks B, const float *__restrict__ depth,
                                                      const float *__restrict__ Tfin, int normalize,
                                                      uint32_t *__restrict__ counts, uint32_t *__restrict__ n_points)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = p < P.n_pixels;
    int item = -1;
    bool has = false;
    float wx = 0.f, wy = 0.f, wz = 0.f;
    if (in) {
        item = item_of_pixel(P, p);
        const ItemParams &I = P.item[item];
        const float T = Tfin[p];
        has = T < 1.0f;
        if (has) {
            const long long lp = p - I.pix_off;
            const int py = (int)(lp / I.W), px = (int)(lp - (long long)py * I.W);
            float D = depth[p];
            if (normalize) D = D / (1.0f - T);
            const float xc = ((float)px + 0.5f - I.cx) / I.fx * D, yc = ((float)py + 0.5f - I.cy) / I.fy * D, zc = D;
            const float *V = I.V;  // rows of [R | t]
            const float ux = xc - V[3], uy = yc - V[7], uz = zc - V[11];
            wx = V[0] * ux + V[4] * uy + V[8] * uz;
            wy = V[1] * ux + V[5] * uy + V[9] * uz;
            wz = V[2] * ux + V[6] * uy + V[10] * uz;
        }
    }
    // lanes of the same item count together
    const unsigned grp = __match_any_sync(0xffffffffu, item);
    const bool leader = lane == __ffs(grp) - 1 && item >= 0;
    const unsigned pts = __ballot_sync(0xffffffffu, has) & grp;
    if (leader && pts) atomicAdd(n_points + item, (uint32_t)__popc(pts));
    for (int b = 0; b < B.n; ++b) {
        const bool inside = has && wx >= B.lo[b][0] && wx < B.hi[b][0] && wy >= B.lo[b][1] && wy < B.hi[b][1] &&
                            wz >= B.lo[b][2] && wz < B.hi[b][2];
        const unsigned m = __ballot_sync(0xffffffffu, inside) & grp;
        if (leader && m) atomicAdd(counts + (long long)item * B.n + b, (uint32_t)__popc(m));
    }
}

cudaError_t launch_fcs_coverage(const BatchParams &P, const FcsBlocks &B, const float *depth, const float *Tfin,
                                int normalize, uint32_t *counts, uint32_t *n_points, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)P.n_items * (size_t)(B.n > 0 ? B.n : 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_points, 0, sizeof(uint32_t) * (size_t)P.n_items, st);
    if (e != cudaSuccess || P.n_pixels == 0) return e;
    count_launch();
    launch_pdl(k_fcs_coverage, dim3((unsigned)((P.n_pixels + 255) / 256)), dim3(256), 0, st, P, B, depth, Tfin, normalize, counts,
                                                                         n_points);
    return cudaGetLastError();
}

}  // namespace lobe
