// densify.cu -- selective densification (Sec. 3.3) with the adaptive density control of the
// 3DGS procedure the paper trains with (appendix "3DGS Training"), as a GPU stream compaction.
//
// Per Gaussian g, from its selective-densification statistic (the summed view-space gradient
// norm acc[g] over cnt[g] views in which g was visible with its mean inside the block, so
// cnt[g] = 0 for every Gaussian outside the block):
//   prune  when logit[g] < prune_logit                               -> no output
//   clone  when cnt > 0, acc / cnt >= grad_threshold and
//          max(log_s) <= max_clone_log_scale                         -> g, then an exact copy
//   split  when cnt > 0, acc / cnt >= grad_threshold and larger      -> n_split children with
//          mean mu + R(q) (s * z_k) (z_k the caller's standard normal draws for g, child k),
//          log-scales log_s - split_log_shrink, the same rotation, opacity and SH
//   keep   otherwise                                                 -> g
// The decisions compare float32 values directly (the mean gradient as acc / cnt in IEEE
// float32, log-scales and logits without exp), so they are exactly reproducible. Outputs keep
// the order of their sources (a single-pass scan of the per-Gaussian output counts).
#include "lookback.cuh"

namespace lobe {

enum : uint8_t { DENS_KEEP = 0, DENS_CLONE = 1, DENS_SPLIT = 2, DENS_PRUNE = 3 };

__global__ void __launch_bounds__(256) k_densify_classify(long long n, const float *__restrict__ log_scales,
                                                          const float *__restrict__ logits,
                                                          const float *__restrict__ acc, const int *__restrict__ cnt,
                                                          lobe_densify_params prm, uint8_t *__restrict__ action,
                                                          uint32_t *__restrict__ n_out)
{
    pdl_wait();
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    uint8_t a = DENS_KEEP;
    if (logits[g] < prm.prune_logit) {
        a = DENS_PRUNE;
    } else if (cnt[g] > 0 && acc[g] / (float)cnt[g] >= prm.grad_threshold) {
        const float m = fmaxf(log_scales[3 * g], fmaxf(log_scales[3 * g + 1], log_scales[3 * g + 2]));
        a = m <= prm.max_clone_log_scale ? DENS_CLONE : DENS_SPLIT;
    }
    action[g] = a;
    n_out[g] = a == DENS_PRUNE ? 0u : a == DENS_CLONE ? 2u : a == DENS_SPLIT ? (uint32_t)prm.n_split : 1u;
}

// One thread per source Gaussian writes the geometry of its outputs at off[g] .. (if they fit
// the capacity); the block's outputs are a contiguous range, whose SH (192 B each, 81% of the
// bytes) the block then copies with consecutive threads on consecutive 16-byte chunks.
constexpr int DE_THREADS = 256;

__global__ void __launch_bounds__(DE_THREADS) k_densify_emit(long long n, lobe_gaussians in,
                                                             const uint8_t *__restrict__ action,
                                                             const uint32_t *__restrict__ off, const uint32_t *total,
                                                             const float *__restrict__ normals, lobe_densify_params prm,
                                                             lobe_params_out out, int *__restrict__ source)
{
    pdl_wait();
    __shared__ uint32_t s_src[DE_THREADS * 4];  // the source of each of the block's outputs (n_split <= 4)
    const long long g0 = (long long)blockIdx.x * DE_THREADS;
    const long long g = g0 + threadIdx.x;
    if ((long long)*total > out.capacity) return;  // the whole grid returns: nothing written
    const long long O0 = off[g0];
    const long long O1 = g0 + DE_THREADS < n ? (long long)off[g0 + DE_THREADS] : (long long)*total;
    const uint8_t a = g < n ? action[g] : DENS_PRUNE;
    if (a != DENS_PRUNE) {
        const int k_out = a == DENS_CLONE ? 2 : a == DENS_SPLIT ? prm.n_split : 1;
        const long long o0 = off[g];
        const float mx = in.means[3 * g], my = in.means[3 * g + 1], mz = in.means[3 * g + 2];
        const float l0 = in.log_scales[3 * g], l1 = in.log_scales[3 * g + 1], l2 = in.log_scales[3 * g + 2];
        const float4 q = reinterpret_cast<const float4 *>(in.quats)[g];
        const float lg = in.opacity_logits[g];
        float R[9];
        if (a == DENS_SPLIT) {  // rotation of the normalised quaternion (w, x, y, z)
            const float qi = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
            const float r = q.x * qi, x = q.y * qi, y = q.z * qi, z = q.w * qi;
            R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - r * z);       R[2] = 2.f * (x * z + r * y);
            R[3] = 2.f * (x * y + r * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - r * x);
            R[6] = 2.f * (x * z - r * y);       R[7] = 2.f * (y * z + r * x);       R[8] = 1.f - 2.f * (x * x + y * y);
        }
        const float s0 = a == DENS_SPLIT ? __expf(l0) : 0.f, s1 = a == DENS_SPLIT ? __expf(l1) : 0.f,
                    s2 = a == DENS_SPLIT ? __expf(l2) : 0.f;
        for (int k = 0; k < k_out; ++k) {
            const long long o = o0 + k;
            s_src[o - O0] = (uint32_t)threadIdx.x;
            float px = mx, py = my, pz = mz, n0 = l0, n1 = l1, n2 = l2;
            if (a == DENS_SPLIT) {
                const float *zk = normals + (g * prm.n_split + k) * 3;
                const float u0 = s0 * zk[0], u1 = s1 * zk[1], u2 = s2 * zk[2];
                px = mx + R[0] * u0 + R[1] * u1 + R[2] * u2;
                py = my + R[3] * u0 + R[4] * u1 + R[5] * u2;
                pz = mz + R[6] * u0 + R[7] * u1 + R[8] * u2;
                n0 = l0 - prm.split_log_shrink;
                n1 = l1 - prm.split_log_shrink;
                n2 = l2 - prm.split_log_shrink;
            }
            out.means[3 * o] = px; out.means[3 * o + 1] = py; out.means[3 * o + 2] = pz;
            out.log_scales[3 * o] = n0; out.log_scales[3 * o + 1] = n1; out.log_scales[3 * o + 2] = n2;
            reinterpret_cast<float4 *>(out.quats)[o] = q;
            out.opacity_logits[o] = lg;
            if (source) source[o] = (int)g;
        }
    }
    __syncthreads();
    // SH of outputs O0 .. O1: 12 float4 each, chunk j = output (j / 12), part (j % 12)
    const int chunks = (int)(O1 - O0) * 12;
    const float4 *src = reinterpret_cast<const float4 *>(in.sh) + 12 * g0;
    float4 *dst = reinterpret_cast<float4 *>(out.sh) + 12 * O0;
    for (int j = threadIdx.x; j < chunks; j += DE_THREADS) {
        const int o = j / 12, c = j - 12 * o;
        dst[j] = src[12 * (int)s_src[o] + c];
    }
}

cudaError_t launch_densify_count(long long n, const lobe_gaussians &in, const float *acc, const int *cnt,
                                 const lobe_densify_params &prm, uint8_t *action, uint32_t *n_out, uint32_t *total,
                                 LB lb, cudaStream_t st)
{
    if (n > 0) {
        count_launch();
        launch_pdl(k_densify_classify, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, n, in.log_scales, in.opacity_logits, acc, cnt,
                                                                        prm, action, n_out);
    }
    scan(LoadPlain{n_out}, nullptr, n, n_out, total, nullptr, nullptr, -1, lb, st, true);
    return cudaGetLastError();
}

cudaError_t launch_densify_emit(long long n, const lobe_gaussians &in, const uint8_t *action, const uint32_t *off,
                                const uint32_t *total, const float *normals, const lobe_densify_params &prm,
                                const lobe_params_out &out, int *source, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    count_launch();
    launch_pdl(k_densify_emit, dim3((unsigned)((n + DE_THREADS - 1) / DE_THREADS)), dim3(DE_THREADS), 0, st, n, in, action, off, total, normals, prm, out, source);
    return cudaGetLastError();
}

}  // namespace lobe
