// peak_probe.cu -- throughput probes of the pipes the compositing kernels are bound by.
//
// The composite and its adjoint are issue-bound on the FP32 pipe (scalar FFMA and packed
// fma.rn.f32x2) with one ex2.approx per evaluated (pixel, splat) pair on the MUFU unit. No
// vendor figure for these is measured on this part, so the roofline of those kernels is
// taken against these probes: every thread runs eight independent dependency chains of one
// instruction kind, enough to cover the pipe's latency at full occupancy.
#include "lobe_internal.cuh"

namespace lobe {

template <int KIND>
__global__ void __launch_bounds__(256) k_peak_probe(int iters, float seed, float *sink)
{
    pdl_wait();
    const float b = seed * 0.999f, c = seed * 1e-3f;
    float s = 0.0f;
    if constexpr (KIND == 1) {
        unsigned long long v[8], bb, cc;
        asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(b), "f"(b));
        asm("mov.b64 %0, {%1, %2};" : "=l"(cc) : "f"(c), "f"(c));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float x = seed + 0.01f * k + 1e-6f * threadIdx.x;
            asm("mov.b64 %0, {%1, %2};" : "=l"(v[k]) : "f"(x), "f"(x));
        }
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v[k]) : "l"(bb), "l"(cc));
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v[k]));
            s += lo + hi;
        }
    } else {
        float a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = seed + 0.01f * k + 1e-6f * threadIdx.x;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (KIND == 0)
                    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(b), "f"(c));
                else
                    asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[k]));
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s += a[k];
    }
    if (s == 1.2345f) sink[threadIdx.x] = s;  // never true in practice; keeps the chains live
}

}  // namespace lobe

using namespace lobe;

extern "C" lobe_status lobe_peak_probe(void *stream, int32_t kind, int32_t blocks, int32_t iters, float *sink)
{
    if (kind < 0 || kind > 2 || blocks <= 0 || iters <= 0 || !sink) return LOBE_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    count_launch();
    cudaError_t e;
    if (kind == 0)
        e = launch_pdl(k_peak_probe<0>, dim3(blocks), dim3(256), 0, st, iters, 1.0001f, sink);
    else if (kind == 1)
        e = launch_pdl(k_peak_probe<1>, dim3(blocks), dim3(256), 0, st, iters, 1.0001f, sink);
    else
        e = launch_pdl(k_peak_probe<2>, dim3(blocks), dim3(256), 0, st, iters, -0.5f, sink);
    return e == cudaSuccess ? LOBE_OK : LOBE_ERR_CUDA;
}
