// FP32 fused multiply-add throughput of the device: the denominator of the
// shooting kernels' roofline (their near sums and Taylor chains run on the
// FP32 pipe, as scalar FFMA and as Blackwell's two-lane fma.rn.f32x2).  Each
// thread runs eight independent FMA chains, a <- a * b + c with |a| settling
// near 1, so that issue, not latency, bounds the launch; nothing is read from
// or written to memory except one store that never happens (it keeps the
// chains from being optimised away).
#include "ml_internal.cuh"

namespace ml {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_THREADS = 256;

template <bool TWO>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(int64_t iters, float *sink)
{
    const float b = 0.99990f, c = 1.0e-4f;
    if constexpr (TWO) {
        f32x2 a[PEAK_CHAINS];
        const f32x2 B = pack2(b, b), C = pack2(c, c);
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k)
            a[k] = pack2(1.0f + 1.0e-3f * k, 1.0f - 1.0e-3f * (threadIdx.x & 7));
#pragma unroll 16
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fma2(a[k], B, C);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) {
            float lo, hi;
            unpack2(a[k], lo, hi);
            s += lo + hi;
        }
        if (s == -1.0f) sink[blockIdx.x] = s;
    } else {
        float a[PEAK_CHAINS];
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = 1.0f + 1.0e-3f * k + 1.0e-4f * (threadIdx.x & 7);
#pragma unroll 16
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = __fmaf_rn(a[k], b, c);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
        if (s == -1.0f) sink[blockIdx.x] = s;
    }
}

cudaError_t launch_fma_peak(bool two_lane, unsigned blocks, int64_t iters, float *sink,
                            cudaStream_t s)
{
    if (two_lane)
        k_fma_peak<true><<<blocks, PEAK_THREADS, 0, s>>>(iters, sink);
    else
        k_fma_peak<false><<<blocks, PEAK_THREADS, 0, s>>>(iters, sink);
    return cudaGetLastError();
}

double fma_peak_flop(bool two_lane, unsigned blocks, int64_t iters)
{
    return 2.0 * (two_lane ? 2.0 : 1.0) * PEAK_CHAINS * (double)iters * (double)blocks * PEAK_THREADS;
}

}  // namespace ml
