// Arithmetic-pipe micro-benchmarks: the sustained rate of FP32 FMA, packed
// f32x2 FMA, FP64 FMA and the sin/cos unit on this GPU, the denominators for
// kernels bound by plain arithmetic rather than by HBM.  Every thread runs 8
// independent dependency chains, so the pipe and not the latency is measured.
#include "kernels_misc.h"

namespace qaoa {

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 8;

template <int KIND>
__global__ void __launch_bounds__(PEAK_THREADS) peak_kernel(float *out, int iters, float seed) {
    const float x = seed + 1e-7f * threadIdx.x, y = 0.5f;
    if (KIND == 0) {
        float a[PEAK_CHAINS];
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = x + c;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = fmaf(a[c], x, y);
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) s += a[c];
        if (s == 12345.f) out[threadIdx.x] = s;
    } else if (KIND == 1) {
        float2 a[PEAK_CHAINS];
        const float2 xx = make_float2(x, x + 1e-3f), yy = make_float2(y, y);
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = make_float2(x + c, x - c);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = __ffma2_rn(a[c], xx, yy);
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) s += a[c].x + a[c].y;
        if (s == 12345.f) out[threadIdx.x] = s;
    } else if (KIND == 2) {
        double a[PEAK_CHAINS];
        const double xd = x, yd = y;
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = xd + c;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = fma(a[c], xd, yd);
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) s += a[c];
        if (s == 12345.0) out[threadIdx.x] = (float)s;
    } else {
        float a[PEAK_CHAINS];
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = x + 0.1f * c;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; ++c) {
                float sn, cs;
                __sincosf(a[c], &sn, &cs);
                a[c] = sn + cs;
            }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) s += a[c];
        if (s == 12345.f) out[threadIdx.x] = s;
    }
}

}  // namespace

// Operations per launch: FMAs (kinds 0, 2), FMA lane pairs (kind 1) or
// sin/cos pairs (kind 3), per thread iters * PEAK_CHAINS.
cudaError_t launch_peak(int kind, int blocks, int iters, float *out, cudaStream_t st) {
    switch (kind) {
        case 0: peak_kernel<0><<<blocks, PEAK_THREADS, 0, st>>>(out, iters, 1.0001f); break;
        case 1: peak_kernel<1><<<blocks, PEAK_THREADS, 0, st>>>(out, iters, 1.0001f); break;
        case 2: peak_kernel<2><<<blocks, PEAK_THREADS, 0, st>>>(out, iters, 1.0001f); break;
        default: peak_kernel<3><<<blocks, PEAK_THREADS, 0, st>>>(out, iters, 0.3f); break;
    }
    return cudaGetLastError();
}

double peak_ops_per_launch(int blocks, int iters) { return (double)blocks * PEAK_THREADS * iters * PEAK_CHAINS; }

}  // namespace qaoa
