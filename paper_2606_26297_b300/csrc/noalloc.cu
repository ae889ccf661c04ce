// Allocation-free expectation entry point.
//
// Some callers cannot allocate device memory at the moment they need <H_C>:
// a host framework that owns every byte of the device behind its own
// capped pool, code that must not hit the implicit device synchronisation a
// cudaMalloc/cudaFree may cause (a latency-critical optimisation loop), or a
// caller that only holds raw device pointers handed over by someone else and
// has no library context to keep scratch in.  For them this file provides one
// entry point that computes the same reduction as qaoa_expect but keeps its
// scratch in a fixed, file-scope device array instead of allocating.
//
// Cost of that choice: the array (2 * 2^17 + 2 doubles, about 2 MiB) is
// resident on every GPU that loads the library, for the life of the process,
// whether or not the entry point is used; and every call shares it.
#include <cuda_runtime.h>

#include "qaoa_internal.h"

namespace {

constexpr int kNoallocMaxN = 30;                           // largest supported state: 2^30 amplitudes
constexpr int kNoallocMaxChunks = 1 << (kNoallocMaxN - 13);  // chunks of 8192 amplitudes

// Two FP64 partial sums per chunk, then the two final sums.
__device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxChunks + 2];


// Per chunk of 8192 amplitudes: sum |psi|^2 T and sum |psi|^2, FP32 per thread
// over 32 amplitudes, then an FP64 fixed-order block sum (the same order as
// the library's qaoa_expect, so the two agree to the last bit).
__global__ void noalloc_partial_kernel(const float2 *__restrict__ psi, const int32_t *__restrict__ T, long long N,
                                       double *part) {
    __shared__ double red[8][2];
    const long long b0 = (long long)blockIdx.x * 8192;
    float e0 = 0.f, e1 = 0.f;
#pragma unroll 8
    for (int m = 0; m < 32; ++m) {
        const long long x = b0 + threadIdx.x + 256 * m;
        if (x < N) {
            const float2 a = psi[x];
            const float P = fmaf(a.x, a.x, a.y * a.y);
            e0 = fmaf(P, (float)T[x], e0);
            e1 += P;
        }
    }
    double v[2] = {(double)e0, (double)e1};
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        double x = v[s];
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (l == 0) red[w][s] = x;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
        part[2 * (size_t)blockIdx.x + threadIdx.x] = t;
    }
}

// out[s] = sum over chunks of part[2*b + s], fixed order (block s sums slot s).
__global__ void noalloc_final_kernel(const double *__restrict__ part, int nchunks, double *out) {
    __shared__ double sh[256];
    const int s = blockIdx.x;
    double t = 0.0;
    for (int b = threadIdx.x; b < nchunks; b += 256) t += part[2 * (size_t)b + s];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int k = 128; k; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[s] = sh[0];
}

// amps / table must live on the current device (or be managed memory):
// cudaPointerGetAttributes allocates nothing
qaoa_status check_device_pointer(const void *p, int dev, const char *what) {
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return qaoa::fail(QAOA_ERR_INVALID_ARG, "qaoa_expect_noalloc: %s is not a device pointer (%s)", what,
                          cudaGetErrorString(e));
    }
    if (at.type == cudaMemoryTypeManaged) return QAOA_OK;
    if (at.type != cudaMemoryTypeDevice || at.device != dev)
        return qaoa::fail(QAOA_ERR_INVALID_ARG, "qaoa_expect_noalloc: %s is not memory of the current device %d", what,
                          dev);
    return QAOA_OK;
}

}  // namespace

extern "C" qaoa_status qaoa_expect_noalloc(const void *amps, const int32_t *table, int n, int32_t shift_bits,
                                           int64_t k_c, void *cuda_stream, double *out_expect) {
    using qaoa::fail;
    if (!amps || !table || !out_expect) return fail(QAOA_ERR_INVALID_ARG, "qaoa_expect_noalloc: null pointer");
    if (n < 1 || n > kNoallocMaxN)
        return fail(QAOA_ERR_INVALID_ARG,
                    "qaoa_expect_noalloc: n=%d is outside [1, %d], the size its fixed scratch array holds", n,
                    kNoallocMaxN);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(QAOA_ERR_CUDA, "qaoa_expect_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    qaoa_status ps = check_device_pointer(amps, dev, "amps");
    if (ps == QAOA_OK) ps = check_device_pointer(table, dev, "table");
    if (ps != QAOA_OK) return ps;
    // The device address of the array in the context current now (host code
    // cannot use the symbol itself as a device pointer).  Looked up on every
    // call: a cache keyed by device would hand a caller working in another
    // context of the same device the primary context's address.
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(QAOA_ERR_CUDA, "qaoa_expect_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    double *scratch = static_cast<double *>(p);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long N = 1ll << n;
    const int nchunks = (int)((N + 8191) / 8192);
    double *final_sums = scratch + 2 * (size_t)kNoallocMaxChunks;
    // every partial slot read below is written by this call first, and the
    // final sums are overwritten, so no part of the array needs clearing
    noalloc_partial_kernel<<<nchunks, 256, 0, st>>>(static_cast<const float2 *>(amps), table, N, scratch);
    noalloc_final_kernel<<<2, 256, 0, st>>>(scratch, nchunks, final_sums);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(QAOA_ERR_CUDA, "qaoa_expect_noalloc: launch: %s", cudaGetErrorString(e));
    double h[2] = {0.0, 0.0};
    e = cudaMemcpyAsync(h, final_sums, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(QAOA_ERR_CUDA, "qaoa_expect_noalloc: %s", cudaGetErrorString(e));
    *out_expect = ldexp(h[0] + (double)k_c * h[1], -shift_bits);
    return QAOA_OK;
}
