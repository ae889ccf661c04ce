// 512-thread TMA-pipelined persistent layer passes (sm_103a): forward pass,
// final forward pass of a gradient evaluation (writes the interleaved
// (psi, lambda) buffer), and reverse pass on that buffer.  Same method and
// fusion as kernels_tma.cu / kernels_rev2.cu (Eq. qaoa_state with boundary
// fusion; adjoint sweep), with 16 amplitudes per thread and three register
// rounds per mixer (see pass3.cuh), so that 16 warps per SM hide latency.
#include <cuda.h>

#include "kernels_tma.h"
#include "pass3.cuh"
#include "tma_util.cuh"

namespace qaoa {

template <int T>
__device__ __forceinline__ void issue_psi3(uint32_t b, const PassArgs &a, const CUtensorMap *m, void *stage,
                                           unsigned long long *mbar) {
    mbar_expect_tx(mbar, 65536u);
    if (T == 0) {
        bulk_load(stage, a.psi + ((size_t)b << 13), 65536u, mbar);
    } else {
        const int nlow = a.lo - 3;
        tma_load_5d(stage, m, (int)(b & ((1u << nlow) - 1u)), (int)(b >> nlow), mbar);
    }
}

template <int T>
__device__ __forceinline__ void issue_pl3(uint32_t b, const PassArgs &a, const CUtensorMap *m, void *stage,
                                          unsigned long long *mbar) {
    mbar_expect_tx(mbar, 131072u);
    if (T == 0) {
        bulk_load(stage, a.pl + ((size_t)b << 13), 131072u, mbar);
    } else {
        const int nlow = a.lo - 3;
        tma_load_5d(stage, m, (int)(b & ((1u << nlow) - 1u)), (int)(b >> nlow), mbar);
    }
}

template <int T>
__device__ __forceinline__ void issue_cost3(uint32_t b, const PassArgs &a, const CUtensorMap *m, int32_t *cstage,
                                            unsigned long long *mbar) {
    mbar_expect_tx(mbar, 32768u);
    if (T == 0) {
        bulk_load(cstage, a.C + ((size_t)b << 13), 32768u, mbar);
    } else {
        const int nlow = a.lo - 3;
        tma_load_5d(cstage, m, (int)(b & ((1u << nlow) - 1u)), (int)(b >> nlow), mbar);
    }
}

// ---------------------------------------------------------------------------
// forward pass: [RX_G(beta_a)] [U_C(gamma)] [RX_G(beta_b)] on psi (in place)
// ---------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(V3_THREADS, 1)
    fwd3_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpsi, const __grid_constant__ CUtensorMap mcost,
                int nblocks, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *stage = reinterpret_cast<float2 *>(smraw);                 // psi block, 64 KB
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 65536);      // table block, 32 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 65536 + 32768);  // transposes, 64 KB
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const bool pre = a.pre.mode != 0, post = a.post.mode != 0, load = !a.init, usec = a.has_cost != 0;
    const uint32_t fa = a.pre.flip ? a.mask : 0u, fb = a.post.flip ? a.mask : 0u;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&mbarc, 1);
    }
    __syncthreads();
    uint32_t parity = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nblocks) {
        if (load) issue_psi3<T>(blockIdx.x, a, &mpsi, stage, &mbar);
        if (usec) issue_cost3<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }
    for (uint32_t b = blockIdx.x; (int)b < nblocks; b += gridDim.x) {
        const size_t base = block_base<T>(b, a.lo);
        float2 v[16];
        if (load) {
            if (!stage_ready(&mbar, parity, status)) return;
            parity ^= 1u;
            if (pre) read_stage3<T, 0>(v, stage, l, w);
            else read_stage3<T, 2>(v, stage, l, w);
            __syncthreads();
            if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
                fence_proxy_async();
                issue_psi3<T>(b + gridDim.x, a, &mpsi, stage, &mbar);
            }
        } else {
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = make_float2(a.amp0, 0.f);
        }
        if (pre) {
            round3<T, 0>(v, a.pre.t, a.mask);
            transpose3<T, 0, 1>(v, xbuf, l, w, fa);
            round3<T, 1>(v, a.pre.t, a.mask);
            transpose3<T, 1, 2>(v, xbuf, l, w, 0u);
            round3<T, 2>(v, a.pre.t, a.mask);
        }
        // arrangement C
        if (usec) {
            int32_t c[16];
            if (!stage_ready(&mbarc, parc, status)) return;
            parc ^= 1u;
            read_cost3<T, 2>(c, cstage, l, w);
            __syncthreads();
            if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
                fence_proxy_async();
                issue_cost3<T>(b + gridDim.x, a, &mcost, cstage, &mbarc);
            }
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = cmul(v[m], cost_phase(c[m], a.phi, a.off, a.kmag, a.precise_phase));
        }
        if (post) {
            round3<T, 2>(v, a.post.t, a.mask);
            transpose3<T, 2, 1>(v, xbuf, l, w, fb);
            round3<T, 1>(v, a.post.t, a.mask);
            transpose3<T, 1, 0>(v, xbuf, l, w, 0u);
            round3<T, 0>(v, a.post.t, a.mask);
            if (!usec) {
#pragma unroll
                for (int m = 0; m < 16; ++m) v[m] = cmul(v[m], a.kend);
            }
            store3<T, 0>(v, a.psi + base, l, w, a.lo);
        } else {
            if (!usec) {
#pragma unroll
                for (int m = 0; m < 16; ++m) v[m] = cmul(v[m], a.kend);
            }
            store3<T, 2>(v, a.psi + base, l, w, a.lo);
        }
    }
}

// ---------------------------------------------------------------------------
// final forward pass of a gradient evaluation.  slots: 0 = sum P T, 1 = sum P,
// 2..4 = X-terms of beta_p in arrangements C, B, A.
// ---------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(V3_THREADS, 1)
    epi3_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpsi, const __grid_constant__ CUtensorMap mcost,
                int nblocks, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *stage = reinterpret_cast<float2 *>(smraw);
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 65536);
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 65536 + 32768);
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    __shared__ double red[V3_THREADS / 32][NSLOT];
    __shared__ unsigned long long smk[16 * 16];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t fa = a.pre.flip ? a.mask : 0u;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&mbarc, 1);
    }
    __syncthreads();
    uint32_t parity = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nblocks) {
        issue_psi3<T>(blockIdx.x, a, &mpsi, stage, &mbar);
        issue_cost3<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }
    for (uint32_t b = blockIdx.x; (int)b < nblocks; b += gridDim.x) {
        const size_t base = block_base<T>(b, a.lo);
        float2 v[16];
        if (!stage_ready(&mbar, parity, status)) return;
        parity ^= 1u;
        read_stage3<T, 0>(v, stage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
            fence_proxy_async();
            issue_psi3<T>(b + gridDim.x, a, &mpsi, stage, &mbar);
        }
        round3<T, 0>(v, a.pre.t, a.mask);
        transpose3<T, 0, 1>(v, xbuf, l, w, fa);
        round3<T, 1>(v, a.pre.t, a.mask);
        transpose3<T, 1, 2>(v, xbuf, l, w, 0u);
        round3<T, 2>(v, a.pre.t, a.mask);
        int32_t c[16];
        if (!stage_ready(&mbarc, parc, status)) return;
        parc ^= 1u;
        read_cost3<T, 2>(c, cstage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
            fence_proxy_async();
            issue_cost3<T>(b + gridDim.x, a, &mcost, cstage, &mbarc);
        }
        float2 P[16], Q[16];
        float e0 = 0.f, e1 = 0.f;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            v[m] = cmul(v[m], a.kend);
            const float pr = fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
            const float cf = (float)c[m];
            e0 = fmaf(pr, cf, e0);
            e1 += pr;
            const float lf = cf * a.cscale;
            P[m] = make_float2(v[m].x, v[m].x * lf);
            Q[m] = make_float2(v[m].y, v[m].y * lf);
        }
        if (a.ktop > 0) {
            const size_t xthread = base + goff<T>(local3<T, 2>(l, 0u, w), a.lo);
            block_topk3<T, 2>(v, xthread, a.lo, a.ktop, a.topk_keys + (size_t)b * a.ktop, smk);
        }
        const float x2 = xterm3<T, 2>(P, Q, a.mask);
        round3_pq<T, 2>(P, Q, -a.pre.t, a.mask);
        transpose3<T, 2, 1>(P, xbuf, l, w, fa);
        transpose3<T, 2, 1>(Q, xbuf, l, w, fa);
        const float x1 = xterm3<T, 1>(P, Q, a.mask);
        round3_pq<T, 1>(P, Q, -a.pre.t, a.mask);
        transpose3<T, 1, 0>(P, xbuf, l, w, 0u);
        transpose3<T, 1, 0>(Q, xbuf, l, w, 0u);
        const float x0 = xterm3<T, 0>(P, Q, a.mask);
        round3_pq<T, 0>(P, Q, -a.pre.t, a.mask);
#pragma unroll
        for (int m = 0; m < 16; ++m) cmul_pq3(P[m], Q[m], a.kend2);
        store3_pq<T, 0>(P, Q, a.pl + base, l, w, a.lo);
        double vals[NSLOT] = {(double)e0, (double)e1, (double)x2, (double)x1, (double)x0, 0.0, 0.0, 0.0};
        block_sum_write3(vals, red, a.partials, b);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// reverse pass on the interleaved buffer.  slots: 0..2 = X-terms of the post
// mixer (A, B, C); 3 = cost term; 4..6 = X-terms of the pre mixer (C, B, A).
// ---------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(V3_THREADS, 1)
    rev3_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpl, const __grid_constant__ CUtensorMap mcost,
                int nblocks, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float4 *stage = reinterpret_cast<float4 *>(smraw);                  // (psi, lambda) block, 128 KB
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 131072);      // table block, 32 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 131072 + 32768);  // transposes, 64 KB
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    __shared__ double red[V3_THREADS / 32][NSLOT];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const bool pre = a.pre.mode != 0, post = a.post.mode != 0;
    const uint32_t fa = a.pre.flip ? a.mask : 0u, fb = a.post.flip ? a.mask : 0u;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&mbarc, 1);
    }
    __syncthreads();
    uint32_t parity = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nblocks) {
        issue_pl3<T>(blockIdx.x, a, &mpl, stage, &mbar);
        if (a.has_cost) issue_cost3<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }
    for (uint32_t b = blockIdx.x; (int)b < nblocks; b += gridDim.x) {
        const size_t base = block_base<T>(b, a.lo);
        float2 P[16], Q[16];
        float acc[NSLOT] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (!stage_ready(&mbar, parity, status)) return;
        parity ^= 1u;
        if (post) read_stage3_pq<T, 0>(P, Q, stage, l, w);
        else read_stage3_pq<T, 2>(P, Q, stage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
            fence_proxy_async();
            issue_pl3<T>(b + gridDim.x, a, &mpl, stage, &mbar);
        }
        if (post) {
            const float t = -a.post.t;
            acc[0] = xterm3<T, 0>(P, Q, a.mask);
            round3_pq<T, 0>(P, Q, t, a.mask);
            transpose3<T, 0, 1>(P, xbuf, l, w, fb);
            transpose3<T, 0, 1>(Q, xbuf, l, w, fb);
            acc[1] = xterm3<T, 1>(P, Q, a.mask);
            round3_pq<T, 1>(P, Q, t, a.mask);
            transpose3<T, 1, 2>(P, xbuf, l, w, 0u);
            transpose3<T, 1, 2>(Q, xbuf, l, w, 0u);
            acc[2] = xterm3<T, 2>(P, Q, a.mask);
            round3_pq<T, 2>(P, Q, t, a.mask);
        }
        // arrangement C
        if (a.has_cost) {
            int32_t c[16];
            if (!stage_ready(&mbarc, parc, status)) return;
            parc ^= 1u;
            read_cost3<T, 2>(c, cstage, l, w);
            __syncthreads();
            if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
                fence_proxy_async();
                issue_cost3<T>(b + gridDim.x, a, &mcost, cstage, &mbarc);
            }
            float g0 = 0.f, g1 = 0.f;
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                // Im(conj(lambda) psi) = lambda.re psi.im - lambda.im psi.re
                const float im = fmaf(P[m].y, Q[m].x, -Q[m].y * P[m].x);
                if (m & 1) g1 = fmaf((float)c[m], im, g1);
                else g0 = fmaf((float)c[m], im, g0);
                cmul_pq3(P[m], Q[m], cost_phase(c[m], a.phi, a.off, a.kmag, a.precise_phase));
            }
            acc[3] = g0 + g1;
        }
        if (pre) {
            const float t = -a.pre.t;
            acc[4] = xterm3<T, 2>(P, Q, a.mask);
            round3_pq<T, 2>(P, Q, t, a.mask);
            transpose3<T, 2, 1>(P, xbuf, l, w, fa);
            transpose3<T, 2, 1>(Q, xbuf, l, w, fa);
            acc[5] = xterm3<T, 1>(P, Q, a.mask);
            round3_pq<T, 1>(P, Q, t, a.mask);
            transpose3<T, 1, 0>(P, xbuf, l, w, 0u);
            transpose3<T, 1, 0>(Q, xbuf, l, w, 0u);
            acc[6] = xterm3<T, 0>(P, Q, a.mask);
            round3_pq<T, 0>(P, Q, t, a.mask);
            if (a.store_psi) {
                if (!a.has_cost) {
#pragma unroll
                    for (int m = 0; m < 16; ++m) cmul_pq3(P[m], Q[m], a.kend);
                }
                store3_pq<T, 0>(P, Q, a.pl + base, l, w, a.lo);
            }
        } else if (a.store_psi) {
            if (!a.has_cost) {
#pragma unroll
                for (int m = 0; m < 16; ++m) cmul_pq3(P[m], Q[m], a.kend);
            }
            store3_pq<T, 2>(P, Q, a.pl + base, l, w, a.lo);
        }
        double vals[NSLOT];
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) vals[s] = (double)acc[s];
        block_sum_write3(vals, red, a.partials, b);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t set_smem3(K kern, int bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_fwd3(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
    const int nblocks = 1 << (a.n - BLOCK_BITS);
    const int smem = 65536 + 32768 + 65536;
    CUtensorMap m, mc;
    std::memset(&m, 0, sizeof m);
    std::memset(&mc, 0, sizeof mc);
    cudaError_t e;
    if (type == 1 && !a.init && (e = make_block_map(&m, a.psi, a.n, a.lo, 8))) return e;
    if (type == 1 && a.has_cost && (e = make_block_map(&mc, a.C, a.n, a.lo, 4))) return e;
    if (grid > nblocks) grid = nblocks;
    if (type == 0) {
        if ((e = set_smem3(fwd3_kernel<0>, smem))) return e;
        fwd3_kernel<0><<<grid, V3_THREADS, smem, st>>>(a, m, mc, nblocks, status);
    } else {
        if ((e = set_smem3(fwd3_kernel<1>, smem))) return e;
        fwd3_kernel<1><<<grid, V3_THREADS, smem, st>>>(a, m, mc, nblocks, status);
    }
    return cudaGetLastError();
}

cudaError_t launch_epi3(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
    const int nblocks = 1 << (a.n - BLOCK_BITS);
    const int smem = 65536 + 32768 + 65536;
    CUtensorMap m, mc;
    std::memset(&m, 0, sizeof m);
    std::memset(&mc, 0, sizeof mc);
    cudaError_t e;
    if (type == 1) {
        if ((e = make_block_map(&m, a.psi, a.n, a.lo, 8))) return e;
        if ((e = make_block_map(&mc, a.C, a.n, a.lo, 4))) return e;
    }
    if (grid > nblocks) grid = nblocks;
    if (type == 0) {
        if ((e = set_smem3(epi3_kernel<0>, smem))) return e;
        epi3_kernel<0><<<grid, V3_THREADS, smem, st>>>(a, m, mc, nblocks, status);
    } else {
        if ((e = set_smem3(epi3_kernel<1>, smem))) return e;
        epi3_kernel<1><<<grid, V3_THREADS, smem, st>>>(a, m, mc, nblocks, status);
    }
    return cudaGetLastError();
}

cudaError_t launch_rev3(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
    const int nblocks = 1 << (a.n - BLOCK_BITS);
    const int smem = 131072 + 32768 + 65536;
    CUtensorMap m, mc;
    std::memset(&m, 0, sizeof m);
    std::memset(&mc, 0, sizeof mc);
    cudaError_t e;
    if (type == 1) {
        if ((e = make_block_map(&m, a.pl, a.n, a.lo, 16))) return e;
        if (a.has_cost && (e = make_block_map(&mc, a.C, a.n, a.lo, 4))) return e;
    }
    if (grid > nblocks) grid = nblocks;
    if (type == 0) {
        if ((e = set_smem3(rev3_kernel<0>, smem))) return e;
        rev3_kernel<0><<<grid, V3_THREADS, smem, st>>>(a, m, mc, nblocks, status);
    } else {
        if ((e = set_smem3(rev3_kernel<1>, smem))) return e;
        rev3_kernel<1><<<grid, V3_THREADS, smem, st>>>(a, m, mc, nblocks, status);
    }
    return cudaGetLastError();
}

}  // namespace qaoa
