// Adjoint-sweep kernels on the interleaved (psi, lambda) layout (sm_103a).
//
// The reverse sweep applies the same inverse gates to psi and to lambda
// (Sec. 2.3 gates undone layer by layer).  Storing the two states
// interleaved, one 16-byte element (psi.re, lambda.re, psi.im, lambda.im)
// per basis index, lets every butterfly and phase multiply advance both
// states with packed f32x2 FMAs: P = (psi.re, lambda.re), Q = (psi.im,
// lambda.im), and (a, b) -> (a - i t b, b - i t a) becomes
//   P_a += t Q_b,  Q_a -= t P_b,  P_b += t Q_a,  Q_b -= t P_a.
// The final forward pass (epi_pl_kernel) forms lambda = H_C psi_p and writes
// the interleaved buffer; rev_pl_kernel undoes one forward pass.  Both are
// persistent and TMA-pipelined like kernels_tma.cu, with bounded waits.
#include <cuda.h>

#include "kernels_tma.h"
#include "pass_body.cuh"
#include "tma_util.cuh"

namespace qaoa {

__device__ __forceinline__ float2 f2s(float s) { return make_float2(s, s); }

// butterflies of every mixed register bit on the packed pair (P, Q)
template <int T, int A>
__device__ __forceinline__ void round_mix_pq(float2 (&P)[32], float2 (&Q)[32], float t, uint32_t mask) {
    const float2 tt = f2s(t), nt = f2s(-t);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        if (!((mask >> regbit<T, A>(i)) & 1u)) continue;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            if (m & (1 << i)) continue;
            const int q = m | (1 << i);
            const float2 pa = P[m], qa = Q[m], pb = P[q], qb = Q[q];
            P[m] = __ffma2_rn(tt, qb, pa);
            Q[m] = __ffma2_rn(nt, pb, qa);
            P[q] = __ffma2_rn(tt, qa, pb);
            Q[q] = __ffma2_rn(nt, pa, qb);
        }
    }
}

// Im<lambda| sum_j X_j |psi> over the mixed register bits (this thread's part):
// per pair, cross(P_a, Q_b) + cross(P_b, Q_a) with cross(u, v) = u.y v.x - u.x v.y.
template <int T, int A>
__device__ __forceinline__ float xterm_pq(const float2 (&P)[32], const float2 (&Q)[32], uint32_t mask) {
    // four independent partial sums keep the FMA dependency chains short
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        if (!((mask >> regbit<T, A>(i)) & 1u)) continue;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            if (m & (1 << i)) continue;
            const int q = m | (1 << i);
            s0 = fmaf(P[m].y, Q[q].x, s0);
            s1 = fmaf(-P[m].x, Q[q].y, s1);
            s2 = fmaf(P[q].y, Q[m].x, s2);
            s3 = fmaf(-P[q].x, Q[m].y, s3);
        }
    }
    return (s0 + s1) + (s2 + s3);
}

// (P, Q) <- (P, Q) * z for a complex scalar z applied to both states
__device__ __forceinline__ void cmul_pq(float2 &P, float2 &Q, float2 z) {
    const float2 p = P, q = Q;
    P = __ffma2_rn(p, f2s(z.x), __fmul2_rn(q, f2s(-z.y)));
    Q = __ffma2_rn(p, f2s(z.y), __fmul2_rn(q, f2s(z.x)));
}

template <int T, int A>
__device__ __forceinline__ void read_stage_pq(float2 (&P)[32], float2 (&Q)[32], const float4 *stage, uint32_t l,
                                              uint32_t w) {
    const uint32_t t = local_idx<T, A>(l, 0u, w);
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const float4 e = stage[t | local_idx<T, A>(0u, (uint32_t)m, 0u)];
        P[m] = make_float2(e.x, e.y);
        Q[m] = make_float2(e.z, e.w);
    }
}

template <int T, int A>
__device__ __forceinline__ void store_pq(const float2 (&P)[32], const float2 (&Q)[32], float4 *__restrict__ p,
                                         uint32_t l, uint32_t w, int lo) {
    float4 *q = p + goff<T>(local_idx<T, A>(l, 0u, w), lo);
#pragma unroll
    for (int m = 0; m < 32; ++m) __stcs(q + roff<T, A>(m, lo), make_float4(P[m].x, P[m].y, Q[m].x, Q[m].y));
}

template <int T, bool TWO>
__device__ __forceinline__ void issue_pl(uint32_t b, const PassArgs &a, const CUtensorMap *map, void *stage,
                                         unsigned long long *mbar) {
    // TWO: the interleaved (psi, lambda) block, 128 KB; else the psi block, 64 KB
    const uint32_t bytes = TWO ? 131072u : 65536u;
    mbar_expect_tx(mbar, bytes);
    if (T == 0) {
        const void *src = TWO ? (const void *)(a.pl + ((size_t)b << 13)) : (const void *)(a.psi + ((size_t)b << 13));
        bulk_load(stage, src, bytes, mbar);
    } else {
        const int nlow = a.lo - 3;
        tma_load_5d(stage, map, (int)(b & ((1u << nlow) - 1u)), (int)(b >> nlow), mbar);
    }
}

template <int T>
__device__ __forceinline__ void issue_cost2(uint32_t b, const PassArgs &a, const CUtensorMap *mcost, int32_t *cstage,
                                            unsigned long long *mbar) {
    mbar_expect_tx(mbar, 8192u * 4u);
    if (T == 0) {
        bulk_load(cstage, a.C + ((size_t)b << 13), 32768u, mbar);
    } else {
        const int nlow = a.lo - 3;
        tma_load_5d(cstage, mcost, (int)(b & ((1u << nlow) - 1u)), (int)(b >> nlow), mbar);
    }
}

// ---------------------------------------------------------------------------
// final forward pass of a gradient evaluation: psi_in -> psi_p = RX_G psi_in;
// E partials, top-K, lambda = H_C psi_p; X-terms of beta_p for group G; undo
// RX_G on (psi, lambda) and write the interleaved (psi_in, lambda_in).
// slots: 0 = sum P T, 1 = sum P, 2 = X-term (Y), 3 = X-term (X)
// ---------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(PASS_THREADS, 1)
    epi_pl_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpsi, const __grid_constant__ CUtensorMap mcost,
                  int nblocks, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *stage = reinterpret_cast<float2 *>(smraw);                 // psi block, 64 KB
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 65536);      // table block, 32 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 65536 + 32768);  // transposes, 64 KB
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    __shared__ double red[PASS_THREADS / 32][NSLOT];
    __shared__ unsigned long long smk[8 * 16];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t fm = a.pre.flip ? a.mask : 0u;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&mbarc, 1);
    }
    __syncthreads();
    uint32_t parity = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nblocks) {
        issue_pl<T, false>(blockIdx.x, a, &mpsi, stage, &mbar);
        issue_cost2<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }
    for (uint32_t b = blockIdx.x; (int)b < nblocks; b += gridDim.x) {
        const size_t base = block_base<T>(b, a.lo);
        float2 v[32];
        if (!stage_ready(&mbar, parity, status)) return;
        parity ^= 1u;
        read_stage<T, 0>(v, stage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
            fence_proxy_async();
            issue_pl<T, false>(b + gridDim.x, a, &mpsi, stage, &mbar);
        }
        round_mix<T, 0>(v, a.pre, a.mask);
        transpose1<T, 0, 1>(v, xbuf, l, w, fm);
        round_mix<T, 1>(v, a.pre, a.mask);
        int32_t c[32];
        if (!stage_ready(&mbarc, parc, status)) return;
        parc ^= 1u;
        read_cost_stage<T, 1>(c, cstage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
            fence_proxy_async();
            issue_cost2<T>(b + gridDim.x, a, &mcost, cstage, &mbarc);
        }
        // psi_p = kend * v; lambda = (T 2^-s) psi_p
        float2 P[32], Q[32];
        float e0 = 0.f, e1 = 0.f;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
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
            const size_t xthread = base + goff<T>(local_idx<T, 1>(l, 0u, w), a.lo);
            block_topk<T, 1>(v, xthread, a.lo, a.ktop, a.topk_keys + (size_t)b * a.ktop, smk);
        }
        const float x1 = xterm_pq<T, 1>(P, Q, a.mask);
        round_mix_pq<T, 1>(P, Q, -a.pre.t, a.mask);
        transpose1<T, 1, 0>(P, xbuf, l, w, fm);
        transpose1<T, 1, 0>(Q, xbuf, l, w, fm);
        const float x0 = xterm_pq<T, 0>(P, Q, a.mask);
        round_mix_pq<T, 0>(P, Q, -a.pre.t, a.mask);
#pragma unroll
        for (int m = 0; m < 32; ++m) cmul_pq(P[m], Q[m], a.kend2);
        store_pq<T, 0>(P, Q, a.pl + base, l, w, a.lo);
        double vals[NSLOT] = {(double)e0, (double)e1, (double)x1, (double)x0, 0.0};
        block_sum_write(vals, red, a.partials, b);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// reverse pass on the interleaved buffer; slots as in kernels_pass.cu
// ---------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(PASS_THREADS, 1)
    rev_pl_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpl, const __grid_constant__ CUtensorMap mcost,
                  int nblocks, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float4 *stage = reinterpret_cast<float4 *>(smraw);                  // (psi, lambda) block, 128 KB
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 131072);      // table block, 32 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 131072 + 32768);  // transposes, 64 KB
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    __shared__ double red[PASS_THREADS / 32][NSLOT];
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
        issue_pl<T, true>(blockIdx.x, a, &mpl, stage, &mbar);
        if (a.has_cost) issue_cost2<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }
    for (uint32_t b = blockIdx.x; (int)b < nblocks; b += gridDim.x) {
        const size_t base = block_base<T>(b, a.lo);
        float2 P[32], Q[32];
        float acc[NSLOT] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (!stage_ready(&mbar, parity, status)) return;
        parity ^= 1u;
        if (post) read_stage_pq<T, 0>(P, Q, stage, l, w);
        else read_stage_pq<T, 1>(P, Q, stage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
            fence_proxy_async();
            issue_pl<T, true>(b + gridDim.x, a, &mpl, stage, &mbar);
        }
        if (post) {
            acc[0] = xterm_pq<T, 0>(P, Q, a.mask);
            round_mix_pq<T, 0>(P, Q, -a.post.t, a.mask);
            transpose1<T, 0, 1>(P, xbuf, l, w, fb);
            transpose1<T, 0, 1>(Q, xbuf, l, w, fb);
            acc[1] = xterm_pq<T, 1>(P, Q, a.mask);
            round_mix_pq<T, 1>(P, Q, -a.post.t, a.mask);
        }
        if (a.has_cost) {
            int32_t c[32];
            if (!stage_ready(&mbarc, parc, status)) return;
            parc ^= 1u;
            read_cost_stage<T, 1>(c, cstage, l, w);
            __syncthreads();
            if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
                fence_proxy_async();
                issue_cost2<T>(b + gridDim.x, a, &mcost, cstage, &mbarc);
            }
            float g = 0.f;
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                // Im(conj(lambda) psi) = lambda.re psi.im - lambda.im psi.re
                g = fmaf((float)c[m], fmaf(P[m].y, Q[m].x, -Q[m].y * P[m].x), g);
                cmul_pq(P[m], Q[m], cost_phase(c[m], a.phi, a.off, a.kmag, a.precise_phase));
            }
            acc[2] = g;
        }
        if (pre) {
            acc[3] = xterm_pq<T, 1>(P, Q, a.mask);
            round_mix_pq<T, 1>(P, Q, -a.pre.t, a.mask);
            transpose1<T, 1, 0>(P, xbuf, l, w, fa);
            transpose1<T, 1, 0>(Q, xbuf, l, w, fa);
            acc[4] = xterm_pq<T, 0>(P, Q, a.mask);
            round_mix_pq<T, 0>(P, Q, -a.pre.t, a.mask);
            if (a.store_psi) {
                if (!a.has_cost) {
#pragma unroll
                    for (int m = 0; m < 32; ++m) cmul_pq(P[m], Q[m], a.kend);
                }
                store_pq<T, 0>(P, Q, a.pl + base, l, w, a.lo);
            }
        } else if (a.store_psi) {
            if (!a.has_cost) {
#pragma unroll
                for (int m = 0; m < 32; ++m) cmul_pq(P[m], Q[m], a.kend);
            }
            store_pq<T, 1>(P, Q, a.pl + base, l, w, a.lo);
        }
        double vals[NSLOT];
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) vals[s] = (double)acc[s];
        block_sum_write(vals, red, a.partials, b);
        __syncthreads();
    }
}

template <typename K>
static cudaError_t set_smem2(K kern, int bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_epi_pl(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
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
        if ((e = set_smem2(epi_pl_kernel<0>, smem))) return e;
        epi_pl_kernel<0><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nblocks, status);
    } else {
        if ((e = set_smem2(epi_pl_kernel<1>, smem))) return e;
        epi_pl_kernel<1><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nblocks, status);
    }
    return cudaGetLastError();
}

cudaError_t launch_rev_pl(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
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
        if ((e = set_smem2(rev_pl_kernel<0>, smem))) return e;
        rev_pl_kernel<0><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nblocks, status);
    } else {
        if ((e = set_smem2(rev_pl_kernel<1>, smem))) return e;
        rev_pl_kernel<1><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nblocks, status);
    }
    return cudaGetLastError();
}

}  // namespace qaoa
