// Building blocks of the 512-thread layer passes (kernels_v3.cu).
//
// A CTA owns a 2^13-amplitude block (same block geometry as pass_common.cuh:
// type 0 = global bits 0..12; type 1 = global bits 0..2 carried + a 10-bit
// group window lo..lo+9).  512 threads hold 16 amplitudes each, so a thread
// needs at most 64 data registers even for two interleaved states and a CTA
// keeps 16 warps in flight.  A thread's lane (5 bits), register slot m
// (4 bits) and warp (4 bits) select the local index in one of three
// arrangements A, B, C; each register round mixes the qubits of one
// arrangement, and transposes through shared memory move between them:
//   type 1  A: lanes {0..4}        regs {11,12 | 5,6}  warps {7..10}   mixes 11,12
//           B: lanes {0,1,2,5,6}   regs {3,4,9,10}     warps {7,8,11,12} mixes 3,4,9,10
//           C: lanes {0..4}        regs {5..8}         warps {9..12}   mixes 5..8
//   type 0  A: lanes {0,1,2,5,6}   regs {3,4 | 7,8}    warps {9..12}   mixes 3,4
//           B: lanes {3..7}        regs {0,1,2,9}      warps {8,10,11,12} mixes 0,1,2,9
//           C: lanes {0..4}        regs {5..8}         warps {9..12}   mixes 5..8
// ("| x" = register bits carried along unmixed).  Arrangements A and C keep
// global bits 0..2 in lanes, B keeps them as a thread-contiguous run.  The
// cost phase is applied in C, where reading a staged table block is
// bank-conflict free.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pass_common.cuh"

namespace qaoa {

constexpr int V3_THREADS = 512;

template <int T, int A>
__device__ __forceinline__ constexpr uint32_t local3(uint32_t l, uint32_t m, uint32_t w) {
    return T == 1 ? (A == 2 ? (l | (m << 5) | (w << 9))
                     : A == 1 ? ((l & 7u) | ((l >> 3) << 5) | ((m & 3u) << 3) | ((m >> 2) << 9) | ((w & 3u) << 7) |
                                 ((w >> 2) << 11))
                              : (l | ((m & 3u) << 11) | ((m >> 2) << 5) | (w << 7)))
                  : (A == 2 ? (l | (m << 5) | (w << 9))
                     : A == 1 ? ((m & 7u) | ((m >> 3) << 9) | (l << 3) | ((w & 1u) << 8) | ((w >> 1) << 10))
                              : (((m & 3u) << 3) | ((m >> 2) << 7) | (l & 7u) | ((l >> 3) << 5) | (w << 9)));
}

// local bit of register bit i
template <int T, int A>
__device__ __forceinline__ constexpr int regbit3(int i) {
    return T == 1 ? (A == 2 ? 5 + i : A == 1 ? (i < 2 ? 3 + i : 7 + i) : (i < 2 ? 11 + i : 3 + i))
                  : (A == 2 ? 5 + i : A == 1 ? (i < 3 ? i : 9) : (i < 2 ? 3 + i : 5 + i));
}

// local bits that round A may mix
template <int T, int A>
__device__ __forceinline__ constexpr uint32_t round_set3() {
    return T == 1 ? (A == 0 ? 0x1800u : A == 1 ? 0x0618u : 0x01E0u) : (A == 0 ? 0x0018u : A == 1 ? 0x0207u : 0x01E0u);
}

template <int T>
__device__ __forceinline__ constexpr uint32_t swz3(uint32_t e) {
    return T == 1 ? (e ^ (((e >> 5) & 1u) << 3)) : (e ^ ((e >> 4) & 7u) ^ (((e >> 5) & 1u) << 3));
}

template <int T, int A>
__device__ __forceinline__ size_t roff3(int m, int lo) {
    return goff<T>(local3<T, A>(0u, (uint32_t)m, 0u), lo);
}

template <int T, int A>
__device__ __forceinline__ bool mixes3(uint32_t mask, int i) {
    return (mask & round_set3<T, A>() & (1u << regbit3<T, A>(i))) != 0u;
}

// ---- one state (psi) ----------------------------------------------------------

template <int T, int A>
__device__ __forceinline__ void round3(float2 (&v)[16], float t, uint32_t mask) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!mixes3<T, A>(mask, i)) continue;
#pragma unroll
        for (int m = 0; m < 16; ++m)
            if (!(m & (1 << i))) bfly_tan(v[m], v[m | (1 << i)], t);
    }
}

template <int T, int A>
__device__ __forceinline__ void read_stage3(float2 (&v)[16], const float2 *stage, uint32_t l, uint32_t w) {
    const uint32_t t = local3<T, A>(l, 0u, w);
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = stage[t | local3<T, A>(0u, (uint32_t)m, 0u)];
}

template <int T, int A>
__device__ __forceinline__ void read_cost3(int32_t (&c)[16], const int32_t *cst, uint32_t l, uint32_t w) {
    const uint32_t t = local3<T, A>(l, 0u, w);
#pragma unroll
    for (int m = 0; m < 16; ++m) c[m] = cst[t | local3<T, A>(0u, (uint32_t)m, 0u)];
}

template <int T, int A>
__device__ __forceinline__ void store3(const float2 (&v)[16], float2 *__restrict__ p, uint32_t l, uint32_t w,
                                       int lo) {
    float2 *q = p + goff<T>(local3<T, A>(l, 0u, w), lo);
#pragma unroll
    for (int m = 0; m < 16; ++m) __stcs(q + roff3<T, A>(m, lo), v[m]);
}

// transpose from arrangement A to B; fm: bit flip applied on the way
template <int T, int A, int B>
__device__ __forceinline__ void transpose3(float2 (&v)[16], float2 *sm, uint32_t l, uint32_t w, uint32_t fm) {
    __syncthreads();
    const uint32_t ta = swz3<T>(local3<T, A>(l, 0u, w) ^ fm);
#pragma unroll
    for (int m = 0; m < 16; ++m) sm[ta ^ swz3<T>(local3<T, A>(0u, (uint32_t)m, 0u))] = v[m];
    __syncthreads();
    const uint32_t tb = swz3<T>(local3<T, B>(l, 0u, w));
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = sm[tb ^ swz3<T>(local3<T, B>(0u, (uint32_t)m, 0u))];
}

// ---- two interleaved states: P = (psi.re, lambda.re), Q = (psi.im, lambda.im) ----

template <int T, int A>
__device__ __forceinline__ void round3_pq(float2 (&P)[16], float2 (&Q)[16], float t, uint32_t mask) {
    const float2 tt = make_float2(t, t), nt = make_float2(-t, -t);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!mixes3<T, A>(mask, i)) continue;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
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

// Im<lambda| sum_j X_j |psi> over the qubits round A mixes (this thread's
// part), with four independent partial sums to keep the FMA chains short.
template <int T, int A>
__device__ __forceinline__ float xterm3(const float2 (&P)[16], const float2 (&Q)[16], uint32_t mask) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!mixes3<T, A>(mask, i)) continue;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
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

__device__ __forceinline__ void cmul_pq3(float2 &P, float2 &Q, float2 z) {
    const float2 p = P, q = Q;
    P = __ffma2_rn(p, make_float2(z.x, z.x), __fmul2_rn(q, make_float2(-z.y, -z.y)));
    Q = __ffma2_rn(p, make_float2(z.y, z.y), __fmul2_rn(q, make_float2(z.x, z.x)));
}

template <int T, int A>
__device__ __forceinline__ void read_stage3_pq(float2 (&P)[16], float2 (&Q)[16], const float4 *stage, uint32_t l,
                                               uint32_t w) {
    const uint32_t t = local3<T, A>(l, 0u, w);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const float4 e = stage[t | local3<T, A>(0u, (uint32_t)m, 0u)];
        P[m] = make_float2(e.x, e.y);
        Q[m] = make_float2(e.z, e.w);
    }
}

template <int T, int A>
__device__ __forceinline__ void store3_pq(const float2 (&P)[16], const float2 (&Q)[16], float4 *__restrict__ p,
                                          uint32_t l, uint32_t w, int lo) {
    float4 *q = p + goff<T>(local3<T, A>(l, 0u, w), lo);
#pragma unroll
    for (int m = 0; m < 16; ++m) __stcs(q + roff3<T, A>(m, lo), make_float4(P[m].x, P[m].y, Q[m].x, Q[m].y));
}

// Deterministic block sum of NSLOT FP64 values over the 16 warps.
__device__ __forceinline__ void block_sum_write3(double (&val)[NSLOT], double (*red)[NSLOT], double *out,
                                                 uint32_t blk) {
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        double x = val[s];
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (l == 0) red[w][s] = x;
    }
    __syncthreads();
    if (threadIdx.x < NSLOT) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < V3_THREADS / 32; ++k) t += red[k][threadIdx.x];
        out[(size_t)blk * NSLOT + threadIdx.x] = t;
    }
}

// Top-K (K <= 16) of the block's |psi|^2 held in arrangement A; same key as
// pass_body.cuh.  smk: shared, >= 16*16 keys.
template <int T, int A>
__device__ __forceinline__ void block_topk3(const float2 (&v)[16], size_t xthread, int lo, int K,
                                            unsigned long long *out, unsigned long long *smk) {
    const uint32_t l = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t taken = 0;
    unsigned long long bk = 0;
    int bm = -1;
    auto scan = [&]() {
        bk = 0;
        bm = -1;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            if ((taken >> m) & 1u) continue;
            const float P = fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
            const unsigned long long x = xthread + roff3<T, A>(m, lo);
            const unsigned long long key = ((unsigned long long)__float_as_uint(P) << 33) | (0x1FFFFFFFFull - x);
            if (key > bk) {
                bk = key;
                bm = m;
            }
        }
    };
    scan();
    for (int r = 0; r < K; ++r) {
        unsigned long long wb = bk;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, wb, o);
            wb = t > wb ? t : wb;
        }
        if (l == 0) smk[w * 16 + r] = wb;
        if (bk == wb && bm >= 0) {
            taken |= 1u << bm;
            scan();
        }
    }
    __syncthreads();
    if (w == 0) {
        // merge the 16 sorted warp lists: lane i (< 16) walks list i
        int head = 0;
        for (int r = 0; r < K; ++r) {
            const unsigned long long mine = (l < 16 && head < K) ? smk[l * 16 + head] : 0ull;
            unsigned long long wb = mine;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const unsigned long long t = __shfl_xor_sync(0xffffffffu, wb, o);
                wb = t > wb ? t : wb;
            }
            if (mine == wb && l < 16) ++head;
            if (l == 0) out[r] = wb;
        }
    }
}

}  // namespace qaoa
