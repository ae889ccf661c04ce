// Register/shared-memory building blocks of a layer pass, shared by the
// direct-load kernels (kernels_pass.cu) and the TMA-pipelined persistent
// kernels (kernels_adjoint.cu).
#pragma once

#include "pass_common.cuh"

namespace qaoa {

template <int T, int A>
__device__ __forceinline__ size_t roff(int m, int loA, int loB) {
    return goff<T>(local_idx<T, A>(0u, (uint32_t)m, 0u), loA, loB);
}

template <int T, int A>
__device__ __forceinline__ void load_arr(float2 (&v)[32], const float2 *__restrict__ p, uint32_t l,
                                         uint32_t w, int loA, int loB) {
    const float2 *q = p + goff<T>(local_idx<T, A>(l, 0u, w), loA, loB);
    if (T == 0 && A == 1) {  // runs of 8 contiguous amplitudes per thread
#pragma unroll
        for (int m = 0; m < 32; m += 2) {
            const float4 t = *reinterpret_cast<const float4 *>(q + roff<T, A>(m, loA, loB));
            v[m] = make_float2(t.x, t.y);
            v[m + 1] = make_float2(t.z, t.w);
        }
    } else {
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = q[roff<T, A>(m, loA, loB)];
    }
}

template <int T, int A>
__device__ __forceinline__ void store_arr(const float2 (&v)[32], float2 *__restrict__ p, uint32_t l,
                                          uint32_t w, int loA, int loB) {
    float2 *q = p + goff<T>(local_idx<T, A>(l, 0u, w), loA, loB);
    if (T == 0 && A == 1) {
#pragma unroll
        for (int m = 0; m < 32; m += 2)
            __stcs(reinterpret_cast<float4 *>(q + roff<T, A>(m, loA, loB)),
                   make_float4(v[m].x, v[m].y, v[m + 1].x, v[m + 1].y));
    } else {
#pragma unroll
        for (int m = 0; m < 32; ++m) __stcs(q + roff<T, A>(m, loA, loB), v[m]);
    }
}

template <int T, int A>
__device__ __forceinline__ void load_cost(int32_t (&c)[32], const int32_t *__restrict__ p, uint32_t l,
                                          uint32_t w, int loA, int loB) {
    const int32_t *q = p + goff<T>(local_idx<T, A>(l, 0u, w), loA, loB);
    if (T == 0 && A == 1) {
#pragma unroll
        for (int m = 0; m < 32; m += 4) {
            const int4 t = __ldg(reinterpret_cast<const int4 *>(q + roff<T, A>(m, loA, loB)));
            c[m] = t.x;
            c[m + 1] = t.y;
            c[m + 2] = t.z;
            c[m + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int m = 0; m < 32; ++m) c[m] = __ldg(q + roff<T, A>(m, loA, loB));
    }
}

// Barrier of a shared-memory transpose.  Type 0 keeps the warp bits (local
// bits 10..12) in both arrangements, and the swizzle and the flip touch bits
// 0..9 only, so each warp writes and reads only its own 1024 slots: a warp
// barrier suffices (the kernels that hand the buffer to a TMA copy afterwards
// synchronise the block themselves).  Type 1 moves amplitudes between warps.
template <int T>
__device__ __forceinline__ void xpose_barrier() {
    if constexpr (T == 0) {
        __syncwarp();
    } else {
        __syncthreads();
    }
}

// Transpose one state from arrangement A to arrangement B through shared
// memory.  fm: local-bit mask of a bit flip X applied on the way (the
// amplitude of local index e lands at e ^ fm).  LEAD = false drops the
// barrier that keeps the writes from overtaking the previous transpose's
// reads, for call sites where a block barrier already lies between the two
// (or where the buffer has not been used yet).
template <int T, int A, int B, bool LEAD = true>
__device__ __forceinline__ void transpose1(float2 (&v)[32], float2 *sm, uint32_t l, uint32_t w, uint32_t fm) {
    if constexpr (LEAD) xpose_barrier<T>();
    const uint32_t ta = swz<T>(local_idx<T, A>(l, 0u, w) ^ fm);
#pragma unroll
    for (int m = 0; m < 32; ++m) sm[ta ^ swz<T>(local_idx<T, A>(0u, (uint32_t)m, 0u))] = v[m];
    xpose_barrier<T>();
    const uint32_t tb = swz<T>(local_idx<T, B>(l, 0u, w));
#pragma unroll
    for (int m = 0; m < 32; ++m) v[m] = sm[tb ^ swz<T>(local_idx<T, B>(0u, (uint32_t)m, 0u))];
}

template <int T, int A, int B>
__device__ __forceinline__ void transpose2(float2 (&v)[32], float2 (&u)[32], float2 *sm, uint32_t l,
                                           uint32_t w, uint32_t fm) {
    __syncthreads();
    const uint32_t ta = swz<T>(local_idx<T, A>(l, 0u, w) ^ fm);
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const uint32_t s = ta ^ swz<T>(local_idx<T, A>(0u, (uint32_t)m, 0u));
        sm[s] = v[m];
        sm[s + 8192] = u[m];
    }
    __syncthreads();
    const uint32_t tb = swz<T>(local_idx<T, B>(l, 0u, w));
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const uint32_t s = tb ^ swz<T>(local_idx<T, B>(0u, (uint32_t)m, 0u));
        v[m] = sm[s];
        u[m] = sm[s + 8192];
    }
}

// Top-K keys of |psi|^2 (P desc, index asc): key = (bits(P) << 33) | (2^33 - 1 - x),
// unique since x is.
// Running top-K (K <= 16) of one warp over the units a persistent CTA visits.
// list (shared, K keys, descending, 0 = empty) holds the warp's best keys so
// far; a unit's amplitudes are ranked only if one of them can still enter the
// list (P not below the list's K-th), which after the first few units is rare.
// scratch: shared, 2K keys.  The union of the warps' lists contains the top K
// of everything the CTA saw, whatever the order of the units.
template <int T, int A>
__device__ __forceinline__ void warp_topk_running(const float2 (&v)[32], size_t xthread, int loA, int loB, int K,
                                                  unsigned long long *list, unsigned long long *scratch) {
    const uint32_t l = threadIdx.x & 31;
    const uint32_t tp = (uint32_t)(list[K - 1] >> 33);
    uint32_t taken = 0;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const uint32_t p = __float_as_uint(fmaf(v[m].x, v[m].x, v[m].y * v[m].y));
        if (p < tp) taken |= 1u << m;
    }
    if (!__any_sync(0xffffffffu, taken != 0xFFFFFFFFu)) return;
    unsigned long long bk = 0;
    int bm = -1;
    auto scan = [&]() {
        uint32_t bp[4] = {0u, 0u, 0u, 0u};
        int bj[4] = {-1, -1, -1, -1};
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            if ((taken >> m) & 1u) continue;
            const uint32_t p = __float_as_uint(fmaf(v[m].x, v[m].x, v[m].y * v[m].y));
            if (bj[m & 3] < 0 || p > bp[m & 3]) {
                bp[m & 3] = p;
                bj[m & 3] = m;
            }
        }
        uint32_t b = bp[0];
        bm = bj[0];
#pragma unroll
        for (int j = 1; j < 4; ++j)
            if (bj[j] >= 0 && (bm < 0 || bp[j] > b || (bp[j] == b && bj[j] < bm))) {
                b = bp[j];
                bm = bj[j];
            }
        bk = 0ull;
        if (bm >= 0) {
            const unsigned long long x = xthread + goff<T>(local_idx<T, A>(0u, (uint32_t)bm, 0u), loA, loB);
            bk = ((unsigned long long)b << 33) | (0x1FFFFFFFFull - x);
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
        if (l == 0) scratch[r] = wb;
        if (bk == wb && bm >= 0) {
            taken |= 1u << bm;
            scan();
        }
    }
    __syncwarp();
    if (l == 0) {
        // merge the two descending lists into scratch[K..2K), then back
        int i = 0, j = 0;
        for (int r = 0; r < K; ++r) scratch[K + r] = list[i] >= scratch[j] ? list[i++] : scratch[j++];
        for (int r = 0; r < K; ++r) list[r] = scratch[K + r];
    }
    __syncwarp();
}

// Read 32 amplitudes of arrangement A from a TMA-staged block (natural local
// order, unswizzled).
template <int T, int A>
__device__ __forceinline__ void read_stage(float2 (&v)[32], const float2 *stage, uint32_t l, uint32_t w) {
    const uint32_t t = local_idx<T, A>(l, 0u, w);
#pragma unroll
    for (int m = 0; m < 32; ++m) v[m] = stage[t | local_idx<T, A>(0u, (uint32_t)m, 0u)];
}

// Read the 32 table entries of arrangement A from a TMA-staged block of the
// objective table (natural local order).
template <int T, int A>
__device__ __forceinline__ void read_cost_stage(int32_t (&c)[32], const int32_t *cst, uint32_t l, uint32_t w) {
    const uint32_t t = local_idx<T, A>(l, 0u, w);
    if (T == 0 && A == 1) {
#pragma unroll
        for (int m = 0; m < 32; m += 4) {
            const int4 q = *reinterpret_cast<const int4 *>(cst + (t | local_idx<T, A>(0u, (uint32_t)m, 0u)));
            c[m] = q.x;
            c[m + 1] = q.y;
            c[m + 2] = q.z;
            c[m + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int m = 0; m < 32; ++m) c[m] = cst[t | local_idx<T, A>(0u, (uint32_t)m, 0u)];
    }
}

}  // namespace qaoa
