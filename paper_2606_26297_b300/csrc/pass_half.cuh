// Half-block layout of the reverse cost-layer pass: a CTA of 128 threads owns
// 2^12 amplitudes (one half of a 2^13 block), so that two CTAs share an SM
// (each with its own TMA stage, table stage and transpose buffer, 112 KB of
// shared memory) and their phases - shared-memory transposes, FMA-bound
// butterflies and X-terms, the cost phase - overlap instead of running in
// lock step as the eight warps of one CTA do.
//
// 12 local bits.  Low group (type 0): local bit i = global bit i; the group
// mixes bits 0..9 and the two warp bits are 10, 11 (the 13-bit arrangements
// without bit 12).  High group (type 1): local bits 0, 1 = global bits 0, 1
// (carried), local bits 2..6 = window A (global loA..loA+4), local bits
// 7..11 = window B (global loB..loB+4); global bit 2 is the lowest bit of the
// unit index, so the two halves of a 2^13 block are neighbouring units (their
// 32-byte rows of lambda meet in L2 before they are written back).
//   type 1  X: lanes {0,1,2,3,4}  regs {7..11}  warps {5,6}
//           Y: lanes {0,1,7,8,9}  regs {2..6}   warps {10,11}
// The (psi, lambda) stage is in natural local order, read in X (32
// consecutive 16-byte elements per warp); the table stage of a high group is
// copied with its dimensions in the order (bits 0,1) x window B x window A,
// which makes the reads of arrangement Y, where the cost phase is applied,
// 32 consecutive int32 per warp.
#pragma once

#include "pass_common.cuh"

namespace qaoa {
namespace half {

constexpr int BITS = 12;
constexpr int THREADS = 128;
constexpr int WARPS = THREADS / 32;

template <int T, int A>
__device__ __forceinline__ constexpr int regbit(int i) {
    return T == 0 ? qaoa::regbit<0, A>(i) : (A == 0 ? 7 + i : 2 + i);
}

template <int T, int A>
__device__ __forceinline__ constexpr uint32_t local_idx(uint32_t l, uint32_t m, uint32_t w) {
    return T == 0 ? qaoa::local_idx<0, A>(l, m, w)
                  : (A == 0 ? (l | (w << 5) | (m << 7)) : ((l & 3u) | ((l >> 2) << 7) | (m << 2) | (w << 10)));
}

// XOR swizzle of the transpose buffer, linear over GF(2).  Type 1: the
// half-warp of arrangement X varies local bits 0..3, that of Y bits 0, 1, 7,
// 8; folding bits 7, 8 into bits 2, 3 gives 16 distinct 8-byte slots mod 16
// in both.  Type 0: the 13-bit swizzle (it touches bits below 10 only).
template <int T>
__device__ __forceinline__ constexpr uint32_t swz(uint32_t e) {
    return T == 0 ? qaoa::swz<0>(e) : (e ^ (((e >> 7) & 3u) << 2));
}

template <int T>
__device__ __forceinline__ constexpr uint32_t full_mask() {
    return T == 0 ? 0x3FFu : 0xFFCu;
}

// global element offset of local index e relative to the unit base
template <int T>
__device__ __forceinline__ size_t goff(uint32_t e, int loA, int loB) {
    return T == 0 ? (size_t)e
                  : ((size_t)(e & 3u) | ((size_t)((e >> 2) & 31u) << loA) | ((size_t)(e >> 7) << loB));
}

// base index of unit b: type 0 blocks of 2^12; type 1 enumerates global bit
// 2, then bits 3..loA-1, loA+5..loB-1, loB+5..n-1
template <int T>
__device__ __forceinline__ size_t unit_base(uint32_t b, int loA, int loB) {
    if (T == 0) return (size_t)b << BITS;
    const int n1 = loA - 3, n2 = loB - loA - 5;
    const size_t b0 = b & 1u, b1 = (b >> 1) & ((1u << n1) - 1u), b2 = (b >> (1 + n1)) & ((1u << n2) - 1u),
                 b3 = b >> (1 + n1 + n2);
    return (b0 << 2) | (b1 << 3) | (b2 << (loA + 5)) | (b3 << (loB + 5));
}

// offset of the table entry of local index (l, m, w) of arrangement Y in the
// table stage: natural order for type 0, (bits 0,1) x B x A for type 1
template <int T>
__device__ __forceinline__ uint32_t cost_slot_y(uint32_t l, uint32_t m, uint32_t w) {
    return T == 0 ? qaoa::local_idx<0, 1>(l, m, w) : (l | (w << 5) | (m << 7));
}

template <int T>
__device__ __forceinline__ void xpose_barrier() {
    if constexpr (T == 0) {
        __syncwarp();  // type 0 keeps the warp bits: each warp moves only its own 1024 amplitudes
    } else {
        __syncthreads();
    }
}

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

template <int T, int A>
__device__ __forceinline__ size_t roff(int m, int loA, int loB) {
    return goff<T>(local_idx<T, A>(0u, (uint32_t)m, 0u), loA, loB);
}

// Deterministic block sum of the first K of NSLOT FP32 values over the four
// warps: warp sums as FP32 TwoSum pairs, then the warps' pairs in FP64 in
// index order.  red: shared [WARPS][NSLOT] pairs.  Writes out[blk*NSLOT+s].
template <int K>
__device__ __forceinline__ void block_sum_write_pairs(const float *val, float2 (*red)[NSLOT], double *out,
                                                      uint32_t blk) {
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < K; ++s) {
        const float2 p = warp_sum_pair(val[s]);
        if (l == 0) red[w][s] = p;
    }
    __syncthreads();
    if (threadIdx.x < NSLOT) {
        double t = 0.0;
        if ((int)threadIdx.x < K) {
#pragma unroll
            for (int k = 0; k < WARPS; ++k) {
                const float2 p = red[k][threadIdx.x];
                t += (double)p.x + (double)p.y;
            }
        }
        out[(size_t)blk * NSLOT + threadIdx.x] = t;
    }
}

// The same sums with FP64 warp shuffles (the pair form spills in the
// register-bound forms whose group does not fill the block).
__device__ __forceinline__ void block_sum_write_f64(const float *val, double (*red)[NSLOT], double *out,
                                                    uint32_t blk) {
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        double x = (double)val[s];
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (l == 0) red[w][s] = x;
    }
    __syncthreads();
    if (threadIdx.x < NSLOT) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < WARPS; ++k) t += red[k][threadIdx.x];
        out[(size_t)blk * NSLOT + threadIdx.x] = t;
    }
}

}  // namespace half
}  // namespace qaoa
