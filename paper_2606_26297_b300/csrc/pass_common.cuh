// Device helpers shared by the layer-pass kernels: block layouts, register
// butterflies for RX(2 beta), the exact fixed-point cost phase, and
// deterministic block reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qaoa_internal.h"

namespace qaoa {

// ---------------------------------------------------------------------------
// Block layout.  A CTA owns 2^13 amplitudes ("block").  Its 13 local bits map
// to global index bits in one of two ways:
//   type 0 (low group):  local bit i  = global bit i, i < 13;
//   type 1 (high group): local bits 0..2 = global bits 0..2 (carried for
//                        coalescing), local bits 3..12 = global bits lo..lo+9.
// 256 threads hold 32 amplitudes each, in one of two arrangements: a thread's
// lane (5 bits), register slot m (5 bits) and warp (3 bits) select the local
// index.  Butterflies act on the 5 register bits; a transpose through shared
// memory swaps which local bits are register bits.
//   type 0  X: lanes {0,1,2,8,9}  regs {3..7}         warps {10,11,12}
//           Y: lanes {3..7}       regs {0,1,2,8,9}    warps {10,11,12}
//   type 1  X: lanes {0,1,2,5,6}  regs {3,4,10,11,12} warps {7,8,9}
//           Y: lanes {0..4}       regs {5..9}         warps {10,11,12}
// Every arrangement keeps global bits 0..2 in lanes or in a thread-contiguous
// run, so global accesses stay in >= 64-byte segments; the cost phase is
// applied in arrangement Y, where reading the staged table is conflict free
// (type 1) or nearly so (type 0, 16-byte reads).
// ---------------------------------------------------------------------------

template <int T, int A>
__device__ __forceinline__ constexpr int regbit(int i) {
    return T == 0 ? (A == 0 ? 3 + i : (i < 3 ? i : 5 + i))
                  : (A == 0 ? (i < 2 ? 3 + i : 8 + i) : 5 + i);
}

template <int T, int A>
__device__ __forceinline__ constexpr uint32_t local_idx(uint32_t l, uint32_t m, uint32_t w) {
    return T == 0 ? (A == 0 ? ((l & 7u) | ((l >> 3) << 8) | (m << 3) | (w << 10))
                            : ((l << 3) | (m & 7u) | ((m >> 3) << 8) | (w << 10)))
                  : (A == 0 ? ((l & 7u) | ((l >> 3) << 5) | ((m & 3u) << 3) | ((m >> 2) << 10) | (w << 7))
                            : (l | (m << 5) | (w << 10)));
}

// XOR swizzle of the shared-memory slot; linear over GF(2), and conflict free
// for 8-byte accesses in both arrangements (16 lanes of a half-warp hit 16
// distinct slots mod 16).
template <int T>
__device__ __forceinline__ constexpr uint32_t swz(uint32_t e) {
    return T == 0 ? (e ^ ((e >> 4) & 7u) ^ (((e >> 8) & 1u) << 3)) : (e ^ (((e >> 5) & 1u) << 3));
}

// Mixed-bit mask of a group that fills its block: type 0 bits 0..9, type 1
// bits 3..12 (every register bit of both arrangements is then mixed).
template <int T>
__device__ __forceinline__ constexpr uint32_t full_mask() {
    return T == 0 ? 0x3FFu : 0x1FF8u;
}

// Global element offset of local index e, relative to the block base.  Type 1:
// local bits 0..2 -> global bits 0..2, local bits 3..7 -> loA.., 8..12 -> loB..
template <int T>
__device__ __forceinline__ size_t goff(uint32_t e, int loA, int loB) {
    return T == 0 ? (size_t)e
                  : ((size_t)(e & 7u) | ((size_t)((e >> 3) & 31u) << loA) | ((size_t)(e >> 8) << loB));
}

// Base index of block b: type 1 blocks enumerate the bits outside the two
// windows and bits 0..2, lowest first (3..loA-1, loA+5..loB-1, loB+5..n-1).
template <int T>
__device__ __forceinline__ size_t block_base(uint32_t b, int loA, int loB) {
    if (T == 0) return (size_t)b << 13;
    const int n1 = loA - 3, n2 = loB - loA - 5;
    const size_t b1 = b & ((1u << n1) - 1u), b2 = (b >> n1) & ((1u << n2) - 1u), b3 = b >> (n1 + n2);
    return (b1 << 3) | (b2 << (loA + 5)) | (b3 << (loB + 5));
}

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// RX(2 beta) pair update without its common factor, tangent form:
// (a, b) <- (a - i t b, b - i t a); the true result is cos(beta) times this.
// For |sin beta| > |cos beta| the pass scalars carry t = tan(beta - pi/2) and
// a flip flag: RX(2 beta) = (-i X) RX(2 beta - pi) on every mixed qubit, and
// the bit flip X of the whole group is applied for free by the transpose
// inside the same mixer (an XOR of the shared-memory slot).
__device__ __forceinline__ void bfly_tan(float2 &a, float2 &b, float t) {
    const float2 na = make_float2(fmaf(t, b.y, a.x), fmaf(-t, b.x, a.y));
    const float2 nb = make_float2(fmaf(t, a.y, b.x), fmaf(-t, a.x, b.y));
    a = na;
    b = nb;
}

// One register round: the butterflies of every mixed register bit.  A
// register bit the group does not mix runs with t = 0, the identity, so that a
// group smaller than its block (mask known only at run time) takes no branch:
// a branch around a round's butterflies forces every amplitude back into the
// register it held before the branch, one move per value, which cost the
// partial-group forms about a third of their instructions.  With the full
// mask (a compile-time constant) the selects fold away.
template <int T, int A>
__device__ __forceinline__ void round_mix(float2 (&v)[32], float t, uint32_t mask) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float ti = ((mask >> regbit<T, A>(i)) & 1u) ? t : 0.f;
#pragma unroll
        for (int m = 0; m < 32; ++m)
            if (!(m & (1 << i))) bfly_tan(v[m], v[m | (1 << i)], ti);
    }
}

// sum over the mixed register bits j of sum_m Im(conj(u_m) v_{m^j}): the part
// of Im <lambda| sum_j X_j |psi> held by this thread in this arrangement.
template <int T, int A>
__device__ __forceinline__ float xterm(const float2 (&u)[32], const float2 (&v)[32], uint32_t mask) {
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        if (!((mask >> regbit<T, A>(i)) & 1u)) continue;
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            if (m & (1 << i)) continue;
            const int q = m | (1 << i);
            // Im(conj(u_m) v_q) + Im(conj(u_q) v_m)
            s = fmaf(u[m].x, v[q].y, s);
            s = fmaf(-u[m].y, v[q].x, s);
            s = fmaf(u[q].x, v[m].y, s);
            s = fmaf(-u[q].y, v[m].x, s);
        }
        acc += s;
    }
    return acc;
}

// exp(-2 pi i t / 2^64) * kmag for t = T * phi + off (mod 2^64).  The turn
// count is exact modular integer arithmetic; it is rounded to 32 bits
// (2^-33 turn) and then to an FP32 angle in [-pi, pi).
__device__ __forceinline__ float2 cost_phase(int32_t tq, unsigned long long phi, unsigned long long off,
                                             float kmag, int precise) {
    const unsigned long long t = (unsigned long long)(long long)tq * phi + off;
    const int32_t hi = (int32_t)((t + 0x80000000ull) >> 32);
    float s, c;
    if (precise) {
        sincospif((float)hi * 4.656612873077393e-10f, &s, &c);  // angle/pi = hi 2^-31
    } else {
        __sincosf((float)hi * 1.4629180792671596e-09f, &s, &c);  // angle = hi 2 pi 2^-32
    }
    return make_float2(c * kmag, -s * kmag);
}

static_assert(sizeof(float2) == sizeof(double), "a pair slot holds one FP64 slot");

// Sum of x over the warp as an unevaluated pair hi + lo: Knuth's TwoSum at
// every level of the butterfly keeps each addition's rounding error, so the
// pair carries the warp sum to about 2^-48 relative without FP64 instructions
// (the FP64 rate of this GPU is a small fraction of its FP32 rate).  TwoSum's
// error term is exact whatever the operand order, so every lane ends with the
// same pair.
__device__ __forceinline__ float2 warp_sum_pair(float x) {
    float hi = x, lo = 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const float s = __fadd_rn(hi, h2);
        const float bv = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(h2, bv));
        hi = s;
        lo = __fadd_rn(__fadd_rn(lo, l2), e);
    }
    return make_float2(hi, lo);
}

// Deterministic block sum of the first K of NSLOT FP32 values (the other
// slots are written as 0): warp sums as FP32 pairs (fixed shuffle tree), then
// the warps' pairs in FP64 in index order.  red: shared [8][NSLOT] pairs.
// Writes out[blk*NSLOT+s].
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
            for (int k = 0; k < PASS_THREADS / 32; ++k) {
                const float2 p = red[k][threadIdx.x];
                t += (double)p.x + (double)p.y;
            }
        }
        out[(size_t)blk * NSLOT + threadIdx.x] = t;
    }
}

// Deterministic block sum of NSLOT FP64 values (fixed shuffle tree, then warps
// in index order).  red: shared [8][NSLOT].  Writes out[blockIdx.x*NSLOT+s].
__device__ __forceinline__ void block_sum_write(double (&val)[NSLOT], double (*red)[NSLOT], double *out,
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
        for (int k = 0; k < PASS_THREADS / 32; ++k) t += red[k][threadIdx.x];
        out[(size_t)blk * NSLOT + threadIdx.x] = t;
    }
}

}  // namespace qaoa
