// Measurement of a statevector by shots (the shot-based objective of Sec. 3.4
// and the final evaluation of Sec. 3.6), as inverse-CDF sampling on exact
// integer weights:
//   q_x = floor(re^2 2^60) + floor(im^2 2^60) (exact squares), Q = sum q_x,
//   shot s: T = floor(R_s Q / 2^64), x_s = min { x : q_0 + ... + q_x > T }.
// The weights use integer arithmetic only (the FP64 pipe of this GPU is a
// small fraction of its integer rate), and integer prefix sums are exact, so
// the blocked order used here gives the same x_s as a sequential scan.  Three
// launches per request:
//   1. weights: one CTA per super-chunk (64 chunks of 256 amplitudes), chunk
//      sums and their inclusive prefix inside the super-chunk, super totals;
//   2. scan: one CTA per item, exclusive prefix of the super totals and Q;
//   3. shots: one warp per shot, a 32-ary search over the super prefixes, a
//      ballot over the 64 chunk prefixes and a warp scan inside the chunk.
// Traffic: one read of the state for (1), one chunk (2 KB) per shot for (3).
#include "kernels_misc.h"
#include "philox.cuh"

namespace qaoa {

namespace {

constexpr int SAMPLE_THREADS = 256;

struct Geo {
    unsigned long long N;
    int ch;      // amplitudes per chunk
    int cps;     // chunks per super-chunk
    int per;     // amplitudes per lane inside a chunk
    long long nsuper;
};

__host__ __device__ inline Geo geo_of(int n) {
    Geo g;
    g.N = 1ull << n;
    g.ch = n >= 8 ? 256 : (1 << n);
    const unsigned long long chunks = g.N / (unsigned long long)g.ch;
    g.cps = chunks >= 64 ? 64 : (int)chunks;
    g.per = g.ch >= 32 ? g.ch / 32 : 1;
    g.nsuper = (long long)(chunks / (unsigned long long)g.cps);
    return g;
}

// Logical right shift of a 32-bit word; shifts of 32 or more give 0.
__device__ __forceinline__ uint32_t shr_clamped(uint32_t x, uint32_t n) {
    uint32_t r;
    asm("shr.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(n));
    return r;
}

// floor(v^2 2^60) for |v| < 2.  With the exponent field E and the 24-bit
// mantissa M (leading 1 included), v = M 2^(E - 150); m8 = M 2^8 < 2^32 is
// the value's bits shifted left by 8 with the top bit set (the shift drops the
// sign and all but the lowest exponent bit, which the top bit overwrites), so
// v^2 2^60 = m8^2 / 2^s with s = 256 - 2E in [2, 256] for E <= 127: one
// 32 x 32 -> 64-bit square and one right shift on its 32-bit halves, where a
// shift of 32 or more clears a word (so |v| < 2^-30, E <= 96, s >= 64, zeros
// and subnormals included, gives 0).  |v| >= 2 and non-finite values
// (E >= 128) lie outside the domain and give an unspecified value: the
// weights pass reports them through top_word instead.
__device__ __forceinline__ unsigned long long sq60(float v) {
    const uint32_t b = __float_as_uint(v);
    const uint32_t m8 = (b << 8) | 0x80000000u;
    const uint32_t E = (b << 1) >> 24;
    const uint32_t s = 256u - 2u * E;
    const unsigned long long w = (unsigned long long)m8 * m8;
    const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
    const uint32_t rlo = s >= 32u ? shr_clamped(hi, s - 32u) : __funnelshift_r(lo, hi, s);
    const uint32_t rhi = shr_clamped(hi, s);
    return ((unsigned long long)rhi << 32) | rlo;
}

__device__ __forceinline__ unsigned long long sq60(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    const int E = (int)(u >> 52);
    const unsigned long long M = E ? ((u & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : (u & 0xFFFFFFFFFFFFFull);
    const int sh = 2 * (E ? E - 1075 : -1074) + 60;  // M^2 < 2^106 as (hi, lo)
    const unsigned long long lo = M * M, hi = __umul64hi(M, M);
    if (sh > -44) return 1ull << 62;
    const int r = -sh;
    if (r >= 128) return 0ull;
    if (r >= 64) return hi >> (r - 64);
    return (lo >> r) | (hi << (64 - r));
}

template <typename E>
__device__ __forceinline__ unsigned long long weight_of(const E &a) {
    return sq60(a.x) + sq60(a.y);
}

// The 32-bit word that holds the top exponent bit of a component, at bit 30:
// it is set exactly when |v| >= 2, v infinite or NaN (float: the value's bits;
// double: their high word).
__device__ __forceinline__ uint32_t top_word(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint32_t top_word(double v) { return (uint32_t)(__double_as_longlong(v) >> 32); }
constexpr uint32_t TOP_EXPONENT_BIT = 0x40000000u;

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// This lane's part of the weight sum of one chunk of ch amplitudes (a warp
// covers the chunk); ORs the components' top words into *top.
template <typename E>
__device__ __forceinline__ unsigned long long lane_chunk_sum(const E *p, int ch, int lane, uint32_t *top) {
    unsigned long long s = 0;
    uint32_t t = 0;
    if constexpr (sizeof(E) == 8) {
        if (ch == 256) {  // complex64: two amplitudes per 16-byte load
            const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 v = p4[lane + 32 * j];
                s += (sq60(v.x) + sq60(v.y)) + (sq60(v.z) + sq60(v.w));
                t |= (top_word(v.x) | top_word(v.y)) | (top_word(v.z) | top_word(v.w));
            }
            *top |= t;
            return s;
        }
    }
    if (ch >= 32) {
#pragma unroll 8
        for (int j = 0; j < ch / 32; ++j) {
            const E a = p[lane + 32 * j];
            s += weight_of(a);
            t |= top_word(a.x) | top_word(a.y);
        }
    } else if (lane < ch) {
        const E a = p[lane];
        s = weight_of(a);
        t = top_word(a.x) | top_word(a.y);
    }
    *top |= t;
    return s;
}

template <typename E>
__global__ void __launch_bounds__(SAMPLE_THREADS) sample_weights_kernel(const SampleItem *__restrict__ items,
                                                                        unsigned int *status) {
    const SampleItem &it = items[blockIdx.y];
    const Geo g = geo_of(it.n);
    if ((long long)blockIdx.x >= g.nsuper) return;
    __shared__ unsigned long long cs[64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const E *amps = static_cast<const E *>(it.amps);
    const unsigned long long sbase = (unsigned long long)blockIdx.x * g.cps * g.ch;
    uint32_t top = 0;
    for (int c = warp; c < g.cps; c += SAMPLE_THREADS / 32) {
        const E *p = amps + sbase + (unsigned long long)c * g.ch;
        const unsigned long long s = warp_sum(lane_chunk_sum(p, g.ch, lane, &top));
        if (lane == 0) cs[c] = s;
    }
    if (top & TOP_EXPONENT_BIT) atomicOr(status, 4u);  // a component outside |v| < 2
    __syncthreads();
    if (warp == 0) {
        const unsigned long long a = 2 * lane < g.cps ? cs[2 * lane] : 0ull;
        const unsigned long long b = 2 * lane + 1 < g.cps ? cs[2 * lane + 1] : 0ull;
        const unsigned long long incl = warp_incl_scan(a + b, lane);
        const unsigned long long excl = incl - a - b;
        unsigned long long *out = it.chunk + (unsigned long long)blockIdx.x * g.cps;
        if (2 * lane < g.cps) out[2 * lane] = excl + a;
        if (2 * lane + 1 < g.cps) out[2 * lane + 1] = incl;
        if (lane == 31) it.sup[blockIdx.x] = incl;
    }
}

// One CTA per item: exclusive prefix of the super totals (in place) and Q.
__global__ void __launch_bounds__(1024) sample_scan_kernel(const SampleItem *__restrict__ items) {
    const SampleItem &it = items[blockIdx.x];
    const Geo g = geo_of(it.n);
    __shared__ unsigned long long wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long per = (g.nsuper + 1023) / 1024;
    const long long lo = (long long)t * per;
    const long long hi = lo + per < g.nsuper ? lo + per : g.nsuper;
    unsigned long long s = 0;
    for (long long i = lo; i < hi; ++i) s += it.sup[i];
    const unsigned long long incl = warp_incl_scan(s, lane);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = wsum[lane];
        const unsigned long long wi = warp_incl_scan(w, lane);
        wsum[lane] = wi - w;
    }
    __syncthreads();
    unsigned long long run = wsum[warp] + incl - s;
    for (long long i = lo; i < hi; ++i) {
        const unsigned long long v = it.sup[i];
        it.sup[i] = run;
        run += v;
    }
    if (t == 1023) *it.total = run;
}

template <typename E>
__global__ void __launch_bounds__(SAMPLE_THREADS) sample_shot_kernel(const SampleItem *__restrict__ items,
                                                                     unsigned int *status) {
    const SampleItem &it = items[blockIdx.y];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ long long tsum[SAMPLE_THREADS / 32];
    long long tv = 0;  // this warp's sum of table values
    // one warp per shot, grid-strided (a launch holds at most 2^22 CTAs)
    for (long long s = (long long)blockIdx.x * (SAMPLE_THREADS / 32) + warp; s < it.shots;
         s += (long long)gridDim.x * (SAMPLE_THREADS / 32)) {
        const Geo g = geo_of(it.n);
        const unsigned long long Q = *it.total;
        const unsigned long long R = it.rand ? it.rand[s] : shot_random(it.seed, it.stream, (uint64_t)s);
        const unsigned long long T = __umul64hi(R, Q);
        // largest super-chunk whose exclusive prefix is <= T (sup[0] = 0 <= T)
        long long lo = 0, hi = g.nsuper;
        while (hi - lo > 1) {
            const long long step = (hi - lo + 31) / 32;
            const long long pos = lo + lane * step;
            const bool pred = pos < hi && it.sup[pos] <= T;
            const unsigned m = __ballot_sync(0xffffffffu, pred);
            lo += (long long)(31 - __clz(m)) * step;
            hi = lo + step < hi ? lo + step : hi;
        }
        const unsigned long long r = T - it.sup[lo];
        // first chunk of the super-chunk whose inclusive prefix exceeds r
        const unsigned long long *inc = it.chunk + (unsigned long long)lo * g.cps;
        const unsigned m1 = __ballot_sync(0xffffffffu, lane < g.cps && inc[lane] > r);
        const unsigned m2 = __ballot_sync(0xffffffffu, lane + 32 < g.cps && inc[lane + 32] > r);
        int c;
        if (m1)
            c = __ffs(m1) - 1;
        else if (m2)
            c = 32 + __ffs(m2) - 1;
        else {
            c = g.cps - 1;  // unreachable with exact sums; recorded
            if (lane == 0) atomicOr(status, 2u);
        }
        const unsigned long long r2 = r - (c ? inc[c - 1] : 0ull);
        // inside the chunk: lane l owns amplitudes [l per, (l+1) per)
        const unsigned long long base = (unsigned long long)lo * g.cps * g.ch + (unsigned long long)c * g.ch;
        const E *p = static_cast<const E *>(it.amps) + base;
        const bool act = g.ch >= 32 || lane < g.ch;
        unsigned long long ls = 0;
        if (act)
            for (int j = 0; j < g.per; ++j) ls += weight_of(p[lane * g.per + j]);
        const unsigned long long li = warp_incl_scan(ls, lane);
        const unsigned m3 = __ballot_sync(0xffffffffu, act && li > r2);
        int L = m3 ? __ffs(m3) - 1 : -1;
        if (L < 0) {
            L = (g.ch >= 32 ? 32 : g.ch) - 1;
            if (lane == 0) atomicOr(status, 2u);
        }
        unsigned long long x = 0;
        if (lane == L) {
            const unsigned long long r3 = r2 - (li - ls);
            unsigned long long acc = 0;
            int j = 0;
            for (; j < g.per - 1; ++j) {
                acc += weight_of(p[lane * g.per + j]);
                if (acc > r3) break;
            }
            x = base + (unsigned long long)(lane * g.per + j);
        }
        x = __shfl_sync(0xffffffffu, x, L);
        if (lane == 0) {
            if (it.idx) it.idx[s] = x;
            if (it.T) {
                const int32_t t = it.T[x];
                tv += t;
                if (it.tval) it.tval[s] = t;
            }
        }
    }
    if (lane == 0) tsum[warp] = tv;
    __syncthreads();
    if (threadIdx.x == 0 && it.tsum) {
        long long a = 0;
        for (int w = 0; w < SAMPLE_THREADS / 32; ++w) a += tsum[w];
        if (a) atomicAdd(reinterpret_cast<unsigned long long *>(it.tsum), (unsigned long long)a);
    }
}

}  // namespace

long long sample_chunk_count(int n) {
    const Geo g = geo_of(n);
    return g.nsuper * g.cps;
}

long long sample_super_count(int n) { return geo_of(n).nsuper; }

constexpr int MAX_GRID_Y = 65535;

cudaError_t launch_sample_weights(const SampleItem *items_dev, int count, int max_n, bool fp64,
                                  unsigned int *status, cudaStream_t st) {
    for (int o = 0; o < count; o += MAX_GRID_Y) {
        const int k = count - o < MAX_GRID_Y ? count - o : MAX_GRID_Y;
        const dim3 grid((unsigned)sample_super_count(max_n), (unsigned)k);
        if (fp64)
            sample_weights_kernel<double2><<<grid, SAMPLE_THREADS, 0, st>>>(items_dev + o, status);
        else
            sample_weights_kernel<float2><<<grid, SAMPLE_THREADS, 0, st>>>(items_dev + o, status);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
    }
    sample_scan_kernel<<<count, 1024, 0, st>>>(items_dev);
    return cudaGetLastError();
}

cudaError_t launch_sample_shots(const SampleItem *items_dev, int count, long long max_shots, bool fp64,
                                unsigned int *status, cudaStream_t st) {
    const long long per_cta = SAMPLE_THREADS / 32;
    long long ctas = (max_shots + per_cta - 1) / per_cta;
    if (ctas > (1ll << 22)) ctas = 1ll << 22;
    for (int o = 0; o < count; o += MAX_GRID_Y) {
        const int k = count - o < MAX_GRID_Y ? count - o : MAX_GRID_Y;
        const dim3 grid((unsigned)ctas, (unsigned)k);
        if (fp64)
            sample_shot_kernel<double2><<<grid, SAMPLE_THREADS, 0, st>>>(items_dev + o, status);
        else
            sample_shot_kernel<float2><<<grid, SAMPLE_THREADS, 0, st>>>(items_dev + o, status);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
    }
    return cudaSuccess;
}

}  // namespace qaoa
