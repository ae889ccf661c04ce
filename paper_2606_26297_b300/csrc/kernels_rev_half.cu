// Reverse (adjoint) pass undoing a cost-layer forward pass, on half blocks of
// 2^12 (psi, lambda) pairs with two CTAs per SM (sm_103a).
//
// Same arithmetic as the 2^13-block form in kernels_adjoint.cu (the reverse
// sweep of Eq. qaoa_state on the interleaved (psi, lambda) buffer, with
//   dE/dbeta_l  = 2 Im <lambda| sum_j X_j |psi>  at the mixers,
//   dE/dgamma_l = 2 Im <lambda| H_C |psi>        at the cost layer),
// but a CTA holds half a block: 128 threads x 32 pairs, 112 KB of shared
// memory (64 KB (psi, lambda) stage, 16 KB table stage, 32 KB transpose
// buffer), so two independent CTAs run on each SM.  With one 256-thread CTA
// per SM every warp waits at the same block barriers and the SM alternates
// between shared-memory-bound transposes and FMA-bound butterflies; two CTAs
// drift apart and overlap them.  The layout is in pass_half.cuh.
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "pass_half.cuh"
#include "tma_util.cuh"

namespace qaoa {
namespace half {

__device__ __forceinline__ float2 f2s(float s) { return make_float2(s, s); }

// butterflies on the packed pair (P, Q); an unmixed bit runs with t = 0 (the
// identity) rather than a branch, which would pin every value to its register
template <int T, int A>
__device__ __forceinline__ void round_mix_pq(float2 (&P)[32], float2 (&Q)[32], float t, uint32_t mask) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float ti = ((mask >> regbit<T, A>(i)) & 1u) ? t : 0.f;
        const float2 tt = f2s(ti), nt = f2s(-ti);
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

// Im<lambda| sum_j X_j |psi> over the mixed register bits, one f32x2 FMA per
// ordered pair (m, m ^ e_j): cross(P_m, Q_{m^e_j}) = (P_m.y, -P_m.x) . Q_{m^e_j}
template <int T, int A>
__device__ __forceinline__ float xterm_pq(const float2 (&P)[32], const float2 (&Q)[32], uint32_t mask) {
    bool on[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) on[i] = (mask >> regbit<T, A>(i)) & 1u;
    float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const float2 r = make_float2(P[m].y, -P[m].x);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if (!on[i]) continue;
            acc[(m + i) & 3] = __ffma2_rn(r, Q[m ^ (1 << i)], acc[(m + i) & 3]);
        }
    }
    return ((acc[0].x + acc[0].y) + (acc[1].x + acc[1].y)) + ((acc[2].x + acc[2].y) + (acc[3].x + acc[3].y));
}

// the same sum as four scalar FMA chains: more instructions, shorter live
// ranges (the forms whose group does not fill the block spill with the packed one)
template <int T, int A>
__device__ __forceinline__ float xterm_pq_chains(const float2 (&P)[32], const float2 (&Q)[32], uint32_t mask) {
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

template <int T, int A, bool PACKED>
__device__ __forceinline__ float xterm_form(const float2 (&P)[32], const float2 (&Q)[32], uint32_t mask) {
    return PACKED ? xterm_pq<T, A>(P, Q, mask) : xterm_pq_chains<T, A>(P, Q, mask);
}

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

// table entries of arrangement Y from the table stage
template <int T>
__device__ __forceinline__ void read_cost_y(int32_t (&c)[32], const int32_t *cst, uint32_t l, uint32_t w) {
    const uint32_t t = cost_slot_y<T>(l, 0u, w);
    if (T == 0) {  // runs of 8 contiguous entries per thread (register bits 0..2)
#pragma unroll
        for (int m = 0; m < 32; m += 4) {
            const int4 q = *reinterpret_cast<const int4 *>(cst + (t | cost_slot_y<T>(0u, (uint32_t)m, 0u)));
            c[m] = q.x;
            c[m + 1] = q.y;
            c[m + 2] = q.z;
            c[m + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int m = 0; m < 32; ++m) c[m] = cst[t | cost_slot_y<T>(0u, (uint32_t)m, 0u)];
    }
}

template <int T, int A>
__device__ __forceinline__ void store_pq(const float2 (&P)[32], const float2 (&Q)[32], float4 *__restrict__ p,
                                         uint32_t l, uint32_t w, int loA, int loB) {
    float4 *q = p + goff<T>(local_idx<T, A>(l, 0u, w), loA, loB);
#pragma unroll
    for (int m = 0; m < 32; ++m)
        __stcs(q + roff<T, A>(m, loA, loB), make_float4(P[m].x, P[m].y, Q[m].x, Q[m].y));
}

template <int T, int A>
__device__ __forceinline__ void store_lam(const float2 (&P)[32], const float2 (&Q)[32], float2 *__restrict__ p,
                                          uint32_t l, uint32_t w, int loA, int loB) {
    float2 *q = p + goff<T>(local_idx<T, A>(l, 0u, w), loA, loB);
#pragma unroll
    for (int m = 0; m < 32; ++m) __stcs(q + roff<T, A>(m, loA, loB), make_float2(P[m].y, Q[m].y));
}

struct Unit {
    uint32_t item, b;
};
__device__ __forceinline__ Unit unit_of(uint32_t u, int nbits) { return {u >> nbits, u & ((1u << nbits) - 1u)}; }

__device__ __forceinline__ void tma_load_5d_c(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                              int c4, unsigned long long *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(mbar))
        : "memory");
}

// Coordinates of a high-group unit b of array `arr`: bits 2..loA-1 (b's low
// loA-2 bits), bits loA+5..loB-1, and the bits above window B (in units of
// the 32-wide window) with the arrays stacked.
__device__ __forceinline__ void unit_coords(uint32_t b, uint32_t arr, const PassArgs &a, int *c_lo, int *c_mid,
                                            int *c_hi) {
    const int n1 = a.loA - 2, n2 = a.loB - a.loA - 5;
    *c_lo = (int)(b & ((1u << n1) - 1u));
    *c_mid = (int)((b >> n1) & ((1u << n2) - 1u));
    *c_hi = (int)(((b >> (n1 + n2)) << 5) + (arr << (a.n - a.loB)));
}

template <int T>
__device__ __forceinline__ void issue_amps(uint32_t u, const PassArgs &a, const CUtensorMap *map, void *stage,
                                           unsigned long long *mbar) {
    const int nbits = a.n - BITS;
    const Unit un = unit_of(u, nbits);
    mbar_expect_tx(mbar, 65536u);
    if (T == 0) {
        bulk_load(stage, a.pl + ((size_t)un.item << a.n) + ((size_t)un.b << BITS), 65536u, mbar);
    } else {
        int cl, cm, ch;
        unit_coords(un.b, un.item, a, &cl, &cm, &ch);
        tma_load_5d_c(stage, map, 0, cl, 0, cm, ch, mbar);  // (bits 0,1) x lo x A x mid x (B, above)
    }
}

template <int T>
__device__ __forceinline__ void issue_table(uint32_t u, const PassArgs &a, const CUtensorMap *mcost, int32_t *cstage,
                                            unsigned long long *mbar) {
    const int nbits = a.n - BITS;
    const Unit un = unit_of(u, nbits);
    const uint32_t tab = a.item_table ? (uint32_t)a.item_table[un.item] : 0u;
    mbar_expect_tx(mbar, 16384u);
    if (T == 0) {
        bulk_load(cstage, a.C + ((size_t)tab << a.n) + ((size_t)un.b << BITS), 16384u, mbar);
    } else {
        int cl, cm, ch;
        unit_coords(un.b, tab, a, &cl, &cm, &ch);
        tma_load_5d_c(cstage, mcost, 0, ch, 0, cl, cm, mbar);  // (bits 0,1) x (B, above) x A x lo x mid
    }
}

// slots: 0,1 = X-terms of the post mixer (arrangements X, Y); 2 = cost term;
// 3,4 = X-terms of the pre mixer (Y, X).  One partial-sum row per unit.
template <int T, bool SPLIT, bool PRE, bool COST, bool POST, bool STORE, bool FULL>
__global__ void __launch_bounds__(THREADS, 2)
    rev_pass_half_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpl,
                         const __grid_constant__ CUtensorMap mcost, int nunits, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    const uint32_t mask = FULL ? full_mask<T>() : a.mask;
    float4 *stage = reinterpret_cast<float4 *>(smraw);                  // (psi, lambda) half block, 64 KB
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 65536);       // table, 16 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 65536 + 16384);   // transposes, 32 KB
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    __shared__ float2 red[WARPS][NSLOT];  // FP32 pairs, or FP64 sums in the same bytes
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const int nbits = a.n - BITS;
    constexpr bool PACKED = FULL && PRE && COST && POST;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&mbarc, 1);
    }
    __syncthreads();
    uint32_t parity = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nunits) {
        issue_amps<T>(blockIdx.x, a, &mpl, stage, &mbar);
        if (COST) issue_table<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }
    for (uint32_t u = blockIdx.x; (int)u < nunits; u += gridDim.x) {
        const Unit un = unit_of(u, nbits);
        const PassScal sc = a.scal[un.item];
        const uint32_t fa = sc.pre_flip ? mask : 0u, fb = sc.post_flip ? mask : 0u;
        const size_t base = unit_base<T>(un.b, a.loA, a.loB);
        float2 P[32], Q[32];
        float acc[NSLOT] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (!stage_ready(&mbar, parity, status)) return;
        parity ^= 1u;
        if (POST) read_stage_pq<T, 0>(P, Q, stage, l, w);
        else read_stage_pq<T, 1>(P, Q, stage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(u + gridDim.x) < nunits) {
            fence_proxy_async();
            issue_amps<T>(u + gridDim.x, a, &mpl, stage, &mbar);
        }
        if (POST) {
            acc[0] = xterm_form<T, 0, PACKED>(P, Q, mask);
            round_mix_pq<T, 0>(P, Q, -sc.post_t, mask);
            transpose1<T, 0, 1, false>(P, xbuf, l, w, fb);  // after the stage-read barrier
            transpose1<T, 0, 1>(Q, xbuf, l, w, fb);
            acc[1] = xterm_form<T, 1, PACKED>(P, Q, mask);
            round_mix_pq<T, 1>(P, Q, -sc.post_t, mask);
        }
        if (COST) {
            int32_t c[32];
            if (!stage_ready(&mbarc, parc, status)) return;
            parc ^= 1u;
            read_cost_y<T>(c, cstage, l, w);
            __syncthreads();
            if (threadIdx.x == 0 && (int)(u + gridDim.x) < nunits) {
                fence_proxy_async();
                issue_table<T>(u + gridDim.x, a, &mcost, cstage, &mbarc);
            }
            float g0 = 0.f, g1 = 0.f;
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                // Im(conj(lambda) psi) = lambda.re psi.im - lambda.im psi.re
                const float im = fmaf(P[m].y, Q[m].x, -Q[m].y * P[m].x);
                if (m & 1) g1 = fmaf((float)c[m], im, g1);
                else g0 = fmaf((float)c[m], im, g0);
                cmul_pq(P[m], Q[m], cost_phase(c[m], sc.phi, sc.off, sc.kmag, a.precise_phase));
            }
            acc[2] = g0 + g1;
        }
        float4 *dst = a.pl + ((size_t)un.item << a.n) + base;
        if (PRE) {
            acc[3] = xterm_form<T, 1, PACKED>(P, Q, mask);
            round_mix_pq<T, 1>(P, Q, -sc.pre_t, mask);
            // with a cost layer the table barrier, without a post mixer the stage-read
            // barrier, lies between the last use of xbuf and this transpose
            transpose1<T, 1, 0, !COST && POST>(P, xbuf, l, w, fa);
            transpose1<T, 1, 0>(Q, xbuf, l, w, fa);
            acc[4] = xterm_form<T, 0, PACKED>(P, Q, mask);
            round_mix_pq<T, 0>(P, Q, -sc.pre_t, mask);
            if (STORE) {
                if (!COST) {
#pragma unroll
                    for (int m = 0; m < 32; ++m) cmul_pq(P[m], Q[m], sc.kend);
                }
                if (SPLIT) store_lam<T, 0>(P, Q, a.lam + ((size_t)un.item << a.n) + base, l, w, a.loA, a.loB);
                else store_pq<T, 0>(P, Q, dst, l, w, a.loA, a.loB);
            }
        } else if (STORE) {
            if (!COST) {
#pragma unroll
                for (int m = 0; m < 32; ++m) cmul_pq(P[m], Q[m], sc.kend);
            }
            if (SPLIT) store_lam<T, 1>(P, Q, a.lam + ((size_t)un.item << a.n) + base, l, w, a.loA, a.loB);
            else store_pq<T, 1>(P, Q, dst, l, w, a.loA, a.loB);
        }
        if constexpr (FULL || !(PRE && COST && POST)) {
            block_sum_write_pairs<5>(acc, red, a.partials, u);
        } else {
            block_sum_write_f64(acc, reinterpret_cast<double(*)[NSLOT]>(red), a.partials, u);
        }
        // no barrier here: the next unit passes one (after its stage read) before it writes red
    }
}

// ---- final forward pass on half blocks ------------------------------------------------------

// RX butterflies of the mixed register bits on one state (tangent form); an
// unmixed bit runs with t = 0
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

template <int T, int A>
__device__ __forceinline__ void read_stage(float2 (&v)[32], const float2 *stage, uint32_t l, uint32_t w) {
    const uint32_t t = local_idx<T, A>(l, 0u, w);
#pragma unroll
    for (int m = 0; m < 32; ++m) v[m] = stage[t | local_idx<T, A>(0u, (uint32_t)m, 0u)];
}

// Running top-K (K <= 16) of one warp over the units a persistent CTA visits:
// key = (bits(P) << 33) | (2^33 - 1 - x), P descending then index ascending.
// list (shared, K keys, descending, 0 = empty) holds the warp's best keys so
// far; a unit's amplitudes are ranked only if one of them can still enter it.
// scratch: shared, 2K keys.
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
            const unsigned long long x = xthread + roff<T, A>(bm, loA, loB);
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
        int i = 0, j = 0;
        for (int r = 0; r < K; ++r) scratch[K + r] = list[i] >= scratch[j] ? list[i++] : scratch[j++];
        for (int r = 0; r < K; ++r) list[r] = scratch[K + r];
    }
    __syncwarp();
}

template <int T>
__device__ __forceinline__ void issue_psi(uint32_t u, const PassArgs &a, const CUtensorMap *map, void *stage,
                                          unsigned long long *mbar) {
    const int nbits = a.n - BITS;
    const Unit un = unit_of(u, nbits);
    mbar_expect_tx(mbar, 32768u);
    if (T == 0) {
        bulk_load(stage, a.psi + ((size_t)un.item << a.n) + ((size_t)un.b << BITS), 32768u, mbar);
    } else {
        int cl, cm, ch;
        unit_coords(un.b, un.item, a, &cl, &cm, &ch);
        tma_load_5d_c(stage, map, 0, cl, 0, cm, ch, mbar);
    }
}

// Final forward pass of a gradient evaluation on half blocks: psi_in ->
// psi_p = RX_G psi_in; E partials, running top-K, lambda = H_C psi_p; X-terms
// of beta_p for group G; undo RX_G on (psi, lambda); write lambda alone
// (SPLIT) or interleaved with psi.  slots: 0 = sum P T, 1 = sum P,
// 2 = X-term (Y), 3 = X-term (X).
template <int T, bool SPLIT, bool TOPK, bool FULL>
__global__ void __launch_bounds__(THREADS, 2)
    final_pass_half_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpsi,
                           const __grid_constant__ CUtensorMap mcost, int nunits, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    const uint32_t mask = FULL ? full_mask<T>() : a.mask;
    float2 *stage = reinterpret_cast<float2 *>(smraw);                 // psi half block, 32 KB
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 32768);      // table, 16 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 32768 + 16384);  // transposes, 32 KB
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    __shared__ float2 red[WARPS][NSLOT];
    __shared__ unsigned long long tk_list[WARPS * 16], tk_scr[WARPS * 32];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const int nbits = a.n - BITS;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&mbarc, 1);
    }
    if (threadIdx.x < WARPS * 16) tk_list[threadIdx.x] = 0ull;
    __syncthreads();
    uint32_t parity = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nunits) {
        issue_psi<T>(blockIdx.x, a, &mpsi, stage, &mbar);
        issue_table<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }
    for (uint32_t u = blockIdx.x; (int)u < nunits; u += gridDim.x) {
        const Unit un = unit_of(u, nbits);
        const PassScal sc = a.scal[un.item];
        const uint32_t fm = sc.pre_flip ? mask : 0u;
        const size_t base = unit_base<T>(un.b, a.loA, a.loB);
        float2 v[32];
        if (!stage_ready(&mbar, parity, status)) return;
        parity ^= 1u;
        read_stage<T, 0>(v, stage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(u + gridDim.x) < nunits) {
            fence_proxy_async();
            issue_psi<T>(u + gridDim.x, a, &mpsi, stage, &mbar);
        }
        round_mix<T, 0>(v, sc.pre_t, mask);
        transpose1<T, 0, 1, false>(v, xbuf, l, w, fm);  // after the stage-read barrier
        round_mix<T, 1>(v, sc.pre_t, mask);
        int32_t c[32];
        if (!stage_ready(&mbarc, parc, status)) return;
        parc ^= 1u;
        read_cost_y<T>(c, cstage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(u + gridDim.x) < nunits) {
            fence_proxy_async();
            issue_table<T>(u + gridDim.x, a, &mcost, cstage, &mbarc);
        }
        // psi_p = kend * v; lambda = (T 2^-s) psi_p
        float2 P[32], Q[32];
        float e0 = 0.f, e1 = 0.f;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            v[m] = cmul(v[m], sc.kend);
            const float pr = fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
            const float cf = (float)c[m];
            e0 = fmaf(pr, cf, e0);
            e1 += pr;
            const float lf = cf * sc.cscale;
            P[m] = make_float2(v[m].x, v[m].x * lf);
            Q[m] = make_float2(v[m].y, v[m].y * lf);
        }
        if (TOPK) {
            const size_t xthread = base + goff<T>(local_idx<T, 1>(l, 0u, w), a.loA, a.loB);
            warp_topk_running<T, 1>(v, xthread, a.loA, a.loB, a.ktop, tk_list + w * 16, tk_scr + w * 32);
        }
        const float x1 = xterm_form<T, 1, FULL && T == 0>(P, Q, mask);
        round_mix_pq<T, 1>(P, Q, -sc.pre_t, mask);
        transpose1<T, 1, 0, false>(P, xbuf, l, w, fm);  // after the table barrier
        transpose1<T, 1, 0>(Q, xbuf, l, w, fm);
        const float x0 = xterm_form<T, 0, FULL && T == 0>(P, Q, mask);
        round_mix_pq<T, 0>(P, Q, -sc.pre_t, mask);
#pragma unroll
        for (int m = 0; m < 32; ++m) cmul_pq(P[m], Q[m], sc.kend2);
        if (SPLIT)
            store_lam<T, 0>(P, Q, a.lam + ((size_t)un.item << a.n) + base, l, w, a.loA, a.loB);
        else
            store_pq<T, 0>(P, Q, a.pl + ((size_t)un.item << a.n) + base, l, w, a.loA, a.loB);
        const float vals[4] = {e0, e1, x1, x0};
        block_sum_write_pairs<4>(vals, red, a.partials, u);
        // no barrier here: the next unit passes one (after its stage read) before it writes red
    }
    // one top-K list per warp: topk_keys[(CTA * WARPS + warp) * K ..]
    if (TOPK && (int)l < a.ktop)
        a.topk_keys[((size_t)blockIdx.x * WARPS + w) * a.ktop + l] = tk_list[w * 16 + l];
}

}  // namespace half

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static int rev_half_units(int n, int nitems) { return nitems << (n - half::BITS); }

static PFN_cuTensorMapEncodeTiled_v12000 g_encode_half = nullptr;

static cudaError_t get_encoder_half() { return tensor_map_encoder(&g_encode_half); }

// High-group half-block views (5-D).  The (psi, lambda) map: (bits 0,1 as
// 8 FP64 words) x (bits 2..loA-1) x (window A) x (bits loA+5..loB-1) x
// (bits loB..n-1, then `count` arrays), box 8 x 1 x 32 x 1 x 32 = 64 KB in
// natural local order.  The table map lists window B (with the bits above
// it) before window A: (bits 0,1) x (bits loB..n-1, arrays) x (window A) x
// (bits 2..loA-1) x (bits loA+5..loB-1), box 4 x 32 x 32 x 1 x 1 = 16 KB in
// the order (bits 0,1) x B x A.
static cudaError_t make_half_pl_map(CUtensorMap *map, const void *base, int n, int loA, int loB, int count) {
    std::memset(map, 0, sizeof(*map));
    cudaError_t e = get_encoder_half();
    if (e) return e;
    const cuuint64_t es = 16;
    cuuint64_t dims[5] = {8ull, 1ull << (loA - 2), 32ull, 1ull << (loB - loA - 5), (1ull << (n - loB)) * (cuuint64_t)count};
    cuuint64_t strides[4] = {4ull * es, es << loA, es << (loA + 5), es << loB};
    cuuint32_t box[5] = {8u, 1u, 32u, 1u, 32u};
    cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
    CUresult r = g_encode_half(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, const_cast<void *>(base), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static cudaError_t make_half_cost_map(CUtensorMap *map, const void *base, int n, int loA, int loB, int count) {
    std::memset(map, 0, sizeof(*map));
    cudaError_t e = get_encoder_half();
    if (e) return e;
    const cuuint64_t es = 4;
    cuuint64_t dims[5] = {4ull, (1ull << (n - loB)) * (cuuint64_t)count, 32ull, 1ull << (loA - 2),
                          1ull << (loB - loA - 5)};
    cuuint64_t strides[4] = {es << loB, es << loA, 4ull * es, es << (loA + 5)};
    cuuint32_t box[5] = {4u, 32u, 32u, 1u, 1u};
    cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
    CUresult r = g_encode_half(map, CU_TENSOR_MAP_DATA_TYPE_INT32, 5, const_cast<void *>(base), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// complex64 half-block view: (bits 0,1 as 4 FP64 words) x ... as the (psi,
// lambda) map, box 4 x 1 x 32 x 1 x 32 = 32 KB
static cudaError_t make_half_psi_map(CUtensorMap *map, const void *base, int n, int loA, int loB, int count) {
    std::memset(map, 0, sizeof(*map));
    cudaError_t e = get_encoder_half();
    if (e) return e;
    const cuuint64_t es = 8;
    cuuint64_t dims[5] = {4ull, 1ull << (loA - 2), 32ull, 1ull << (loB - loA - 5), (1ull << (n - loB)) * (cuuint64_t)count};
    cuuint64_t strides[4] = {4ull * es, es << loA, es << (loA + 5), es << loB};
    cuuint32_t box[5] = {4u, 1u, 32u, 1u, 32u};
    cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
    CUresult r = g_encode_half(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, const_cast<void *>(base), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr int HALF_SMEM = 65536 + 16384 + 32768;
constexpr int HALF_FINAL_SMEM = 32768 + 16384 + 32768;

template <int T, bool SPLIT, bool TOPK, bool FULL>
static cudaError_t half_final_f(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid, int nunits,
                                unsigned int *status, cudaStream_t st) {
    auto k = half::final_pass_half_kernel<T, SPLIT, TOPK, FULL>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, HALF_FINAL_SMEM);
    if (e) return e;
    k<<<grid, half::THREADS, HALF_FINAL_SMEM, st>>>(a, m, mc, nunits, status);
    return cudaGetLastError();
}

template <int T, bool SPLIT, bool TOPK>
static cudaError_t half_final(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid, int nunits,
                              unsigned int *status, cudaStream_t st) {
    const uint32_t full = T == 0 ? 0x3FFu : 0xFFCu;
    return a.mask == full ? half_final_f<T, SPLIT, TOPK, true>(a, m, mc, grid, nunits, status, st)
                          : half_final_f<T, SPLIT, TOPK, false>(a, m, mc, grid, nunits, status, st);
}

cudaError_t launch_final_pass_half(int type, const PassArgs &a_in, int grid, unsigned int *status, cudaStream_t st) {
    PassArgs a = a_in;
    if (type == 1) a.mask = a_in.mask >> 1;
    const int nunits = rev_half_units(a.n, a.nitems);
    CUtensorMap m, mc;
    std::memset(&m, 0, sizeof m);
    std::memset(&mc, 0, sizeof mc);
    cudaError_t e;
    if (type == 1) {
        if ((e = make_half_psi_map(&m, a.psi, a.n, a.loA, a.loB, a.nitems))) return e;
        if ((e = make_half_cost_map(&mc, a.C, a.n, a.loA, a.loB, a.ntables))) return e;
    }
    if (grid > nunits) grid = nunits;
    const int key = (type ? 4 : 0) | (a.split ? 2 : 0) | (a.ktop > 0 ? 1 : 0);
    switch (key) {
        case 0: return half_final<0, false, false>(a, m, mc, grid, nunits, status, st);
        case 1: return half_final<0, false, true>(a, m, mc, grid, nunits, status, st);
        case 2: return half_final<0, true, false>(a, m, mc, grid, nunits, status, st);
        case 3: return half_final<0, true, true>(a, m, mc, grid, nunits, status, st);
        case 4: return half_final<1, false, false>(a, m, mc, grid, nunits, status, st);
        case 5: return half_final<1, false, true>(a, m, mc, grid, nunits, status, st);
        case 6: return half_final<1, true, false>(a, m, mc, grid, nunits, status, st);
        default: return half_final<1, true, true>(a, m, mc, grid, nunits, status, st);
    }
}

template <int T, bool SPLIT, bool PRE, bool COST, bool POST, bool STORE, bool FULL>
static cudaError_t half_launch_f(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid,
                                 int nunits, unsigned int *status, cudaStream_t st) {
    auto k = half::rev_pass_half_kernel<T, SPLIT, PRE, COST, POST, STORE, FULL>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, HALF_SMEM);
    if (e) return e;
    k<<<grid, half::THREADS, HALF_SMEM, st>>>(a, m, mc, nunits, status);
    return cudaGetLastError();
}

template <int T, bool SPLIT, bool PRE, bool COST, bool POST, bool STORE>
static cudaError_t half_launch(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid, int nunits,
                               unsigned int *status, cudaStream_t st) {
    const uint32_t full = T == 0 ? 0x3FFu : 0xFFCu;
    return a.mask == full ? half_launch_f<T, SPLIT, PRE, COST, POST, STORE, true>(a, m, mc, grid, nunits, status, st)
                          : half_launch_f<T, SPLIT, PRE, COST, POST, STORE, false>(a, m, mc, grid, nunits, status, st);
}

template <int T, bool SPLIT>
static cudaError_t half_shape(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid, int nunits,
                              unsigned int *status, cudaStream_t st) {
    const int key = (a.has_pre ? 8 : 0) | (a.has_cost ? 4 : 0) | (a.has_post ? 2 : 0) | (a.store ? 1 : 0);
    switch (key) {
        case 15: return half_launch<T, SPLIT, true, true, true, true>(a, m, mc, grid, nunits, status, st);
        case 6: return half_launch<T, SPLIT, false, true, true, false>(a, m, mc, grid, nunits, status, st);
        case 3: return half_launch<T, SPLIT, false, false, true, true>(a, m, mc, grid, nunits, status, st);
        default: return cudaErrorInvalidValue;  // no schedule produces another shape
    }
}

// a.mask is given in the 13-bit local positions of the schedule (type 1:
// window bits 3..12); the half-block layout has them one bit lower.
cudaError_t launch_rev_pass_half(int type, const PassArgs &a_in, int grid, unsigned int *status, cudaStream_t st) {
    PassArgs a = a_in;
    if (type == 1) a.mask = a_in.mask >> 1;
    const int nunits = rev_half_units(a.n, a.nitems);
    CUtensorMap m, mc;
    std::memset(&m, 0, sizeof m);
    std::memset(&mc, 0, sizeof mc);
    cudaError_t e;
    if (type == 1) {
        if ((e = make_half_pl_map(&m, a.pl, a.n, a.loA, a.loB, a.nitems))) return e;
        if (a.has_cost && (e = make_half_cost_map(&mc, a.C, a.n, a.loA, a.loB, a.ntables))) return e;
    }
    if (grid > nunits) grid = nunits;
    if (type == 0)
        return a.split ? half_shape<0, true>(a, m, mc, grid, nunits, status, st)
                       : half_shape<0, false>(a, m, mc, grid, nunits, status, st);
    return a.split ? half_shape<1, true>(a, m, mc, grid, nunits, status, st)
                   : half_shape<1, false>(a, m, mc, grid, nunits, status, st);
}

}  // namespace qaoa
