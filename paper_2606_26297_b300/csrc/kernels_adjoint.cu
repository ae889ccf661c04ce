// Final forward pass and reverse (adjoint) passes on the interleaved
// (psi, lambda) layout (sm_103a).
//
// The reverse sweep undoes the gates of Eq. qaoa_state layer by layer on both
// psi and lambda = H_C psi_p, and accumulates the exact derivatives
//   dE/dbeta_l  = 2 Im <lambda| sum_j X_j |psi>  (at the mixer of layer l),
//   dE/dgamma_l = 2 Im <lambda| H_C |psi>        (at the cost layer l),
// the exact counterpart of the gradient that Sec. 4.2 estimates by SPSA.
// Storing the two states interleaved, one 16-byte element (psi.re,
// lambda.re, psi.im, lambda.im) per basis index, lets every butterfly and
// phase multiply advance both states with packed f32x2 FMAs: with
// P = (psi.re, lambda.re) and Q = (psi.im, lambda.im), (a, b) -> (a - i t b,
// b - i t a) becomes P_a += t Q_b, Q_a -= t P_b, P_b += t Q_a, Q_b -= t P_a;
// rows of 8 elements are 128 bytes.
//
// Both kernels are persistent (one CTA per SM walking the (item, block)
// units of a batch) and TMA-pipelined: the next unit's amplitudes (a 64 KB
// psi block or a 128 KB (psi, lambda) block) and its 32 KB table block are
// brought into shared memory by cp.async.bulk[.tensor] while the current unit
// is computed.  Every mbarrier wait is bounded; a timeout sets the status word.
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "pass_body.cuh"
#include "tma_util.cuh"

namespace qaoa {

__device__ __forceinline__ float2 f2s(float s) { return make_float2(s, s); }

// butterflies of every mixed register bit on the packed pair (P, Q); an
// unmixed bit runs with t = 0 (the identity) rather than a branch, as in
// round_mix
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

// The same sum with one f32x2 FMA per ordered pair (m, m ^ e_j):
// cross(P_m, Q_{m^e_j}) = (P_m.y, -P_m.x) . Q_{m^e_j}, the swapped, negated
// P_m formed once per m, four packed accumulators.  Fewer instructions (one
// evaluation at n = 30: 131.4 -> 124.8 ms of reverse passes) but longer live
// ranges of Q: used only in the full-mask forms, where it does not spill.
template <int T, int A>
__device__ __forceinline__ float xterm_pq_packed(const float2 (&P)[32], const float2 (&Q)[32], uint32_t mask) {
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

// X-term in the form a kernel shape takes: packed where it spills nothing
// (full groups of the cost-layer reverse pass and of the low-group final
// pass), four scalar chains otherwise
template <int T, int A, bool PACKED>
__device__ __forceinline__ float xterm_form(const float2 (&P)[32], const float2 (&Q)[32], uint32_t mask) {
    return PACKED ? xterm_pq_packed<T, A>(P, Q, mask) : xterm_pq<T, A>(P, Q, mask);
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
                                         uint32_t l, uint32_t w, int loA, int loB) {
    float4 *q = p + goff<T>(local_idx<T, A>(l, 0u, w), loA, loB);
#pragma unroll
    for (int m = 0; m < 32; ++m)
        __stcs(q + roff<T, A>(m, loA, loB), make_float4(P[m].x, P[m].y, Q[m].x, Q[m].y));
}

// store lambda alone from the packed pair (P, Q)
template <int T, int A>
__device__ __forceinline__ void store_lam(const float2 (&P)[32], const float2 (&Q)[32], float2 *__restrict__ p,
                                          uint32_t l, uint32_t w, int loA, int loB) {
    float2 *q = p + goff<T>(local_idx<T, A>(l, 0u, w), loA, loB);
#pragma unroll
    for (int m = 0; m < 32; ++m) __stcs(q + roff<T, A>(m, loA, loB), make_float2(P[m].y, Q[m].y));
}

// unit u of a launch: item u >> nbits, block u & (2^nbits - 1)
struct Unit {
    uint32_t item, b;
};
__device__ __forceinline__ Unit unit_of(uint32_t u, int nbits) { return {u >> nbits, u & ((1u << nbits) - 1u)}; }

// Tensor-map coordinates of high-group block b of array `arr` (item or table
// index): dims (bits 0..2) x (bits 3..loA-1) x (window A) x (bits
// loA+5..loB-1) x (window B and above, arrays stacked); the box covers bits
// 0..2 and both windows.
__device__ __forceinline__ void tile_coords(uint32_t b, uint32_t arr, const PassArgs &a, int *c1, int *c3,
                                            int *c4) {
    const int n1 = a.loA - 3, n2 = a.loB - a.loA - 5;
    *c1 = (int)(b & ((1u << n1) - 1u));
    *c3 = (int)((b >> n1) & ((1u << n2) - 1u));
    *c4 = (int)(((b >> (n1 + n2)) << 5) + (arr << (a.n - a.loB)));
}

// Issue the copy of a unit's amplitudes: the psi block (64 KB) or the
// interleaved (psi, lambda) block (128 KB).  High-group tensor maps stack the
// items of a batch along their outermost dimension.
template <int T, bool PL>
__device__ __forceinline__ void issue_amps(uint32_t u, const PassArgs &a, const CUtensorMap *map, void *stage,
                                           unsigned long long *mbar) {
    const int nbits = a.n - BLOCK_BITS;
    const Unit un = unit_of(u, nbits);
    const uint32_t bytes = PL ? 131072u : 65536u;
    mbar_expect_tx(mbar, bytes);
    if (T == 0) {
        const size_t off = ((size_t)un.item << a.n) + ((size_t)un.b << 13);
        const void *src = PL ? (const void *)(a.pl + off) : (const void *)(a.psi + off);
        bulk_load(stage, src, bytes, mbar);
    } else {
        int c1, c3, c4;
        tile_coords(un.b, un.item, a, &c1, &c3, &c4);
        tma_load_5d(stage, map, c1, c3, c4, mbar);
    }
}

template <int T>
__device__ __forceinline__ void issue_table(uint32_t u, const PassArgs &a, const CUtensorMap *mcost, int32_t *cstage,
                                            unsigned long long *mbar) {
    const int nbits = a.n - BLOCK_BITS;
    const Unit un = unit_of(u, nbits);
    const uint32_t tab = a.item_table ? (uint32_t)a.item_table[un.item] : 0u;
    mbar_expect_tx(mbar, 32768u);
    if (T == 0) {
        bulk_load(cstage, a.C + ((size_t)tab << a.n) + ((size_t)un.b << 13), 32768u, mbar);
    } else {
        int c1, c3, c4;
        tile_coords(un.b, tab, a, &c1, &c3, &c4);
        tma_load_5d(cstage, mcost, c1, c3, c4, mbar);
    }
}

// ---------------------------------------------------------------------------
// final forward pass of a gradient evaluation: psi_in -> psi_p = RX_G psi_in;
// E partials, top-K, lambda = H_C psi_p; X-terms of beta_p for group G; undo
// RX_G on (psi, lambda) and write the interleaved (psi_in, lambda_in).
// slots: 0 = sum P T, 1 = sum P, 2 = X-term (Y), 3 = X-term (X)
// ---------------------------------------------------------------------------
template <int T, bool SPLIT, bool TOPK, bool FULL>
__global__ void __launch_bounds__(PASS_THREADS, 1)
    final_pass_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpsi,
                      const __grid_constant__ CUtensorMap mcost, int nunits, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    const uint32_t mask = FULL ? full_mask<T>() : a.mask;
    float2 *stage = reinterpret_cast<float2 *>(smraw);                 // psi block, 64 KB
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 65536);      // table block, 32 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 65536 + 32768);  // transposes, 64 KB
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    __shared__ float2 red[PASS_THREADS / 32][NSLOT];
    __shared__ unsigned long long tk_list[8 * 16], tk_scr[8 * 32];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const int nbits = a.n - BLOCK_BITS;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&mbarc, 1);
    }
    if (threadIdx.x < 8 * 16) tk_list[threadIdx.x] = 0ull;
    __syncthreads();
    uint32_t parity = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nunits) {
        issue_amps<T, false>(blockIdx.x, a, &mpsi, stage, &mbar);
        issue_table<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }
    for (uint32_t u = blockIdx.x; (int)u < nunits; u += gridDim.x) {
        const Unit un = unit_of(u, nbits);
        const PassScal sc = a.scal[un.item];
        const uint32_t fm = sc.pre_flip ? mask : 0u;
        const size_t base = block_base<T>(un.b, a.loA, a.loB);
        float2 v[32];
        if (!stage_ready(&mbar, parity, status)) return;
        parity ^= 1u;
        read_stage<T, 0>(v, stage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(u + gridDim.x) < nunits) {
            fence_proxy_async();
            issue_amps<T, false>(u + gridDim.x, a, &mpsi, stage, &mbar);
        }
        round_mix<T, 0>(v, sc.pre_t, mask);
        transpose1<T, 0, 1, false>(v, xbuf, l, w, fm);  // after the stage-read barrier
        round_mix<T, 1>(v, sc.pre_t, mask);
        int32_t c[32];
        if (!stage_ready(&mbarc, parc, status)) return;
        parc ^= 1u;
        read_cost_stage<T, 1>(c, cstage, l, w);
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
    // one top-K list per warp: topk_keys[(CTA * 8 + warp) * K ..]
    if (TOPK && (int)l < a.ktop)
        a.topk_keys[((size_t)blockIdx.x * (PASS_THREADS / 32) + w) * a.ktop + l] = tk_list[w * 16 + l];
}

// ---------------------------------------------------------------------------
// reverse pass on the interleaved buffer: undoes one forward pass on
// (psi, lambda).  slots: 0,1 = X-terms of the post mixer (arrangements X, Y);
// 2 = cost term; 3,4 = X-terms of the pre mixer (Y, X).
// ---------------------------------------------------------------------------
template <int T, bool SPLIT, bool PRE, bool COST, bool POST, bool STORE, bool FULL>
__global__ void __launch_bounds__(PASS_THREADS, 1)
    rev_pass_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpl,
                    const __grid_constant__ CUtensorMap mcost, int nunits, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    const uint32_t mask = FULL ? full_mask<T>() : a.mask;
    float4 *stage = reinterpret_cast<float4 *>(smraw);                  // (psi, lambda) block, 128 KB
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 131072);      // table block, 32 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 131072 + 32768);  // transposes, 64 KB
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    __shared__ float2 red[PASS_THREADS / 32][NSLOT];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const int nbits = a.n - BLOCK_BITS;
    constexpr bool pre = PRE, post = POST;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&mbarc, 1);
    }
    __syncthreads();
    uint32_t parity = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nunits) {
        issue_amps<T, true>(blockIdx.x, a, &mpl, stage, &mbar);
        if (COST) issue_table<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }
    for (uint32_t u = blockIdx.x; (int)u < nunits; u += gridDim.x) {
        const Unit un = unit_of(u, nbits);
        const PassScal sc = a.scal[un.item];
        const uint32_t fa = sc.pre_flip ? mask : 0u, fb = sc.post_flip ? mask : 0u;
        const size_t base = block_base<T>(un.b, a.loA, a.loB);
        float2 P[32], Q[32];
        float acc[NSLOT] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (!stage_ready(&mbar, parity, status)) return;
        parity ^= 1u;
        if (post) read_stage_pq<T, 0>(P, Q, stage, l, w);
        else read_stage_pq<T, 1>(P, Q, stage, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && (int)(u + gridDim.x) < nunits) {
            fence_proxy_async();
            issue_amps<T, true>(u + gridDim.x, a, &mpl, stage, &mbar);
        }
        if (post) {
            acc[0] = xterm_form<T, 0, FULL && PRE && COST && POST>(P, Q, mask);
            round_mix_pq<T, 0>(P, Q, -sc.post_t, mask);
            transpose1<T, 0, 1, false>(P, xbuf, l, w, fb);  // after the stage-read barrier
            transpose1<T, 0, 1>(Q, xbuf, l, w, fb);
            acc[1] = xterm_form<T, 1, FULL && PRE && COST && POST>(P, Q, mask);
            round_mix_pq<T, 1>(P, Q, -sc.post_t, mask);
        }
        if (COST) {
            int32_t c[32];
            if (!stage_ready(&mbarc, parc, status)) return;
            parc ^= 1u;
            read_cost_stage<T, 1>(c, cstage, l, w);
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
        if (pre) {
            acc[3] = xterm_form<T, 1, FULL && PRE && COST && POST>(P, Q, mask);
            round_mix_pq<T, 1>(P, Q, -sc.pre_t, mask);
            // with a cost layer the table barrier, without a post mixer the stage-read
            // barrier, lies between the last use of xbuf and this transpose
            transpose1<T, 1, 0, !COST && POST>(P, xbuf, l, w, fa);
            transpose1<T, 1, 0>(Q, xbuf, l, w, fa);
            acc[4] = xterm_form<T, 0, FULL && PRE && COST && POST>(P, Q, mask);
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
        } else {  // the FP64 tree: the pair form spills in these register-bound forms
            double vals[NSLOT];
#pragma unroll
            for (int s = 0; s < NSLOT; ++s) vals[s] = (double)acc[s];
            block_sum_write(vals, reinterpret_cast<double(*)[NSLOT]>(red), a.partials, u);
        }
        // no barrier here: the next unit passes one (after its stage read) before it writes red
    }
}

// ---------------------------------------------------------------------------
// reverse pass of a middle forward pass (mixer only) with stored states:
// lambda alone is carried back through the mixer (undo the group's RX,
// return to true scale) and written, alone or interleaved with the stored
// input state psi_in; the X-terms of the mixer are taken at the pass input
// against psi_in, once with lambda in arrangement Y and once, after a
// transpose, in arrangement X.  slots: 0 = X-term (Y bits), 1 = X-term (X
// bits).
// ---------------------------------------------------------------------------

// A persistent TMA-pipelined kernel (one CTA per SM): the lambda block and the
// stored psi_in block of a unit are staged in shared memory by bulk/tensor
// copies, the next unit's copies are issued as soon as each stage has been
// read, and both X-term sums read psi_in from the stage (one read of psi_in
// from HBM).  A direct-load form with two CTAs per SM took 8% longer per
// gradient evaluation at n = 30 (load latency with 16 warps per SM).
template <int T>
__device__ __forceinline__ void issue_block8(uint32_t u, const PassArgs &a, const CUtensorMap *map,
                                             const float2 *arr, float2 *stage, unsigned long long *mbar) {
    const int nbits = a.n - BLOCK_BITS;
    const Unit un = unit_of(u, nbits);
    mbar_expect_tx(mbar, 65536u);
    if (T == 0) {
        bulk_load(stage, arr + ((size_t)un.item << a.n) + ((size_t)un.b << 13), 65536u, mbar);
    } else {
        int c1, c3, c4;
        tile_coords(un.b, un.item, a, &c1, &c3, &c4);
        tma_load_5d(stage, map, c1, c3, c4, mbar);
    }
}

// X-terms of the mixed register bits with lambda in registers (arrangement A)
// and psi read from a staged block; PL: also write (psi, lambda) interleaved
template <int T, int A, bool PL>
__device__ __forceinline__ float xterm_staged(const float2 (&v)[32], const float2 *pst, float4 *__restrict__ pl,
                                              uint32_t l, uint32_t w, int loA, int loB, uint32_t mask) {
    const uint32_t ts = local_idx<T, A>(l, 0u, w);
    const size_t t = goff<T>(ts, loA, loB);
    bool on[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) on[i] = (mask >> regbit<T, A>(i)) & 1u;
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const float2 ps = pst[ts | local_idx<T, A>(0u, (uint32_t)m, 0u)];
        if (PL) __stcs(pl + t + roff<T, A>(m, loA, loB), make_float4(ps.x, v[m].x, ps.y, v[m].y));
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if (!on[i]) continue;
            const float2 la = v[m ^ (1 << i)];
            s0 = fmaf(la.x, ps.y, s0);
            s1 = fmaf(-la.y, ps.x, s1);
        }
    }
    return s0 + s1;
}

template <int T, bool PLOUT, bool FULL>
__global__ void __launch_bounds__(PASS_THREADS, 1)
    rev_mid_tma_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mlam,
                       const __grid_constant__ CUtensorMap mpsi, int nunits, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    const uint32_t mask = FULL ? full_mask<T>() : a.mask;
    float2 *lst = reinterpret_cast<float2 *>(smraw);            // lambda block, 64 KB
    float2 *pst = reinterpret_cast<float2 *>(smraw + 65536);    // stored psi_in block, 64 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 131072);  // transposes, 64 KB
    __shared__ __align__(8) unsigned long long mbl, mbp;
    __shared__ float2 red[PASS_THREADS / 32][NSLOT];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const int nbits = a.n - BLOCK_BITS;
    if (threadIdx.x == 0) {
        mbar_init(&mbl, 1);
        mbar_init(&mbp, 1);
    }
    __syncthreads();
    uint32_t parl = 0, parp = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nunits) {
        issue_block8<T>(blockIdx.x, a, &mlam, a.lam, lst, &mbl);
        issue_block8<T>(blockIdx.x, a, &mpsi, a.psi_src, pst, &mbp);
    }
    for (uint32_t u = blockIdx.x; (int)u < nunits; u += gridDim.x) {
        const Unit un = unit_of(u, nbits);
        const PassScal sc = a.scal[un.item];
        const uint32_t fb = sc.post_flip ? mask : 0u;
        const size_t base = block_base<T>(un.b, a.loA, a.loB);
        const bool more = (int)(u + gridDim.x) < nunits;
        float2 v[32];
        if (!stage_ready(&mbl, parl, status)) return;
        parl ^= 1u;
        read_stage<T, 0>(v, lst, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && more) {
            fence_proxy_async();
            issue_block8<T>(u + gridDim.x, a, &mlam, a.lam, lst, &mbl);
        }
        round_mix<T, 0>(v, -sc.post_t, mask);
        transpose1<T, 0, 1, false>(v, xbuf, l, w, fb);  // after the stage-read barrier
        round_mix<T, 1>(v, -sc.post_t, mask);
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], sc.kend);
        if (!stage_ready(&mbp, parp, status)) return;
        parp ^= 1u;
        float4 *plo = a.pl + ((size_t)un.item << a.n) + base;
        const float xy = xterm_staged<T, 1, false>(v, pst, plo, l, w, a.loA, a.loB, mask);
        if (!PLOUT) store_arr<T, 1>(v, a.lam + ((size_t)un.item << a.n) + base, l, w, a.loA, a.loB);
        transpose1<T, 1, 0>(v, xbuf, l, w, 0u);
        const float xx = xterm_staged<T, 0, PLOUT>(v, pst, plo, l, w, a.loA, a.loB, mask);
        __syncthreads();
        if (threadIdx.x == 0 && more) {
            fence_proxy_async();
            issue_block8<T>(u + gridDim.x, a, &mpsi, a.psi_src, pst, &mbp);
        }
        const float vals[2] = {xy, xx};
        block_sum_write_pairs<2>(vals, red, a.partials, u);
        // no barrier here: the next unit passes one (after its stage read) before it writes red
    }
}

// forward cost-layer pass (pre mixer, cost, post mixer), persistent, two CTAs
// per SM: the psi block is staged by TMA and, once read, the same stage serves
// as the transpose buffer; the next unit's psi copy is issued after the last
// transpose, the next table copy as soon as the table stage has been read.
// Against the direct-load form this cuts the forward passes of one n = 30,
// p = 8 evaluation from 66.6 to 64.2 ms; for the mixer-only passes (already
// near the HBM bound) the same form gains nothing, and with one CTA per SM and
// a separate transpose buffer it was slower.
template <int T, bool FULL>
__global__ void __launch_bounds__(PASS_THREADS, 2)
    fwd_cost_tma_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpsi,
                        const __grid_constant__ CUtensorMap mcost, int nunits, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    const uint32_t mask = FULL ? full_mask<T>() : a.mask;
    float2 *pst = reinterpret_cast<float2 *>(smraw);            // psi block / transposes, 64 KB
    int32_t *cst = reinterpret_cast<int32_t *>(smraw + 65536);  // table block, 32 KB
    __shared__ __align__(8) unsigned long long mbp, mbc;
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const int nbits = a.n - BLOCK_BITS;
    if (threadIdx.x == 0) {
        mbar_init(&mbp, 1);
        mbar_init(&mbc, 1);
    }
    __syncthreads();
    uint32_t parp = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nunits) {
        issue_block8<T>(blockIdx.x, a, &mpsi, a.psi, pst, &mbp);
        issue_table<T>(blockIdx.x, a, &mcost, cst, &mbc);
    }
    for (uint32_t u = blockIdx.x; (int)u < nunits; u += gridDim.x) {
        const Unit un = unit_of(u, nbits);
        const PassScal sc = a.scal[un.item];
        const size_t base = block_base<T>(un.b, a.loA, a.loB);
        const bool more = (int)(u + gridDim.x) < nunits;
        float2 *po = (a.psi_out ? a.psi_out : a.psi) + ((size_t)un.item << a.n) + base;
        float2 v[32];
        if (!stage_ready(&mbp, parp, status)) return;
        parp ^= 1u;
        read_stage<T, 0>(v, pst, l, w);
        round_mix<T, 0>(v, sc.pre_t, mask);
        transpose1<T, 0, 1>(v, pst, l, w, sc.pre_flip ? mask : 0u);
        round_mix<T, 1>(v, sc.pre_t, mask);
        int32_t c[32];
        if (!stage_ready(&mbc, parc, status)) return;
        parc ^= 1u;
        read_cost_stage<T, 1>(c, cst, l, w);
        __syncthreads();
        if (threadIdx.x == 0 && more) {
            fence_proxy_async();
            issue_table<T>(u + gridDim.x, a, &mcost, cst, &mbc);
        }
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], cost_phase(c[m], sc.phi, sc.off, sc.kmag, a.precise_phase));
        round_mix<T, 1>(v, sc.post_t, mask);
        transpose1<T, 1, 0, false>(v, pst, l, w, sc.post_flip ? mask : 0u);  // after the table barrier
        __syncthreads();
        if (threadIdx.x == 0 && more) {
            fence_proxy_async();
            issue_block8<T>(u + gridDim.x, a, &mpsi, a.psi, pst, &mbp);
        }
        round_mix<T, 0>(v, sc.post_t, mask);
        store_arr<T, 0>(v, po, l, w, a.loA, a.loB);
    }
}

// Diagnostic of the bounded waits every TMA-pipelined kernel uses: one CTA
// announces a 16-byte transaction on an mbarrier and issues no copy, so the
// phase never completes; stage_ready() gives up after its limit (about 2 s of
// clock, then a second bounded wait), records the timeout in the status word
// and the CTA returns.  Nothing is left in flight.
__global__ void wait_probe_kernel(unsigned int *status) {
    __shared__ __align__(8) unsigned long long mbar;
    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(&mbar, 16u);
    if (!stage_ready(&mbar, 0u, status)) return;
}

// ---------------------------------------------------------------------------
// host side: tensor maps and launchers
// ---------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static cudaError_t get_encoder() { return tensor_map_encoder(&g_encode); }

// 5-D view of high-group blocks: (bits 0..2) x (bits 3..loA-1) x (window A,
// bits loA..loA+4) x (bits loA+5..loB-1) x (bits loB..n-1, then `count`
// consecutive arrays of 2^n elements); the box is 8 x 1 x 32 x 1 x 32, i.e.
// bits 0..2 and both windows.  esize: 16 (interleaved psi/lambda, described as
// pairs of 8-byte elements in dim 0), 8 (complex64) or 4 (int32).
static cudaError_t make_block_map(CUtensorMap *map, const void *base, int n, int loA, int loB, int esize,
                                  int count) {
    std::memset(map, 0, sizeof(*map));
    cudaError_t e = get_encoder();
    if (e) return e;
    const cuuint64_t es = (cuuint64_t)esize;
    const cuuint64_t d0 = esize == 16 ? 16ull : 8ull;
    cuuint64_t dims[5] = {d0, 1ull << (loA - 3), 32ull, 1ull << (loB - loA - 5),
                          (1ull << (n - loB)) * (cuuint64_t)count};
    cuuint64_t strides[4] = {8ull * es, es << loA, es << (loA + 5), es << loB};
    cuuint32_t box[5] = {(cuuint32_t)d0, 1u, 32u, 1u, 32u};
    cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
    CUresult r = g_encode(map, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_INT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5,
                          const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename K>
static cudaError_t set_smem(K kern, int bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int T, bool SPLIT, bool TOPK, bool FULL>
static cudaError_t final_launch_f(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid,
                                  int nunits, int smem, unsigned int *status, cudaStream_t st) {
    cudaError_t e = set_smem(final_pass_kernel<T, SPLIT, TOPK, FULL>, smem);
    if (e) return e;
    final_pass_kernel<T, SPLIT, TOPK, FULL><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nunits, status);
    return cudaGetLastError();
}

template <int T, bool SPLIT, bool TOPK>
static cudaError_t final_launch(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid, int nunits,
                                int smem, unsigned int *status, cudaStream_t st) {
    return a.mask == full_mask<T>() ? final_launch_f<T, SPLIT, TOPK, true>(a, m, mc, grid, nunits, smem, status, st)
                                    : final_launch_f<T, SPLIT, TOPK, false>(a, m, mc, grid, nunits, smem, status, st);
}

cudaError_t launch_final_pass(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
    const int nunits = a.nitems << (a.n - BLOCK_BITS);
    const int smem = 65536 + 32768 + 65536;
    CUtensorMap m, mc;
    std::memset(&m, 0, sizeof m);
    std::memset(&mc, 0, sizeof mc);
    cudaError_t e;
    if (type == 1) {
        if ((e = make_block_map(&m, a.psi, a.n, a.loA, a.loB, 8, a.nitems))) return e;
        if ((e = make_block_map(&mc, a.C, a.n, a.loA, a.loB, 4, a.ntables))) return e;
    }
    if (grid > nunits) grid = nunits;
    const int key = (type ? 4 : 0) | (a.split ? 2 : 0) | (a.ktop > 0 ? 1 : 0);
    switch (key) {
        case 0: return final_launch<0, false, false>(a, m, mc, grid, nunits, smem, status, st);
        case 1: return final_launch<0, false, true>(a, m, mc, grid, nunits, smem, status, st);
        case 2: return final_launch<0, true, false>(a, m, mc, grid, nunits, smem, status, st);
        case 3: return final_launch<0, true, true>(a, m, mc, grid, nunits, smem, status, st);
        case 4: return final_launch<1, false, false>(a, m, mc, grid, nunits, smem, status, st);
        case 5: return final_launch<1, false, true>(a, m, mc, grid, nunits, smem, status, st);
        case 6: return final_launch<1, true, false>(a, m, mc, grid, nunits, smem, status, st);
        default: return final_launch<1, true, true>(a, m, mc, grid, nunits, smem, status, st);
    }
}

template <int T, bool SPLIT, bool PRE, bool COST, bool POST, bool STORE, bool FULL>
static cudaError_t rev_launch_f(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid, int nunits,
                                int smem, unsigned int *status, cudaStream_t st) {
    cudaError_t e = set_smem(rev_pass_kernel<T, SPLIT, PRE, COST, POST, STORE, FULL>, smem);
    if (e) return e;
    rev_pass_kernel<T, SPLIT, PRE, COST, POST, STORE, FULL><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nunits,
                                                                                               status);
    return cudaGetLastError();
}

template <int T, bool SPLIT, bool PRE, bool COST, bool POST, bool STORE>
static cudaError_t rev_launch(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid, int nunits,
                              int smem, unsigned int *status, cudaStream_t st) {
    return a.mask == full_mask<T>()
               ? rev_launch_f<T, SPLIT, PRE, COST, POST, STORE, true>(a, m, mc, grid, nunits, smem, status, st)
               : rev_launch_f<T, SPLIT, PRE, COST, POST, STORE, false>(a, m, mc, grid, nunits, smem, status, st);
}

// One instantiation per pass shape the schedules produce: a cost-layer pass
// (mixer, cost, mixer), the first pass (cost, mixer; nothing to store) and,
// without stored states, a mixer-only pass.
template <int T, bool SPLIT>
static cudaError_t rev_shape(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid, int nunits,
                             int smem, unsigned int *status, cudaStream_t st) {
    const int key = (a.has_pre ? 8 : 0) | (a.has_cost ? 4 : 0) | (a.has_post ? 2 : 0) | (a.store ? 1 : 0);
    switch (key) {
        case 15: return rev_launch<T, SPLIT, true, true, true, true>(a, m, mc, grid, nunits, smem, status, st);
        case 6: return rev_launch<T, SPLIT, false, true, true, false>(a, m, mc, grid, nunits, smem, status, st);
        case 3: return rev_launch<T, SPLIT, false, false, true, true>(a, m, mc, grid, nunits, smem, status, st);
        default: return cudaErrorInvalidValue;  // no schedule produces another shape
    }
}

static cudaError_t rev_dispatch(int type, const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid,
                                int nunits, int smem, unsigned int *status, cudaStream_t st) {
    if (type == 0)
        return a.split ? rev_shape<0, true>(a, m, mc, grid, nunits, smem, status, st)
                       : rev_shape<0, false>(a, m, mc, grid, nunits, smem, status, st);
    return a.split ? rev_shape<1, true>(a, m, mc, grid, nunits, smem, status, st)
                   : rev_shape<1, false>(a, m, mc, grid, nunits, smem, status, st);
}

cudaError_t launch_rev_pass(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
    const int nunits = a.nitems << (a.n - BLOCK_BITS);
    const int smem = 131072 + 32768 + 65536;
    CUtensorMap m, mc;
    std::memset(&m, 0, sizeof m);
    std::memset(&mc, 0, sizeof mc);
    cudaError_t e;
    if (type == 1) {
        if ((e = make_block_map(&m, a.pl, a.n, a.loA, a.loB, 16, a.nitems))) return e;
        if (a.has_cost && (e = make_block_map(&mc, a.C, a.n, a.loA, a.loB, 4, a.ntables))) return e;
    }
    if (grid > nunits) grid = nunits;
    return rev_dispatch(type, a, m, mc, grid, nunits, smem, status, st);
}

template <int T, bool PLOUT, bool FULL>
static cudaError_t mid_launch_f(const PassArgs &a, const CUtensorMap &ml, const CUtensorMap &mp, int grid,
                                int nunits, unsigned int *status, cudaStream_t st) {
    const int smem = 3 * 65536;
    cudaError_t e = set_smem(rev_mid_tma_kernel<T, PLOUT, FULL>, smem);
    if (e) return e;
    rev_mid_tma_kernel<T, PLOUT, FULL><<<grid, PASS_THREADS, smem, st>>>(a, ml, mp, nunits, status);
    return cudaGetLastError();
}

template <int T, bool PLOUT>
static cudaError_t mid_launch(const PassArgs &a, const CUtensorMap &ml, const CUtensorMap &mp, int grid,
                              int nunits, unsigned int *status, cudaStream_t st) {
    return a.mask == full_mask<T>() ? mid_launch_f<T, PLOUT, true>(a, ml, mp, grid, nunits, status, st)
                                    : mid_launch_f<T, PLOUT, false>(a, ml, mp, grid, nunits, status, st);
}

cudaError_t launch_rev_mid(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
    const int nunits = a.nitems << (a.n - BLOCK_BITS);
    CUtensorMap ml, mp;
    std::memset(&ml, 0, sizeof ml);
    std::memset(&mp, 0, sizeof mp);
    cudaError_t e;
    if (type == 1) {
        if ((e = make_block_map(&ml, a.lam, a.n, a.loA, a.loB, 8, a.nitems))) return e;
        if ((e = make_block_map(&mp, a.psi_src, a.n, a.loA, a.loB, 8, a.nitems))) return e;
    }
    if (grid > nunits) grid = nunits;
    if (type == 0)
        return a.pl_out ? mid_launch<0, true>(a, ml, mp, grid, nunits, status, st)
                        : mid_launch<0, false>(a, ml, mp, grid, nunits, status, st);
    return a.pl_out ? mid_launch<1, true>(a, ml, mp, grid, nunits, status, st)
                    : mid_launch<1, false>(a, ml, mp, grid, nunits, status, st);
}

template <int T, bool FULL>
static cudaError_t fct_launch_f(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid,
                                int nunits, unsigned int *status, cudaStream_t st) {
    const int smem = 65536 + 32768;
    cudaError_t e = set_smem(fwd_cost_tma_kernel<T, FULL>, smem);
    if (e) return e;
    fwd_cost_tma_kernel<T, FULL><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nunits, status);
    return cudaGetLastError();
}

template <int T>
static cudaError_t fct_launch(const PassArgs &a, const CUtensorMap &m, const CUtensorMap &mc, int grid, int nunits,
                              unsigned int *status, cudaStream_t st) {
    return a.mask == full_mask<T>() ? fct_launch_f<T, true>(a, m, mc, grid, nunits, status, st)
                                    : fct_launch_f<T, false>(a, m, mc, grid, nunits, status, st);
}

cudaError_t launch_fwd_cost_tma(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
    const int nunits = a.nitems << (a.n - BLOCK_BITS);
    CUtensorMap m, mc;
    std::memset(&m, 0, sizeof m);
    std::memset(&mc, 0, sizeof mc);
    cudaError_t e;
    if (type == 1) {
        if ((e = make_block_map(&m, a.psi, a.n, a.loA, a.loB, 8, a.nitems))) return e;
        if ((e = make_block_map(&mc, a.C, a.n, a.loA, a.loB, 4, a.ntables))) return e;
    }
    if (grid > nunits) grid = nunits;
    return type == 0 ? fct_launch<0>(a, m, mc, grid, nunits, status, st)
                     : fct_launch<1>(a, m, mc, grid, nunits, status, st);
}

cudaError_t launch_wait_probe(unsigned int *status, cudaStream_t st) {
    wait_probe_kernel<<<1, 128, 0, st>>>(status);
    return cudaGetLastError();
}

}  // namespace qaoa
