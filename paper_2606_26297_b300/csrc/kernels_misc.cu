// Objective-table build (Sec. 2.1-2.2), expectation and top-K over a stored
// state, the shared-memory-resident small-n evaluator, and the DQAOA
// factorisation check (Sec. 3.2).
#include "kernels_misc.h"
#include "pass_common.cuh"
#include "schedule.cuh"

namespace qaoa {

// ---------------------------------------------------------------------------
// objective table: T[x] = c_off + sum l_i z_i + sum_{i<j} b_ij z_i z_j (exact
// int64, stored as int32)
// ---------------------------------------------------------------------------
constexpr int MAXT = 8;

// x = x_lo | x_mid << nlo | x_top << (nlo + t).  A thread owns one (x_lo,
// x_top) and walks the 2^t values of x_mid in Gray-code order.  With the
// objective split as
//   F(x) = K(x_lo, x_top) + F_mid(x_mid) + sum_{j in mid} z_j W_j(x_lo, x_top),
//   W_j = sum_{i not in mid} b_ij z_i,
// flipping mid bit j changes the last sum by +/-W_j, F_mid (the objective of
// the mid bits alone, shared by the CTA) is a table lookup, and K is fixed.
__global__ void cost_build_kernel(CostBuildArgs a) {
    extern __shared__ long long shc[];  // ell[n], bs[n*n] (symmetric), fmid[2^t], wsh[t][blockDim]
    const int n = a.n, nlo = a.nlo, t = a.t;
    long long *ell = shc;
    long long *bs = shc + n;
    long long *fmid = bs + n * n;
    long long *wsh = fmid + (1 << t);
    for (int k = threadIdx.x; k < n; k += blockDim.x) ell[k] = a.ell[k];
    for (int k = threadIdx.x; k < n * n; k += blockDim.x) {
        const int i = k / n, j = k % n;
        bs[k] = i < j ? a.b[k] : (j < i ? a.b[j * n + i] : 0);
    }
    __syncthreads();
    // F_mid over the mid bits alone (linear + mid-mid couplings)
    for (int u = threadIdx.x; u < (1 << t); u += blockDim.x) {
        long long f = 0;
        for (int k = 0; k < t; ++k) {
            if (!((u >> k) & 1)) continue;
            f += ell[nlo + k];
            for (int k2 = k + 1; k2 < t; ++k2)
                if ((u >> k2) & 1) f += bs[(nlo + k) * n + nlo + k2];
        }
        fmid[u] = f;
    }
    const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long xlo = gt & ((1ull << nlo) - 1ull), top = gt >> nlo;
    const unsigned long long x0 = xlo | (top << (nlo + t));
    // K(x0): the objective of the fixed bits
    long long K = a.c_off;
    for (int i = 0; i < n; ++i) {
        if (!((x0 >> i) & 1ull)) continue;
        K += ell[i];
        for (int j = i + 1; j < n; ++j)
            if ((x0 >> j) & 1ull) K += bs[i * n + j];
    }
    for (int k = 0; k < t; ++k) {
        const int j = nlo + k;
        long long wj = 0;
        for (int i = 0; i < n; ++i)
            if (((x0 >> i) & 1ull)) wj += bs[i * n + j];
        wsh[k * blockDim.x + threadIdx.x] = wj;
    }
    __syncthreads();
    long long cross = 0;
    unsigned mid = 0;
    long long best = K + fmid[0];
    unsigned long long bestx = x0;
    a.T[x0] = (int32_t)best;
    const unsigned cnt = 1u << t;
    for (unsigned u = 1; u < cnt; ++u) {
        const int k = __ffs(u) - 1;
        const long long wk = wsh[k * blockDim.x + threadIdx.x];
        const bool was = (mid >> k) & 1u;
        cross += was ? -wk : wk;
        mid ^= 1u << k;
        const long long F = K + fmid[mid] + cross;
        const unsigned long long x = x0 | ((unsigned long long)mid << nlo);
        a.T[x] = (int32_t)F;
        if (F < best || (F == best && x < bestx)) {
            best = F;
            bestx = x;
        }
    }
    // block argmin (value, then index)
    __shared__ long long sv[256];
    __shared__ unsigned long long sx[256];
    sv[threadIdx.x] = best;
    sx[threadIdx.x] = bestx;
    __syncthreads();
    for (int s = blockDim.x >> 1; s; s >>= 1) {
        if ((int)threadIdx.x < s) {
            const long long ov = sv[threadIdx.x + s];
            const unsigned long long ox = sx[threadIdx.x + s];
            if (ov < sv[threadIdx.x] || (ov == sv[threadIdx.x] && ox < sx[threadIdx.x])) {
                sv[threadIdx.x] = ov;
                sx[threadIdx.x] = ox;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.blk_val[blockIdx.x] = sv[0];
        a.blk_idx[blockIdx.x] = sx[0];
    }
}

__global__ void argmin_reduce_kernel(const long long *val, const unsigned long long *idx, int m,
                                     long long *oval, unsigned long long *oidx) {
    __shared__ long long sv[256];
    __shared__ unsigned long long sx[256];
    long long bv = LLONG_MAX;
    unsigned long long bx = ~0ull;
    for (int k = threadIdx.x; k < m; k += 256)
        if (val[k] < bv || (val[k] == bv && idx[k] < bx)) {
            bv = val[k];
            bx = idx[k];
        }
    sv[threadIdx.x] = bv;
    sx[threadIdx.x] = bx;
    __syncthreads();
    for (int s = 128; s; s >>= 1) {
        if ((int)threadIdx.x < s) {
            const long long ov = sv[threadIdx.x + s];
            const unsigned long long ox = sx[threadIdx.x + s];
            if (ov < sv[threadIdx.x] || (ov == sv[threadIdx.x] && ox < sx[threadIdx.x])) {
                sv[threadIdx.x] = ov;
                sx[threadIdx.x] = ox;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *oval = sv[0];
        *oidx = sx[0];
    }
}

cudaError_t launch_cost_build(CostBuildArgs a, int *nblocks_out, cudaStream_t st) {
    const int n = a.n;
    a.nlo = n < 12 ? n : 12;
    a.t = (n - a.nlo) < MAXT ? (n - a.nlo) : MAXT;
    const unsigned long long threads = 1ull << (n - a.t);
    const int bs = threads < 256 ? (int)threads : 256;
    const unsigned long long grid = threads / bs;
    const int smem = (n + n * n + (1 << a.t) + a.t * bs) * (int)sizeof(long long);
    cost_build_kernel<<<(unsigned)grid, bs, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    argmin_reduce_kernel<<<1, 256, 0, st>>>(a.blk_val, a.blk_idx, (int)grid, a.min_val, a.min_idx);
    *nblocks_out = (int)grid;
    return cudaGetLastError();
}

cudaError_t launch_argmin_reduce(const long long *val, const unsigned long long *idx, int m, long long *oval,
                                 unsigned long long *oidx, cudaStream_t st) {
    argmin_reduce_kernel<<<1, 256, 0, st>>>(val, idx, m, oval, oidx);
    return cudaGetLastError();
}

int cost_build_blocks(int n) {
    const int nlo = n < 12 ? n : 12;
    const int t = (n - nlo) < MAXT ? (n - nlo) : MAXT;
    const unsigned long long threads = 1ull << (n - t);
    const int bs = threads < 256 ? (int)threads : 256;
    return (int)(threads / bs);
}

// ---------------------------------------------------------------------------
// <H_C> and top-K over a stored complex64 state (chunks of 8192 amplitudes)
// ---------------------------------------------------------------------------
__global__ void expect_kernel(const float2 *__restrict__ psi, const int32_t *__restrict__ T, long long N,
                              double *partials) {
    __shared__ double red[8][NSLOT];
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
    double vals[NSLOT] = {(double)e0, (double)e1, 0.0, 0.0, 0.0};
    block_sum_write(vals, red, partials, blockIdx.x);
}

// Per-chunk top-K (K <= 64) by key (P desc, index asc).
__global__ void topk_chunk_kernel(const float2 *__restrict__ psi, long long N, int K,
                                  unsigned long long *out) {
    __shared__ unsigned long long smk[8 * 64];
    const uint32_t l = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long b0 = (long long)blockIdx.x * 8192;
    float P[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const long long x = b0 + threadIdx.x + 256 * m;
        if (x < N) {
            const float2 a = psi[x];
            P[m] = fmaf(a.x, a.x, a.y * a.y);
        } else {
            P[m] = -1.f;
        }
    }
    uint32_t taken = 0;
    unsigned long long bk = 0;
    int bm = -1;
    auto scan = [&]() {
        bk = 0;
        bm = -1;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            if (((taken >> m) & 1u) || P[m] < 0.f) continue;
            const unsigned long long x = (unsigned long long)(b0 + threadIdx.x + 256 * m);
            const unsigned long long key = ((unsigned long long)__float_as_uint(P[m]) << 33) | (0x1FFFFFFFFull - x);
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
        if (l == 0) smk[w * 64 + r] = wb;
        if (bk == wb && bm >= 0) {
            taken |= 1u << bm;
            scan();
        }
    }
    __syncthreads();
    if (w == 0) {
        int head = 0;
        for (int r = 0; r < K; ++r) {
            const unsigned long long mine = (l < 8 && head < K) ? smk[l * 64 + head] : 0ull;
            unsigned long long wb = mine;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const unsigned long long t = __shfl_xor_sync(0xffffffffu, wb, o);
                wb = t > wb ? t : wb;
            }
            if (l < 8 && mine == wb && wb != 0ull) ++head;
            if (l == 0) out[(size_t)blockIdx.x * K + r] = wb;
        }
    }
}

cudaError_t launch_expect(const float2 *psi, const int32_t *T, int n, double *partials, cudaStream_t st) {
    const long long N = 1ll << n;
    const unsigned grid = (unsigned)((N + 8191) / 8192);
    expect_kernel<<<grid, 256, 0, st>>>(psi, T, N, partials);
    return cudaGetLastError();
}

// out[i] = amps[idx[i]] (element size esize = 8 or 16 bytes); an index
// outside the state sets *bad and leaves out[i] untouched.
__global__ void gather_kernel(const unsigned char *__restrict__ amps, int esize, unsigned long long N,
                              const unsigned long long *__restrict__ idx, int count, unsigned char *out,
                              unsigned int *bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const unsigned long long x = idx[i];
    if (x >= N) {
        atomicOr(bad, 1u);
        return;
    }
    if (esize == 16)
        reinterpret_cast<double2 *>(out)[i] = reinterpret_cast<const double2 *>(amps)[x];
    else
        reinterpret_cast<float2 *>(out)[i] = reinterpret_cast<const float2 *>(amps)[x];
}

cudaError_t launch_gather(const void *amps, int esize, int n, const unsigned long long *idx, int count, void *out,
                          unsigned int *bad, cudaStream_t st) {
    gather_kernel<<<(count + 255) / 256, 256, 0, st>>>(static_cast<const unsigned char *>(amps), esize,
                                                        1ull << n, idx, count, static_cast<unsigned char *>(out),
                                                        bad);
    return cudaGetLastError();
}

cudaError_t launch_topk_chunks(const float2 *psi, int n, int K, unsigned long long *out, cudaStream_t st) {
    const long long N = 1ll << n;
    const unsigned grid = (unsigned)((N + 8191) / 8192);
    topk_chunk_kernel<<<grid, 256, 0, st>>>(psi, N, K, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// small-n evaluator: one CTA per item, the whole state in shared memory,
// all p layers forward (Eq. qaoa_state), <H_C>, optional top-K, and the
// adjoint sweep.  R = float (complex64) or double (complex128).
// ---------------------------------------------------------------------------
template <typename R>
struct Cx;
template <>
struct Cx<float> {
    using T = float2;
    __device__ static T mk(float a, float b) { return make_float2(a, b); }
};
template <>
struct Cx<double> {
    using T = double2;
    __device__ static T mk(double a, double b) { return make_double2(a, b); }
};

template <typename R>
__device__ __forceinline__ typename Cx<R>::T small_phase(int32_t tq, unsigned long long phi,
                                                          unsigned long long off, int precise);
template <>
__device__ __forceinline__ float2 small_phase<float>(int32_t tq, unsigned long long phi,
                                                      unsigned long long off, int precise) {
    return cost_phase(tq, phi, off, 1.0f, precise);
}
template <>
__device__ __forceinline__ double2 small_phase<double>(int32_t tq, unsigned long long phi,
                                                        unsigned long long off, int) {
    const unsigned long long t = (unsigned long long)(long long)tq * phi + off;
    const double a = (double)(long long)t * 1.0842021724855044e-19;  // turns*2 in [-1,1): 2^-63
    double s, c;
    sincospi(a, &s, &c);
    return make_double2(c, -s);
}

template <typename C2>
__device__ __forceinline__ C2 cm(C2 a, C2 b) {
    C2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// deterministic block sum for 512 threads (16 warps); result valid in all threads
__device__ __forceinline__ double bsum512(double x, double *sh) {
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 16; ++k) t += sh[k];
    return t;
}

template <typename R>
__global__ void __launch_bounds__(512, 1) small_kernel(const SmallItem *__restrict__ items) {
    using C2 = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[16];
    __shared__ unsigned long long bestk[16];
    const SmallItem &it = items[blockIdx.x];
    const int n = it.n, p = it.p;
    const int N = 1 << n, H = N >> 1;
    C2 *psi = reinterpret_cast<C2 *>(smraw);
    C2 *lam = psi + N;
    int32_t *T = reinterpret_cast<int32_t *>(lam + (it.grad ? N : 0));
    const int tid = threadIdx.x;
    for (int x = tid; x < N; x += 512) {
        T[x] = it.T[x];
        psi[x] = Cx<R>::mk((R)it.amp0, (R)0);
    }
    for (int l = 0; l < p; ++l) {
        __syncthreads();
        for (int x = tid; x < N; x += 512) psi[x] = cm(psi[x], small_phase<R>(T[x], it.phi[l], it.off[l], it.precise));
        const R c = (R)it.cb[l], s = (R)it.sb[l];
        for (int j = 0; j < n; ++j) {
            __syncthreads();
            for (int k = tid; k < H; k += 512) {
                const int lowm = (1 << j) - 1;
                const int x = ((k & ~lowm) << 1) | (k & lowm), y = x | (1 << j);
                const C2 a = psi[x], b = psi[y];
                psi[x] = Cx<R>::mk(c * a.x + s * b.y, c * a.y - s * b.x);  // c a - i s b
                psi[y] = Cx<R>::mk(c * b.x + s * a.y, c * b.y - s * a.x);  // c b - i s a
            }
        }
    }
    __syncthreads();
    // <H_C>
    double e0 = 0.0, e1 = 0.0;
    for (int x = tid; x < N; x += 512) {
        const double P = (double)psi[x].x * psi[x].x + (double)psi[x].y * psi[x].y;
        e0 += P * (double)T[x];
        e1 += P;
    }
    e0 = bsum512(e0, red);
    e1 = bsum512(e1, red);
    if (tid == 0) it.out[0] = (e0 + (double)it.k_c * e1) * it.cscale;
    if (it.psi_out) {
        for (int x = tid; x < N; x += 512) {
            if (sizeof(R) == 4) reinterpret_cast<float2 *>(it.psi_out)[x] = make_float2((float)psi[x].x, (float)psi[x].y);
            else reinterpret_cast<double2 *>(it.psi_out)[x] = make_double2((double)psi[x].x, (double)psi[x].y);
        }
    }
    // top-K by (P desc, x asc): K rounds of block argmax
    if (it.ktop > 0) {
        unsigned long long taken_last = ~0ull;  // key taken in the previous round
        for (int r = 0; r < it.ktop; ++r) {
            unsigned long long bk = 0;
            for (int x = tid; x < N; x += 512) {
                const float P = (float)((double)psi[x].x * psi[x].x + (double)psi[x].y * psi[x].y);
                const unsigned long long key = ((unsigned long long)__float_as_uint(P) << 33) | (0x1FFFFFFFFull - x);
                if (key < taken_last && key > bk) bk = key;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const unsigned long long t = __shfl_xor_sync(0xffffffffu, bk, o);
                bk = t > bk ? t : bk;
            }
            __syncthreads();
            if ((tid & 31) == 0) bestk[tid >> 5] = bk;
            __syncthreads();
            unsigned long long b = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) b = bestk[k] > b ? bestk[k] : b;
            if (tid == 0) it.topk[r] = b;
            taken_last = b;
        }
    }
    if (!it.grad) return;
    // adjoint sweep: lambda = H_C psi (shifted by k_c 2^-s)
    for (int x = tid; x < N; x += 512) {
        const R f = (R)((double)T[x] * it.cscale);
        lam[x] = Cx<R>::mk(f * psi[x].x, f * psi[x].y);
    }
    for (int l = p - 1; l >= 0; --l) {
        const R c = (R)it.cb[l], s = (R)it.sb[l];
        double xt = 0.0;
        for (int j = 0; j < n; ++j) {
            __syncthreads();
            for (int k = tid; k < H; k += 512) {
                const int lowm = (1 << j) - 1;
                const int x = ((k & ~lowm) << 1) | (k & lowm), y = x | (1 << j);
                const C2 a = psi[x], b = psi[y], la = lam[x], lb = lam[y];
                // Im(conj(la) b) + Im(conj(lb) a)
                xt += (double)(la.x * b.y - la.y * b.x) + (double)(lb.x * a.y - lb.y * a.x);
                // undo: RX(-2 beta): (a, b) <- (c a + i s b, c b + i s a)
                psi[x] = Cx<R>::mk(c * a.x - s * b.y, c * a.y + s * b.x);
                psi[y] = Cx<R>::mk(c * b.x - s * a.y, c * b.y + s * a.x);
                lam[x] = Cx<R>::mk(c * la.x - s * lb.y, c * la.y + s * lb.x);
                lam[y] = Cx<R>::mk(c * lb.x - s * la.y, c * lb.y + s * la.x);
            }
        }
        xt = bsum512(xt, red);
        if (tid == 0) it.out[1 + p + l] = 2.0 * xt;
        __syncthreads();
        double g = 0.0;
        for (int x = tid; x < N; x += 512) {
            const C2 a = psi[x], la = lam[x];
            g += (double)T[x] * (double)(la.x * a.y - la.y * a.x);
            C2 ph = small_phase<R>(T[x], it.phi[l], it.off[l], it.precise);
            ph.y = -ph.y;  // inverse phase
            psi[x] = cm(a, ph);
            lam[x] = cm(la, ph);
        }
        g = bsum512(g, red);
        if (tid == 0) it.out[1 + l] = 2.0 * it.cscale * g;
    }
}

// Recompute the angle-dependent fields of small items from device angles
// (used inside captured optimisation steps).
__global__ void small_prep_kernel(SmallItem *items, int count, const double *gamma, const double *beta, int p,
                                  const int *item_s, const long long *item_kc) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count * p) return;
    const int it = idx / p, l = idx % p;
    const double g = gamma[(size_t)it * p + l], b = beta[(size_t)it * p + l];
    const unsigned long long phi = phase_multiplier(g, item_s[it]);
    items[it].phi[l] = phi;
    items[it].off[l] = (unsigned long long)item_kc[it] * phi;
    items[it].cb[l] = cos(b);
    items[it].sb[l] = sin(b);
}

cudaError_t launch_small_prep(SmallItem *items, int count, const double *gamma, const double *beta, int p,
                              const int *item_s, const long long *item_kc, cudaStream_t st) {
    const int total = count * p;
    small_prep_kernel<<<(total + 127) / 128, 128, 0, st>>>(items, count, gamma, beta, p, item_s, item_kc);
    return cudaGetLastError();
}

int small_smem_bytes(int n, bool fp64, bool grad) {
    const int N = 1 << n;
    const int c2 = fp64 ? 16 : 8;
    return N * c2 * (grad ? 2 : 1) + N * 4;
}

cudaError_t launch_small(const SmallItem *items_dev, int count, int max_n, bool fp64, bool grad,
                         cudaStream_t st) {
    const int smem = small_smem_bytes(max_n, fp64, grad);
    cudaError_t e;
    if (fp64) {
        if ((e = cudaFuncSetAttribute(small_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
            return e;
        small_kernel<double><<<count, 512, smem, st>>>(items_dev);
    } else {
        if ((e = cudaFuncSetAttribute(small_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
            return e;
        small_kernel<float><<<count, 512, smem, st>>>(items_dev);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// DQAOA factorisation check (Sec. 3.2): for every x,
//   T[x] == c_off + sum_m L_m[u_m(x)] + sum_{m<m'} sum_{a in m} z_a V_{m,m'}[u_m'(x)][a]
// with u_m(x) the bits of QPU m's variables (exact integers).  The phase
// factors then agree as well: the library's phase is the turn count
// (T + k_c) phi mod 2^64, which is additive, so the integer identity implies
// e^{-i g F} = e^{-i g F_local} e^{-i g F_cross} up to the rounding of the
// phase routine itself.  That rounding is measured on a sample (the first x
// of every 1024) instead of at every x.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 phase_ll(long long v, unsigned long long phi, unsigned long long off) {
    const unsigned long long t = (unsigned long long)v * phi + off;
    const int32_t hi = (int32_t)((t + 0x80000000ull) >> 32);
    float s, c;
    __sincosf((float)hi * 1.4629180792671596e-09f, &s, &c);
    return make_float2(c, -s);
}

// |e^{-i g (T + k_c)} - e^{-i g (loc + k_c)} e^{-i g cross}| (max norm) with the
// library's phase routine, for one sampled entry
__device__ __forceinline__ float phase_split_err(long long tx, long long loc, long long cross, const FactArgs &a) {
    const float2 pf = phase_ll(tx + a.k_c, a.phi, 0ull);
    const float2 pl = phase_ll(loc + a.k_c, a.phi, 0ull);
    const float2 pc = phase_ll(cross, a.phi, 0ull);
    const float2 pp = cmul(pl, pc);
    return fmaxf(fabsf(pf.x - pp.x), fabsf(pf.y - pp.y));
}

__global__ void fact_check_kernel(FactArgs a) {
    __shared__ int qof[64], pos[64], qstart[17], qsize[16];
    __shared__ unsigned long long cnt_sh;
    __shared__ unsigned int err_sh;
    if (threadIdx.x < (unsigned)a.n) {
        qof[threadIdx.x] = a.qpu_of[threadIdx.x];
        pos[threadIdx.x] = a.pos_in_q[threadIdx.x];
    }
    if (threadIdx.x <= (unsigned)a.M) qstart[threadIdx.x] = a.q_start[threadIdx.x];
    if (threadIdx.x == 0) {
        cnt_sh = 0;
        err_sh = 0;
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)a.M) qsize[threadIdx.x] = qstart[threadIdx.x + 1] - qstart[threadIdx.x];
    __syncthreads();
    const long long N = 1ll << a.n;
    unsigned long long bad = 0;
    float maxerr = 0.f;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < N;
         x += (long long)gridDim.x * blockDim.x) {
        unsigned int u[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) u[m] = 0;
        for (int i = 0; i < a.n; ++i)
            if ((x >> i) & 1ll) {
                const int m = qof[i];
#pragma unroll
                for (int mm = 0; mm < 16; ++mm)
                    if (mm == m) u[mm] |= 1u << pos[i];
            }
        long long loc = a.c_off, cross = 0;
        for (int m = 0; m < a.M; ++m) {
            unsigned int um = 0;
#pragma unroll
            for (int mm = 0; mm < 16; ++mm)
                if (mm == m) um = u[mm];
            loc += a.Ltab[a.L_off[m] + um];
            for (int m2 = m + 1; m2 < a.M; ++m2) {
                unsigned int u2 = 0;
#pragma unroll
                for (int mm = 0; mm < 16; ++mm)
                    if (mm == m2) u2 = u[mm];
                const long long *Vrow = a.V + a.V_off[m * 16 + m2] + (size_t)u2 * qsize[m];
                for (int q = 0; q < qsize[m]; ++q)
                    if ((um >> q) & 1u) cross += Vrow[q];
            }
        }
        const int32_t tx = a.T[x];
        if ((long long)tx != loc + cross) ++bad;
        if ((x & 1023) == 0) maxerr = fmaxf(maxerr, phase_split_err(tx, loc, cross, a));
    }
    atomicAdd(&cnt_sh, bad);
    atomicMax(&err_sh, __float_as_uint(maxerr));
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(a.mismatches, cnt_sh);
        atomicMax(a.max_err_bits, err_sh);
    }
}

// Contiguous allocation (QPU m owns bits [s_m, s_m + c_m)).  x = u0 + 2^c0 hi
// with u0 the field of QPU 0.  The part of the split that does not depend on
// u0 (the local tables of QPUs 1..M-1 and their mutual cross terms) is formed
// once per hi by fact_hi_kernel; for each row hi the check forms
// W[q] = sum_{m >= 1} V_{0,m}[u_m][q] (QPU 0 variable q's cross coupling to
// the other QPUs' set variables) and two subset-sum tables of W over the low
// and high 8 bits of u0, so that the cross term of x is two table reads.
__global__ void fact_hi_kernel(FactArgs a, long long *Hhi) {
    const unsigned long long hi = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c0 = a.c0;
    if (hi >= (1ull << (a.n - c0))) return;
    long long h = a.c_off;
    for (int m = 1; m < a.M; ++m) {
        const int sm = a.q_start[m], cm = a.q_start[m + 1] - sm;
        const unsigned um = (unsigned)((hi >> (sm - c0)) & ((1u << cm) - 1u));
        h += a.Ltab[a.L_off[m] + um];
        for (int m2 = m + 1; m2 < a.M; ++m2) {
            const int s2 = a.q_start[m2], c2 = a.q_start[m2 + 1] - s2;
            const unsigned u2 = (unsigned)((hi >> (s2 - c0)) & ((1u << c2) - 1u));
            const long long *Vrow = a.V + a.V_off[m * 16 + m2] + (size_t)u2 * cm;
            for (int q = 0; q < cm; ++q)
                if ((um >> q) & 1u) h += Vrow[q];
        }
    }
    Hhi[hi] = h;
}

// A CTA checks rows hi = blockIdx.x, blockIdx.x + gridDim.x, ... (the bits
// above QPU 0); per row it forms W[q] and the subset-sum tables of W over the
// low and high 8 bits of u0, the latter from four 16-entry tables over 4 bits
// each (one add per entry).  Counts and the error bound are reduced once per
// CTA; every sum is an exact integer and the bound a maximum, so the result
// does not depend on the grid.
__global__ void __launch_bounds__(256) fact_check_contig_kernel(FactArgs a, const long long *__restrict__ Hhi,
                                                                long long nhi) {
    __shared__ long long wrow[16];
    __shared__ long long nib[4][16];
    __shared__ long long tlo[256], thi[256];
    __shared__ unsigned long long cnt_sh;
    __shared__ unsigned int err_sh;
    const int c0 = a.c0;
    const int klo = c0 < 8 ? c0 : 8;
    if (threadIdx.x == 0) {
        cnt_sh = 0;
        err_sh = 0;
    }
    unsigned long long bad = 0;
    float maxerr = 0.f;
    for (long long hi = blockIdx.x; hi < nhi; hi += gridDim.x) {
        __syncthreads();  // the previous row's table readers are done
        if (threadIdx.x < 16) {
            const int q = threadIdx.x;
            long long w = 0;
            if (q < c0)
                for (int m2 = 1; m2 < a.M; ++m2) {
                    const int s2 = a.q_start[m2], c2 = a.q_start[m2 + 1] - s2;
                    const unsigned u2 = (unsigned)((hi >> (s2 - c0)) & ((1u << c2) - 1u));
                    w += a.V[a.V_off[m2] + (size_t)u2 * c0 + q];
                }
            wrow[q] = w;  // 0 beyond QPU 0's c0 variables
        }
        __syncthreads();
        if (threadIdx.x < 64) {
            const int j = threadIdx.x >> 4, k = threadIdx.x & 15;
            long long t = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if ((k >> b) & 1) t += wrow[4 * j + b];
            nib[j][k] = t;
        }
        __syncthreads();
        {
            const int k = threadIdx.x;  // 256 threads: one entry of each table
            tlo[k] = nib[0][k & 15] + nib[1][k >> 4];
            thi[k] = nib[2][k & 15] + nib[3][k >> 4];
        }
        __syncthreads();
        const long long H = Hhi[hi];
        const int32_t *Tr = a.T + (hi << c0);
        for (unsigned u0 = threadIdx.x; u0 < (1u << c0); u0 += blockDim.x) {
            const long long cross = tlo[u0 & ((1u << klo) - 1u)] + thi[u0 >> klo];
            const long long loc = H + a.Ltab[u0];
            const int32_t tx = Tr[u0];
            if ((long long)tx != loc + cross) ++bad;
            if (((((unsigned long long)hi << c0) | u0) & 1023ull) == 0) maxerr = fmaxf(maxerr, phase_split_err(tx, loc, cross, a));
        }
    }
    // warp then CTA reduction of the counts and the error bound
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
        maxerr = fmaxf(maxerr, __shfl_xor_sync(0xffffffffu, maxerr, o));
    }
    if ((threadIdx.x & 31u) == 0) {
        if (bad) atomicAdd(&cnt_sh, bad);
        atomicMax(&err_sh, __float_as_uint(maxerr));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (cnt_sh) atomicAdd(a.mismatches, cnt_sh);
        atomicMax(a.max_err_bits, err_sh);
    }
}

// Contiguous allocation with QPU 0 of at least 10 variables: a warp checks
// tiles of 1024 consecutive x, each inside one row hi (bits 0..9 of u0 vary,
// its bits 10..c0-1 are fixed).  Lane l owns x = 128 k + 4 l + e (k = 0..7,
// e = 0..3): eight 16-byte table loads per lane, each instruction reading 512
// contiguous bytes, and the next tile's loads issued before the current one is
// checked.  Lanes 0..c0-1 compute the row's W_q (fact_w) and the warp shares
// them by shuffles, so no block barrier is needed: the cross term of an entry
// is the lane's sum over bits 2..6 (from l), plus the tile's bits >= 10, plus
// the constants of bits 7..9 (from k) and 0, W0, W1, W0 + W1 (from e).
__device__ __forceinline__ long long fact_w(const FactArgs &a, long long hi, int q) {
    long long w = 0;
    const int c0 = a.c0;
    for (int m2 = 1; m2 < a.M; ++m2) {
        const int s2 = a.q_start[m2], c2 = a.q_start[m2 + 1] - s2;
        const unsigned u2 = (unsigned)((hi >> (s2 - c0)) & ((1u << c2) - 1u));
        w += a.V[a.V_off[m2] + (size_t)u2 * c0 + q];
    }
    return w;
}

__global__ void __launch_bounds__(256, 2) fact_check_tiles_kernel(FactArgs a, const long long *__restrict__ Hhi,
                                                               long long ntiles) {
    __shared__ unsigned long long cnt_sh;
    __shared__ unsigned int err_sh;
    const int c0 = a.c0;
    const unsigned l = threadIdx.x & 31u;
    if (threadIdx.x == 0) {
        cnt_sh = 0;
        err_sh = 0;
    }
    unsigned long long bad = 0;
    float maxerr = 0.f;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    long long tile = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int4 nxt[8];
    if (tile < ntiles) {
#pragma unroll
        for (int k = 0; k < 8; ++k) nxt[k] = __ldcs(reinterpret_cast<const int4 *>(a.T + (tile << 10) + 128 * k + 4 * l));
    }
    for (; tile < ntiles; tile += nwarps) {
        int4 cur[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) cur[k] = nxt[k];
        if (tile + nwarps < ntiles) {
            const int32_t *src = a.T + ((tile + nwarps) << 10) + 4 * l;
#pragma unroll
            for (int k = 0; k < 8; ++k) nxt[k] = __ldcs(reinterpret_cast<const int4 *>(src + 128 * k));
        }
        const long long x0 = tile << 10;
        const long long hi = x0 >> c0;
        const unsigned uc = (unsigned)(x0 & ((1ll << c0) - 1));
        const long long wl = (int)l < c0 ? fact_w(a, hi, (int)l) : 0ll;
        // bits >= 10 of the tile (the same for the whole warp)
        long long chi = ((int)l >= 10 && ((uc >> l) & 1u)) ? wl : 0ll;
#pragma unroll
        for (int o = 8; o; o >>= 1) chi += __shfl_xor_sync(0xffffffffu, chi, o);
        long long w[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) w[q] = __shfl_sync(0xffffffffu, wl, q);
        long long cl = __shfl_sync(0xffffffffu, chi, 0);
#pragma unroll
        for (int q = 2; q < 7; ++q)
            if ((l >> (q - 2)) & 1u) cl += w[q];
        const long long H = Hhi[hi] + cl;
        const long long w01 = w[0] + w[1];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long ck = H + ((k & 1) ? w[7] : 0ll) + ((k & 2) ? w[8] : 0ll) + ((k & 4) ? w[9] : 0ll);
            const longlong2 l01 = __ldg(reinterpret_cast<const longlong2 *>(a.Ltab + uc + 128 * k + 4 * l));
            const longlong2 l23 = __ldg(reinterpret_cast<const longlong2 *>(a.Ltab + uc + 128 * k + 4 * l + 2));
            bad += (long long)cur[k].x != ck + l01.x;
            bad += (long long)cur[k].y != ck + l01.y + w[0];
            bad += (long long)cur[k].z != ck + l23.x + w[1];
            bad += (long long)cur[k].w != ck + l23.y + w01;
        }
        // phase rounding sampled on the first x of the tile
        if (l == 0) maxerr = fmaxf(maxerr, phase_split_err(cur[0].x, Hhi[hi] + a.Ltab[uc], cl, a));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
        maxerr = fmaxf(maxerr, __shfl_xor_sync(0xffffffffu, maxerr, o));
    }
    __syncthreads();  // cnt_sh / err_sh initialised before the first atomic
    if (l == 0) {
        if (bad) atomicAdd(&cnt_sh, bad);
        atomicMax(&err_sh, __float_as_uint(maxerr));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (cnt_sh) atomicAdd(a.mismatches, cnt_sh);
        atomicMax(a.max_err_bits, err_sh);
    }
}

bool fact_check_uses_tiles(const FactArgs &a) { return a.contiguous && a.c0 >= 10 && a.n - a.c0 >= 1; }

cudaError_t launch_fact_check(const FactArgs &a, cudaStream_t st) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (a.contiguous) {
        const unsigned long long nhi = 1ull << (a.n - a.c0);
        fact_hi_kernel<<<(unsigned)((nhi + 255) / 256), 256, 0, st>>>(a, a.hhi);
        if (fact_check_uses_tiles(a)) {
            // one warp per tile at a time, 8 per CTA; two CTAs per SM stay resident
            // (128 registers), each warp with two tiles of loads in flight
            const long long ntiles = 1ll << (a.n - 10);
            const long long ctas = (ntiles + 7) / 8;
            const long long grid = ctas < 2ll * sms ? ctas : 2ll * sms;
            fact_check_tiles_kernel<<<(unsigned)grid, 256, 0, st>>>(a, a.hhi, ntiles);
        } else {
            const long long grid = nhi < 2048 ? (long long)nhi : 2048;  // rows per CTA: nhi / 2048 from n - c0 = 11
            fact_check_contig_kernel<<<(unsigned)grid, 256, 0, st>>>(a, a.hhi, (long long)nhi);
        }
    } else {
        fact_check_kernel<<<(unsigned)(8 * sms), 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace qaoa
