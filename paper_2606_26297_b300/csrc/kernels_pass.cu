// Layer-pass kernels of the QAOA statevector path (sm_103a).
//
// One pass streams the state through HBM once and, per 2^13-amplitude block
// held by a CTA, applies a fused sequence on one qubit group G (<= 10 qubits):
//     [RX_G(2 beta_a)] [U_C(gamma) (diagonal phase)] [RX_G(2 beta_b)]
// which realises, across passes, the state of Eq. qaoa_state: consecutive
// layers share their boundary group, so layer l's last group, the cost layer
// l+1 and layer l+1's first group run in one pass (U_C is diagonal and the
// RX of different qubits commute, Sec. 2.3).
//
// Forward pass: psi in -> psi out (in place).  With EPI (final pass of a
// gradient evaluation) it also forms lambda = H_C psi_p, the FP64 partial sums
// of <H_C> (Eq. qaoa_expectation_expanded), the top-K candidates, and the
// first reverse step, and writes lambda instead of psi.
// Reverse pass: undoes one forward pass on (psi, lambda) and accumulates
// 2 Im<lambda| sum_j X_j |psi> (d/d beta) and 2 Im<lambda|H_C|psi> (d/d gamma)
// as block partial sums.
#include "pass_body.cuh"

namespace qaoa {

// ---------------------------------------------------------------------------
// forward pass
// ---------------------------------------------------------------------------
template <int T, bool EPI>
__global__ void __launch_bounds__(PASS_THREADS, EPI ? 1 : 2) fwd_pass_kernel(const PassArgs a) {
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red[PASS_THREADS / 32][NSLOT];
    __shared__ unsigned long long smk[8 * 16];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const size_t base = block_base<T>(blockIdx.x, a.lo);
    float2 *pb = a.psi + base;
    const int32_t *cb = a.C + base;
    const bool pre = a.pre.mode != 0;
    float2 v[32];

    if (a.init) {
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = make_float2(a.amp0, 0.f);
    } else if (pre) {
        load_arr<T, 0>(v, pb, l, w, a.lo);
    } else {
        load_arr<T, 1>(v, pb, l, w, a.lo);
    }
    if (pre) {
        round_mix<T, 0>(v, a.pre, a.mask);
        transpose1<T, 0, 1>(v, sm, l, w, a.pre.flip ? a.mask : 0u);
        round_mix<T, 1>(v, a.pre, a.mask);
    }
    // arrangement Y
    if (a.has_cost) {
        int32_t c[32];
        load_cost<T, 1>(c, cb, l, w, a.lo);
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], cost_phase(c[m], a.phi, a.off, a.kmag, a.precise_phase));
    }
    if constexpr (!EPI) {
        if (a.post.mode) {
            round_mix<T, 1>(v, a.post, a.mask);
            transpose1<T, 1, 0>(v, sm, l, w, a.post.flip ? a.mask : 0u);
            round_mix<T, 0>(v, a.post, a.mask);
            if (!a.has_cost) {
#pragma unroll
                for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], a.kend);
            }
            store_arr<T, 0>(v, pb, l, w, a.lo);
        } else {
            if (!a.has_cost) {
#pragma unroll
                for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], a.kend);
            }
            store_arr<T, 1>(v, pb, l, w, a.lo);
        }
    } else {
        // psi_p = kend * v  (arrangement Y)
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], a.kend);
        float2 u[32];
        float e0 = 0.f, e1 = 0.f;
        {
            int32_t c[32];
            load_cost<T, 1>(c, cb, l, w, a.lo);
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                const float P = fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
                const float cf = (float)c[m];
                e0 = fmaf(P, cf, e0);
                e1 += P;
                u[m] = cscale(v[m], cf * a.cscale);  // lambda = H_C psi (shifted by k_c 2^-s)
            }
        }
        if (a.ktop > 0) {
            const size_t xthread = base + goff<T>(local_idx<T, 1>(l, 0u, w), a.lo);
            block_topk<T, 1>(v, xthread, a.lo, a.ktop, a.topk_keys + (size_t)blockIdx.x * a.ktop, smk);
        }
        const float x1 = xterm<T, 1>(u, v, a.mask);
        const MixOp ip = {a.pre.mode, a.pre.flip, -a.pre.t};
        round_mix<T, 1>(u, ip, a.mask);
        round_mix<T, 1>(v, ip, a.mask);
        transpose2<T, 1, 0>(v, u, sm, l, w, a.pre.flip ? a.mask : 0u);
        const float x0 = xterm<T, 0>(u, v, a.mask);
        round_mix<T, 0>(u, ip, a.mask);
#pragma unroll
        for (int m = 0; m < 32; ++m) u[m] = cmul(u[m], a.kend2);
        store_arr<T, 0>(u, a.lam + base, l, w, a.lo);
        double vals[NSLOT] = {(double)e0, (double)e1, (double)x1, (double)x0, 0.0};
        block_sum_write(vals, red, a.partials, blockIdx.x);
    }
}

// ---------------------------------------------------------------------------
// reverse (adjoint) pass: inverse of one forward pass on (psi, lambda)
// slots: 0,1 = X-terms of the post mixer (arrangement X, Y); 2 = cost term;
//        3,4 = X-terms of the pre mixer (arrangement Y, X)
// ---------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(PASS_THREADS, 1) rev_pass_kernel(const PassArgs a) {
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red[PASS_THREADS / 32][NSLOT];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const size_t base = block_base<T>(blockIdx.x, a.lo);
    float2 *pb = a.psi + base;
    float2 *lb = a.lam + base;
    const int32_t *cb = a.C + base;
    const bool pre = a.pre.mode != 0, post = a.post.mode != 0;
    float2 v[32], u[32];
    float acc[NSLOT] = {0.f, 0.f, 0.f, 0.f, 0.f};

    if (post) {
        load_arr<T, 0>(v, pb, l, w, a.lo);
        load_arr<T, 0>(u, lb, l, w, a.lo);
        const MixOp ib = {a.post.mode, a.post.flip, -a.post.t};
        acc[0] = xterm<T, 0>(u, v, a.mask);
        round_mix<T, 0>(v, ib, a.mask);
        round_mix<T, 0>(u, ib, a.mask);
        transpose2<T, 0, 1>(v, u, sm, l, w, a.post.flip ? a.mask : 0u);
        acc[1] = xterm<T, 1>(u, v, a.mask);
        round_mix<T, 1>(v, ib, a.mask);
        round_mix<T, 1>(u, ib, a.mask);
    } else {
        load_arr<T, 1>(v, pb, l, w, a.lo);
        load_arr<T, 1>(u, lb, l, w, a.lo);
    }
    // arrangement Y
    if (a.has_cost) {
        int32_t c[32];
        load_cost<T, 1>(c, cb, l, w, a.lo);
        float g = 0.f;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            g = fmaf((float)c[m], fmaf(u[m].x, v[m].y, -u[m].y * v[m].x), g);
            const float2 ph = cost_phase(c[m], a.phi, a.off, a.kmag, a.precise_phase);
            v[m] = cmul(v[m], ph);
            u[m] = cmul(u[m], ph);
        }
        acc[2] = g;
    }
    if (pre) {
        const MixOp ia = {a.pre.mode, a.pre.flip, -a.pre.t};
        acc[3] = xterm<T, 1>(u, v, a.mask);
        round_mix<T, 1>(v, ia, a.mask);
        round_mix<T, 1>(u, ia, a.mask);
        transpose2<T, 1, 0>(v, u, sm, l, w, a.pre.flip ? a.mask : 0u);
        acc[4] = xterm<T, 0>(u, v, a.mask);
        round_mix<T, 0>(v, ia, a.mask);
        round_mix<T, 0>(u, ia, a.mask);
        if (a.store_psi) {
            if (!a.has_cost) {
#pragma unroll
                for (int m = 0; m < 32; ++m) {
                    v[m] = cmul(v[m], a.kend);
                    u[m] = cmul(u[m], a.kend);
                }
            }
            store_arr<T, 0>(v, pb, l, w, a.lo);
            store_arr<T, 0>(u, lb, l, w, a.lo);
        }
    } else if (a.store_psi) {
        if (!a.has_cost) {
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                v[m] = cmul(v[m], a.kend);
                u[m] = cmul(u[m], a.kend);
            }
        }
        store_arr<T, 1>(v, pb, l, w, a.lo);
        store_arr<T, 1>(u, lb, l, w, a.lo);
    }
    double vals[NSLOT];
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) vals[s] = (double)acc[s];
    block_sum_write(vals, red, a.partials, blockIdx.x);
}

// ---------------------------------------------------------------------------
// deterministic column sums of per-block partials: out[s] = sum_b in[b*nslot+s]
// ---------------------------------------------------------------------------
__global__ void reduce_partials_kernel(const double *__restrict__ in, int nblocks, int nslot,
                                       double *__restrict__ out) {
    __shared__ double sh[256];
    const int s = blockIdx.x;
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) t += in[(size_t)b * nslot + s];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int k = 128; k; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[s] = sh[0];
}

// K-way merge of sorted (descending) key lists of length K.  CTA c merges
// lists [c*LPC, (c+1)*LPC) and writes its K best keys to out[c*K ...].
__global__ void topk_merge_kernel(const unsigned long long *__restrict__ in, int nlists, int K,
                                  unsigned long long *__restrict__ out) {
    __shared__ unsigned long long wbest[8];
    __shared__ int wowner[8];
    __shared__ int winner;
    const int lpc = blockDim.x;
    const int list = blockIdx.x * lpc + threadIdx.x;
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int head = 0;
    for (int r = 0; r < K; ++r) {
        const unsigned long long mine = (list < nlists && head < K) ? in[(size_t)list * K + head] : 0ull;
        unsigned long long b = mine;
        int owner = threadIdx.x;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
            const int to = __shfl_xor_sync(0xffffffffu, owner, o);
            if (t > b || (t == b && to < owner)) {
                b = t;
                owner = to;
            }
        }
        if (l == 0) {
            wbest[w] = b;
            wowner[w] = owner;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long bb = wbest[0];
            int oo = wowner[0];
            for (int k = 1; k < nw; ++k)
                if (wbest[k] > bb) {
                    bb = wbest[k];
                    oo = wowner[k];
                }
            out[(size_t)blockIdx.x * K + r] = bb;
            winner = bb ? oo : -1;
        }
        __syncthreads();
        if ((int)threadIdx.x == winner) ++head;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t ensure_smem(K kern, int bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_fwd_pass(int type, bool epi, const PassArgs &a, cudaStream_t st) {
    const unsigned grid = 1u << (a.n - BLOCK_BITS);
    const int smem = (epi ? 2 : 1) * 8192 * (int)sizeof(float2);
    cudaError_t e;
    if (type == 0) {
        if (epi) {
            if ((e = ensure_smem(fwd_pass_kernel<0, true>, smem))) return e;
            fwd_pass_kernel<0, true><<<grid, PASS_THREADS, smem, st>>>(a);
        } else {
            if ((e = ensure_smem(fwd_pass_kernel<0, false>, smem))) return e;
            fwd_pass_kernel<0, false><<<grid, PASS_THREADS, smem, st>>>(a);
        }
    } else {
        if (epi) {
            if ((e = ensure_smem(fwd_pass_kernel<1, true>, smem))) return e;
            fwd_pass_kernel<1, true><<<grid, PASS_THREADS, smem, st>>>(a);
        } else {
            if ((e = ensure_smem(fwd_pass_kernel<1, false>, smem))) return e;
            fwd_pass_kernel<1, false><<<grid, PASS_THREADS, smem, st>>>(a);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_rev_pass(int type, const PassArgs &a, cudaStream_t st) {
    const unsigned grid = 1u << (a.n - BLOCK_BITS);
    const int smem = 2 * 8192 * (int)sizeof(float2);
    cudaError_t e;
    if (type == 0) {
        if ((e = ensure_smem(rev_pass_kernel<0>, smem))) return e;
        rev_pass_kernel<0><<<grid, PASS_THREADS, smem, st>>>(a);
    } else {
        if ((e = ensure_smem(rev_pass_kernel<1>, smem))) return e;
        rev_pass_kernel<1><<<grid, PASS_THREADS, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double *partials, int nblocks, int nslot, double *out,
                                   cudaStream_t st) {
    reduce_partials_kernel<<<nslot, 256, 0, st>>>(partials, nblocks, nslot, out);
    return cudaGetLastError();
}

// Repeatedly merge until one list remains.  `in` holds nlists lists of K keys;
// `out` must hold ceil(nlists/256)*K keys and is used as ping-pong scratch
// together with `in` (which is overwritten).  The final list is left in
// whichever buffer *nout points to: 0 = in, 1 = out.
cudaError_t launch_topk_merge(const unsigned long long *in_c, int nlists, int k, unsigned long long *out,
                              int *nout, int *nlaunch, cudaStream_t st) {
    *nlaunch = 0;
    unsigned long long *bufs[2] = {const_cast<unsigned long long *>(in_c), out};
    int cur = 0;
    while (nlists > 1) {
        const int threads = nlists >= 256 ? 256 : ((nlists + 31) / 32) * 32;
        const int ctas = (nlists + threads - 1) / threads;
        topk_merge_kernel<<<ctas, threads, 0, st>>>(bufs[cur], nlists, k, bufs[1 - cur]);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
        cur = 1 - cur;
        nlists = ctas;
        ++*nlaunch;
    }
    *nout = cur;
    return cudaSuccess;
}

}  // namespace qaoa
