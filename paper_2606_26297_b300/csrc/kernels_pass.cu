// Forward layer-pass kernel (direct global loads), partial-sum reduction and
// top-K merge (sm_103a).
//
// One pass streams the state through HBM once and, per 2^13-amplitude block
// held by a CTA, applies a fused sequence on one qubit group G (<= 10 qubits):
//     [RX_G(2 beta_a)] [U_C(gamma) (diagonal phase)] [RX_G(2 beta_b)]
// which realises, across passes, the state of Eq. qaoa_state: consecutive
// layers share their boundary group, so layer l's last group, the cost layer
// l+1 and layer l+1's first group run in one pass (U_C is diagonal and the
// RX of different qubits commute, Sec. 2.3).  A launch covers every item of
// a batch (grid = items x blocks); item i has its own angles (PassScal).
#include "pass_body.cuh"

namespace qaoa {

template <int T, bool INIT, bool PRE, bool COST, bool POST, bool FULL>
__global__ void __launch_bounds__(PASS_THREADS, 2) fwd_pass_kernel(const PassArgs a) {
    const uint32_t mask = FULL ? full_mask<T>() : a.mask;
    extern __shared__ __align__(16) float2 sm[];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const int nbits = a.n - BLOCK_BITS;
    const uint32_t item = blockIdx.x >> nbits, b = blockIdx.x & ((1u << nbits) - 1u);
    const PassScal sc = a.scal[item];
    const size_t base = block_base<T>(b, a.loA, a.loB);
    const float2 *pb = a.psi + ((size_t)item << a.n) + base;
    float2 *po = (a.psi_out ? a.psi_out : a.psi) + ((size_t)item << a.n) + base;
    const int32_t *cb = a.C + ((size_t)(a.item_table ? a.item_table[item] : 0) << a.n) + base;
    float2 v[32];
    if (INIT) {
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = make_float2(a.amp0, 0.f);
    } else if (PRE) {
        load_arr<T, 0>(v, pb, l, w, a.loA, a.loB);
    } else {
        load_arr<T, 1>(v, pb, l, w, a.loA, a.loB);
    }
    if (PRE) {
        round_mix<T, 0>(v, sc.pre_t, mask);
        transpose1<T, 0, 1, false>(v, sm, l, w, sc.pre_flip ? mask : 0u);  // first use of sm
        round_mix<T, 1>(v, sc.pre_t, mask);
    }
    // arrangement Y
    if (COST) {
        int32_t c[32];
        load_cost<T, 1>(c, cb, l, w, a.loA, a.loB);
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], cost_phase(c[m], sc.phi, sc.off, sc.kmag, a.precise_phase));
    }
    if (POST) {
        round_mix<T, 1>(v, sc.post_t, mask);
        transpose1<T, 1, 0, PRE>(v, sm, l, w, sc.post_flip ? mask : 0u);  // first use of sm without PRE
        round_mix<T, 0>(v, sc.post_t, mask);
        if (!COST) {
#pragma unroll
            for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], sc.kend);
        }
        store_arr<T, 0>(v, po, l, w, a.loA, a.loB);
    } else {
        if (!COST) {
#pragma unroll
            for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], sc.kend);
        }
        store_arr<T, 1>(v, po, l, w, a.loA, a.loB);
    }
}

// out[(item)*NSLOT + s] = sum over blocks b of in[(item*nblocks + b)*NSLOT + s],
// in a fixed order (deterministic).  One CTA per (item, slot).
__global__ void reduce_partials_kernel(const double *__restrict__ in, int nblocks, double *__restrict__ out) {
    __shared__ double sh[256];
    const int item = blockIdx.x / NSLOT, s = blockIdx.x % NSLOT;
    const double *src = in + (size_t)item * nblocks * NSLOT;
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) t += src[(size_t)b * NSLOT + s];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int k = 128; k; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)item * NSLOT + s] = sh[0];
}

// First stage of the per-pass partial sums when an item has many units: CTA
// (c, item) sums units [256 c, 256 c + 256) of the item for every slot; warp s
// takes slot s, its lanes the units lane, lane + 32, ... in order, then a
// fixed shuffle tree.  out[(item * nchunks + c) * NSLOT + s].  The chunking is
// fixed, so the sums do not depend on the GPU's size.
constexpr int REDUCE_CHUNK = 256;
static_assert(NSLOT * 32 == 256, "one warp per slot");
__global__ void __launch_bounds__(256) reduce_chunks_kernel(const double *__restrict__ in, int nblocks, int nchunks,
                                                            double *__restrict__ out) {
    const int item = blockIdx.y, c = blockIdx.x;
    const int l = threadIdx.x & 31, s = threadIdx.x >> 5;
    const double *src = in + ((size_t)item * nblocks + (size_t)c * REDUCE_CHUNK) * NSLOT + s;
    const int rows = min(REDUCE_CHUNK, nblocks - c * REDUCE_CHUNK);
    double t = 0.0;
    for (int r = l; r < rows; r += 32) t += src[(size_t)r * NSLOT];
#pragma unroll
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) out[((size_t)item * nchunks + c) * NSLOT + s] = t;
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
        unsigned long long bk = mine;
        int owner = threadIdx.x;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, bk, o);
            const int to = __shfl_xor_sync(0xffffffffu, owner, o);
            if (t > bk || (t == bk && to < owner)) {
                bk = t;
                owner = to;
            }
        }
        if (l == 0) {
            wbest[w] = bk;
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

template <int T, bool INIT, bool PRE, bool COST, bool POST, bool FULL>
static cudaError_t fwd_launch_f(const PassArgs &a, cudaStream_t st) {
    const unsigned grid = (unsigned)a.nitems << (a.n - BLOCK_BITS);
    const int smem = 8192 * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(fwd_pass_kernel<T, INIT, PRE, COST, POST, FULL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e) return e;
    fwd_pass_kernel<T, INIT, PRE, COST, POST, FULL><<<grid, PASS_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// a full group (every register bit mixed) gets code without per-bit tests
template <int T, bool INIT, bool PRE, bool COST, bool POST>
static cudaError_t fwd_launch(const PassArgs &a, cudaStream_t st) {
    return a.mask == full_mask<T>() ? fwd_launch_f<T, INIT, PRE, COST, POST, true>(a, st)
                                    : fwd_launch_f<T, INIT, PRE, COST, POST, false>(a, st);
}

// One instantiation per pass shape (first pass, mixer only, cost layer, ...):
// specialised code keeps each shape's registers and instruction stream lean
// (about 12% faster forward passes than one kernel branching at run time).
template <int T>
static cudaError_t fwd_dispatch(const PassArgs &a, cudaStream_t st) {
    const int key = (a.init ? 8 : 0) | (a.has_pre ? 4 : 0) | (a.has_cost ? 2 : 0) | (a.has_post ? 1 : 0);
    switch (key) {
        case 1: return fwd_launch<T, false, false, false, true>(a, st);
        case 7: return fwd_launch<T, false, true, true, true>(a, st);
        case 11: return fwd_launch<T, true, false, true, true>(a, st);
        case 8: return fwd_launch<T, true, false, false, false>(a, st);
        case 4: return fwd_launch<T, false, true, false, false>(a, st);
        case 9: return fwd_launch<T, true, false, false, true>(a, st);
        default: return cudaErrorInvalidValue;  // no schedule produces another shape
    }
}

cudaError_t launch_fwd_pass(int type, const PassArgs &a, cudaStream_t st) {
    return type == 0 ? fwd_dispatch<0>(a, st) : fwd_dispatch<1>(a, st);
}

cudaError_t launch_reduce_partials(const double *partials, int nitems, int nblocks, double *out, cudaStream_t st) {
    reduce_partials_kernel<<<nitems * NSLOT, 256, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

int reduce_chunk_count(int nblocks) {
    const int nchunks = (nblocks + REDUCE_CHUNK - 1) / REDUCE_CHUNK;
    return nchunks >= 64 ? nchunks : 0;  // from 2^14 units (n >= 27): below, the one-stage sum is as fast
}

cudaError_t launch_reduce_partials_chunked(const double *partials, int nitems, int nblocks, double *scratch,
                                           double *out, int *launches, cudaStream_t st) {
    const int nchunks = reduce_chunk_count(nblocks);
    if (nchunks == 0 || nitems > 65535 || !scratch) {
        *launches = 1;
        return launch_reduce_partials(partials, nitems, nblocks, out, st);
    }
    reduce_chunks_kernel<<<dim3((unsigned)nchunks, (unsigned)nitems), 256, 0, st>>>(partials, nblocks, nchunks, scratch);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    *launches = 2;
    return launch_reduce_partials(scratch, nitems, nchunks, out, st);
}

// Repeatedly merge until one list remains.  `in` holds nlists lists of K keys;
// `out` must hold ceil(nlists/256)*K keys; the two buffers are used as
// ping-pong scratch (`in` is overwritten).  *nout: 0 = the final list is in
// `in`, 1 = in `out`; *nlaunch: kernels launched.
cudaError_t launch_topk_merge(const unsigned long long *in_c, int nlists, int k, unsigned long long *out, int *nout,
                              int *nlaunch, cudaStream_t st) {
    unsigned long long *bufs[2] = {const_cast<unsigned long long *>(in_c), out};
    int cur = 0;
    *nlaunch = 0;
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
