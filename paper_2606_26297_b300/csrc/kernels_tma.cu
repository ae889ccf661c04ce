// TMA-pipelined persistent layer-pass kernels (sm_103a).
//
// Same arithmetic as the direct-load kernels in kernels_pass.cu (one fused
// [RX_G(beta_a)] [U_C(gamma)] [RX_G(beta_b)] step per 2^13-amplitude block,
// Eq. qaoa_state with boundary fusion), but each CTA is persistent (one per
// SM) and the amplitudes of its next block are brought into shared memory by
// the Tensor Memory Accelerator (cp.async.bulk.tensor for a high-group block,
// a 64 KB cp.async.bulk for a low-group block) while the current block is
// computed.  Completion is tracked by an mbarrier with transaction counts;
// every wait is bounded and a timeout sets the status word instead of hanging.
#include <cuda.h>

#include "pass_body.cuh"
#include "kernels_tma.h"
#include "tma_util.cuh"

namespace qaoa {

// Issue the copies of block b (psi, and lambda when TWO) into the stage.
template <int T, bool TWO>
__device__ __forceinline__ void issue_block(uint32_t b, const PassArgs &a, const CUtensorMap *mpsi,
                                            const CUtensorMap *mlam, float2 *stage, unsigned long long *mbar) {
    mbar_expect_tx(mbar, (TWO ? 2u : 1u) * 8192u * 8u);
    if (T == 0) {
        bulk_load(stage, a.psi + ((size_t)b << 13), 65536u, mbar);
        if (TWO) bulk_load(stage + 8192, a.lam + ((size_t)b << 13), 65536u, mbar);
    } else {
        const int nlow = a.lo - 3;
        const int c1 = (int)(b & ((1u << nlow) - 1u)), c4 = (int)(b >> nlow);
        tma_load_5d(stage, mpsi, c1, c4, mbar);
        if (TWO) tma_load_5d(stage + 8192, mlam, c1, c4, mbar);
    }
}

// Issue the copy of block b of the objective table (32 KB).
template <int T>
__device__ __forceinline__ void issue_cost(uint32_t b, const PassArgs &a, const CUtensorMap *mcost,
                                           int32_t *cstage, unsigned long long *mbar) {
    mbar_expect_tx(mbar, 8192u * 4u);
    if (T == 0) {
        bulk_load(cstage, a.C + ((size_t)b << 13), 32768u, mbar);
    } else {
        const int nlow = a.lo - 3;
        tma_load_5d(cstage, mcost, (int)(b & ((1u << nlow) - 1u)), (int)(b >> nlow), mbar);
    }
}

// ---------------------------------------------------------------------------
// forward pass (EPI: final pass of a gradient evaluation)
// ---------------------------------------------------------------------------
template <int T, bool EPI>
__global__ void __launch_bounds__(PASS_THREADS, 1)
    fwd_tma_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpsi, const __grid_constant__ CUtensorMap mcost,
                   int nblocks, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *stage = reinterpret_cast<float2 *>(smraw);                       // psi block, 64 KB
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 65536);            // table block, 32 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 65536 + 32768);        // transposes, 64 KB
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    __shared__ double red[PASS_THREADS / 32][NSLOT];
    __shared__ unsigned long long smk[8 * 16];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const bool pre = a.pre.mode != 0;
    const bool load = !a.init;
    const bool usec = a.has_cost || EPI;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&mbarc, 1);
    }
    __syncthreads();
    uint32_t parity = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nblocks) {
        if (load) issue_block<T, false>(blockIdx.x, a, &mpsi, nullptr, stage, &mbar);
        if (usec) issue_cost<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }

    for (uint32_t b = blockIdx.x; (int)b < nblocks; b += gridDim.x) {
        const size_t base = block_base<T>(b, a.lo);
        float2 *pb = a.psi + base;
        float2 v[32];
        int32_t c[32];
        if (load) {
            if (!stage_ready(&mbar, parity, status)) return;
            parity ^= 1u;
            if (pre) read_stage<T, 0>(v, stage, l, w);
            else read_stage<T, 1>(v, stage, l, w);
            __syncthreads();
            if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
                fence_proxy_async();
                issue_block<T, false>(b + gridDim.x, a, &mpsi, nullptr, stage, &mbar);
            }
        } else {
#pragma unroll
            for (int m = 0; m < 32; ++m) v[m] = make_float2(a.amp0, 0.f);
        }
        if (pre) {
            round_mix<T, 0>(v, a.pre, a.mask);
            transpose1<T, 0, 1>(v, xbuf, l, w, a.pre.flip ? a.mask : 0u);
            round_mix<T, 1>(v, a.pre, a.mask);
        }
        if (usec) {
            if (!stage_ready(&mbarc, parc, status)) return;
            parc ^= 1u;
            read_cost_stage<T, 1>(c, cstage, l, w);
            __syncthreads();
            if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
                fence_proxy_async();
                issue_cost<T>(b + gridDim.x, a, &mcost, cstage, &mbarc);
            }
        }
        if (a.has_cost) {
#pragma unroll
            for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], cost_phase(c[m], a.phi, a.off, a.kmag, a.precise_phase));
        }
        if constexpr (!EPI) {
            if (a.post.mode) {
                round_mix<T, 1>(v, a.post, a.mask);
                transpose1<T, 1, 0>(v, xbuf, l, w, a.post.flip ? a.mask : 0u);
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
#pragma unroll
            for (int m = 0; m < 32; ++m) v[m] = cmul(v[m], a.kend);
            float2 u[32];
            float e0 = 0.f, e1 = 0.f;
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                const float P = fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
                const float cf = (float)c[m];
                e0 = fmaf(P, cf, e0);
                e1 += P;
                u[m] = cscale(v[m], cf * a.cscale);
            }
            if (a.ktop > 0) {
                const size_t xthread = base + goff<T>(local_idx<T, 1>(l, 0u, w), a.lo);
                block_topk<T, 1>(v, xthread, a.lo, a.ktop, a.topk_keys + (size_t)b * a.ktop, smk);
            }
            const float x1 = xterm<T, 1>(u, v, a.mask);
            const MixOp ip = {a.pre.mode, a.pre.flip, -a.pre.t};
            round_mix<T, 1>(u, ip, a.mask);
            round_mix<T, 1>(v, ip, a.mask);
            transpose1<T, 1, 0>(v, xbuf, l, w, a.pre.flip ? a.mask : 0u);
            transpose1<T, 1, 0>(u, xbuf, l, w, a.pre.flip ? a.mask : 0u);
            const float x0 = xterm<T, 0>(u, v, a.mask);
            round_mix<T, 0>(u, ip, a.mask);
#pragma unroll
            for (int m = 0; m < 32; ++m) u[m] = cmul(u[m], a.kend2);
            store_arr<T, 0>(u, a.lam + base, l, w, a.lo);
            double vals[NSLOT] = {(double)e0, (double)e1, (double)x1, (double)x0, 0.0};
            block_sum_write(vals, red, a.partials, b);
            __syncthreads();  // red reused by the next block
        }
    }
}

// ---------------------------------------------------------------------------
// reverse (adjoint) pass; slots as in kernels_pass.cu
// ---------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(PASS_THREADS, 1)
    rev_tma_kernel(const PassArgs a, const __grid_constant__ CUtensorMap mpsi, const __grid_constant__ CUtensorMap mlam,
                   const __grid_constant__ CUtensorMap mcost, int nblocks, unsigned int *status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *stage = reinterpret_cast<float2 *>(smraw);                         // psi [8192], lambda [8192]
    int32_t *cstage = reinterpret_cast<int32_t *>(smraw + 131072);             // table block, 32 KB
    float2 *xbuf = reinterpret_cast<float2 *>(smraw + 131072 + 32768);         // transposes, 64 KB
    __shared__ __align__(8) unsigned long long mbar, mbarc;
    __shared__ double red[PASS_THREADS / 32][NSLOT];
    const uint32_t l = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const bool pre = a.pre.mode != 0, post = a.post.mode != 0;
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&mbarc, 1);
    }
    __syncthreads();
    uint32_t parity = 0, parc = 0;
    if (threadIdx.x == 0 && (int)blockIdx.x < nblocks) {
        issue_block<T, true>(blockIdx.x, a, &mpsi, &mlam, stage, &mbar);
        if (a.has_cost) issue_cost<T>(blockIdx.x, a, &mcost, cstage, &mbarc);
    }

    for (uint32_t b = blockIdx.x; (int)b < nblocks; b += gridDim.x) {
        const size_t base = block_base<T>(b, a.lo);
        float2 *pb = a.psi + base;
        float2 *lb = a.lam + base;
        float2 v[32], u[32];
        float acc[NSLOT] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (!stage_ready(&mbar, parity, status)) return;
        parity ^= 1u;
        if (post) {
            read_stage<T, 0>(v, stage, l, w);
            read_stage<T, 0>(u, stage + 8192, l, w);
        } else {
            read_stage<T, 1>(v, stage, l, w);
            read_stage<T, 1>(u, stage + 8192, l, w);
        }
        __syncthreads();
        if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
            fence_proxy_async();
            issue_block<T, true>(b + gridDim.x, a, &mpsi, &mlam, stage, &mbar);
        }
        if (post) {
            const MixOp ib = {a.post.mode, a.post.flip, -a.post.t};
            acc[0] = xterm<T, 0>(u, v, a.mask);
            round_mix<T, 0>(v, ib, a.mask);
            round_mix<T, 0>(u, ib, a.mask);
            transpose1<T, 0, 1>(v, xbuf, l, w, a.post.flip ? a.mask : 0u);
            transpose1<T, 0, 1>(u, xbuf, l, w, a.post.flip ? a.mask : 0u);
            acc[1] = xterm<T, 1>(u, v, a.mask);
            round_mix<T, 1>(v, ib, a.mask);
            round_mix<T, 1>(u, ib, a.mask);
        }
        if (a.has_cost) {
            int32_t c[32];
            if (!stage_ready(&mbarc, parc, status)) return;
            parc ^= 1u;
            read_cost_stage<T, 1>(c, cstage, l, w);
            __syncthreads();
            if (threadIdx.x == 0 && (int)(b + gridDim.x) < nblocks) {
                fence_proxy_async();
                issue_cost<T>(b + gridDim.x, a, &mcost, cstage, &mbarc);
            }
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
            transpose1<T, 1, 0>(v, xbuf, l, w, a.pre.flip ? a.mask : 0u);
            transpose1<T, 1, 0>(u, xbuf, l, w, a.pre.flip ? a.mask : 0u);
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
        block_sum_write(vals, red, a.partials, b);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static cudaError_t get_encoder() {
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return cudaSuccess;
}

// 5-D view of a high-group block: (carried bits 0..2) x (bits 3..lo-1) x
// (group bits 0..4) x (group bits 5..9) x (bits lo+10..n-1), elements of
// `esize` bytes (16: interleaved (psi, lambda), 8: complex64 amplitudes,
// 4: int32 table entries).
cudaError_t make_block_map(CUtensorMap *map, const void *base, int n, int lo, int esize) {
    std::memset(map, 0, sizeof(*map));
    cudaError_t e = get_encoder();
    if (e) return e;
    // 16-byte elements are described as pairs of 8-byte elements in dim 0
    const cuuint64_t es = (cuuint64_t)esize;
    const cuuint64_t d0 = esize == 16 ? 16ull : 8ull;
    cuuint64_t dims[5] = {d0, 1ull << (lo - 3), 32ull, 32ull, 1ull << (n - lo - 10)};
    cuuint64_t strides[4] = {8ull * es, es << lo, es << (lo + 5), es << (lo + 10)};
    cuuint32_t box[5] = {(cuuint32_t)d0, 1u, 32u, 32u, 1u};
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

cudaError_t launch_fwd_tma(int type, bool epi, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
    const int nblocks = 1 << (a.n - BLOCK_BITS);
    const int smem = 65536 + 32768 + 65536;
    CUtensorMap m, mc;
    std::memset(&m, 0, sizeof m);
    std::memset(&mc, 0, sizeof mc);
    cudaError_t e;
    if (type == 1 && !a.init && (e = make_block_map(&m, a.psi, a.n, a.lo, 8))) return e;
    if (type == 1 && (a.has_cost || epi) && (e = make_block_map(&mc, a.C, a.n, a.lo, 4))) return e;
    if (grid > nblocks) grid = nblocks;
    if (type == 0) {
        if (epi) {
            if ((e = set_smem(fwd_tma_kernel<0, true>, smem))) return e;
            fwd_tma_kernel<0, true><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nblocks, status);
        } else {
            if ((e = set_smem(fwd_tma_kernel<0, false>, smem))) return e;
            fwd_tma_kernel<0, false><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nblocks, status);
        }
    } else {
        if (epi) {
            if ((e = set_smem(fwd_tma_kernel<1, true>, smem))) return e;
            fwd_tma_kernel<1, true><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nblocks, status);
        } else {
            if ((e = set_smem(fwd_tma_kernel<1, false>, smem))) return e;
            fwd_tma_kernel<1, false><<<grid, PASS_THREADS, smem, st>>>(a, m, mc, nblocks, status);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_rev_tma(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st) {
    const int nblocks = 1 << (a.n - BLOCK_BITS);
    const int smem = 131072 + 32768 + 65536;
    CUtensorMap mp, ml, mc;
    std::memset(&mp, 0, sizeof mp);
    std::memset(&ml, 0, sizeof ml);
    std::memset(&mc, 0, sizeof mc);
    cudaError_t e;
    if (type == 1) {
        if ((e = make_block_map(&mp, a.psi, a.n, a.lo, 8))) return e;
        if ((e = make_block_map(&ml, a.lam, a.n, a.lo, 8))) return e;
        if (a.has_cost && (e = make_block_map(&mc, a.C, a.n, a.lo, 4))) return e;
    }
    if (grid > nblocks) grid = nblocks;
    if (type == 0) {
        if ((e = set_smem(rev_tma_kernel<0>, smem))) return e;
        rev_tma_kernel<0><<<grid, PASS_THREADS, smem, st>>>(a, mp, ml, mc, nblocks, status);
    } else {
        if ((e = set_smem(rev_tma_kernel<1>, smem))) return e;
        rev_tma_kernel<1><<<grid, PASS_THREADS, smem, st>>>(a, mp, ml, mc, nblocks, status);
    }
    return cudaGetLastError();
}

}  // namespace qaoa
