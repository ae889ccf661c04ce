// Objective-table build on the tensor cores (tcgen05, sm_103a).
//
// The table of Eq. qubo_canonical_work, F(x) = c0 + sum_i l_i z_i +
// sum_{i<j} b_ij z_i z_j over all 2^n basis indices (the diagonal of H_C,
// Eq. cost_hamiltonian_raw), is split by x = x_lo + 2^{n_lo} x_hi into
//   F(x) = A_lo(x_lo) + A_hi(x_hi) + sum_{j < n_hi} W(x_lo, j) z_j(x_hi),
//   W(x_lo, j) = sum_{i < n_lo} z_i(x_lo) b_{i, n_lo + j},
// where A_lo holds c0, the low variables' linear terms and their couplings, and
// A_hi the same for the high variables.  The cross term is a dense product
// W (2^{n_lo} x 16) times Z_hi^T (16 x 2^{n_hi}, the 0/1 bits of x_hi), done by
// tcgen05.mma kind::f16 in 128 x 64 tiles with FP32 accumulators in tensor
// memory.  Exactness: W is cut into balanced base-2^11 digits (|digit| <= 1024,
// exact in f16); each digit's product sums at most 16 terms of magnitude
// <= 1024, so every FP32 accumulator is an exact integer (< 2^24); the epilogue
// recombines the digits in integers modulo 2^32, which gives the int32 table
// entry exactly.  The result is bit-identical to the integer definition for
// every fixed-point table.  Each finished tile is staged in shared memory and
// written by one tensor store (cp.async.bulk.tensor), double-buffered.
#include <climits>
#include <cstring>

#include <cuda_fp16.h>

#include "kernels_misc.h"
#include "tma_util.cuh"

namespace qaoa {

namespace {

constexpr int TM = 128;         // rows (x_lo) per tile
constexpr int TN = 64;          // columns (x_hi) per tile
constexpr int KP = 16;          // padded contraction length (n_hi <= 16)
constexpr int OPB = TM * KP * 2;  // bytes of one 128 x 16 f16 operand tile (4 KB)
constexpr int STILE_OFF = 24 * 1024;  // output tiles, after the operands (at most 4 x 4 + 4 KB + 256 B)
constexpr int TABLE_SMEM = STILE_OFF + 2 * TM * TN * 4;  // 88 KB: two CTAs per SM, not three

// ---- PTX wrappers ----------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (=|+=) A[smem] * B[smem]^T, M = 128, N = 128, K = 16, f16 in, f32 out
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory operand descriptor, K-major without swizzle: 8-row x 16-byte
// core matrices, K-adjacent core matrices 128 B apart (leading byte offset),
// 8-row groups 256 B apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t op_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
           (1ull << 46);
}

// kind::f16 instruction descriptor: D = F32, A = B = F16, both K-major, N, M.
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

// byte offset of element (r, k) of a 128 x 16 operand tile in the core-matrix layout
__device__ __forceinline__ uint32_t op_off(uint32_t r, uint32_t k) {
    return (r >> 3) * 256u + (k >> 3) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

}  // namespace

// ---- prep: A_lo, A_hi, W digits ---------------------------------------------------------
// One thread per index u < max(2^{n_lo}, 2^{n_hi}).  bsym: n x n, b_ij for i < j.
__global__ void table_prep_kernel(TableMmaArgs a) {
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = a.n, nlo = a.nlo, nhi = a.nhi;
    if (u < (1ll << nlo)) {
        long long f = a.c_off;
        for (int i = 0; i < nlo; ++i) {
            if (!((u >> i) & 1)) continue;
            f += a.ell[i];
            for (int k = i + 1; k < nlo; ++k)
                if ((u >> k) & 1) f += a.b[i * n + k];
        }
        a.alo[u] = f;
        for (int j = 0; j < KP; ++j) {
            long long w = 0;
            if (j < nhi)
                for (int i = 0; i < nlo; ++i)
                    if ((u >> i) & 1) w += a.b[i * n + nlo + j];
            // balanced base-2^11 digits, least significant first
            for (int d = 0; d < a.digits; ++d) {
                const long long r = ((w % 2048) + 2048) % 2048;
                const long long dig = r >= 1024 ? r - 2048 : r;
                a.wdig[((size_t)d << nlo) * KP + (size_t)u * KP + j] = __int2half_rn((int)dig);
                w = (w - dig) / 2048;
            }
        }
    }
    if (u < (1ll << nhi)) {
        long long f = 0;
        for (int j = 0; j < nhi; ++j) {
            if (!((u >> j) & 1)) continue;
            f += a.ell[nlo + j];
            for (int k = j + 1; k < nhi; ++k)
                if ((u >> k) & 1) f += a.b[(nlo + j) * n + nlo + k];
        }
        a.ahi[u] = f;
    }
}

// ---- the tile kernel ----------------------------------------------------------------------
// 256 threads, two CTAs per SM (each holds DIG x 64 tensor-memory columns,
// at most 256, so both allocations fit the SM's 512 columns and neither waits:
// the CTAs overlap one another's operand, MMA and epilogue latencies).  Warp w
// reads tensor-memory lanes 32 (w mod 4) .. +31 (tile rows, x_lo) and columns
// 32 (w / 4) .. +31 of the 64-column tile, one digit at a time.  The epilogue
// works modulo 2^32: T itself fits in int32, so wrapping int32 sums of A_lo,
// A_hi and the digit products give T exactly whatever the size of the parts.
// DIG = number of base-2^11 digits of W (1..4).
template <int DIG>
__global__ void __launch_bounds__(256, 2) table_mma_kernel(TableMmaArgs a, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *opA = smem;                                  // DIG x 4 KB
    unsigned char *opB = smem + DIG * OPB;                      // 2 KB (64 x 16 f16)
    int32_t *ahi_t = reinterpret_cast<int32_t *>(opB + OPB);    // 64 entries, mod 2^32
    int32_t *stiles = reinterpret_cast<int32_t *>(smem + STILE_OFF);  // two 128 x 64 output tiles
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tslot;
    __shared__ int32_t rv[8];
    __shared__ unsigned long long rx[8];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    constexpr uint32_t ncols = DIG == 1 ? 64u : (DIG == 2 ? 128u : 256u);
    if (warp == 0) tmem_alloc(&tslot, ncols);
    if (tid == 0) mbar_init(&mbar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const int nlo = a.nlo, nhi = a.nhi;
    const long long NT = 1ll << (nhi - 6);
    const long long ntiles = 1ll << (a.n - 13);
    const uint32_t row = (warp & 3u) * 32u + lane;  // tile row of this thread
    const int col0 = (int)(warp >> 2) * 32;         // first tile column of this thread
    const uint32_t kstep = 1u << (nlo - 7);         // (x >> 7) step of one column
    int32_t best = INT_MAX;
    uint32_t bestk = 0xFFFFFFFFu;  // x >> 7 of the best entry (row fixed per thread)
    long long cur_mt = -1;
    uint32_t parity = 0;
    bool ok = true;
    int it = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const long long mt = t / NT, nt = t % NT;
        // the output tile of this iteration reuses the buffer stored two tiles ago:
        // that store must have read it (its bulk group is the older of at most two)
        if (tid == 0) bulk_wait_read<1>();
        // operands: threads 0..127 write row `tid` of the A tiles, 0..63 row `tid` of B
        if (tid < 128) {
            if (mt != cur_mt) {
#pragma unroll
                for (int d = 0; d < DIG; ++d) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(a.wdig + ((size_t)d << nlo) * KP +
                                                                       (size_t)(mt * TM + tid) * KP);
                    const uint4 lo = src[0], hi = src[1];
                    *reinterpret_cast<uint4 *>(opA + d * OPB + op_off(tid, 0)) = lo;
                    *reinterpret_cast<uint4 *>(opA + d * OPB + op_off(tid, 8)) = hi;
                }
            }
            if (tid < TN) {
                const unsigned long long xh = (unsigned long long)(nt * TN + tid);
                uint32_t wds[KP / 2];
#pragma unroll
                for (int k = 0; k < KP; k += 2) {
                    const uint32_t b0 = (k < nhi && ((xh >> k) & 1ull)) ? 0x3C00u : 0u;  // f16 1.0
                    const uint32_t b1 = (k + 1 < nhi && ((xh >> (k + 1)) & 1ull)) ? 0x3C00u : 0u;
                    wds[k / 2] = b0 | (b1 << 16);
                }
                *reinterpret_cast<uint4 *>(opB + op_off(tid, 0)) = make_uint4(wds[0], wds[1], wds[2], wds[3]);
                *reinterpret_cast<uint4 *>(opB + op_off(tid, 8)) = make_uint4(wds[4], wds[5], wds[6], wds[7]);
                ahi_t[tid] = (int32_t)a.ahi[xh];
            }
            fence_proxy_async();
        }
        cur_mt = mt;
        // x = x_lo + 2^nlo x_hi, x_lo = mt 128 + row; read before the barrier so the load overlaps the MMA
        const unsigned long long xlo = (unsigned long long)(mt * TM + row);
        const int32_t alo = (int32_t)a.alo[xlo];
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            const uint64_t bdesc = op_desc(smem_u32(opB));
#pragma unroll
            for (int d = 0; d < DIG; ++d)
                mma_f16(tmem + (uint32_t)(d * TN), op_desc(smem_u32(opA + d * OPB)), bdesc, IDESC, 0u);
            mma_commit(&mbar);
        }
        ok = mbar_wait_bounded(&mbar, parity);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(a.status, 1u);
            mbar_wait_bounded(&mbar, parity);  // a last bounded chance for the MMAs in flight
            ok = false;
            break;
        }
        parity ^= 1u;
        tc_fence_after();
        // epilogue: digits one at a time into the integer sums u (modulo 2^32,
        // so a digit of weight 2^(11 d) >= 2^32 adds nothing).  An exact integer
        // |acc| <= 2^14 plus 1.5 * 2^23 has the bit pattern acc + 0x4B400000;
        // the constant times 2^(11 d) of every digit is taken off once, so a
        // digit costs one FADD and one shift-add.
        constexpr uint32_t kOff = 0x4B400000u * (1u + (DIG > 1 ? (1u << 11) : 0u) + (DIG > 2 ? (1u << 22) : 0u));
        const uint32_t base = (uint32_t)alo - kOff;
        uint32_t u[32];
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
            const int4 h = *reinterpret_cast<const int4 *>(ahi_t + col0 + j);
            u[j] = base + (uint32_t)h.x;
            u[j + 1] = base + (uint32_t)h.y;
            u[j + 2] = base + (uint32_t)h.z;
            u[j + 3] = base + (uint32_t)h.w;
        }
#pragma unroll
        for (int d = 0; d < (DIG < 3 ? DIG : 3); ++d) {
            float acc[32];
            tmem_ld32(tmem + (((warp & 3u) * 32u) << 16) + (uint32_t)(d * TN + col0), acc);
#pragma unroll
            for (int j = 0; j < 32; ++j) u[j] += (uint32_t)__float_as_int(acc[j] + 12582912.0f) << (11 * d);
        }
        // the tile goes to shared memory in the box order of the table's 2-D view
        // (x_lo inner, x_hi outer; 32 lanes write 32 consecutive words), then one
        // tensor store per tile
        int32_t *st = stiles + (it & 1) * (TM * TN) + col0 * TM + row;
        int32_t m = INT_MAX;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            st[j * TM] = (int32_t)u[j];
            m = min(m, (int32_t)u[j]);
        }
        fence_proxy_async();
        // argmin (value, then index): the index grows with j within the tile, so
        // only the first j holding the tile's minimum can improve (best, bestk)
        if (m <= best) {
            int jm = 0;
#pragma unroll
            for (int j = 31; j >= 0; --j)
                if ((int32_t)u[j] == m) jm = j;
            const uint32_t k = (((uint32_t)(nt * TN + col0) << (nlo - 7)) | (uint32_t)mt) + (uint32_t)jm * kstep;
            if (m < best || k < bestk) {
                best = m;
                bestk = k;
            }
        }
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tma_store_2d(&tmap, stiles + (it & 1) * (TM * TN), (int)(mt * TM), (int)(nt * TN));
            bulk_commit();
        }
    }
    // shared memory stays allocated until every store of the CTA has completed
    if (tid == 0) bulk_wait_all();
    // CTA argmin (value, then index)
    unsigned long long bestx = bestk == 0xFFFFFFFFu ? ~0ull : (((unsigned long long)bestk << 7) | row);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const int32_t ov = __shfl_xor_sync(0xffffffffu, best, o);
        const unsigned long long ox = __shfl_xor_sync(0xffffffffu, bestx, o);
        if (ov < best || (ov == best && ox < bestx)) {
            best = ov;
            bestx = ox;
        }
    }
    if (lane == 0) {
        rv[warp] = best;
        rx[warp] = bestx;
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < 8; ++w)
            if (rv[w] < rv[0] || (rv[w] == rv[0] && rx[w] < rx[0])) {
                rv[0] = rv[w];
                rx[0] = rx[w];
            }
        a.blk_val[blockIdx.x] = rv[0];
        a.blk_idx[blockIdx.x] = rx[0];
    }
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

int table_mma_digits(long long wmax) {
    // balanced base-2^11 digits: d digits cover |w| <= 1024 (2^{11 d} - 1) / (2^11 - 1)
    int d = 1;
    long long cover = 1024;
    while (d < 4 && wmax > cover) {
        cover = cover * 2048 + 1024;
        ++d;
    }
    return wmax > cover ? -1 : d;
}

cudaError_t launch_table_mma(TableMmaArgs a, int grid, cudaStream_t st) {
    a.nhi = a.n - 7 < KP ? a.n - 7 : KP;
    a.nlo = a.n - a.nhi;
    const long long m = 1ll << (a.nlo > a.nhi ? a.nlo : a.nhi);
    table_prep_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    const long long ntiles = 1ll << (a.n - 13);
    if (grid > ntiles) grid = (int)ntiles;
    // the table as a 2-D int32 tensor: x_lo (2^nlo, contiguous) x x_hi (2^nhi)
    CUtensorMap tmap;
    {
        PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
        if ((e = tensor_map_encoder(&encode))) return e;
        std::memset(&tmap, 0, sizeof(tmap));
        cuuint64_t dims[2] = {1ull << a.nlo, 1ull << a.nhi};
        cuuint64_t strides[1] = {4ull << a.nlo};
        cuuint32_t box[2] = {(cuuint32_t)TM, (cuuint32_t)TN};
        cuuint32_t estr[2] = {1u, 1u};
        const CUresult r = encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, a.T, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    // two CTAs per SM: the dynamic shared memory request keeps a third CTA off
    // the SM, so a tensor-memory allocation (at most 256 columns) never waits
    const int smem = TABLE_SMEM;
    switch (a.digits) {
        case 1:
            if ((e = cudaFuncSetAttribute(table_mma_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
                return e;
            table_mma_kernel<1><<<grid, 256, smem, st>>>(a, tmap);
            break;
        case 2:
            if ((e = cudaFuncSetAttribute(table_mma_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
                return e;
            table_mma_kernel<2><<<grid, 256, smem, st>>>(a, tmap);
            break;
        case 3:
            if ((e = cudaFuncSetAttribute(table_mma_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
                return e;
            table_mma_kernel<3><<<grid, 256, smem, st>>>(a, tmap);
            break;
        case 4:
            if ((e = cudaFuncSetAttribute(table_mma_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
                return e;
            table_mma_kernel<4><<<grid, 256, smem, st>>>(a, tmap);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    if ((e = cudaGetLastError())) return e;
    return launch_argmin_reduce(a.blk_val, a.blk_idx, grid, a.min_val, a.min_idx, st);
}

}  // namespace qaoa
