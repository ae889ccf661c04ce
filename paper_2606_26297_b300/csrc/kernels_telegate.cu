// Gate-level simulation of the distributed (TeleGate) QAOA circuit of Sec.
// 3.3: n data qubits plus the two communication qubits (bits n and n + 1),
// mid-circuit measurement, reset and classical feed-forward.  One CTA runs one
// trajectory with the whole 2^(n+2) state in shared memory (n <= 12: 128 KB)
// and interprets the op list; measurements reduce P(1) over the CTA, draw
// their random number from Philox4x32-10 and collapse the state.  At the end
// the CTA folds out the communication qubits (they finish in basis states)
// and measures the overlap with the monolithic state.
#include <cmath>

#include "kernels_misc.h"
#include "philox.cuh"

namespace qaoa {

namespace {

constexpr int TG_THREADS = 1024;

__device__ __forceinline__ uint32_t pair_lo(uint32_t k, int q) {
    return ((k >> q) << (q + 1)) | (k & ((1u << q) - 1u));
}

// FP64 sum over the CTA (every thread passes its part; all threads get the sum)
__device__ double cta_sum(double v, double *red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < TG_THREADS / 32; ++w) t += red[w];  // fixed order: same bits in every thread
    return t;
}

__global__ void __launch_bounds__(TG_THREADS, 1) telegate_kernel(const TgOp *__restrict__ ops, int nops, int n,
                                                                unsigned long long seed, int traj0,
                                                                float2 *data_out, const float2 *__restrict__ mono,
                                                                double *fid_out) {
    extern __shared__ float2 psi[];
    __shared__ double red[TG_THREADS / 32];
    __shared__ int slots[2];
    const uint32_t N = 1u << (n + 2);
    const uint32_t t = (uint32_t)(traj0 + (int)blockIdx.x);
    for (uint32_t x = threadIdx.x; x < N; x += TG_THREADS) psi[x] = make_float2(x == 0 ? 1.f : 0.f, 0.f);
    if (threadIdx.x < 2) slots[threadIdx.x] = 0;
    __syncthreads();
    for (int i = 0; i < nops; ++i) {
        const TgOp op = ops[i];
        const int q = op.q0;
        const uint32_t bit = 1u << q;
        switch (op.kind) {
            case TG_PHASE:
            case TG_GPHASE:
                for (uint32_t x = threadIdx.x; x < N; x += TG_THREADS)
                    if (op.kind == TG_GPHASE || (x & bit)) {
                        const float2 a = psi[x];
                        psi[x] = make_float2(a.x * op.c - a.y * op.s, a.x * op.s + a.y * op.c);
                    }
                break;
            case TG_RX:
            case TG_H:
            case TG_X:
                for (uint32_t k = threadIdx.x; k < N / 2; k += TG_THREADS) {
                    const uint32_t lo = pair_lo(k, q), hi = lo | bit;
                    const float2 a = psi[lo], b = psi[hi];
                    if (op.kind == TG_RX) {  // (a, b) -> (c a - i s b, -i s a + c b)
                        psi[lo] = make_float2(op.c * a.x + op.s * b.y, op.c * a.y - op.s * b.x);
                        psi[hi] = make_float2(op.s * a.y + op.c * b.x, -op.s * a.x + op.c * b.y);
                    } else if (op.kind == TG_H) {
                        const float r = 0.70710678118654752f;
                        psi[lo] = make_float2(r * (a.x + b.x), r * (a.y + b.y));
                        psi[hi] = make_float2(r * (a.x - b.x), r * (a.y - b.y));
                    } else {
                        psi[lo] = b;
                        psi[hi] = a;
                    }
                }
                break;
            case TG_Z:
                for (uint32_t x = threadIdx.x; x < N; x += TG_THREADS)
                    if (x & bit) psi[x] = make_float2(-psi[x].x, -psi[x].y);
                break;
            case TG_CNOT: {
                const uint32_t tb = 1u << op.q1;
                for (uint32_t k = threadIdx.x; k < N / 2; k += TG_THREADS) {
                    const uint32_t lo = pair_lo(k, op.q1);
                    if (lo & bit) {
                        const float2 a = psi[lo];
                        psi[lo] = psi[lo | tb];
                        psi[lo | tb] = a;
                    }
                }
                break;
            }
            case TG_MEASURE:
            case TG_RESET: {
                double part = 0.0;
                for (uint32_t x = threadIdx.x; x < N; x += TG_THREADS)
                    if (x & bit) part += (double)psi[x].x * psi[x].x + (double)psi[x].y * psi[x].y;
                const double p1 = cta_sum(part, red);
                int m;
                if (op.kind == TG_MEASURE) {
                    const Philox4 w = philox4x32_10((uint32_t)op.midx, t, 0u, 0x54454C45u, (uint32_t)seed,
                                                    (uint32_t)(seed >> 32));
                    const double u = (double)((((uint64_t)w.w[1] << 32) | w.w[0]) >> 11) * 0x1p-53;
                    m = u < p1 ? 1 : 0;
                } else {
                    m = p1 > 0.5 ? 1 : 0;
                }
                const double pm = m ? p1 : 1.0 - p1;
                const float sc = pm > 0.0 ? (float)(1.0 / sqrt(pm)) : 0.f;
                for (uint32_t k = threadIdx.x; k < N / 2; k += TG_THREADS) {
                    const uint32_t lo = pair_lo(k, q), hi = lo | bit;
                    const float2 keep = m ? psi[hi] : psi[lo];
                    const float2 v = make_float2(keep.x * sc, keep.y * sc);
                    if (op.kind == TG_RESET) {  // the kept value moves to |0>
                        psi[lo] = v;
                        psi[hi] = make_float2(0.f, 0.f);
                    } else {
                        psi[lo] = m ? make_float2(0.f, 0.f) : v;
                        psi[hi] = m ? v : make_float2(0.f, 0.f);
                    }
                }
                if (op.kind == TG_MEASURE && threadIdx.x == 0) slots[op.q1] = m;
                break;
            }
            case TG_XIF:
            case TG_ZIF:
                if (slots[op.q1]) {
                    if (op.kind == TG_ZIF) {
                        for (uint32_t x = threadIdx.x; x < N; x += TG_THREADS)
                            if (x & bit) psi[x] = make_float2(-psi[x].x, -psi[x].y);
                    } else {
                        for (uint32_t k = threadIdx.x; k < N / 2; k += TG_THREADS) {
                            const uint32_t lo = pair_lo(k, q);
                            const float2 a = psi[lo];
                            psi[lo] = psi[lo | bit];
                            psi[lo | bit] = a;
                        }
                    }
                }
                break;
            default:
                break;
        }
        __syncthreads();
    }
    // fold out the communication qubits and take the overlap with the monolithic state
    const uint32_t D = 1u << n;
    double re = 0.0, im = 0.0;
    for (uint32_t x = threadIdx.x; x < D; x += TG_THREADS) {
        float2 d = psi[x];
        for (uint32_t c = 1; c < 4; ++c) {
            d.x += psi[x | (c << n)].x;
            d.y += psi[x | (c << n)].y;
        }
        if (data_out) data_out[(size_t)blockIdx.x * D + x] = d;
        if (mono) {
            const float2 m = mono[x];
            re += (double)m.x * d.x + (double)m.y * d.y;
            im += (double)m.x * d.y - (double)m.y * d.x;
        }
    }
    const double sre = cta_sum(re, red);
    const double sim = cta_sum(im, red);
    if (threadIdx.x == 0 && fid_out) fid_out[blockIdx.x] = sre * sre + sim * sim;
}

}  // namespace

int telegate_smem_bytes(int n) { return (int)(sizeof(float2) << (n + 2)); }

cudaError_t launch_telegate(const TgOp *ops, int nops, int n, unsigned long long seed, int traj0, int count,
                            float2 *data_out, const float2 *mono, double *fid_out, cudaStream_t st) {
    const int smem = telegate_smem_bytes(n);
    cudaError_t e = cudaFuncSetAttribute(telegate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e) return e;
    telegate_kernel<<<count, TG_THREADS, smem, st>>>(ops, nops, n, seed, traj0, data_out, mono, fid_out);
    return cudaGetLastError();
}

}  // namespace qaoa
