// Argument blocks and launchers of kernels_misc.cu.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "qaoa_internal.h"

namespace qaoa {

struct CostBuildArgs {
    int n, nlo, t;
    const long long *ell;      // [n]    fixed-point linear coefficients (device)
    const long long *b;        // [n*n]  fixed-point couplings, upper triangle (device)
    long long c_off;           // c0_q - k_c
    int32_t *T;                // [2^n]  table out
    long long *blk_val;        // [blocks] per-CTA minimum
    unsigned long long *blk_idx;
    long long *min_val;        // final minimum (device scalar)
    unsigned long long *min_idx;
};
cudaError_t launch_cost_build(CostBuildArgs a, int *nblocks_out, cudaStream_t st);
int cost_build_blocks(int n);
cudaError_t launch_argmin_reduce(const long long *val, const unsigned long long *idx, int m, long long *oval,
                                 unsigned long long *oidx, cudaStream_t st);

// Tensor-core table build (kernels_table_mma.cu), n >= 14.
struct TableMmaArgs {
    int n, nlo, nhi, digits;
    const long long *ell;      // [n]    fixed-point linear coefficients (device)
    const long long *b;        // [n*n]  fixed-point couplings, upper triangle (device)
    long long c_off;           // c0_q - k_c
    long long *alo;            // [2^nlo] objective of the low variables (+ c_off)
    long long *ahi;            // [2^nhi] objective of the high variables
    __half *wdig;              // [digits][2^nlo][16] base-2^11 digits of W
    int32_t *T;                // [2^n] table out
    long long *blk_val;        // [grid] per-CTA minimum
    unsigned long long *blk_idx;
    long long *min_val;        // final minimum (device scalar)
    unsigned long long *min_idx;
    unsigned int *status;      // set if a bounded wait expired
};
int table_mma_digits(long long wmax);  // -1 if W does not fit 4 digits
cudaError_t launch_table_mma(TableMmaArgs a, int grid, cudaStream_t st);

cudaError_t launch_expect(const float2 *psi, const int32_t *T, int n, double *partials, cudaStream_t st);
cudaError_t launch_gather(const void *amps, int esize, int n, const unsigned long long *idx, int count, void *out,
                          unsigned int *bad, cudaStream_t st);
cudaError_t launch_topk_chunks(const float2 *psi, int n, int K, unsigned long long *out, cudaStream_t st);

constexpr int SMALL_MAXP = 64;
constexpr int SMALL_MAXN = 12;

// One small-n evaluation (n <= 12): the whole state lives in shared memory.
struct SmallItem {
    const int32_t *T;          // table (device)
    void *psi_out;             // optional final state (complex64 or complex128), device
    double *out;               // [1 + 2p]: E, dE/dgamma[p], dE/dbeta[p] (device)
    unsigned long long *topk;  // [ktop] keys (device)
    int n, p, grad, ktop, precise;
    float amp0;
    double cscale;             // 2^-s
    long long k_c;
    unsigned long long phi[SMALL_MAXP], off[SMALL_MAXP];
    double cb[SMALL_MAXP], sb[SMALL_MAXP];  // cos, sin of beta_l
};
int small_smem_bytes(int n, bool fp64, bool grad);
cudaError_t launch_small(const SmallItem *items_dev, int count, int max_n, bool fp64, bool grad,
                         cudaStream_t st);
cudaError_t launch_small_prep(SmallItem *items, int count, const double *gamma, const double *beta, int p,
                              const int *item_s, const long long *item_kc, cudaStream_t st);

// One state measured by shots (kernels_sample.cu).  Device pointers.
struct SampleItem {
    const void *amps;                  // [2^n] complex64 (float2) or complex128 (double2)
    const int32_t *T;                  // [2^n] objective table, or null (no costs)
    unsigned long long *chunk;         // [sample_chunk_count(n)] scratch
    unsigned long long *sup;           // [sample_super_count(n)] scratch
    unsigned long long *total;         // [1] Q = sum of the weights
    const unsigned long long *rand;    // [shots] random integers, or null: Philox(seed, stream, s)
    unsigned long long *idx;           // [shots] measured indices, or null
    int32_t *tval;                     // [shots] table values of the measured indices, or null
    long long *tsum;                   // [1] += sum of the table values (zeroed by the caller), or null
    unsigned long long seed, stream;
    long long shots;
    int n;
};
long long sample_chunk_count(int n);
long long sample_super_count(int n);
// weights + per-item scan; then the caller checks Q and the status (bit 4: a
// component with |v| >= 2, infinite or NaN) and launches the shots
cudaError_t launch_sample_weights(const SampleItem *items_dev, int count, int max_n, bool fp64,
                                  unsigned int *status, cudaStream_t st);
cudaError_t launch_sample_shots(const SampleItem *items_dev, int count, long long max_shots, bool fp64,
                                unsigned int *status, cudaStream_t st);

// One operation of the distributed (TeleGate) circuit (kernels_telegate.cu).
enum TgKind { TG_PHASE = 0, TG_RX, TG_H, TG_X, TG_Z, TG_CNOT, TG_MEASURE, TG_XIF, TG_ZIF, TG_GPHASE, TG_RESET };
struct TgOp {
    int32_t kind;
    int32_t q0, q1;  // qubit; second qubit (CNOT target) or outcome slot (MEASURE, XIF, ZIF)
    int32_t midx;    // running index of a MEASURE (its random-number counter)
    float c, s;      // cos and sin of the angle (PHASE, GPHASE: e^{i theta}; RX: exp(-i theta X))
};
int telegate_smem_bytes(int n);
cudaError_t launch_telegate(const TgOp *ops, int nops, int n, unsigned long long seed, int traj0, int count,
                            float2 *data_out, const float2 *mono, double *fid_out, cudaStream_t st);

// arithmetic-pipe micro-benchmarks (kernels_peak.cu)
cudaError_t launch_peak(int kind, int blocks, int iters, float *out, cudaStream_t st);
double peak_ops_per_launch(int blocks, int iters);

struct FactArgs {
    const int32_t *T;
    int n, M;
    const int *qpu_of;        // [n]
    const int *pos_in_q;      // [n] position of variable i inside its QPU
    const int *q_start;       // [M+1] prefix sums of QPU sizes
    const long long *Ltab;    // concatenated per-QPU local tables
    const long long *L_off;   // [M]
    const long long *V;       // concatenated pair tables V_{m,m'}[u'][a]
    const long long *V_off;   // [16*16]
    long long c_off;          // c0_q - k_c
    long long k_c;
    unsigned long long phi;   // probe phase multiplier
    unsigned long long *mismatches;
    unsigned int *max_err_bits;
    int contiguous;           // QPU m owns the contiguous bit range [q_start[m], q_start[m+1])
    int c0;                   // size of QPU 0 (contiguous case)
    long long *hhi;           // [2^(n - c0)] scratch of the contiguous case
};
cudaError_t launch_fact_check(const FactArgs &a, cudaStream_t st);

}  // namespace qaoa
