// Internal declarations shared by the host code and the CUDA launchers of the
// QAOA statevector library.  Nothing here is part of the C ABI (include/qaoa.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "qaoa.h"

namespace qaoa {

// ---- errors ---------------------------------------------------------------
void set_error(const char *fmt, ...);
qaoa_status fail(qaoa_status st, const char *fmt, ...);

// ---- canonical QUBO (Sec. 2.1) and its fixed-point form --------------------
struct Canonical {
    int n = 0;
    double c0 = 0.0;
    std::vector<double> ell;  // l_i = f_i + H_ii                  (Eq. canonical_linear)
    std::vector<double> b;    // b[i*n+j] = H_ij + H_ji, i<j, else 0 (Eq. canonical_quadratic)
    bool integer = false;     // every coefficient is an integer (exact table)
};

// Fixed-point objective: F(x) * 2^s = c0_q + sum ell_q z + sum b_q z z  (exact integers),
// and the stored table is T[x] = F(x) 2^s - k_c, |T| < 2^31.
struct FixedPoint {
    int s = 0;
    int64_t k_c = 0;
    int64_t c0_q = 0;
    std::vector<int64_t> ell_q;
    std::vector<int64_t> b_q;  // n*n, upper triangle
    int64_t lo_bound = 0, hi_bound = 0;  // bounds of F 2^s over all x
};

qaoa_status canonicalize(const qaoa_qubo *q, Canonical *out);
qaoa_status make_fixed_point(const Canonical &c, FixedPoint *out);

// Sec. 3.1 allocation helpers and Sec. 3.2 classification.
qaoa_status partition(int n, int M, const int32_t *caps, const int32_t *manual, int32_t *qpu_of);
qaoa_status graph_aware(const Canonical &c, int M, const std::vector<int32_t> &caps, int32_t *qpu_of);
void classify(const Canonical &c, const int32_t *qpu_of, int64_t *n_local, int64_t *n_cross,
              int64_t *n_cross_all);

// ---- layer-pass arguments ----------------------------------------------------

constexpr int NSLOT = 8;
constexpr int BLOCK_BITS = 13;
constexpr int PASS_THREADS = 256;

// Angle-dependent scalars of one pass for one item (one parameter set).  The
// mixer is the butterfly (a, b) -> (a - i t b, b - i t a) with common factor
// cos(beta') where beta' = beta (flip = 0, t = tan beta) or beta - pi/2
// (flip = 1: t = tan(beta - pi/2), then the group bit flip X and a factor -i).
// The cost phase is exp(-2 pi i (T phi + off) / 2^64) * kmag (any complex scalar
// folded into it has its phase in `off`).  kend: scalar applied before a store
// when the pass has no cost phase; kend2: the final pass's lambda scalar.
struct PassScal {
    float pre_t, post_t;
    int pre_flip, post_flip;
    unsigned long long phi, off;
    float kmag, cscale;  // cscale = 2^-s of the item's table
    float2 kend, kend2;
};

// Structural arguments of one layer pass, shared by the items of a launch.
// Item i's state is psi + i * 2^n (pl likewise); its table is
// C + item_table[i] * 2^n (item_table null: table 0 for all).
struct PassArgs {
    float2 *psi;                    // forward: input state (in place unless psi_out is set)
    float2 *psi_out;                // forward: output state, or null for in place
    float4 *pl;                     // interleaved (psi.re, lambda.re, psi.im, lambda.im) per index
    const float2 *psi_src;          // stored forward state read by a reverse pass (split mode)
    float2 *lam;                    // lambda alone (stored-state adjoint)
    int split;                      // final / reverse pass: write lambda alone to lam
    int pl_out;                     // mixer-only reverse pass: write (psi_in, lambda) interleaved to pl
    const int32_t *C;
    const int *item_table;
    const PassScal *scal;           // [nitems]
    double *partials;               // [item][block][NSLOT] per-block FP64 partial sums
    unsigned long long *topk_keys;  // [block][ktop] candidate keys (final pass, single item)
    int n;
    int loA, loB;                   // window offsets of a high-group pass (local bits 3..7, 8..12)
    uint32_t mask;                  // which of the 13 block bits are mixed
    int nitems, ntables;
    int init;                       // synthesise |+>^n instead of loading psi
    int has_pre, has_cost, has_post;
    int store;                      // write the result back (reverse passes)
    int precise_phase;              // 1: sincospif, 0: hardware sin/cos
    int ktop;                       // top-K candidates per block (final pass), 0 = off
    float amp0;                     // 2^{-n/2}
};

// Launchers.  grid: persistent CTAs (TMA kernels); status: device word set to
// a non-zero value if a bounded wait expired.
cudaError_t launch_fwd_pass(int type, const PassArgs &a, cudaStream_t st);
cudaError_t launch_final_pass(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);
cudaError_t launch_rev_pass(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);
// the same pass on half blocks of 2^12 amplitudes (two CTAs per SM; grid =
// 2 x SMs); one partial-sum row per half block
cudaError_t launch_rev_pass_half(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);
cudaError_t launch_final_pass_half(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);
cudaError_t launch_rev_mid(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);
cudaError_t launch_wait_probe(unsigned int *status, cudaStream_t st);
cudaError_t launch_fwd_cost_tma(int type, const PassArgs &a, int grid, unsigned int *status, cudaStream_t st);
cudaError_t launch_reduce_partials(const double *partials, int nitems, int nblocks, double *out,
                                   cudaStream_t st);
// Two stages when an item has at least 64 chunks of 256 units (scratch holds
// nitems * reduce_chunk_count(nblocks) * NSLOT doubles), else the one-stage
// sum; *launches = kernels launched.
int reduce_chunk_count(int nblocks);
cudaError_t launch_reduce_partials_chunked(const double *partials, int nitems, int nblocks, double *scratch,
                                           double *out, int *launches, cudaStream_t st);
cudaError_t launch_topk_merge(const unsigned long long *in, int nlists, int k,
                              unsigned long long *out, int *nout, int *nlaunch, cudaStream_t st);

}  // namespace qaoa
