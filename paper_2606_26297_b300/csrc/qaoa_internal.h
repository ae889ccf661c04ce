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

// Phase multiplier for U_C(gamma): the table entry T contributes
// (T + k_c) * phi turns (mod 2^64, units of 2^-64 turn), with
// phi = round(gamma 2^-s / (2 pi) 2^64) mod 2^64.
uint64_t phase_multiplier(double gamma, int s);

// Sec. 3.1 allocation helpers and Sec. 3.2 classification.
qaoa_status partition(int n, int M, const int32_t *caps, const int32_t *manual, int32_t *qpu_of);
void classify(const Canonical &c, const int32_t *qpu_of, int64_t *n_local, int64_t *n_cross,
              int64_t *n_cross_all);

// ---- device-side argument blocks ---------------------------------------------

// One mixer application: RX(2 beta) on every mixed qubit, as the butterfly
// (a, b) -> (a - i t b, b - i t a) with common factor cos(beta') where
// beta' = beta (flip = 0, t = tan beta) or beta' = beta - pi/2 (flip = 1,
// t = tan(beta - pi/2), followed by the group bit flip X and a factor -i).
// mode 0: no mixer; 1: mixer present.
struct MixOp {
    int mode;
    int flip;
    float t;
};

// Arguments of one layer pass over a 2^13-element block per CTA.
struct PassArgs {
    float2 *psi;            // state (read and/or written)
    float2 *lam;            // adjoint state
    float4 *pl;             // interleaved (psi.re, lambda.re, psi.im, lambda.im) per index
    const int32_t *C;       // objective table T
    double *partials;       // [block][NSLOT] per-block FP64 partial sums
    unsigned long long *topk_keys;  // [block][ktop] candidate keys (epilogue only)
    int n;
    int lo;                 // window offset of a high-group pass
    uint32_t mask;          // which of the 13 block bits are mixed
    int init;               // synthesise |+>^n instead of loading psi
    int has_cost;
    int store_psi;          // write psi back (reverse passes)
    int precise_phase;      // 1: sincospif, 0: hardware sin/cos
    int ktop;               // top-K candidates per block (epilogue), 0 = off
    MixOp pre, post;
    unsigned long long phi; // phase turns per table unit
    unsigned long long off; // phase turns offset (k_c * phi)
    float amp0;             // 2^{-n/2}
    float kmag;             // real factor of the cost multiplier (the phase of any folded
                            // complex scalar is already part of `off`)
    float2 kend;            // complex scalar applied before the store when there is no cost
    float2 kend2;           // epilogue: scalar applied to lambda before its store
    float cscale;           // 2^-s
};

constexpr int NSLOT = 8;
constexpr int BLOCK_BITS = 13;
constexpr int PASS_THREADS = 256;

// Launchers (kernels_pass.cu).
cudaError_t launch_fwd_pass(int type, bool epilogue, const PassArgs &a, cudaStream_t st);
cudaError_t launch_rev_pass(int type, const PassArgs &a, cudaStream_t st);
cudaError_t launch_reduce_partials(const double *partials, int nblocks, int nslot, double *out,
                                   cudaStream_t st);
cudaError_t launch_topk_merge(const unsigned long long *in, int nlists, int k,
                              unsigned long long *out, int *nout, int *nlaunch, cudaStream_t st);

}  // namespace qaoa
