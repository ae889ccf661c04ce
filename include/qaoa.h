/*
 * qaoa.h - C ABI of the B300 (sm_103a) QAOA statevector library.
 *
 * The library evolves the depth-p QAOA state of a QUBO over all 2^n basis
 * states on one GPU and returns the expectation, its exact gradient, and the
 * most probable bitstrings.  Problem statement and notation follow the paper
 * (arXiv 2606.26297):
 *   - input QUBO (H, f, c0), F(z) = c0 + f^T z + z^T H z      Sec. 2.1, Eq. qubo_input_form
 *   - canonical form l_i = f_i + H_ii, b_ij = H_ij + H_ji      Eqs. canonical_linear, canonical_quadratic
 *   - cost Hamiltonian, eigenvalue F(z) on |z>                 Sec. 2.2, Eq. cost_hamiltonian_raw
 *   - state U_M(b_p)U_C(g_p)...U_M(b_1)U_C(g_1)|+>^n           Sec. 2.3, Eq. qaoa_state
 *   - U_C(g) = exp(-i g H_C), U_M(b) = exp(-i b sum_j X_j)     Eqs. qaoa_cost_unitary, qaoa_mixer_unitary
 *   - objective sum_z P(z) F(z)                                Eqs. qaoa_expectation_expanded, training_objective_mean_cost
 *   - QPU allocation and local/cross couplings                 Sec. 3.1, Sec. 3.2, Eq. local_cross_rule
 *
 * Conventions shared by every call:
 *   - Variable z_{i+1} of the paper is bit i of the basis index x
 *     (x = sum_i z_{i+1} 2^i).  The logical bitstring z_1..z_n of Sec. 3.6 is
 *     bit 0 first.
 *   - Angles are double; gamma[l-1] = gamma_l and beta[l-1] = beta_l.  The
 *     paper's interleaved vector x = [gamma_1, beta_1, ...] (Sec. 3.4) is split
 *     into these two arrays by the caller.
 *   - Amplitudes are complex64 (float re, float im interleaved), 2^n of them,
 *     in index order.  The phase of U_C is exactly exp(-i g F(x)), c0 included.
 *   - Every call returns a qaoa_status.  No call aborts the process; on error
 *     the thread-local message of qaoa_last_error() says what failed, and
 *     output arguments are left unspecified.
 *   - Host pointers are read or written before the call returns.  Device work
 *     is ordered on the context's CUDA stream; calls that return host values
 *     synchronise that stream.
 *   - Handles are owned by the library and released with qaoa_*_destroy;
 *     every other buffer belongs to the caller.
 *   - Sizes: 1 <= n <= 33 (the state of n=33 is 64 GiB).  Gradients need 3
 *     states + the 4-byte cost table in device memory, or about p + 2 states
 *     with stored forward states (options.adjoint_mode).
 */
#ifndef QAOA_H
#define QAOA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QAOA_OK = 0,
    QAOA_ERR_INVALID_ARG = 1,   /* null pointer, bad size, n out of range, k out of range */
    QAOA_ERR_OUT_OF_MEMORY = 2, /* device allocation failed or exceeds the memory budget */
    QAOA_ERR_RANGE = 3,         /* integer objective does not fit the 32-bit table */
    QAOA_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed */
    QAOA_ERR_TIMEOUT = 5,       /* a bounded device-side wait expired (status word set by a kernel) */
    QAOA_ERR_ALLOCATION = 6     /* QPU allocation rejected (Sec. 3.1, validate_allocation) */
} qaoa_status;

/* Coefficient type of the caller's H and f arrays. */
typedef enum {
    QAOA_I32 = 0, /* int32_t; the objective table is exact */
    QAOA_F32 = 1, /* float */
    QAOA_F64 = 2  /* double */
} qaoa_dtype;

/* A QUBO in the input form of Sec. 2.1 (Eq. qubo_input_form).
 * H: n*n coefficients, row-major, host memory, any (non-symmetric) matrix.
 * f: n coefficients, host memory, or NULL for f = 0.
 * c0: the constant term. */
typedef struct {
    int32_t n;
    qaoa_dtype dtype;
    const void *H;
    const void *f;
    double c0;
} qaoa_qubo;

/* Adjoint (gradient) strategy. */
typedef enum {
    QAOA_ADJ_AUTO = 0,      /* stored states when they fit in free device memory (and the
                               memory budget) with a 4 GiB margin; when only some fit, the
                               inputs of the last mixer-only passes that fit are kept and the
                               rest of the reverse sweep uncomputes; else uncompute */
    QAOA_ADJ_UNCOMPUTE = 1, /* the reverse sweep recomputes earlier states by U^dagger on an
                               interleaved (psi, lambda) buffer: 3 states of memory */
    QAOA_ADJ_STORE = 2      /* the forward sweep keeps the states the reverse sweep needs (about
                               p + 2 states for 3 qubit groups); the reverse passes of mixer-only
                               passes then carry lambda alone */
} qaoa_adjoint_mode;

/* Options of a context.  Zero-initialised means "defaults". */
typedef struct {
    int32_t adjoint_mode;   /* qaoa_adjoint_mode */
    int32_t profile;        /* 1: time every pass kernel with CUDA events (see qaoa_profile_read) */
    int64_t memory_budget;  /* bytes of device memory the context may hold; 0 = free memory */
    int32_t max_fused_qubits; /* qubits per mixer pass: 0 = default (10), else 3..10 */
    int32_t state_fp64;     /* 1: complex128 states and arithmetic (n <= 12 only) */
    int32_t table_build;    /* objective table: 0 = tensor cores (tcgen05) for n >= 14 and the
                               SIMT Gray-code kernel below that; 1 = the SIMT kernel for every n */
    int32_t autotune;       /* 1: the first evaluation of each state size n >= 13 times every
                               fusion width (qaoa_autotune) and the context keeps the fastest;
                               ignored when max_fused_qubits is set */
    int32_t reverse_blocks; /* final forward pass and reverse passes of cost-layer passes:
                               0 = half blocks of 2^12 amplitudes (two 128-thread CTAs per SM)
                               for the low qubit group, blocks of 2^13 (one 256-thread CTA per
                               SM) for the others; 1 = blocks of 2^13 for every group; 2 = half
                               blocks for every group.  The same results up to the rounding of
                               the partial sums. */
    int32_t reserved[3];    /* must be zero */
} qaoa_options;

typedef struct qaoa_ctx_s *qaoa_ctx;     /* device, stream, options, scratch, plan cache */
typedef struct qaoa_cost_s *qaoa_cost;   /* device objective table + canonical QUBO */
typedef struct qaoa_state_s *qaoa_state; /* device statevector, complex64 */

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream) on which every launch of this context is
 * ordered; the caller keeps ownership of the stream.  `opt` may be NULL. */
qaoa_status qaoa_ctx_create(int device, void *cuda_stream, const qaoa_options *opt, qaoa_ctx *out);
void qaoa_ctx_destroy(qaoa_ctx ctx);

/* Thread-local description of the last error (never NULL). */
const char *qaoa_last_error(void);

/* ---- objective table ---------------------------------------------------- */

/* Canonicalise `q` (Sec. 2.1, Eqs. canonical_linear, canonical_quadratic) and
 * build on the device the table of F(x) for all 2^n basis indices (the
 * diagonal of H_C, Sec. 2.2, Eq. cost_hamiltonian_raw).
 * Storage: int32 fixed point, F(x) = (T[x] + k_c) * 2^-s.  Integer QUBOs use
 * s = 0 and are exact (QAOA_ERR_RANGE if the range of F exceeds 2^31).  Real
 * QUBOs round each canonical coefficient to a multiple of 2^-s, with s the
 * largest value that keeps T in int32; the per-entry error is at most
 * (1 + n + n(n-1)/2) * 2^-(s+1).  The inputs are copied; `q` may be freed
 * after the call.  Also records the brute-force minimum (Sec. 3.7). */
qaoa_status qaoa_build_cost(qaoa_ctx ctx, const qaoa_qubo *q, qaoa_cost *out);
void qaoa_cost_destroy(qaoa_cost cost);

/* Table metadata: n, fractional bits s, offset k_c (F = (T + k_c) 2^-s), the
 * brute-force minimiser (smallest index among ties) and its value. */
qaoa_status qaoa_cost_info(qaoa_cost cost, int32_t *n, int32_t *shift_bits, int64_t *k_c,
                           uint64_t *argmin_idx, double *min_cost);

/* Copy the int32 table T (2^n entries) into host memory `table`. */
qaoa_status qaoa_cost_copy_to_host(qaoa_ctx ctx, qaoa_cost cost, int32_t *table);

/* Device address of the int32 table T (2^n entries, index order) and its
 * entry count.  The table stays owned by the cost handle and is meant to be
 * read (for example handed to qaoa_expect_noalloc); every call that takes the
 * handle reads it as it then stands, so a caller that writes through this
 * pointer changes the objective of every later call (the factorisation check
 * reports such an edit as mismatching entries). */
qaoa_status qaoa_cost_device_ptr(qaoa_cost cost, const int32_t **table, int64_t *count);

/* ---- forward evolution -------------------------------------------------- */

/* Evolve |+>^n through p layers (Eq. qaoa_state).  gamma, beta: host arrays
 * of p doubles, p >= 0.  *inout: a state handle for the same n, or NULL, in
 * which case a new state is allocated and returned. */
qaoa_status qaoa_forward(qaoa_ctx ctx, qaoa_cost cost, int p, const double *gamma,
                         const double *beta, qaoa_state *inout);
void qaoa_state_destroy(qaoa_state state);

/* Copy the 2^n amplitudes into host memory `amps`: 2 * 2^n floats for a
 * complex64 state, or 2 * 2^n doubles (passed through this float pointer) for
 * a complex128 state (options.state_fp64). */
qaoa_status qaoa_state_copy_to_host(qaoa_ctx ctx, qaoa_state state, float *amps);

/* Device address of the amplitudes (complex64, 2^n) and their count; the
 * pointer stays owned by the state. */
qaoa_status qaoa_state_device_ptr(qaoa_state state, void **amps, int64_t *count);

/* Amplitudes at `count` basis indices: idx is a host array of count indices
 * (each < 2^n, else QAOA_ERR_INVALID_ARG); out is a host array of count
 * complex values (2 floats each, or 2 doubles for a complex128 state).  For
 * reading a few entries of a state too large to copy to the host. */
qaoa_status qaoa_state_gather(qaoa_ctx ctx, qaoa_state state, const uint64_t *idx, int count, void *out);

/* <H_C> = sum_x |psi_x|^2 F(x) (Eq. qaoa_expectation_expanded), reduced
 * deterministically in FP64 (same inputs give the same bits). */
qaoa_status qaoa_expect(qaoa_ctx ctx, qaoa_cost cost, qaoa_state state, double *out_expect);

/* The k most probable bitstrings (1 <= k <= 64), ordered by probability
 * descending then index ascending (the elite set of Sec. 3.6, ranked by exact
 * probability).  idx, prob, cost_out: host arrays of k.  argmin_idx and
 * min_cost (either may be NULL) receive the brute-force minimiser of F
 * (Sec. 3.7); prob_argmin (may be NULL) its probability in this state. */
qaoa_status qaoa_topk(qaoa_ctx ctx, qaoa_cost cost, qaoa_state state, int k, uint64_t *idx,
                      float *prob, double *cost_out, uint64_t *argmin_idx, double *min_cost,
                      float *prob_argmin);

/* ---- gradient ----------------------------------------------------------- */

/* E(gamma, beta) and its exact gradient dE/dgamma_l, dE/dbeta_l by a reverse
 * (adjoint) sweep over the layers (the exact counterpart of the objective of
 * Sec. 3.4, Eq. training_objective_mean_cost, whose gradient Sec. 4.2
 * estimates by SPSA).  gamma, beta: host, p doubles each; out_expect: host
 * double; dgamma, dbeta: host, p doubles each.  Optional top-K of the final
 * state: k_top = 0 disables it; otherwise top_idx/top_prob are host arrays of
 * k_top (<= 64), same ordering as qaoa_topk.  Device memory: one state plus
 * the context's adjoint buffer (allocated on first use and kept); with
 * adjoint_mode AUTO also the stored forward states that fit (see
 * qaoa_adjoint_mode), which the context releases when a later allocation of
 * it (a state, a table, another n) would not fit otherwise. */
qaoa_status qaoa_grad(qaoa_ctx ctx, qaoa_cost cost, int p, const double *gamma,
                      const double *beta, double *out_expect, double *dgamma, double *dbeta,
                      int k_top, uint64_t *top_idx, float *top_prob);

/* ---- batched evaluation (Sec. 4.3: many parameter vectors per request) -- */

/* B parameter sets evaluated in one request: item b uses cost handle
 * costs[item_cost[b]] (item_cost may be NULL: all items use costs[0]), angles
 * gamma[b*p .. b*p+p-1], beta[b*p ..].  Outputs expect[b], dgamma[b*p + l],
 * dbeta[b*p + l]; dgamma/dbeta may be NULL for forward-only evaluation.
 * All pointers are host memory.  Cost handles may differ in n (ragged batch):
 * the items of one n share each pass launch; the groups of different n run on
 * internal streams forked from and joined back into the context's stream, so
 * they overlap on the GPU (the call returns after all of them). */
qaoa_status qaoa_grad_batch(qaoa_ctx ctx, int nq, const qaoa_cost *costs, const int32_t *item_cost,
                            int B, int p, const double *gamma, const double *beta,
                            double *expect, double *dgamma, double *dbeta);

/* ---- parameter optimisation (Sec. 3.4) ---------------------------------- */

/* Hyper-parameters of qaoa_optimize_adam.  Zero fields take the defaults
 * lr = 0.01, beta1 = 0.9, beta2 = 0.999, eps = 1e-8. */
typedef struct {
    double lr, beta1, beta2, eps;
    int32_t iterations;    /* Adam steps, >= 1 */
    int32_t disable_graph; /* 1: launch every step eagerly instead of replaying a CUDA graph */
    int32_t reserved[6];
} qaoa_adam_options;

/* Minimise the objective of Sec. 3.4 (Eq. training_objective_mean_cost,
 * evaluated exactly rather than from shots) for B parameter sets at once with
 * Adam on the exact adjoint gradient: theta <- theta - lr mhat/(sqrt(vhat)+eps)
 * with bias-corrected moments, theta = (gamma, beta) of each item.  Items and
 * costs as in qaoa_grad_batch.  gamma, beta: host, B*p doubles each, read as
 * the starting point and overwritten with the final parameters.
 * history: host, iterations*B doubles or NULL; history[t*B + b] = E of item b
 * at the parameters before step t+1.  final_expect: host, B doubles or NULL;
 * E at the final parameters.  The first step runs eagerly; the remaining
 * iterations-1 steps replay one CUDA graph of a whole step (scalars, passes,
 * reductions, gradient assembly, Adam update), with no host work between
 * steps.  Runs on a stream owned by the context; `ctx`'s stream is ordered
 * after it on return. */
qaoa_status qaoa_optimize_adam(qaoa_ctx ctx, int nq, const qaoa_cost *costs, const int32_t *item_cost,
                               int B, int p, double *gamma, double *beta,
                               const qaoa_adam_options *opt, double *history, double *final_expect);

/* ---- measurement by shots (Sec. 3.4 shot objective, Sec. 3.6 final evaluation) */

/* A state handle holding `amps` (host, 2^n complex64 values, or complex128
 * with fp64 = 1 and n <= 12), copied to the device.  1 <= n <= 33.  For
 * measuring a state the caller made. */
qaoa_status qaoa_state_from_host(qaoa_ctx ctx, int n, int fp64, const void *amps, qaoa_state *out);

/* Measure `state` with `shots` shots (1 <= shots <= 2^34), the circuit
 * execution whose counts Sec. 3.4 turns into the sampled mean cost and Sec.
 * 3.6 into the final distribution.  Inverse-CDF sampling on exact integer
 * weights: q_x = floor(re^2 2^60) + floor(im^2 2^60) with the squares of the
 * stored components taken exactly, Q = sum_x q_x; shot s with 64-bit random
 * integer R_s lands on the smallest x whose prefix q_0 + ... + q_x exceeds
 * floor(R_s Q / 2^64).  R_s = rand[s]
 * (host array of `shots` integers) or, with rand = NULL, the counter-based
 * Philox4x32-10 (Salmon et al., SC 2011): counter (s lo, s hi, stream lo,
 * stream hi), key (seed lo, seed hi), R = out0 + 2^32 out1.
 * Outputs (host, each may be NULL): idx[s] = x_s; cost_out[s] = F(x_s) from
 * the cost table (needs `cost`, of the same n); *mean_cost = mean of F over
 * the shots (needs `cost`), summed exactly in integers.  QAOA_ERR_RANGE if
 * the state's total probability is outside [0.25, 4] or a component has
 * magnitude >= 2 or is infinite or NaN.  Device scratch: about
 * 2^n / 32 bytes plus 8 bytes per shot for each output kept. */
qaoa_status qaoa_sample(qaoa_ctx ctx, qaoa_cost cost, qaoa_state state, int64_t shots, uint64_t seed,
                        uint64_t stream, const uint64_t *rand, uint64_t *idx, double *cost_out,
                        double *mean_cost);

/* Final distribution metrics of Sec. 3.6 from measured indices. */
typedef struct {
    int64_t shots, distinct;      /* shots, distinct bitstrings seen */
    double mean_cost;             /* sampled mean cost */
    double best_cost;             /* lowest sampled cost */
    uint64_t best_index;          /* smallest index with that cost */
    double p_best_index;          /* frequency of best_index */
    double p_best_cost;           /* frequency of all shots with best_cost */
    double low_cost_mass;         /* frequency of shots with cost <= best_cost + margin */
    double p_ref_cost, p_ref_index;  /* frequency of the reference cost (within tol) / index; NaN without one */
    int32_t best_cost_matches_ref;   /* |best_cost - ref_cost| <= tol; -1 without a reference */
    int32_t best_index_matches_ref;  /* best_index == ref_index; -1 without a reference */
} qaoa_sample_metrics;

/* Host only.  idx, cost: host arrays of `shots` measured indices and their
 * costs (as qaoa_sample returns them).  The elite set (Sec. 3.6, the top
 * sampled bitstrings with their costs and counts) orders distinct indices by
 * count descending, then cost ascending, then index ascending, and fills
 * elite_idx/elite_cost/elite_count (host, `elite` entries each; entries past
 * the distinct count get index ~0, cost NaN, count 0; NULL allowed when
 * elite = 0).  has_ref = 1 adds the reference-based quantities for the
 * classical optimum (ref_cost, ref_index), costs compared within tol. */
qaoa_status qaoa_sample_stats(int64_t shots, const uint64_t *idx, const double *cost, double margin, int elite,
                              uint64_t *elite_idx, double *elite_cost, int64_t *elite_count, int has_ref,
                              double ref_cost, uint64_t ref_index, double tol, qaoa_sample_metrics *out);

/* Hyper-parameters of qaoa_optimize_spsa.  Zero fields take the defaults
 * lr = 0.01, beta1 = 0.9, beta2 = 0.999, eps = 1e-8, c = 0.1, averaging = 1;
 * c_decay is used as given (0 keeps c_k = c). */
typedef struct {
    double lr, beta1, beta2, eps;  /* Adam */
    double c, c_decay;             /* perturbation size c_k = c / (k + 1)^c_decay at iteration k = 0, 1, ... */
    int32_t iterations;            /* >= 1 */
    int32_t shots;                 /* shots per objective evaluation; 0 = exact expectation */
    int32_t averaging;             /* independent shot estimates averaged per evaluation, 1..512 */
    int32_t pad;
    uint64_t seed;                 /* Philox key of the perturbations and the shots */
    int32_t reserved[6];           /* must be zero */
} qaoa_spsa_options;

/* Sec. 3.4: Adam on the SPSA gradient estimate, for B starts at once.  At
 * iteration k every start b draws one perturbation D (+-1 per entry of its
 * interleaved x = [gamma_1, beta_1, ...]; entry i is -1 when bit 0 of word 0
 * of Philox4x32-10 at counter (i, b, k, 0x53505341), key (seed lo, seed hi),
 * is set), evaluates J at x + c_k D and x - c_k D as one batch of 2B items,
 * forms g_i = (J+ - J-) / (2 c_k D_i) and takes one bias-corrected Adam step.
 * J is the exact expectation (shots = 0) or the mean cost of `averaging` x
 * `shots` shots of the item's state measured as by qaoa_sample with
 * stream = k 2^32 + b 2^10 + (0 for +, 1 for -) 2^9 + pass.  Items and costs
 * as in qaoa_grad_batch (B < 2^22).  gamma, beta: host, B*p doubles each,
 * read as the start and overwritten with the result.  history: host,
 * iterations*B*2 doubles or NULL; history[(k*B + b)*2 + 0/1] = J+/J-.
 * final_expect: host, B doubles or NULL: exact E at the final parameters. */
qaoa_status qaoa_optimize_spsa(qaoa_ctx ctx, int nq, const qaoa_cost *costs, const int32_t *item_cost,
                               int B, int p, double *gamma, double *beta, const qaoa_spsa_options *opt,
                               double *history, double *final_expect);

/* ---- depth progression and multi-start search (Sec. 3.5, Algorithm 1) ---- */

typedef struct {
    int32_t p_max;          /* depths 1 .. p_max, p_max <= 64 */
    int32_t optimizer;      /* 0 = SPSA-Adam (qaoa_optimize_spsa), 1 = Adam on the exact gradient */
    int32_t iterations;     /* optimiser steps per start, >= 1 */
    int32_t shots;          /* SPSA: shots per objective evaluation, 0 = exact expectation */
    int32_t averaging;      /* SPSA: shot estimates averaged per evaluation; 0 -> 1 */
    int32_t random_starts;  /* random initial points per depth (>= 1) */
    int32_t warm_perturb;   /* perturbed copies of the lifted previous best, depths >= 2 */
    int32_t include_warm;   /* 1: the lifted previous best itself is a start, depths >= 2 */
    int32_t final_shots;    /* shots of every candidate's final evaluation, >= 1 */
    int32_t use_reference;  /* 1: rank by agreement with the brute-force optimum first */
    double lr, beta1, beta2, eps;   /* Adam; zero fields -> 0.01, 0.9, 0.999, 1e-8 */
    double c, c_decay;              /* SPSA perturbation as in qaoa_spsa_options */
    double warm_sigma;              /* standard deviation of the warm-start perturbations */
    double gamma_range, beta_range; /* random starts: gamma ~ U[0, gamma_range), beta ~ U[0, beta_range) */
    double margin;                  /* low-cost mass margin (qaoa_sample_stats) */
    double tol;                     /* cost tolerance of the reference comparison */
    uint64_t seed;
    int32_t reserved[8];            /* must be zero */
} qaoa_solve_options;

typedef struct {
    int32_t best_p;               /* depth of the selected candidate */
    int32_t runs;                 /* optimisation runs over all depths */
    double expect;                /* exact <H_C> at the selected parameters */
    qaoa_sample_metrics metrics;  /* final evaluation of the selected candidate */
} qaoa_solve_result;

/* Algorithm 1 (Sec. 3.5) on one cost handle.  For p = 1 .. p_max: the starts
 * are the previous depth's best lifted to depth p by linear interpolation
 * (INTERP of Zhou et al., PRX 10, 021067: x'_i = (i-1)/p x_{i-1} +
 * (p-i+1)/p x_i, x_0 = x_{p+1} = 0, for gamma and beta) if include_warm,
 * warm_perturb copies of it plus warm_sigma N(0, 1) per entry, and
 * random_starts random points, in that order; all starts of a depth are
 * optimised as one batch (the paper's parallel restarts), then each result is
 * measured with final_shots shots and scored with qaoa_sample_stats; the
 * candidates are ranked lexicographically (Sec. 3.5): with use_reference,
 * best cost equals the brute-force optimum, best index equals it, mass on the
 * optimum cost, probability of the optimum index (larger first); then best
 * sampled cost (smaller first), mass on it, probability of the best index
 * (larger first), mean cost (smaller first), and without a reference the gap
 * mean - best (smaller first); ties keep the earlier start.  The best of each
 * depth warm-starts the next; the depth representatives are ranked the same
 * way.  Random numbers: Philox4x32-10 with key (seed lo, seed hi) and counter
 * (i, j, p, 0x52414E44) for entry i of the interleaved x of start j at depth
 * p (uniform u = (w0 + 2^32 w1) >> 11 times 2^-53), counter (i, j, p,
 * 0x57415250) for the perturbations (Box-Muller on the uniforms of (w0, w1)
 * and (w2, w3)); SPSA at depth p uses seed + p 0x9E3779B97F4A7C15; the final
 * evaluation of start j at depth p uses shot stream 0xF000000000000000 +
 * p 2^32 + j.
 * Outputs (host): gamma, beta: p_max doubles each, the first best_p set (the
 * rest 0); elite (>= 0) entries of elite_idx/elite_cost/elite_count for the
 * selected candidate (as qaoa_sample_stats; NULL allowed when elite = 0);
 * depth_metrics: p_max entries or NULL, each depth's representative; *out. */
qaoa_status qaoa_solve(qaoa_ctx ctx, qaoa_cost cost, const qaoa_solve_options *opt, double *gamma,
                       double *beta, int elite, uint64_t *elite_idx, double *elite_cost, int64_t *elite_count,
                       qaoa_sample_metrics *depth_metrics, qaoa_solve_result *out);

/* qaoa_optimize_adam continuing an earlier run, for checkpointed optimisation
 * (the paper records the optimiser history, Sec. 3.4; the state needed to
 * resume it is the moments and the step count).  m, v: host, B*2p doubles
 * each, in/out: m[b*2p + l] and m[b*2p + p + l] are the first moments of
 * gamma_l and beta_l of item b (v the second moments); zeros start a fresh
 * run.  step: host, in/out: Adam steps taken before this call (the bias
 * correction continues from it); it is advanced by `iterations`.  Running
 * k1 iterations and then k2 more with the returned gamma, beta, m, v and step
 * equals k1 + k2 iterations in one call.  history[t*B + b] counts the
 * iterations of this call. */
qaoa_status qaoa_optimize_adam_resume(qaoa_ctx ctx, int nq, const qaoa_cost *costs, const int32_t *item_cost,
                                      int B, int p, double *gamma, double *beta, const qaoa_adam_options *opt,
                                      double *history, double *final_expect, double *m, double *v,
                                      int32_t *step);

/* ---- autotuning ---------------------------------------------------------- */

/* Pick the fusion width (qubits per mixer pass) for states of cost's n by
 * timing one forward + adjoint evaluation at depth p (linear-ramp angles) for
 * each width in {10, 9, 8, 7, 6, 5} (<= n) with CUDA events on the context
 * stream.  The fastest width is returned in *best_k and kept by the context
 * for that n (used when options.autotune = 1 and max_fused_qubits = 0).
 * At the chosen width it then times the adjoint with stored forward states
 * (the AUTO choice: uncompute where they do not fit) against the uncompute
 * sweep and keeps the faster form for that n (used when options.autotune = 1
 * and adjoint_mode = AUTO).  ms_by_k (host, 8 doubles, may be NULL):
 * ms_by_k[k - 3] = time for width k (k = 5..10), NaN where not timed; the
 * slots of widths 3 and 4, which are never tuned, receive the times of the
 * two adjoint forms: ms_by_k[0] stored (AUTO), ms_by_k[1] uncompute.  n <= 12
 * is rejected (the shared-memory kernel has no passes).  Sec. 4.1 compiles a
 * circuit once and reuses it; this is the counterpart for the pass plan. */
qaoa_status qaoa_autotune(qaoa_ctx ctx, qaoa_cost cost, int p, int32_t *best_k, double *ms_by_k);

/* ---- schedule (host only) ------------------------------------------------ */

/* One pass of the schedule of an evaluation, as qaoa_plan_describe reports it. */
typedef struct {
    int32_t kind;        /* 0 forward; 1 final forward pass (E, top-K, lambda = H_C psi and the
                            first reverse group); 2 reverse pass on the interleaved (psi, lambda)
                            buffer; 3 reverse pass of a mixer-only pass on lambda alone against a
                            stored forward state */
    int32_t group_type;  /* 0 low qubit group (block = bits 0..12), 1 high group */
    int32_t loA, loB;    /* high group: first global bits of its two 5-bit windows */
    uint32_t mask;       /* mixed local bits of the group */
    int32_t pre_layer, cost_layer, post_layer;  /* 0-based layers of the pass's mixer before
                                                   the cost layer, its cost layer and its mixer
                                                   after it; -1 none */
    int32_t in_slot, out_slot, psi_slot;        /* stored forward states: slot >= 0, -1 the
                                                   working state, -2 none */
    int32_t lambda_alone_out;  /* kinds 1, 2: writes lambda alone (for a kind-3 pass next) */
    int32_t interleaved_out;   /* kind 3: writes (psi, lambda) interleaved (for a kind-2 pass next) */
    int32_t slot_param[8];     /* what each partial-sum slot adds to: -1 nothing, -2 the
                                  expectation sums, l < p: dE/dbeta_l, p + l: dE/dgamma_l */
    double bytes_per_amp;      /* algorithmic bytes per amplitude the pass moves */
} qaoa_pass_info;

/* The pass schedule of one evaluation of n qubits at depth p (Eq. qaoa_state;
 * with grad = 1 the adjoint sweep): the n qubits in groups of at most
 * max_fused_qubits (3..10), 1 + p(G-1) forward passes (consecutive layers share
 * their boundary group), then the reverse passes in reverse order.  stored_mids:
 * how many mixer-only passes keep their input for the reverse sweep (-1 all,
 * 0 none: the uncompute sweep; the automatic adjoint choice picks this from the
 * free memory), the last ones of the forward sweep.  A diagnostic of the plan
 * the library runs; no device is touched.  out: host array of `capacity`
 * entries (may be NULL to query the count); *count (required) receives the
 * number of passes, *nslots the stored states, *nmids the mixer-only passes
 * (both may be NULL).  QAOA_ERR_INVALID_ARG for n outside [13, 33], p < 0,
 * a width outside [3, 10] or too small a capacity. */
qaoa_status qaoa_plan_describe(int n, int p, int grad, int max_fused_qubits, int stored_mids,
                               qaoa_pass_info *out, int capacity, int32_t *count, int32_t *nslots,
                               int32_t *nmids);

/* ---- DQAOA bookkeeping (host) and the GPU factorisation invariant ------- */

/* QPU allocation of Sec. 3.1.  caps: M capacities, or NULL for balanced
 * capacities (floor(n/M) + [m < n mod M], make_balanced_capacities).
 * manual: n QPU indices in [0, M), or NULL for the contiguous allocation
 * (QPU 0 takes the first caps[0] variables, then QPU 1, ...).  The result
 * is validated (every variable once, no capacity exceeded, every QPU used);
 * QAOA_ERR_ALLOCATION if not.  qpu_of: host output, n entries. */
qaoa_status qaoa_partition(int n, int M, const int32_t *caps, const int32_t *manual, int32_t *qpu_of);

/* Graph-aware allocation (Sec. 3.1), host only: the weighted interaction
 * graph has edge weight |b_ij| (canonical couplings of the QUBO *q); QPUs are
 * filled in order, QPU m opening with the unassigned variable of largest
 * weighted degree towards the unassigned variables and then taking the
 * unassigned variable with the largest total weight to its members (ties:
 * larger weighted degree towards the unassigned variables, then smaller
 * index) until it holds min(caps[m], unassigned - QPUs still to open).  caps:
 * M capacities, or NULL for balanced ones.  qpu_of: host output, n entries;
 * the result is validated as by qaoa_partition. */
qaoa_status qaoa_partition_graph(const qaoa_qubo *q, int M, const int32_t *caps, int32_t *qpu_of);

/* Allocation candidates and their selection (Sec. 3.1), host only: the
 * contiguous (kind 0), graph-aware (kind 1) and, when manual != NULL, the
 * manual (kind 2) allocation are scored by their cross-QPU couplings
 * b_ij != 0; the fewest wins, ties resolved in the order manual, graph-aware,
 * contiguous.  Outputs (host): qpu_of (n) and *kind of the selected one;
 * cross[3] and remote_cx[3] (may be NULL) per kind, remote_cx = 2 cross p,
 * -1 for a kind not built. */
qaoa_status qaoa_allocation_candidates(const qaoa_qubo *q, int M, const int32_t *caps, const int32_t *manual,
                                       int p, int32_t *qpu_of, int32_t *kind, int64_t *cross,
                                       int64_t *remote_cx);

/* Classify the couplings b_ij != 0 (i<j) of `cost` as local (q(i) = q(j)) or
 * cross-QPU (Eq. local_cross_rule), and estimate the remote CNOTs as
 * 2 * cross * p (Sec. 3.1).  n_pairs_all (may be NULL) receives the cross
 * count over all pairs, zero coefficients included.  Host only. */
qaoa_status qaoa_classify(qaoa_cost cost, const int32_t *qpu_of, int p, int64_t *n_local,
                          int64_t *n_cross, int64_t *remote_cx_est, int64_t *n_cross_all_pairs);

/* GPU check that, for every x, the table splits as
 *   T[x] + k_c == c0 + sum_m L_m[field_m(x)] + X(x)
 * with L_m the objective of QPU m's own variables and local couplings and X
 * the sum of the cross-QPU couplings (Sec. 3.2), i.e. that the cost phase
 * factorises into local and cross-QPU parts.  All in exact integer arithmetic
 * on the fixed-point coefficients.  *mismatches = number of x that differ.
 * The phase routine works on the turn count (T + k_c) phi mod 2^64, which is
 * additive, so wherever the integers split the phases split too, up to the
 * routine's own rounding; *max_phase_err (may be NULL) measures that rounding,
 * max |e^{-i g F} - e^{-i g F_local} e^{-i g F_cross}| at g = gamma_probe over
 * the sampled x (the first of every 1024 consecutive indices). */
qaoa_status qaoa_check_factorisation(qaoa_ctx ctx, qaoa_cost cost, const int32_t *qpu_of,
                                     double gamma_probe, int64_t *mismatches, double *max_phase_err);

/* ---- explicit distributed circuit (Sec. 3.3) ------------------------------ */

typedef struct {
    int64_t ops;           /* operations in the circuit */
    int64_t local_zz;      /* couplings implemented locally, summed over the layers */
    int64_t cross_zz;      /* couplings across QPUs, summed over the layers */
    int64_t remote_cx;     /* remote CNOTs = 2 cross_zz (the estimate 2 cross p of Sec. 3.1) */
    int64_t measurements;  /* mid-circuit measurements, 2 per remote CNOT */
    int64_t resets;        /* communication-qubit resets, 2 per remote CNOT */
    int64_t feedforward;   /* outcome-controlled Pauli corrections, 2 per remote CNOT */
} qaoa_telegate_counts;

/* Simulate the distributed QAOA circuit gate by gate (Sec. 3.3) for
 * `trajectories` independent measurement records, to confirm that the
 * TeleGate protocol reproduces the monolithic state and to count its
 * overhead.  n data qubits (n <= 12) plus two communication qubits cA = bit
 * n, cB = bit n + 1; every data qubit starts in |+>; each layer applies the
 * global phase -g c0, a phase -g (l_i + sum_j b_ij / 2) on every qubit i, for
 * each coupling b_ij != 0 (i < j) CNOT(i, j), phase +g b_ij / 2 on j,
 * CNOT(i, j), and RX(2 beta) on every data qubit; a CNOT between qubits on
 * different QPUs (qpu_of, host, n entries) is a remote CNOT: reset cA and cB
 * (they are in basis states), H cA, CNOT cA -> cB, CNOT i -> cA, measure cA
 * (m1), CNOT cB -> j, H cB, measure cB (m2), X^m1 on j, Z^m2 on i.
 * Measurement k of trajectory t draws u = ((w0 + 2^32 w1) >> 11) 2^-53 from
 * Philox4x32-10 at counter (k, t, 0, 0x54454C45), key (seed lo, seed hi),
 * and gives 1 when u < P(1).  Outputs (host): fidelity[t] =
 * |<psi_mono | psi_t>|^2 against the library's own monolithic state
 * (qaoa_forward); amps (NULL allowed): trajectories x 2^n complex64
 * data-qubit states (the communication qubits folded out); *counts. */
qaoa_status qaoa_telegate_simulate(qaoa_ctx ctx, qaoa_cost cost, const int32_t *qpu_of, int p,
                                   const double *gamma, const double *beta, int trajectories, uint64_t seed,
                                   double *fidelity, float *amps, qaoa_telegate_counts *counts);

/* ---- allocation-free expectation -----------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory when they evaluate <H_C>: a host
 * framework that owns all device memory behind a capped pool of its own, a
 * latency-critical loop that cannot afford the implicit device
 * synchronisation a cudaMalloc or cudaFree may trigger, or code that holds
 * only raw device pointers and no qaoa_ctx to keep scratch in.
 *
 * Same result as qaoa_expect (the same reduction, in the same order):
 * sum_x |psi_x|^2 (T[x] + k_c) 2^-shift_bits.
 *   amps:        device pointer, 2^n complex64 amplitudes (caller-owned)
 *   table:       device pointer, the 2^n int32 table T of a qaoa_cost
 *                (qaoa_cost_device_ptr / qaoa_cost_info give T, s and k_c)
 *   n:           1 <= n <= 30; larger n is rejected with QAOA_ERR_INVALID_ARG
 *   shift_bits, k_c: the fixed-point parameters s and k_c of that table
 *   cuda_stream: cudaStream_t the work is ordered on (NULL = default stream);
 *                the call synchronises it before returning
 *   out_expect:  host pointer, receives the expectation
 * Memory: allocates nothing.  Its scratch is one fixed device array of
 * 2 * 2^17 + 2 doubles (about 2 MiB) defined in the library, present on every
 * GPU that loads the library until the process exits.  All calls share that
 * array, so calls that overlap on the GPU (two host threads, or two streams
 * without ordering between them) race and may return wrong values; order them.
 * The array keeps the previous call's contents, but every value a call reads
 * is written earlier in the same call.  Every call looks up the array's
 * device address in the context current at the call (cudaGetSymbolAddress;
 * the lookup allocates nothing), so a caller that works in a context of its
 * own gets that context's copy of the array; amps and table must be device
 * (or managed) memory of the current device, else QAOA_ERR_INVALID_ARG.
 * The call copies its result to the host and synchronises cuda_stream, so it
 * cannot be issued on a stream that is being captured into a CUDA graph. */
qaoa_status qaoa_expect_noalloc(const void *amps, const int32_t *table, int n, int32_t shift_bits,
                                int64_t k_c, void *cuda_stream, double *out_expect);

/* ---- profiling ---------------------------------------------------------- */

/* With options.profile = 1, every kernel launch of the given kind is timed
 * with CUDA events on the context stream.  kind: 0 = forward mixer pass,
 * 1 = reverse (adjoint) pass, 2 = objective table build, 3 = small-n resident
 * kernel, 4 = factorisation check, 6 = measurement weights and prefix scan,
 * 7 = measurement shots; kind 5 counts every kernel the context launched
 * (timed or not; ms and bytes are 0).  Every layer pass is also counted under
 * the kind of the one kernel that ran it: 8 = direct-load forward pass,
 * 9 = TMA-staged forward pass with a cost layer, 10 = final forward pass,
 * 11 = reverse pass of a cost-layer pass, 12 = reverse pass of a mixer-only
 * pass, 13 and 14 = kinds 10 and 11 on half blocks (kind 0 sums 8, 9, 10, 13;
 * kind 1 sums 11, 12, 14).  Returns launches, summed
 * milliseconds and summed algorithmic bytes (bytes the method must move) since
 * the last reset; reset = 1 clears the counters after reading. */
qaoa_status qaoa_profile_read(qaoa_ctx ctx, int kind, int64_t *launches, double *ms,
                              double *bytes, int reset);

/* Diagnostic of the failure path of the device-side waits (the paper has no
 * counterpart).  Every TMA-pipelined pass kernel waits for its copies with a
 * bounded wait: after about 2 s it records QAOA_ERR_TIMEOUT in the context's
 * status word and returns, instead of hanging the GPU.  This call launches one
 * CTA that waits on a copy that is never issued, so the wait must expire: it
 * returns QAOA_ERR_TIMEOUT (the expected result, after about 4 s) and leaves
 * the context usable; QAOA_OK would mean the wait did not give up. */
qaoa_status qaoa_wait_probe(qaoa_ctx ctx);

/* Sustained rate of one arithmetic pipe of this GPU, the denominator for
 * kernels bound by plain arithmetic rather than by memory (the paper has no
 * counterpart: this is measurement support).  kind: 0 = FP32 FMA, 1 = packed
 * f32x2 FMA, 2 = FP64 FMA, 3 = fast sin/cos pairs.  Runs 8 CTAs per SM of
 * independent FMA (or sin/cos) chains on the context stream, timed with CUDA
 * events after a warm-up launch.  *ops_per_s: instructions' lane operations
 * per second (one FMA, one f32x2 FMA lane pair, or one sin/cos pair);
 * *flops_per_s: 2 per FMA, 4 per f32x2 FMA, 1 per sin/cos pair.  Either may be
 * NULL. */
qaoa_status qaoa_peak_probe(qaoa_ctx ctx, int kind, double *ops_per_s, double *flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* QAOA_H */
