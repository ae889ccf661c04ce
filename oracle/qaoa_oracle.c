/*
 * FP64 CPU oracle for the QAOA statevector hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * path never does.  It shares no code, header or constant with the CUDA
 * library.
 *
 * Every routine follows the paper (Sec. 2.1-2.3) in its own notation:
 *   - canonical coefficients l_i = f_i + H_ii, b_ij = H_ij + H_ji
 *     (Eqs. canonical_linear, canonical_quadratic);
 *   - the objective F(z) = c0 + sum l_i z_i + sum_{i<j} b_ij z_i z_j
 *     (Eq. qubo_canonical_work), which is the eigenvalue of H_C on |z>
 *     (Eq. cost_hamiltonian_raw);
 *   - the state |gamma,beta> = U_M(beta_p)U_C(gamma_p)...U_M(beta_1)U_C(gamma_1)|+>^n
 *     (Eq. qaoa_state) with U_C(g) = exp(-i g H_C) (Eq. qaoa_cost_unitary) and
 *     U_M(b) = exp(-i b sum_j X_j) (Eqs. qaoa_mixer_hamiltonian,
 *     qaoa_mixer_unitary), i.e. RX(2b) on every qubit (Sec. 3.3);
 *   - the expectation sum_z P(z) F(z) (Eq. qaoa_expectation_expanded).
 *
 * Conventions: variable z_{i+1} of the paper is bit i of the basis index x
 * (x = sum_i z_{i+1} 2^i).  Amplitudes are complex double, stored as
 * interleaved (re, im) pairs.  The phase of U_C is exactly exp(-i g F(x)) with
 * the constant c0 included.
 *
 * Loops over basis states are parallelised with OpenMP; every sum uses a
 * fixed chunking so results do not depend on the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Fixed chunk for deterministic reductions: chunk sums are formed
 * independently, then added in index order. */
#define ORACLE_CHUNK 4096

/* ---- Sec. 2.1: canonical form ------------------------------------------ */

/* H is n*n row-major.  f may be NULL (treated as zero).
 * ell[i] = f_i + H_ii (Eq. canonical_linear).
 * b is n*n; b[i*n+j] = H_ij + H_ji for i<j (Eq. canonical_quadratic), zero
 * elsewhere. */
void oracle_canonicalize(int n, const double *H, const double *f, double *ell, double *b)
{
    for (int i = 0; i < n; ++i) {
        ell[i] = (f ? f[i] : 0.0) + H[(size_t)i * n + i];
        for (int j = 0; j < n; ++j) b[(size_t)i * n + j] = 0.0;
    }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            b[(size_t)i * n + j] = H[(size_t)i * n + j] + H[(size_t)j * n + i];
}

/* F(z) for one basis index x, by the double sum of Eq. qubo_canonical_work. */
double oracle_cost_one(int n, double c0, const double *ell, const double *b, uint64_t x)
{
    double F = c0;
    for (int i = 0; i < n; ++i) {
        if (!((x >> i) & 1)) continue;
        F += ell[i];
        for (int j = i + 1; j < n; ++j)
            if ((x >> j) & 1) F += b[(size_t)i * n + j];
    }
    return F;
}

/* F(x) for every x in [0, 2^n). */
void oracle_cost_table(int n, double c0, const double *ell, const double *b, double *F)
{
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) F[x] = oracle_cost_one(n, c0, ell, b, (uint64_t)x);
}

/* F at a list of sampled indices. */
void oracle_cost_sampled(int n, double c0, const double *ell, const double *b,
                         const uint64_t *xs, int64_t m, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; ++k) out[k] = oracle_cost_one(n, c0, ell, b, xs[k]);
}

/* ---- Sec. 2.3: gates ------------------------------------------------------ */

/* psi_x <- exp(-i g F_x) psi_x   (Eq. qaoa_cost_unitary; H_C diagonal with
 * eigenvalues F, Eq. cost_hamiltonian_raw).  g may be negative (inverse). */
static void apply_cost(int64_t N, const double *F, double g, cplx *psi)
{
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
        double th = -g * F[x];
        psi[x] *= cos(th) + I * sin(th);
    }
}

/* exp(-i b X_j) on qubit j: for each pair (x with bit j = 0, y = x | 2^j),
 * (psi_x, psi_y) <- (cos b psi_x - i sin b psi_y, -i sin b psi_x + cos b psi_y).
 * This is RX(2b) (Sec. 3.3). */
static void apply_rx(int n, int j, double b, cplx *psi)
{
    const int64_t half = (int64_t)1 << (n - 1);
    const int64_t low = ((int64_t)1 << j) - 1;
    const double c = cos(b), s = sin(b);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < half; ++k) {
        int64_t x = ((k & ~low) << 1) | (k & low); /* insert a 0 at bit j */
        int64_t y = x | ((int64_t)1 << j);
        cplx a = psi[x], bb = psi[y];
        psi[x] = c * a - I * s * bb;
        psi[y] = -I * s * a + c * bb;
    }
}

/* U_M(b) = exp(-i b sum_j X_j) = prod_j exp(-i b X_j) (Eq. qaoa_mixer_unitary). */
static void apply_mixer(int n, double b, cplx *psi)
{
    for (int j = 0; j < n; ++j) apply_rx(n, j, b, psi);
}

/* |gamma,beta> of Eq. qaoa_state, written into psi (2^n complex). */
void oracle_evolve(int n, const double *F, int p, const double *gamma, const double *beta,
                   double *psi_out)
{
    const int64_t N = (int64_t)1 << n;
    cplx *psi = (cplx *)psi_out;
    const double amp = 1.0 / sqrt((double)N);
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) psi[x] = amp; /* |+>^n */
    for (int l = 0; l < p; ++l) {
        apply_cost(N, F, gamma[l], psi);
        apply_mixer(n, beta[l], psi);
    }
}

/* sum_x |psi_x|^2 F_x (Eq. qaoa_expectation_expanded). */
double oracle_expectation(int n, const double *F, const double *psi_in)
{
    const int64_t N = (int64_t)1 << n;
    const cplx *psi = (const cplx *)psi_in;
    const int64_t nchunk = (N + ORACLE_CHUNK - 1) / ORACLE_CHUNK;
    double *part = (double *)malloc(sizeof(double) * nchunk);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nchunk; ++c) {
        double s = 0.0;
        int64_t hi = (c + 1) * ORACLE_CHUNK < N ? (c + 1) * ORACLE_CHUNK : N;
        for (int64_t x = c * ORACLE_CHUNK; x < hi; ++x) {
            double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
            s += pr * F[x];
        }
        part[c] = s;
    }
    double E = 0.0;
    for (int64_t c = 0; c < nchunk; ++c) E += part[c];
    free(part);
    return E;
}

/* sum_x conj(a_x) b_{x xor 2^j}, summed over j = 0..n-1: <a| sum_j X_j |b>,
 * evaluated by explicit bit flips. */
static cplx inner_mixer(int n, const cplx *a, const cplx *b)
{
    const int64_t N = (int64_t)1 << n;
    const int64_t nchunk = (N + ORACLE_CHUNK - 1) / ORACLE_CHUNK;
    cplx *part = (cplx *)malloc(sizeof(cplx) * nchunk);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nchunk; ++c) {
        cplx s = 0.0;
        int64_t hi = (c + 1) * ORACLE_CHUNK < N ? (c + 1) * ORACLE_CHUNK : N;
        for (int64_t x = c * ORACLE_CHUNK; x < hi; ++x)
            for (int j = 0; j < n; ++j) s += conj(a[x]) * b[x ^ ((int64_t)1 << j)];
        part[c] = s;
    }
    cplx S = 0.0;
    for (int64_t c = 0; c < nchunk; ++c) S += part[c];
    free(part);
    return S;
}

/* sum_x conj(a_x) F_x b_x = <a|H_C|b>. */
static cplx inner_cost(int n, const double *F, const cplx *a, const cplx *b)
{
    const int64_t N = (int64_t)1 << n;
    const int64_t nchunk = (N + ORACLE_CHUNK - 1) / ORACLE_CHUNK;
    cplx *part = (cplx *)malloc(sizeof(cplx) * nchunk);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nchunk; ++c) {
        cplx s = 0.0;
        int64_t hi = (c + 1) * ORACLE_CHUNK < N ? (c + 1) * ORACLE_CHUNK : N;
        for (int64_t x = c * ORACLE_CHUNK; x < hi; ++x) s += conj(a[x]) * F[x] * b[x];
        part[c] = s;
    }
    cplx S = 0.0;
    for (int64_t c = 0; c < nchunk; ++c) S += part[c];
    free(part);
    return S;
}

/*
 * Exact gradient of E(gamma, beta) = <gamma,beta|H_C|gamma,beta> by the
 * textbook adjoint (reverse) sweep.  Let psi be the final state and
 * lam = H_C psi.  Walking the layers backwards, at the point just after
 * U_M(beta_l):      dE/dbeta_l  = 2 Im <lam| sum_j X_j |psi>,
 * then both states are multiplied by U_M(beta_l)^dagger = U_M(-beta_l); at the
 * point just after U_C(gamma_l): dE/dgamma_l = 2 Im <lam| H_C |psi>,
 * then both are multiplied by U_C(gamma_l)^dagger.  (The derivative of
 * exp(-i t A) is -i A exp(-i t A), and 2 Re(-i w) = 2 Im w.)
 * The parameter vector is x = [gamma_1, beta_1, ..., gamma_p, beta_p]
 * (Sec. 3.4); here gamma and beta are passed as separate arrays.
 * Returns E.  Scratch: two 2^n complex buffers allocated here.
 */
double oracle_grad_adjoint(int n, const double *F, int p, const double *gamma,
                           const double *beta, double *dgamma, double *dbeta)
{
    const int64_t N = (int64_t)1 << n;
    cplx *psi = (cplx *)malloc(sizeof(cplx) * N);
    cplx *lam = (cplx *)malloc(sizeof(cplx) * N);
    oracle_evolve(n, F, p, gamma, beta, (double *)psi);
    double E = oracle_expectation(n, F, (const double *)psi);
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) lam[x] = F[x] * psi[x];
    for (int l = p - 1; l >= 0; --l) {
        dbeta[l] = 2.0 * cimag(inner_mixer(n, lam, psi));
        apply_mixer(n, -beta[l], psi);
        apply_mixer(n, -beta[l], lam);
        dgamma[l] = 2.0 * cimag(inner_cost(n, F, lam, psi));
        apply_cost(N, F, -gamma[l], psi);
        apply_cost(N, F, -gamma[l], lam);
    }
    free(psi);
    free(lam);
    return E;
}
