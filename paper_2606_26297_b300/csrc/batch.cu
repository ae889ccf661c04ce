// Device-side bookkeeping of batched evaluations: per-pass scalars from
// device-resident angles, assembly of E and its gradient from the partial
// sums, and the Adam update (the optimiser of Sec. 3.4, here driven by the
// exact gradient).  All of it runs inside a captured CUDA graph without the
// host.
#include "schedule.cuh"

namespace qaoa {

__global__ void prep_scalars_kernel(DevPlan d) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // pass * nitems + item
    if (idx >= d.npasses * d.nitems) return;
    const int pass = idx / d.nitems, item = idx % d.nitems;
    pass_scalars(d.plan[pass], d.gamma + (size_t)item * d.p, d.beta + (size_t)item * d.p, d.item_s[item],
                 d.item_kc[item], d.scal + idx, d.slot_scale + (size_t)idx * NSLOT);
}

cudaError_t launch_prep_scalars(const DevPlan &d, cudaStream_t st) {
    const int total = d.npasses * d.nitems;
    prep_scalars_kernel<<<(total + 127) / 128, 128, 0, st>>>(d);
    return cudaGetLastError();
}

// One thread per item: E = 2^-s (S0 + k_c S1); dE/dbeta_l = sum 2 v scale over
// the slots mapped to beta_l; dE/dgamma_l = sum 2 2^-s v scale.  Passes and
// slots are visited in a fixed order (deterministic).
__global__ void assemble_kernel(DevPlan d, const double *sums, double *E, double *dg, double *db) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= d.nitems) return;
    const int p = d.p;
    const double cs = ldexp(1.0, -d.item_s[item]);
    for (int l = 0; l < p; ++l) {
        dg[(size_t)item * p + l] = 0.0;
        db[(size_t)item * p + l] = 0.0;
    }
    double S0 = 0.0, S1 = 0.0;
    for (int pass = 0; pass < d.npasses; ++pass) {
        const PassPlan &pl = d.plan[pass];
        if (pl.sum_index < 0) continue;
        const double *v = sums + ((size_t)pl.sum_index * d.nitems + item) * NSLOT;
        const double *sc = d.slot_scale + ((size_t)pass * d.nitems + item) * NSLOT;
        for (int s = 0; s < NSLOT; ++s) {
            const int prm = pl.slot_param[s];
            if (prm == -2) {
                if (s == 0) S0 = v[s];
                else S1 = v[s];
            } else if (prm >= 0 && prm < p) {
                db[(size_t)item * p + prm] += 2.0 * v[s] * sc[s];
            } else if (prm >= p) {
                dg[(size_t)item * p + prm - p] += 2.0 * cs * v[s] * sc[s];
            }
        }
    }
    E[item] = cs * (S0 + (double)d.item_kc[item] * S1);
}

cudaError_t launch_assemble(const DevPlan &d, const double *sums, double *E, double *dgamma, double *dbeta,
                            cudaStream_t st) {
    assemble_kernel<<<(d.nitems + 127) / 128, 128, 0, st>>>(d, sums, E, dgamma, dbeta);
    return cudaGetLastError();
}

// Adam on theta = (gamma, beta): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
// theta <- theta - lr mhat / (sqrt(vhat) + eps), with bias-corrected moments
// at step t (the device counter, advanced by the last thread).  The
// objective of the step is appended to the history.
__global__ void adam_kernel(AdamArgs a) {
    const int np = a.nitems * a.p;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = *a.step + 1;
    if (idx < 2 * np) {
        const bool isg = idx < np;
        const int k = isg ? idx : idx - np;
        const int item = k / a.p, l = k % a.p;
        double *th = isg ? a.gamma : a.beta;
        const double g = isg ? a.dgamma[(size_t)item * a.gstride + l] : a.dbeta[(size_t)item * a.gstride + l];
        double &m = a.m[idx];
        double &v = a.v[idx];
        m = a.beta1 * m + (1.0 - a.beta1) * g;
        v = a.beta2 * v + (1.0 - a.beta2) * g * g;
        const double mh = m / (1.0 - pow(a.beta1, (double)t));
        const double vh = v / (1.0 - pow(a.beta2, (double)t));
        th[k] -= a.lr * mh / (sqrt(vh) + a.eps);
    }
    const int row = t - 1 - a.step0;
    if (a.history && idx < a.nitems && row >= 0 && row < a.max_steps)
        a.history[(size_t)row * a.nitems + idx] = a.E[(size_t)idx * a.estride];
}

__global__ void adam_step_kernel(int *step) { *step += 1; }

cudaError_t launch_adam(const AdamArgs &a, cudaStream_t st) {
    const int total = 2 * a.nitems * a.p;
    adam_kernel<<<(total + 127) / 128, 128, 0, st>>>(a);
    adam_step_kernel<<<1, 1, 0, st>>>(a.step);
    return cudaGetLastError();
}

}  // namespace qaoa
