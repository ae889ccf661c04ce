// Layer-pass schedule and the angle-dependent scalars of every pass.
//
// The n qubits are split into G groups of <= 10 (the mixer of Eq.
// qaoa_mixer_unitary factorises over qubits).  Group 0 owns the low bits
// (blocks of 13 contiguous bits); every other group owns two 5-bit windows
// loA..loA+4 and loB..loB+4 (block local bits 3..7 and 8..12) and carries
// global bits 0..2 for coalescing.  From n = 24 on, each high group takes one
// window in the lower and one in the upper half of the high bits: a block
// whose ten bits were all among the top bits would touch 2^10 rows 2^{n-10}
// elements apart, i.e. about a thousand 2 MiB pages per CTA, and B300 then
// streams at half its bandwidth (measured: 3.1 TB/s for bits 20..29 of a
// 2^30 state against 5.5 TB/s for bits {10..14, 25..29}).  Layers visit the
// groups in alternating order (A,B,C | C,B,A | ...), so the pass that ends
// layer l also applies U_C(gamma_{l+1}) (diagonal, Eq. qaoa_cost_unitary) and
// the same group's mixer of layer l+1: 1 + p(G-1) forward passes in all.
//
// pass_scalars() is __host__ __device__: the host uses it for single
// evaluations, and a device kernel (batch.cu) recomputes it from
// device-resident angles inside a captured CUDA graph.
#pragma once

#include <cmath>
#include <cstdint>
#include <vector>

#include "qaoa_internal.h"

namespace qaoa {

struct Group {
    int type;       // 0: low group (block = global bits 0..12), 1: high group
    int loA, loB;   // window offsets (type 1): local bits 3..7 -> loA.., 8..12 -> loB..
    uint32_t mask;  // mixed local bits
    int kX, kY;     // mixed bits in the register rounds of arrangements X and Y
};

// One pass as executed.  kind 0: forward; 1: final forward pass of a gradient
// evaluation; 2: reverse pass undoing a forward pass on (psi, lambda); 3:
// reverse pass of a middle (mixer-only) forward pass that advances lambda
// alone, reading psi from a stored forward state.
//
// State buffers: slot >= 0 is a stored forward state, SLOT_W the working
// state, SLOT_NONE no buffer.  Without stored states every pass works in place
// and the reverse sweep uncomputes psi on the interleaved (psi, lambda)
// buffer.  With them (three or more qubit groups) the forward pass f reads
// in_slot and writes out_slot, keeping the input of each kept mixer-only pass
// (all of them, or the last few when memory holds only those); the reverse of
// a kept mixer-only pass (kind 3) reads psi from psi_slot and carries lambda
// alone, writing it interleaved with psi (pl_out) when the next reverse pass
// runs on the interleaved buffer.  A pass of kind 1 or 2 writes lambda alone
// (split_out) when the next reverse pass is a kept mixer-only one.
constexpr int SLOT_W = -1, SLOT_NONE = -2;
struct PassPlan {
    int kind;
    int split_out;             // final / cost-layer reverse / uncomputing reverse pass: write lambda alone
    int in_slot, out_slot, psi_slot;
    int pl_out;
    int type, loA, loB;
    uint32_t mask;
    int kX, kY;
    int init;
    int la, lc, lb;            // layers (0-based) of pre mixer, cost, post mixer; -1 none
    int slot_param[NSLOT];     // -1 none, -2 expectation sums, l: dE/dbeta_l, p+l: dE/dgamma_l
    int sum_index;             // row of this pass in the partial-sum table, -1 none
};

// register bits of arrangements X and Y (see pass_common.cuh)
constexpr uint32_t REGS_X[2] = {0x0F8u, 0x1C18u};  // type 0: bits 3..7; type 1: {3,4,10,11,12}
constexpr uint32_t REGS_Y[2] = {0x307u, 0x3E0u};   // type 0: {0,1,2,8,9}; type 1: bits 5..9

inline uint32_t window_mask(int loA, int loB, int q0, int k) {
    uint32_t m = 0;
    for (int q = q0; q < q0 + k; ++q) {
        if (q >= loA && q < loA + 5) m |= 1u << (3 + q - loA);
        else m |= 1u << (8 + q - loB);
    }
    return m;
}

// Groups of the schedule.  Returns an empty vector if no valid layout exists
// (never for 13 <= n <= 33 and 3 <= maxq <= 10).
inline std::vector<Group> make_groups(int n, int maxq) {
    const int G = (n + maxq - 1) / maxq;
    std::vector<int> k(G);
    for (int g = 0; g < G; ++g) k[g] = n / G + (g < n % G ? 1 : 0);
    std::vector<Group> gs(G);
    gs[0] = Group{};
    gs[0].type = 0;
    gs[0].mask = (1u << k[0]) - 1u;
    // high qubits [k0, n): the lower halves of the groups first, then the upper halves
    const bool split = n >= 24 && G >= 2;
    int qa = k[0];
    int qb = k[0];
    if (split)
        for (int g = 1; g < G; ++g) qb += (k[g] + 1) / 2;
    for (int g = 1; g < G; ++g) {
        Group &gr = gs[g];
        gr.type = 1;
        bool ok = false;
        if (split) {
            const int a = (k[g] + 1) / 2, b = k[g] - a;
            int sA = qa - (5 - a);
            if (sA < 3) sA = 3;
            int sB = qb < n - 5 ? qb : n - 5;
            if (sA <= qa && sA + 5 >= qa + a && sB <= qb && sB + 5 >= qb + b && sA + 5 <= sB) {
                gr.loA = sA;
                gr.loB = sB;
                gr.mask = 0;
                for (int q = qa; q < qa + a; ++q) gr.mask |= 1u << (3 + q - sA);
                for (int q = qb; q < qb + b; ++q) gr.mask |= 1u << (8 + q - sB);
                ok = true;
            }
            qa += a;
            qb += b;
            if (!ok) return {};
        } else {
            const int lo = qa < n - 10 ? qa : n - 10;
            gr.loA = lo;
            gr.loB = lo + 5;
            gr.mask = window_mask(gr.loA, gr.loB, qa, k[g]);
            qa += k[g];
        }
    }
    for (Group &gr : gs) {
        gr.kX = __builtin_popcount(gr.mask & REGS_X[gr.type]);
        gr.kY = __builtin_popcount(gr.mask & REGS_Y[gr.type]);
    }
    return gs;
}

// Forward schedule, then (grad) the reverse passes in reverse order; the
// reverse of the final pass is fused into it.  stored_mids: how many
// mixer-only passes keep their input for the reverse sweep (-1: all; 0: none,
// the uncompute sweep).  The kept ones are the last of the forward sweep, which
// the reverse sweep meets first; their reverse passes carry lambda alone, the
// others uncompute psi on the interleaved buffer, and each reverse pass writes
// the form the next one reads.  *nslots receives the number of stored states
// (with -1, the inputs of all mixer-only passes); *nmids the number of
// mixer-only passes.
inline std::vector<PassPlan> make_plan(int n, int p, bool grad, int maxq, int stored_mids = 0,
                                       int *nslots = nullptr, int *nmids = nullptr) {
    const std::vector<Group> gs = make_groups(n, maxq);
    if (gs.empty()) return {};
    const int G = (int)gs.size();
    struct D {
        int group, init, epi, la, lc, lb;
    };
    std::vector<D> f;
    auto order = [&](int l, int i) { return (l % 2 == 0) ? i : G - 1 - i; };
    if (p == 0) {
        f.push_back({0, 1, 0, -1, -1, -1});
    } else {
        f.push_back({order(0, 0), 1, 0, -1, 0, 0});
        for (int l = 0; l < p; ++l) {
            for (int i = 1; i < G - 1; ++i) f.push_back({order(l, i), 0, 0, -1, -1, l});
            const int last = order(l, G - 1);
            if (l + 1 < p) f.push_back({last, 0, 0, l, l + 1, l + 1});
            else if (grad) f.push_back({last, 0, 1, l, -1, -1});
            else f.push_back({last, 0, 0, -1, -1, l});
        }
    }
    const int F = (int)f.size();
    auto is_middle = [&](int i) { return !f[i].init && !f[i].epi && f[i].la < 0 && f[i].lc < 0 && f[i].lb >= 0; };
    int M = 0;
    for (int i = 0; i < F; ++i) M += is_middle(i) ? 1 : 0;
    if (nmids) *nmids = M;
    int keep = (grad && G >= 3) ? (stored_mids < 0 ? M : (stored_mids < M ? stored_mids : M)) : 0;
    // the last `keep` mixer-only passes keep their input
    std::vector<char> kept(F, 0);
    for (int i = F - 1, left = keep; i >= 0 && left > 0; --i)
        if (is_middle(i)) {
            kept[i] = 1;
            --left;
        }
    std::vector<int> in_slot(F, SLOT_NONE), out_slot(F, SLOT_W);
    int ns = 0;
    for (int i = 0; i < F; ++i) {
        in_slot[i] = i == 0 ? SLOT_NONE : out_slot[i - 1];
        if (f[i].epi) {
            out_slot[i] = SLOT_NONE;
        } else if (i + 1 < F && kept[i + 1]) {
            out_slot[i] = ns++;
        }
    }
    if (nslots) *nslots = ns;
    // form each reverse pass reads: lambda alone (a kept mixer-only pass) or the
    // interleaved buffer (every other pass); a reverse pass writes what the next
    // one reads, the final pass what the first reverse pass reads
    auto reads_lambda_alone = [&](int i) { return i >= 0 && kept[i] != 0; };
    std::vector<PassPlan> plan;
    int rows = 0;
    auto base = [&](const D &d, int kind) {
        PassPlan pl{};
        const Group &g = gs[d.group];
        pl.kind = kind;
        pl.split_out = 0;
        pl.in_slot = pl.out_slot = pl.psi_slot = SLOT_W;
        pl.type = g.type;
        pl.loA = g.loA;
        pl.loB = g.loB;
        pl.mask = g.mask;
        pl.kX = g.kX;
        pl.kY = g.kY;
        pl.init = d.init;
        pl.la = d.la;
        pl.lc = d.lc;
        pl.lb = d.lb;
        for (int s = 0; s < NSLOT; ++s) pl.slot_param[s] = -1;
        pl.sum_index = -1;
        return pl;
    };
    for (int i = 0; i < F; ++i) {
        const D &d = f[i];
        PassPlan pl = base(d, d.epi ? 1 : 0);
        pl.in_slot = in_slot[i];
        pl.out_slot = out_slot[i];
        if (d.epi) {
            pl.slot_param[0] = pl.slot_param[1] = -2;
            pl.slot_param[2] = pl.slot_param[3] = d.la;
            pl.sum_index = rows++;
            pl.split_out = reads_lambda_alone(i - 1) ? 1 : 0;
        }
        plan.push_back(pl);
    }
    if (grad)
        for (int i = (int)f.size() - 2; i >= 0; --i) {
            const bool mid = kept[i] != 0;
            PassPlan pl = base(f[i], mid ? 3 : 2);
            pl.psi_slot = mid ? in_slot[i] : SLOT_NONE;
            const bool next_alone = reads_lambda_alone(i - 1);
            pl.pl_out = mid && i >= 1 && !next_alone;
            pl.split_out = !mid && next_alone ? 1 : 0;
            if (f[i].lb >= 0) pl.slot_param[0] = pl.slot_param[1] = f[i].lb;
            if (f[i].lc >= 0) pl.slot_param[2] = p + f[i].lc;
            if (f[i].la >= 0) pl.slot_param[3] = pl.slot_param[4] = f[i].la;
            pl.sum_index = rows++;
            plan.push_back(pl);
        }
    return plan;
}

// The final pass and the reverse passes of cost-layer passes run on half
// blocks of 2^12 amplitudes when the context asks for it for every group.  The
// low group keeps its arrangements there, but in a high group the register
// bits of arrangement X are window B and those of Y window A (13-bit local
// bits 8..12 and 3..7), so a group that does not fill its block splits its
// mixed bits between X and Y differently; the scalars of those passes count
// them this way.
inline void use_half_block_counts(std::vector<PassPlan> &plan) {
    for (PassPlan &pl : plan)
        if ((pl.kind == 1 || pl.kind == 2) && pl.type == 1) {
            pl.kX = __builtin_popcount(pl.mask & 0x1F00u);
            pl.kY = __builtin_popcount(pl.mask & 0x00F8u);
        }
}

inline int plan_rows(const std::vector<PassPlan> &plan) {
    int r = 0;
    for (const auto &pl : plan) r += pl.sum_index >= 0;
    return r;
}

// ---- host/device scalar arithmetic ---------------------------------------------

struct HdCx {
    double re, im;
};
__host__ __device__ inline HdCx hc_mul(HdCx a, HdCx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ inline HdCx hc_conj(HdCx a) { return {a.re, -a.im}; }
__host__ __device__ inline double hc_norm(HdCx a) { return a.re * a.re + a.im * a.im; }
__host__ __device__ inline HdCx hc_inv(HdCx a) {
    const double d = hc_norm(a);
    return {a.re / d, -a.im / d};
}
__host__ __device__ inline HdCx hc_div(HdCx a, HdCx b) { return hc_mul(a, hc_inv(b)); }
__host__ __device__ inline HdCx hc_pow(HdCx f, int k) {
    HdCx r{1.0, 0.0};
    for (int i = 0; i < k; ++i) r = hc_mul(r, f);
    return r;
}
__host__ __device__ inline float2 hc_f2(HdCx z) { return make_float2((float)z.re, (float)z.im); }

// 64 x 64 -> 128-bit product
__host__ __device__ inline void mul64(unsigned long long a, unsigned long long b, unsigned long long *hi,
                                      unsigned long long *lo) {
#ifdef __CUDA_ARCH__
    *lo = a * b;
    *hi = __umul64hi(a, b);
#else
    const unsigned __int128 t = (unsigned __int128)a * b;
    *lo = (unsigned long long)t;
    *hi = (unsigned long long)(t >> 64);
#endif
}

// Phase multiplier for U_C(gamma): a table entry T contributes (T + k_c) * phi
// turns (units of 2^-64 turn, modulo 2^64), with
//   phi = round(gamma 2^-s / (2 pi) 2^64) mod 2^64.
// |gamma| = M 2^E exactly (M < 2^53); phi = round(M * K * 2^(E - s + 64 - 256))
// with K = floor(2^256 / (2 pi)), evaluated on 64-bit limbs.
__host__ __device__ inline unsigned long long phase_multiplier(double gamma, int s) {
    // floor(2^256 / (2 pi)), little-endian 64-bit limbs
    const unsigned long long K[4] = {0x7f9458eaf7aef158ull, 0x36d8a5664f10e410ull, 0x7f09d5f47d4d3770ull,
                                     0x28be60db9391054aull};
    if (gamma == 0.0 || !isfinite(gamma)) return 0ull;
    int e2;
    const double m = frexp(fabs(gamma), &e2);                   // |gamma| = m 2^e2, m in [0.5, 1)
    const unsigned long long M = (unsigned long long)ldexp(m, 53);  // exact 53-bit integer
    const int E = e2 - 53;
    unsigned long long P[5] = {0, 0, 0, 0, 0};
    unsigned long long carry = 0;
    for (int i = 0; i < 4; ++i) {
        unsigned long long hi, lo;
        mul64(M, K[i], &hi, &lo);
        const unsigned long long t = lo + carry;
        P[i] = t;
        carry = hi + (t < lo ? 1ull : 0ull);
    }
    P[4] = carry;
    const int sh = E - s + 64 - 256;
    unsigned long long phi = 0;
    if (sh >= 0) {
        phi = sh < 64 ? (P[0] << sh) : 0ull;
    } else {
        const int r = -sh;
        if (r > 320) return 0ull;
        // round: add 2^(r-1), then shift right by r
        const int wb = (r - 1) / 64, bb = (r - 1) % 64;
        unsigned long long c2 = 0;
        for (int i = 0; i < 5; ++i) {
            const unsigned long long add = (i == wb) ? (1ull << bb) : 0ull;
            const unsigned long long t = P[i] + add;
            const unsigned long long t2 = t + c2;
            c2 = (t < P[i] ? 1ull : 0ull) + (t2 < t ? 1ull : 0ull);
            P[i] = t2;
        }
        const int w = r / 64, b = r % 64;
        const unsigned long long lo = w < 5 ? P[w] : 0ull, hi = (w + 1) < 5 ? P[w + 1] : 0ull;
        phi = b == 0 ? lo : ((lo >> b) | (hi << (64 - b)));
    }
    return gamma < 0 ? (0ull - phi) : phi;
}

// turns offset (units of 2^-64 turn) that multiplies the phase by e^{i arg z}
__host__ __device__ inline unsigned long long turns_of_arg(HdCx z) {
    double x = -atan2(z.im, z.re) / (2.0 * 3.14159265358979323846) * 18446744073709551616.0;
    if (x >= 9.2233720368547758e18) x -= 18446744073709551616.0;
    return (unsigned long long)(long long)llrint(x);
}

struct HdMix {
    float t;
    int flip;
    HdCx f;  // common factor of one level: true = f * computed
};

// RX(2 beta) = cos(beta) (1 - i tan(beta) X) if |cos| >= |sin|,
// else (-i X) RX(2 beta - pi) = -i sin(beta) X (1 - i tan(beta - pi/2) X).
__host__ __device__ inline HdMix mix_of(double beta) {
    HdMix m;
    const double c = cos(beta), s = sin(beta);
    if (fabs(c) >= fabs(s)) {
        m.flip = 0;
        m.t = (float)(s / c);
        m.f = {c, 0.0};
    } else {
        m.flip = 1;
        m.t = (float)(-c / s);
        m.f = {0.0, -s};
    }
    return m;
}

// Scalars of pass `pl` for one parameter set (gamma, beta: p entries each) on
// a table with fixed-point parameters (s, k_c).  The computed amplitudes are
// tracked as true * S: each forward mixer level divides by f, each inverse
// level by conj(f); the phase multiplier absorbs the accumulated scalars so
// that every stored state is at true scale, and slot_scale[s] converts each
// partial sum back to true scale.
__host__ __device__ inline void pass_scalars(const PassPlan &pl, const double *gamma, const double *beta, int s,
                                             long long k_c, PassScal *sc, double *slot_scale) {
    const int k = pl.kX + pl.kY;
    sc->pre_t = sc->post_t = 0.f;
    sc->pre_flip = sc->post_flip = 0;
    sc->phi = sc->off = 0ull;
    sc->kmag = 1.f;
    sc->cscale = (float)ldexp(1.0, -s);
    sc->kend = make_float2(1.f, 0.f);
    sc->kend2 = make_float2(1.f, 0.f);
    for (int q = 0; q < NSLOT; ++q) slot_scale[q] = 0.0;
    HdMix ma{}, mb{};
    if (pl.la >= 0) {
        ma = mix_of(beta[pl.la]);
        sc->pre_t = ma.t;
        sc->pre_flip = ma.flip;
    }
    if (pl.lb >= 0) {
        mb = mix_of(beta[pl.lb]);
        sc->post_t = mb.t;
        sc->post_flip = mb.flip;
    }
    const HdCx one{1.0, 0.0};
    HdCx S = one;
    if (pl.kind == 0 || pl.kind == 1) {
        if (pl.la >= 0) S = hc_div(S, hc_pow(ma.f, k));
        if (pl.lc >= 0) {
            const unsigned long long phi = phase_multiplier(gamma[pl.lc], s);
            const HdCx post = pl.lb >= 0 ? hc_pow(mb.f, k) : one;
            const HdCx Kf = hc_div(post, S);
            sc->phi = phi;
            sc->off = (unsigned long long)k_c * phi + turns_of_arg(Kf);
            sc->kmag = (float)sqrt(hc_norm(Kf));
            S = post;
        }
        if (pl.lb >= 0) S = hc_div(S, hc_pow(mb.f, k));
        if (pl.kind == 0) {
            if (pl.lc < 0) sc->kend = hc_f2(hc_inv(S));
        } else {
            sc->kend = hc_f2(hc_inv(S));  // psi_p = kend * computed
            HdCx Sl = one;
            slot_scale[0] = slot_scale[1] = 1.0;
            slot_scale[2] = 1.0;
            Sl = hc_div(Sl, hc_pow(hc_conj(ma.f), pl.kY));
            slot_scale[3] = 1.0 / hc_norm(Sl);
            Sl = hc_div(Sl, hc_pow(hc_conj(ma.f), pl.kX));
            sc->kend2 = hc_f2(hc_inv(Sl));
        }
    } else if (pl.kind == 3) {
        // lambda alone: undo the mixer, return to true scale, then both
        // X-term halves at the pass input against the stored psi
        S = hc_div(S, hc_pow(hc_conj(mb.f), k));
        sc->kend = hc_f2(hc_inv(S));
        slot_scale[0] = slot_scale[1] = 1.0;
    } else {
        if (pl.lb >= 0) {
            slot_scale[0] = 1.0 / hc_norm(S);
            S = hc_div(S, hc_pow(hc_conj(mb.f), pl.kX));
            slot_scale[1] = 1.0 / hc_norm(S);
            S = hc_div(S, hc_pow(hc_conj(mb.f), pl.kY));
        }
        if (pl.lc >= 0) {
            slot_scale[2] = 1.0 / hc_norm(S);
            const unsigned long long phi = phase_multiplier(gamma[pl.lc], s);
            const HdCx pre = pl.la >= 0 ? hc_pow(hc_conj(ma.f), k) : one;
            const HdCx Kf = hc_div(pre, S);
            sc->phi = 0ull - phi;
            sc->off = (0ull - (unsigned long long)k_c * phi) + turns_of_arg(Kf);
            sc->kmag = (float)sqrt(hc_norm(Kf));
            S = hc_mul(S, Kf);
        }
        if (pl.la >= 0) {
            slot_scale[3] = 1.0 / hc_norm(S);
            S = hc_div(S, hc_pow(hc_conj(ma.f), pl.kY));
            slot_scale[4] = 1.0 / hc_norm(S);
            S = hc_div(S, hc_pow(hc_conj(ma.f), pl.kX));
        }
        if (pl.lc < 0) sc->kend = hc_f2(hc_inv(S));
    }
}

// Algorithmic bytes per amplitude of a pass (what the method must move).
inline double pass_bytes_per_amp(const PassPlan &pl) {
    if (pl.kind == 0) return (pl.init ? 0.0 : 8.0) + 8.0 + (pl.lc >= 0 ? 4.0 : 0.0);
    if (pl.kind == 1) return 8.0 + 4.0 + (pl.split_out ? 8.0 : 16.0);
    if (pl.kind == 3) return 8.0 + 8.0 + (pl.pl_out ? 16.0 : 8.0);  // psi_in, lambda in, lambda (+psi) out
    return 16.0 + (pl.init ? 0.0 : (pl.split_out ? 8.0 : 16.0)) + (pl.lc >= 0 ? 4.0 : 0.0);
}

// Device side (batch.cu): recompute every pass's scalars from device angles,
// assemble E and the gradient from the partial sums, and the Adam update.
struct DevPlan {
    const PassPlan *plan;  // [npasses]
    int npasses, p, nitems;
    const double *gamma, *beta;        // [nitems][p]
    const int *item_s;                 // [nitems] fixed-point shift of the item's table
    const long long *item_kc;          // [nitems]
    PassScal *scal;                    // [npasses][nitems]
    double *slot_scale;                // [npasses][nitems][NSLOT]
};
cudaError_t launch_prep_scalars(const DevPlan &d, cudaStream_t st);
cudaError_t launch_assemble(const DevPlan &d, const double *sums /*[rows][nitems][NSLOT]*/, double *E,
                            double *dgamma, double *dbeta, cudaStream_t st);

struct AdamArgs {
    double *gamma, *beta;        // [nitems][p], updated in place
    const double *dgamma, *dbeta;  // gradient of item i, parameter l at [i * gstride + l]
    int gstride;
    double *m, *v;               // [2][nitems][p] moments
    int *step;                   // device step counter
    const double *E;             // objective of item i at E[i * estride]
    int estride;
    double *history;             // [max_steps][nitems] or null
    int max_steps, nitems, p;
    int step0;                   // steps taken before this run (history rows count from it)
    double lr, beta1, beta2, eps;
};
cudaError_t launch_adam(const AdamArgs &a, cudaStream_t st);

}  // namespace qaoa
