// C ABI of the QAOA statevector library (include/qaoa.h): handles, the layer
// pass schedule, gradient assembly, and the DQAOA entry points.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <memory>
#include <vector>

#include "kernels_misc.h"
#include "kernels_tma.h"
#include "qaoa_internal.h"

using namespace qaoa;
using cd = std::complex<double>;

namespace qaoa {
const char *last_error();
}

#define CUDA_TRY(expr)                                                                      \
    do {                                                                                    \
        cudaError_t e__ = (expr);                                                           \
        if (e__ != cudaSuccess)                                                             \
            return fail(e__ == cudaErrorMemoryAllocation ? QAOA_ERR_OUT_OF_MEMORY : QAOA_ERR_CUDA, \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e__), __FILE__, __LINE__); \
    } while (0)

#define QAOA_TRY(expr)                 \
    do {                               \
        qaoa_status s__ = (expr);      \
        if (s__ != QAOA_OK) return s__; \
    } while (0)

namespace {

// growable device buffer
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    qaoa_status ensure(size_t bytes, int64_t *held, int64_t budget) {
        if (bytes <= cap) return QAOA_OK;
        if (budget > 0 && *held - (int64_t)cap + (int64_t)bytes > budget)
            return fail(QAOA_ERR_OUT_OF_MEMORY, "memory budget of %lld bytes exceeded", (long long)budget);
        if (p) cudaFree(p);
        p = nullptr;
        *held -= (int64_t)cap;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(QAOA_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
        cap = bytes;
        *held += (int64_t)bytes;
        return QAOA_OK;
    }
    template <typename T>
    T *as() const {
        return reinterpret_cast<T *>(p);
    }
};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double bytes;
};

}  // namespace

struct qaoa_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    qaoa_options opt{};
    int64_t held = 0;
    DevBuf work_psi, lam, pl, partials, pass_sums, topk_a, topk_b, items, small_out, misc;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> ev_free;
    int64_t prof_launches[5] = {0, 0, 0, 0, 0};
    double prof_ms[5] = {0, 0, 0, 0, 0};
    double prof_bytes[5] = {0, 0, 0, 0, 0};
    int64_t launches_total = 0;  // every kernel launched by this context
    int num_sms = 148;
    DevBuf status;               // device status word of the bounded waits
};

struct qaoa_cost_s {
    int device = 0;
    int n = 0;
    Canonical can;
    FixedPoint fp;
    int32_t *T = nullptr;
    uint64_t argmin = 0;
    int64_t minval = 0;
    ~qaoa_cost_s() {
        if (T) cudaFree(T);
    }
};

struct qaoa_state_s {
    int device = 0;
    int n = 0;
    bool fp64 = false;
    void *amps = nullptr;
    ~qaoa_state_s() {
        if (amps) cudaFree(amps);
    }
};

namespace {

// ---- profiling -----------------------------------------------------------------
cudaEvent_t get_event(qaoa_ctx c) {
    if (!c->ev_free.empty()) {
        cudaEvent_t e = c->ev_free.back();
        c->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct ProfScope {
    qaoa_ctx c;
    int kind;
    double bytes;
    cudaEvent_t a = nullptr;
    ProfScope(qaoa_ctx c_, int kind_, double bytes_) : c(c_), kind(kind_), bytes(bytes_) {
        if (c->opt.profile) {
            a = get_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~ProfScope() {
        if (c->opt.profile) {
            cudaEvent_t b = get_event(c);
            cudaEventRecord(b, c->stream);
            c->pending.push_back({kind, a, b, bytes});
        }
    }
};

void drain_profile(qaoa_ctx c) {
    if (c->pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto &r : c->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        c->prof_launches[r.kind] += 1;
        c->prof_ms[r.kind] += ms;
        c->prof_bytes[r.kind] += r.bytes;
        c->ev_free.push_back(r.a);
        c->ev_free.push_back(r.b);
    }
    c->pending.clear();
}

qaoa_status set_device(int dev) {
    CUDA_TRY(cudaSetDevice(dev));
    return QAOA_OK;
}

// ---- layer-pass schedule (Eq. qaoa_state with boundary fusion) -----------------------

struct Group {
    int type;      // 0: low group (block = global bits 0..12), 1: high group
    int lo;        // window offset (type 1)
    uint32_t mask; // mixed local bits
    int kX, kY;    // mixed bits in the register rounds of arrangements X and Y (256-thread kernels)
    int k3[3];     // mixed bits in rounds A, B, C (512-thread kernels)
};

struct PassDesc {
    int group;
    bool init = false, epi = false;
    int la = -1, lc = -1, lb = -1;  // layers (0-based) of pre mixer, cost, post mixer
};

constexpr uint32_t REGS_X[2] = {0x0F8u, 0x1C18u};  // type 0: bits 3..7; type 1: {3,4,10,11,12}
constexpr uint32_t REGS_Y[2] = {0x307u, 0x3E0u};   // type 0: {0,1,2,8,9}; type 1: bits 5..9
constexpr uint32_t ROUND3[2][3] = {{0x0018u, 0x0207u, 0x01E0u}, {0x1800u, 0x0618u, 0x01E0u}};

std::vector<Group> make_groups(int n, int maxq) {
    const int G = (n + maxq - 1) / maxq;
    std::vector<Group> gs;
    int q0 = 0;
    for (int g = 0; g < G; ++g) {
        const int k = n / G + (g < n % G ? 1 : 0);
        Group gr{};
        if (g == 0) {
            gr.type = 0;
            gr.lo = 0;
            gr.mask = (1u << k) - 1u;
        } else {
            gr.type = 1;
            gr.lo = std::min(q0, n - 10);
            gr.mask = 0;
            for (int q = q0; q < q0 + k; ++q) gr.mask |= 1u << (3 + q - gr.lo);
        }
        gr.kX = __builtin_popcount(gr.mask & REGS_X[gr.type]);
        gr.kY = __builtin_popcount(gr.mask & REGS_Y[gr.type]);
        for (int r = 0; r < 3; ++r) gr.k3[r] = __builtin_popcount(gr.mask & ROUND3[gr.type][r]);
        gs.push_back(gr);
        q0 += k;
    }
    return gs;
}

std::vector<PassDesc> make_schedule(int G, int p, bool grad) {
    std::vector<PassDesc> s;
    auto order = [&](int l) {  // layer l (0-based): ascending for even l, descending for odd l
        std::vector<int> o(G);
        for (int g = 0; g < G; ++g) o[g] = (l % 2 == 0) ? g : G - 1 - g;
        return o;
    };
    if (p == 0) {  // |+>^n only
        PassDesc d;
        d.group = 0;
        d.init = true;
        s.push_back(d);
        return s;
    }
    {
        PassDesc d;
        d.group = order(0)[0];
        d.init = true;
        d.lc = 0;
        d.lb = 0;
        s.push_back(d);
    }
    for (int l = 0; l < p; ++l) {
        auto o = order(l);
        for (int g = 1; g < G - 1; ++g) {
            PassDesc d;
            d.group = o[g];
            d.lb = l;
            s.push_back(d);
        }
        PassDesc d;
        d.group = o[G - 1];
        if (l + 1 < p) {
            d.la = l;
            d.lc = l + 1;
            d.lb = l + 1;
        } else if (grad) {
            d.la = l;
            d.epi = true;
        } else {
            d.lb = l;  // final mixer of a forward-only run
        }
        s.push_back(d);
    }
    return s;
}

struct Mix {
    MixOp op;
    cd f;  // common factor of one level (true = f * computed)
};

Mix mix_of(double beta) {
    Mix m{};
    const double c = std::cos(beta), s = std::sin(beta);
    m.op.mode = 1;
    if (std::fabs(c) >= std::fabs(s)) {  // RX(2 beta) = cos(beta) (1 - i tan(beta) X)
        m.op.flip = 0;
        m.op.t = (float)(s / c);
        m.f = cd(c, 0.0);
    } else {  // RX(2 beta) = -i X RX(2 beta - pi) = -i sin(beta) X (1 - i tan(beta - pi/2) X)
        m.op.flip = 1;
        m.op.t = (float)(-c / s);
        m.f = cd(0.0, -s);
    }
    return m;
}

cd cpow_int(cd f, int k) {
    cd r(1.0, 0.0);
    for (int i = 0; i < k; ++i) r *= f;
    return r;
}

float2 f2(cd z) { return make_float2((float)z.real(), (float)z.imag()); }

// turns offset (units of 2^-64 turn) that multiplies the phase by e^{i arg z}
uint64_t turns_of_arg(cd z) {
    const double turns = -std::arg(z) / (2.0 * M_PI);  // e^{-2 pi i t} = e^{i arg z}
    const double sc = turns * 18446744073709551616.0;   // 2^64
    return (uint64_t)(int64_t)std::llround(sc);
}

struct PassRun {
    PassArgs args;
    int type;
    bool epi;
    bool has_partials;
    double slot_scale[NSLOT];
    int slot_param[NSLOT];  // 0..p-1: beta_l ; p..2p-1: gamma_l ; -1 none ; -2: E slots
    double bytes;
};

// forward pass arguments (psi in place)
PassRun fwd_args(const Group &g, const PassDesc &d, const qaoa_cost_s *cost, const double *gamma,
                 const double *beta, float2 *psi, float2 *lam, double *partials,
                 unsigned long long *topk, int ktop, int p) {
    PassRun r{};
    PassArgs &a = r.args;
    a.psi = psi;
    a.lam = lam;
    a.C = cost->T;
    a.partials = partials;
    a.topk_keys = topk;
    a.n = cost->n;
    a.lo = g.lo;
    a.mask = g.mask;
    a.init = d.init;
    a.has_cost = d.lc >= 0;
    a.store_psi = 1;
    a.precise_phase = 0;
    a.ktop = d.epi ? ktop : 0;
    a.amp0 = (float)std::pow(2.0, -0.5 * cost->n);
    a.cscale = (float)std::ldexp(1.0, -cost->fp.s);
    a.kmag = 1.f;
    a.kend = make_float2(1.f, 0.f);
    a.kend2 = make_float2(1.f, 0.f);
    const int k = g.kX + g.kY;
    cd S(1.0, 0.0);  // computed = true * S
    Mix ma{}, mb{};
    if (d.la >= 0) {
        ma = mix_of(beta[d.la]);
        a.pre = ma.op;
        S /= cpow_int(ma.f, k);
    }
    if (d.lb >= 0) {
        mb = mix_of(beta[d.lb]);
        a.post = mb.op;
    }
    if (d.lc >= 0) {
        const uint64_t phi = phase_multiplier(gamma[d.lc], cost->fp.s);
        const cd Kf = (d.lb >= 0 ? cpow_int(mb.f, k) : cd(1.0, 0.0)) / S;
        a.phi = phi;
        a.off = (uint64_t)cost->fp.k_c * phi + turns_of_arg(Kf);
        a.kmag = (float)std::abs(Kf);
        S = (d.lb >= 0 ? cpow_int(mb.f, k) : cd(1.0, 0.0));
    }
    if (d.lb >= 0) S /= cpow_int(mb.f, k);
    for (int s = 0; s < NSLOT; ++s) {
        r.slot_scale[s] = 0.0;
        r.slot_param[s] = -1;
    }
    const double N = std::ldexp(1.0, cost->n);
    if (!d.epi) {
        if (d.lc < 0) a.kend = f2(1.0 / S);
        r.has_partials = false;
        r.bytes = N * ((d.init ? 0.0 : 8.0) + 8.0 + (d.lc >= 0 ? 4.0 : 0.0));
    } else {
        // S = 1/fa^k after the pre mixer; psi_p = fa^k * computed
        a.kend = f2(1.0 / S);
        cd Sl(1.0, 0.0);
        r.slot_param[0] = -2;
        r.slot_param[1] = -2;
        r.slot_scale[2] = 1.0;
        r.slot_param[2] = d.la;
        Sl /= cpow_int(std::conj(ma.f), g.kY);
        r.slot_scale[3] = 1.0 / std::norm(Sl);
        r.slot_param[3] = d.la;
        Sl /= cpow_int(std::conj(ma.f), g.kX);
        a.kend2 = f2(1.0 / Sl);
        r.has_partials = true;
        r.bytes = N * (8.0 + 4.0 + 8.0);
    }
    r.type = g.type;
    r.epi = d.epi;
    (void)p;
    return r;
}

// reverse pass arguments: undo forward pass d on (psi, lambda)
PassRun rev_args(const Group &g, const PassDesc &d, const qaoa_cost_s *cost, const double *gamma,
                 const double *beta, float2 *psi, float2 *lam, double *partials, int p) {
    PassRun r{};
    PassArgs &a = r.args;
    a.psi = psi;
    a.lam = lam;
    a.C = cost->T;
    a.partials = partials;
    a.n = cost->n;
    a.lo = g.lo;
    a.mask = g.mask;
    a.has_cost = d.lc >= 0;
    a.store_psi = d.init ? 0 : 1;
    a.precise_phase = 0;
    a.cscale = (float)std::ldexp(1.0, -cost->fp.s);
    a.kmag = 1.f;
    a.kend = make_float2(1.f, 0.f);
    const int k = g.kX + g.kY;
    Mix ma{}, mb{};
    if (d.la >= 0) {
        ma = mix_of(beta[d.la]);
        a.pre = ma.op;
    }
    if (d.lb >= 0) {
        mb = mix_of(beta[d.lb]);
        a.post = mb.op;
    }
    for (int s = 0; s < NSLOT; ++s) {
        r.slot_scale[s] = 0.0;
        r.slot_param[s] = -1;
    }
    cd S(1.0, 0.0);
    if (d.lb >= 0) {
        r.slot_scale[0] = 1.0 / std::norm(S);
        r.slot_param[0] = d.lb;
        S /= cpow_int(std::conj(mb.f), g.kX);
        r.slot_scale[1] = 1.0 / std::norm(S);
        r.slot_param[1] = d.lb;
        S /= cpow_int(std::conj(mb.f), g.kY);
    }
    if (d.lc >= 0) {
        r.slot_scale[2] = 1.0 / std::norm(S);
        r.slot_param[2] = p + d.lc;
        const uint64_t phi = phase_multiplier(gamma[d.lc], cost->fp.s);
        const cd Kf = (d.la >= 0 ? cpow_int(std::conj(ma.f), k) : cd(1.0, 0.0)) / S;
        a.phi = (uint64_t)0 - phi;
        a.off = (uint64_t)0 - (uint64_t)cost->fp.k_c * phi + turns_of_arg(Kf);
        a.kmag = (float)std::abs(Kf);
        S *= Kf;
    }
    if (d.la >= 0) {
        r.slot_scale[3] = 1.0 / std::norm(S);
        r.slot_param[3] = d.la;
        S /= cpow_int(std::conj(ma.f), g.kY);
        r.slot_scale[4] = 1.0 / std::norm(S);
        r.slot_param[4] = d.la;
        S /= cpow_int(std::conj(ma.f), g.kX);
    }
    if (d.lc < 0) a.kend = f2(1.0 / S);
    r.has_partials = true;
    r.type = g.type;
    r.epi = false;
    const double N = std::ldexp(1.0, cost->n);
    r.bytes = N * (16.0 + (a.store_psi ? 16.0 : 0.0) + (d.lc >= 0 ? 4.0 : 0.0));
    return r;
}

// Arguments of the 512-thread kernels.  Same scalar bookkeeping as fwd_args /
// rev_args (computed = true * S), with three register rounds per mixer:
// forward mixers run rounds A, B, C (pre) and C, B, A (post).
PassRun fwd3_args(const Group &g, const PassDesc &d, const qaoa_cost_s *cost, const double *gamma,
                  const double *beta, float2 *psi, float4 *pl, double *partials, unsigned long long *topk, int ktop) {
    PassRun r{};
    PassArgs &a = r.args;
    a.psi = psi;
    a.pl = pl;
    a.C = cost->T;
    a.partials = partials;
    a.topk_keys = topk;
    a.n = cost->n;
    a.lo = g.lo;
    a.mask = g.mask;
    a.init = d.init;
    a.has_cost = d.lc >= 0;
    a.store_psi = 1;
    a.ktop = d.epi ? ktop : 0;
    a.amp0 = (float)std::pow(2.0, -0.5 * cost->n);
    a.cscale = (float)std::ldexp(1.0, -cost->fp.s);
    a.kmag = 1.f;
    a.kend = make_float2(1.f, 0.f);
    a.kend2 = make_float2(1.f, 0.f);
    const int k = g.kX + g.kY;
    cd S(1.0, 0.0);
    Mix ma{}, mb{};
    if (d.la >= 0) {
        ma = mix_of(beta[d.la]);
        a.pre = ma.op;
        S /= cpow_int(ma.f, k);
    }
    if (d.lb >= 0) {
        mb = mix_of(beta[d.lb]);
        a.post = mb.op;
    }
    if (d.lc >= 0) {
        const uint64_t phi = phase_multiplier(gamma[d.lc], cost->fp.s);
        const cd Kf = (d.lb >= 0 ? cpow_int(mb.f, k) : cd(1.0, 0.0)) / S;
        a.phi = phi;
        a.off = (uint64_t)cost->fp.k_c * phi + turns_of_arg(Kf);
        a.kmag = (float)std::abs(Kf);
        S = (d.lb >= 0 ? cpow_int(mb.f, k) : cd(1.0, 0.0));
    }
    if (d.lb >= 0) S /= cpow_int(mb.f, k);
    for (int s = 0; s < NSLOT; ++s) {
        r.slot_scale[s] = 0.0;
        r.slot_param[s] = -1;
    }
    const double N = std::ldexp(1.0, cost->n);
    if (!d.epi) {
        if (d.lc < 0) a.kend = f2(1.0 / S);
        r.has_partials = false;
        r.bytes = N * ((d.init ? 0.0 : 8.0) + 8.0 + (d.lc >= 0 ? 4.0 : 0.0));
    } else {
        a.kend = f2(1.0 / S);
        cd Sl(1.0, 0.0);
        r.slot_param[0] = -2;
        r.slot_param[1] = -2;
        const int order[3] = {2, 1, 0};  // lambda undo: rounds C, B, A -> slots 2, 3, 4
        for (int j = 0; j < 3; ++j) {
            r.slot_scale[2 + j] = 1.0 / std::norm(Sl);
            r.slot_param[2 + j] = d.la;
            Sl /= cpow_int(std::conj(ma.f), g.k3[order[j]]);
        }
        a.kend2 = f2(1.0 / Sl);
        r.has_partials = true;
        r.bytes = N * (8.0 + 4.0 + 16.0);
    }
    r.type = g.type;
    r.epi = d.epi;
    return r;
}

PassRun rev3_args(const Group &g, const PassDesc &d, const qaoa_cost_s *cost, const double *gamma,
                  const double *beta, float4 *pl, double *partials, int p) {
    PassRun r{};
    PassArgs &a = r.args;
    a.pl = pl;
    a.C = cost->T;
    a.partials = partials;
    a.n = cost->n;
    a.lo = g.lo;
    a.mask = g.mask;
    a.has_cost = d.lc >= 0;
    a.store_psi = d.init ? 0 : 1;
    a.cscale = (float)std::ldexp(1.0, -cost->fp.s);
    a.kmag = 1.f;
    a.kend = make_float2(1.f, 0.f);
    const int k = g.kX + g.kY;
    Mix ma{}, mb{};
    if (d.la >= 0) {
        ma = mix_of(beta[d.la]);
        a.pre = ma.op;
    }
    if (d.lb >= 0) {
        mb = mix_of(beta[d.lb]);
        a.post = mb.op;
    }
    for (int s = 0; s < NSLOT; ++s) {
        r.slot_scale[s] = 0.0;
        r.slot_param[s] = -1;
    }
    cd S(1.0, 0.0);
    if (d.lb >= 0) {  // undo the post mixer: rounds A, B, C -> slots 0, 1, 2
        for (int j = 0; j < 3; ++j) {
            r.slot_scale[j] = 1.0 / std::norm(S);
            r.slot_param[j] = d.lb;
            S /= cpow_int(std::conj(mb.f), g.k3[j]);
        }
    }
    if (d.lc >= 0) {
        r.slot_scale[3] = 1.0 / std::norm(S);
        r.slot_param[3] = p + d.lc;
        const uint64_t phi = phase_multiplier(gamma[d.lc], cost->fp.s);
        const cd Kf = (d.la >= 0 ? cpow_int(std::conj(ma.f), k) : cd(1.0, 0.0)) / S;
        a.phi = (uint64_t)0 - phi;
        a.off = (uint64_t)0 - (uint64_t)cost->fp.k_c * phi + turns_of_arg(Kf);
        a.kmag = (float)std::abs(Kf);
        S *= Kf;
    }
    if (d.la >= 0) {  // undo the pre mixer: rounds C, B, A -> slots 4, 5, 6
        const int order[3] = {2, 1, 0};
        for (int j = 0; j < 3; ++j) {
            r.slot_scale[4 + j] = 1.0 / std::norm(S);
            r.slot_param[4 + j] = d.la;
            S /= cpow_int(std::conj(ma.f), g.k3[order[j]]);
        }
    }
    if (d.lc < 0) a.kend = f2(1.0 / S);
    r.has_partials = true;
    r.type = g.type;
    r.epi = false;
    const double N = std::ldexp(1.0, cost->n);
    r.bytes = N * (16.0 + (a.store_psi ? 16.0 : 0.0) + (d.lc >= 0 ? 4.0 : 0.0));
    return r;
}

qaoa_status ensure_scratch(qaoa_ctx c, int n, int npasses, int ktop, bool grad) {
    const size_t N = (size_t)1 << n;
    const int nb = n >= BLOCK_BITS ? (1 << (n - BLOCK_BITS)) : 1;
    QAOA_TRY(c->work_psi.ensure(N * sizeof(float2), &c->held, c->opt.memory_budget));
    if (grad && n >= BLOCK_BITS) {
        if (c->opt.pass_variant == 1) QAOA_TRY(c->lam.ensure(N * sizeof(float2), &c->held, c->opt.memory_budget));
        else QAOA_TRY(c->pl.ensure(N * sizeof(float4), &c->held, c->opt.memory_budget));
    }
    QAOA_TRY(c->partials.ensure((size_t)nb * NSLOT * sizeof(double), &c->held, c->opt.memory_budget));
    QAOA_TRY(c->pass_sums.ensure((size_t)(npasses + 1) * NSLOT * sizeof(double), &c->held, c->opt.memory_budget));
    const int kk = std::max(ktop, 1);
    QAOA_TRY(c->topk_a.ensure((size_t)nb * kk * 8 + 64, &c->held, c->opt.memory_budget));
    QAOA_TRY(c->topk_b.ensure((size_t)((nb + 255) / 256 + 1) * kk * 8 + 64, &c->held, c->opt.memory_budget));
    return QAOA_OK;
}

// Decode top-K keys: x = 2^33-1 - low33, P = float bits of the high part.
void decode_keys(const unsigned long long *keys, int k, uint64_t *idx, float *prob) {
    for (int i = 0; i < k; ++i) {
        const unsigned long long key = keys[i];
        if (idx) idx[i] = 0x1FFFFFFFFull - (key & 0x1FFFFFFFFull);
        if (prob) {
            uint32_t b = (uint32_t)(key >> 33);
            float f;
            std::memcpy(&f, &b, 4);
            prob[i] = f;
        }
    }
}

// Evolve with the pass schedule on a complex64 buffer; optional gradient.
qaoa_status run_passes(qaoa_ctx c, const qaoa_cost_s *cost, int p, const double *gamma,
                       const double *beta, float2 *psi, bool grad, double *E, double *dg, double *db,
                       int ktop, uint64_t *top_idx, float *top_prob) {
    const int n = cost->n;
    const int maxq = c->opt.max_fused_qubits ? c->opt.max_fused_qubits : 10;
    const auto groups = make_groups(n, maxq);
    const auto sched = make_schedule((int)groups.size(), p, grad);
    const int nb = 1 << (n - BLOCK_BITS);
    const int npasses = (int)sched.size() * (grad ? 2 : 1);
    QAOA_TRY(ensure_scratch(c, n, npasses, grad ? ktop : 0, grad));
    const bool use_tma = c->opt.pass_variant != 1;
    float2 *lam = (grad && !use_tma) ? c->lam.as<float2>() : nullptr;
    float4 *pl = (grad && use_tma) ? c->pl.as<float4>() : nullptr;
    double *partials = c->partials.as<double>();
    double *sums = c->pass_sums.as<double>();
    // variant 0 (default): forward passes with direct loads (256 threads, two
    // CTAs per SM), final pass and reverse sweep TMA-pipelined on the
    // interleaved (psi, lambda) buffer
    const int variant = c->opt.pass_variant;
    std::vector<PassRun> runs;
    if (variant == 3) {
        for (const auto &d : sched)
            runs.push_back(fwd3_args(groups[d.group], d, cost, gamma, beta, psi, c->pl.as<float4>(), partials,
                                     c->topk_a.as<unsigned long long>(), ktop));
        if (grad)
            for (int i = (int)sched.size() - 2; i >= 0; --i)
                runs.push_back(rev3_args(groups[sched[i].group], sched[i], cost, gamma, beta, c->pl.as<float4>(),
                                         partials, p));
    } else {
        for (const auto &d : sched)
            runs.push_back(fwd_args(groups[d.group], d, cost, gamma, beta, psi, lam, partials,
                                    c->topk_a.as<unsigned long long>(), ktop, p));
        if (grad)
            for (int i = (int)sched.size() - 2; i >= 0; --i)
                runs.push_back(rev_args(groups[sched[i].group], sched[i], cost, gamma, beta, psi, lam, partials, p));
    }
    for (auto &r : runs) {
        r.args.pl = pl;
        if (use_tma && r.epi) r.bytes = std::ldexp(28.0, n);  // psi + table in, (psi, lambda) out
        if (variant == 3) r.args.psi = psi;
    }
    if (use_tma) {
        QAOA_TRY(c->status.ensure(16, &c->held, c->opt.memory_budget));
        CUDA_TRY(cudaMemsetAsync(c->status.p, 0, 16, c->stream));
    }
    int ns = 0;
    std::vector<int> sum_index(runs.size(), -1);
    for (size_t i = 0; i < runs.size(); ++i) {
        const PassRun &r = runs[i];
        const bool rev = grad && i >= sched.size();
        {
            ProfScope ps(c, rev ? 1 : 0, r.bytes);
            cudaError_t e;
            unsigned int *stw = c->status.as<unsigned int>();
            if (variant == 3)
                e = rev ? launch_rev3(r.type, r.args, c->num_sms, stw, c->stream)
                        : (r.epi ? launch_epi3(r.type, r.args, c->num_sms, stw, c->stream)
                                 : launch_fwd3(r.type, r.args, c->num_sms, stw, c->stream));
            else if (use_tma)
                e = rev ? launch_rev_pl(r.type, r.args, c->num_sms, stw, c->stream)
                        : (r.epi ? launch_epi_pl(r.type, r.args, c->num_sms, stw, c->stream)
                                 : (variant == 0 ? launch_fwd_pass(r.type, false, r.args, c->stream)
                                                 : launch_fwd_tma(r.type, false, r.args, c->num_sms, stw, c->stream)));
            else
                e = rev ? launch_rev_pass(r.type, r.args, c->stream)
                        : launch_fwd_pass(r.type, r.epi, r.args, c->stream);
            c->launches_total += 1;
            if (e) return fail(QAOA_ERR_CUDA, "pass launch failed: %s", cudaGetErrorString(e));
        }
        if (r.has_partials) {
            CUDA_TRY(launch_reduce_partials(partials, nb, NSLOT, sums + (size_t)ns * NSLOT, c->stream));
            c->launches_total += 1;
            sum_index[i] = ns++;
        }
    }
    unsigned int hstatus = 0;
    if (use_tma) CUDA_TRY(cudaMemcpyAsync(&hstatus, c->status.p, 4, cudaMemcpyDeviceToHost, c->stream));
    if (!grad) {
        if (use_tma) {
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            if (hstatus) return fail(QAOA_ERR_TIMEOUT, "a bounded wait of a layer-pass kernel expired");
        }
        return QAOA_OK;
    }
    std::vector<double> h((size_t)ns * NSLOT);
    std::vector<unsigned long long> keys(std::max(ktop, 1));
    if (ktop > 0) {
        int which = 0;
        int nl = 0;
        CUDA_TRY(launch_topk_merge(c->topk_a.as<unsigned long long>(), nb, ktop,
                                   c->topk_b.as<unsigned long long>(), &which, &nl, c->stream));
        c->launches_total += nl;
        const unsigned long long *src = which ? c->topk_b.as<unsigned long long>() : c->topk_a.as<unsigned long long>();
        CUDA_TRY(cudaMemcpyAsync(keys.data(), src, (size_t)ktop * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(h.data(), sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (hstatus) return fail(QAOA_ERR_TIMEOUT, "a bounded wait of a layer-pass kernel expired");
    const double cs = std::ldexp(1.0, -cost->fp.s);
    for (int l = 0; l < p; ++l) dg[l] = db[l] = 0.0;
    double S0 = 0, S1 = 0;
    for (size_t i = 0; i < runs.size(); ++i) {
        if (sum_index[i] < 0) continue;
        const double *v = &h[(size_t)sum_index[i] * NSLOT];
        const PassRun &r = runs[i];
        for (int s = 0; s < NSLOT; ++s) {
            const int prm = r.slot_param[s];
            if (prm == -2) {
                if (s == 0) S0 = v[s];
                else S1 = v[s];
            } else if (prm >= 0 && prm < p) {
                db[prm] += 2.0 * v[s] * r.slot_scale[s];
            } else if (prm >= p) {
                dg[prm - p] += 2.0 * cs * v[s] * r.slot_scale[s];
            }
        }
    }
    *E = cs * (S0 + (double)cost->fp.k_c * S1);
    if (ktop > 0) decode_keys(keys.data(), ktop, top_idx, top_prob);
    return QAOA_OK;
}

// Fill one small-n item (n <= 12).
void fill_small(SmallItem &it, const qaoa_cost_s *cost, int p, const double *gamma, const double *beta) {
    std::memset(&it, 0, sizeof(it));
    it.T = cost->T;
    it.n = cost->n;
    it.p = p;
    it.amp0 = (float)std::pow(2.0, -0.5 * cost->n);
    it.cscale = std::ldexp(1.0, -cost->fp.s);
    it.k_c = cost->fp.k_c;
    for (int l = 0; l < p; ++l) {
        it.phi[l] = phase_multiplier(gamma[l], cost->fp.s);
        it.off[l] = (uint64_t)cost->fp.k_c * it.phi[l];
        it.cb[l] = std::cos(beta[l]);
        it.sb[l] = std::sin(beta[l]);
    }
}

qaoa_status run_small(qaoa_ctx c, const std::vector<SmallItem> &items, bool fp64, bool grad, int max_n) {
    QAOA_TRY(c->items.ensure(items.size() * sizeof(SmallItem), &c->held, c->opt.memory_budget));
    CUDA_TRY(cudaMemcpyAsync(c->items.p, items.data(), items.size() * sizeof(SmallItem), cudaMemcpyHostToDevice,
                             c->stream));
    double bytes = 0;
    for (auto &it : items) bytes += std::ldexp(4.0, it.n);
    ProfScope ps(c, 3, bytes);
    CUDA_TRY(launch_small(c->items.as<SmallItem>(), (int)items.size(), max_n, fp64, grad, c->stream));
    c->launches_total += 1;
    return QAOA_OK;
}

qaoa_status check_angles(int p, const double *gamma, const double *beta) {
    if (p < 0) return fail(QAOA_ERR_INVALID_ARG, "p=%d < 0", p);
    if (p > 0 && (!gamma || !beta)) return fail(QAOA_ERR_INVALID_ARG, "gamma/beta is null");
    for (int l = 0; l < p; ++l)
        if (!std::isfinite(gamma[l]) || !std::isfinite(beta[l]))
            return fail(QAOA_ERR_INVALID_ARG, "non-finite angle at layer %d", l + 1);
    return QAOA_OK;
}

}  // namespace

// ============================================================================
// ABI
// ============================================================================
extern "C" {

const char *qaoa_last_error(void) { return qaoa::last_error(); }

qaoa_status qaoa_ctx_create(int device, void *cuda_stream, const qaoa_options *opt, qaoa_ctx *out) {
    if (!out) return fail(QAOA_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    int count = 0;
    CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(QAOA_ERR_INVALID_ARG, "device %d not present (%d devices)", device, count);
    QAOA_TRY(set_device(device));
    auto *c = new qaoa_ctx_s();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (opt) c->opt = *opt;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (c->opt.pass_variant < 0 || c->opt.pass_variant > 3) {
        delete c;
        return fail(QAOA_ERR_INVALID_ARG, "pass_variant must be 0, 1, 2 or 3");
    }
    if (c->opt.max_fused_qubits != 0 && (c->opt.max_fused_qubits < 3 || c->opt.max_fused_qubits > 10)) {
        delete c;
        return fail(QAOA_ERR_INVALID_ARG, "max_fused_qubits must be 0 or in [3, 10]");
    }
    *out = c;
    return QAOA_OK;
}

void qaoa_ctx_destroy(qaoa_ctx c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &r : c->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->ev_free) cudaEventDestroy(e);
    delete c;
}

qaoa_status qaoa_build_cost(qaoa_ctx c, const qaoa_qubo *q, qaoa_cost *out) {
    if (!c || !q || !out) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    QAOA_TRY(set_device(c->device));
    std::unique_ptr<qaoa_cost_s> h(new qaoa_cost_s());
    QAOA_TRY(canonicalize(q, &h->can));
    QAOA_TRY(make_fixed_point(h->can, &h->fp));
    const int n = q->n;
    h->n = n;
    h->device = c->device;
    const size_t N = (size_t)1 << n;
    {
        cudaError_t e = cudaMalloc(&h->T, N * sizeof(int32_t));
        if (e) {
            cudaGetLastError();
            h->T = nullptr;
            return fail(QAOA_ERR_OUT_OF_MEMORY, "objective table (%zu bytes): %s", N * 4, cudaGetErrorString(e));
        }
    }
    const int nblk = cost_build_blocks(n);
    const size_t coef_bytes = (size_t)(n + n * n) * 8;
    QAOA_TRY(c->misc.ensure(coef_bytes + (size_t)nblk * 16 + 64, &c->held, c->opt.memory_budget));
    std::vector<long long> coef(n + n * n);
    for (int i = 0; i < n; ++i) coef[i] = h->fp.ell_q[i];
    for (int k = 0; k < n * n; ++k) coef[n + k] = h->fp.b_q[k];
    char *m = c->misc.as<char>();
    CUDA_TRY(cudaMemcpyAsync(m, coef.data(), coef_bytes, cudaMemcpyHostToDevice, c->stream));
    CostBuildArgs a{};
    a.n = n;
    a.ell = reinterpret_cast<long long *>(m);
    a.b = reinterpret_cast<long long *>(m) + n;
    a.c_off = h->fp.c0_q - h->fp.k_c;
    a.T = h->T;
    a.blk_val = reinterpret_cast<long long *>(m + coef_bytes);
    a.blk_idx = reinterpret_cast<unsigned long long *>(m + coef_bytes + (size_t)nblk * 8);
    a.min_val = reinterpret_cast<long long *>(m + coef_bytes + (size_t)nblk * 16);
    a.min_idx = reinterpret_cast<unsigned long long *>(m + coef_bytes + (size_t)nblk * 16 + 8);
    int nb = 0;
    {
        ProfScope ps(c, 2, (double)N * 4.0);
        CUDA_TRY(launch_cost_build(a, &nb, c->stream));
        c->launches_total += 2;
    }
    long long mv = 0;
    unsigned long long mi = 0;
    CUDA_TRY(cudaMemcpyAsync(&mv, a.min_val, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(&mi, a.min_idx, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    h->minval = mv;
    h->argmin = mi;
    *out = h.release();
    return QAOA_OK;
}

void qaoa_cost_destroy(qaoa_cost cost) {
    if (!cost) return;
    cudaSetDevice(cost->device);
    delete cost;
}

qaoa_status qaoa_cost_info(qaoa_cost cost, int32_t *n, int32_t *shift_bits, int64_t *k_c, uint64_t *argmin_idx,
                           double *min_cost) {
    if (!cost) return fail(QAOA_ERR_INVALID_ARG, "cost is null");
    if (n) *n = cost->n;
    if (shift_bits) *shift_bits = cost->fp.s;
    if (k_c) *k_c = cost->fp.k_c;
    if (argmin_idx) *argmin_idx = cost->argmin;
    if (min_cost) *min_cost = std::ldexp((double)(cost->minval + cost->fp.k_c), -cost->fp.s);
    return QAOA_OK;
}

qaoa_status qaoa_cost_copy_to_host(qaoa_ctx c, qaoa_cost cost, int32_t *table) {
    if (!c || !cost || !table) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    QAOA_TRY(set_device(c->device));
    CUDA_TRY(cudaMemcpyAsync(table, cost->T, ((size_t)1 << cost->n) * 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return QAOA_OK;
}

qaoa_status qaoa_forward(qaoa_ctx c, qaoa_cost cost, int p, const double *gamma, const double *beta,
                         qaoa_state *inout) {
    if (!c || !cost || !inout) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    QAOA_TRY(check_angles(p, gamma, beta));
    QAOA_TRY(set_device(c->device));
    const int n = cost->n;
    const bool fp64 = c->opt.state_fp64 != 0;  // complex128 state (n <= 12 only)
    if (fp64 && n > SMALL_MAXN) return fail(QAOA_ERR_INVALID_ARG, "complex128 states are limited to n <= 12");
    if (n <= SMALL_MAXN && p > SMALL_MAXP) return fail(QAOA_ERR_INVALID_ARG, "p=%d > %d for n <= 12", p, SMALL_MAXP);
    qaoa_state st = *inout;
    std::unique_ptr<qaoa_state_s> fresh;
    if (st) {
        if (st->n != n || st->fp64 != fp64) return fail(QAOA_ERR_INVALID_ARG, "state does not match (n or precision)");
    } else {
        fresh.reset(new qaoa_state_s());
        fresh->n = n;
        fresh->fp64 = fp64;
        fresh->device = c->device;
        const size_t bytes = ((size_t)1 << n) * (fp64 ? 16 : 8);
        cudaError_t e = cudaMalloc(&fresh->amps, bytes);
        if (e) {
            cudaGetLastError();
            fresh->amps = nullptr;
            return fail(QAOA_ERR_OUT_OF_MEMORY, "state (%zu bytes): %s", bytes, cudaGetErrorString(e));
        }
        st = fresh.get();
    }
    if (n <= SMALL_MAXN) {
        std::vector<SmallItem> items(1);
        fill_small(items[0], cost, p, gamma, beta);
        QAOA_TRY(c->small_out.ensure(8 * (1 + 2 * (size_t)p) + 64, &c->held, c->opt.memory_budget));
        items[0].out = c->small_out.as<double>();
        items[0].psi_out = st->amps;
        QAOA_TRY(run_small(c, items, fp64, false, n));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    } else {
        QAOA_TRY(run_passes(c, cost, p, gamma, beta, (float2 *)st->amps, false, nullptr, nullptr, nullptr, 0,
                            nullptr, nullptr));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    if (fresh) *inout = fresh.release();
    return QAOA_OK;
}

void qaoa_state_destroy(qaoa_state s) {
    if (!s) return;
    cudaSetDevice(s->device);
    delete s;
}

qaoa_status qaoa_state_copy_to_host(qaoa_ctx c, qaoa_state s, float *amps) {
    if (!c || !s || !amps) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    QAOA_TRY(set_device(c->device));
    const size_t bytes = ((size_t)1 << s->n) * (s->fp64 ? 16 : 8);
    CUDA_TRY(cudaMemcpyAsync(amps, s->amps, bytes, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return QAOA_OK;
}

qaoa_status qaoa_state_device_ptr(qaoa_state s, void **amps, int64_t *count) {
    if (!s) return fail(QAOA_ERR_INVALID_ARG, "state is null");
    if (amps) *amps = s->amps;
    if (count) *count = (int64_t)1 << s->n;
    return QAOA_OK;
}

qaoa_status qaoa_expect(qaoa_ctx c, qaoa_cost cost, qaoa_state s, double *out) {
    if (!c || !cost || !s || !out) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    if (s->n != cost->n) return fail(QAOA_ERR_INVALID_ARG, "state and cost differ in n");
    if (s->fp64) return fail(QAOA_ERR_INVALID_ARG, "qaoa_expect takes complex64 states; complex128 states report E from qaoa_grad");
    QAOA_TRY(set_device(c->device));
    const int n = s->n;
    const int nb = (int)((((size_t)1 << n) + 8191) / 8192);
    QAOA_TRY(c->partials.ensure((size_t)nb * NSLOT * 8, &c->held, c->opt.memory_budget));
    QAOA_TRY(c->pass_sums.ensure(NSLOT * 8 * 2, &c->held, c->opt.memory_budget));
    CUDA_TRY(launch_expect((const float2 *)s->amps, cost->T, n, c->partials.as<double>(), c->stream));
    c->launches_total += 2;
    CUDA_TRY(launch_reduce_partials(c->partials.as<double>(), nb, NSLOT, c->pass_sums.as<double>(), c->stream));
    double h[NSLOT];
    CUDA_TRY(cudaMemcpyAsync(h, c->pass_sums.p, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    *out = std::ldexp(h[0] + (double)cost->fp.k_c * h[1], -cost->fp.s);
    return QAOA_OK;
}

qaoa_status qaoa_topk(qaoa_ctx c, qaoa_cost cost, qaoa_state s, int k, uint64_t *idx, float *prob,
                      double *cost_out, uint64_t *argmin_idx, double *min_cost, float *prob_argmin) {
    if (!c || !cost || !s || !idx) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    if (k < 1 || k > 64) return fail(QAOA_ERR_INVALID_ARG, "k=%d not in [1, 64]", k);
    if (s->n != cost->n) return fail(QAOA_ERR_INVALID_ARG, "state and cost differ in n");
    if (s->fp64) return fail(QAOA_ERR_INVALID_ARG, "qaoa_topk takes complex64 states");
    const int n = s->n;
    if (((int64_t)1 << n) < k) return fail(QAOA_ERR_INVALID_ARG, "k=%d exceeds 2^n", k);
    QAOA_TRY(set_device(c->device));
    const int nb = (int)((((size_t)1 << n) + 8191) / 8192);
    QAOA_TRY(c->topk_a.ensure((size_t)nb * k * 8 + 64, &c->held, c->opt.memory_budget));
    QAOA_TRY(c->topk_b.ensure((size_t)((nb + 255) / 256 + 1) * k * 8 + 64, &c->held, c->opt.memory_budget));
    CUDA_TRY(launch_topk_chunks((const float2 *)s->amps, n, k, c->topk_a.as<unsigned long long>(), c->stream));
    int which = 0;
    int nl = 0;
    CUDA_TRY(launch_topk_merge(c->topk_a.as<unsigned long long>(), nb, k, c->topk_b.as<unsigned long long>(), &which,
                               &nl, c->stream));
    c->launches_total += 1 + nl;
    std::vector<unsigned long long> keys(k);
    const void *src = which ? c->topk_b.p : c->topk_a.p;
    CUDA_TRY(cudaMemcpyAsync(keys.data(), src, (size_t)k * 8, cudaMemcpyDeviceToHost, c->stream));
    std::vector<int32_t> tv(k);
    float2 amp_min = make_float2(0, 0);
    CUDA_TRY(cudaMemcpyAsync(&amp_min, (const float2 *)s->amps + cost->argmin, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    decode_keys(keys.data(), k, idx, prob);
    if (cost_out) {
        for (int i = 0; i < k; ++i)
            CUDA_TRY(cudaMemcpyAsync(&tv[i], cost->T + idx[i], 4, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < k; ++i) cost_out[i] = std::ldexp((double)tv[i] + (double)cost->fp.k_c, -cost->fp.s);
    }
    if (argmin_idx) *argmin_idx = cost->argmin;
    if (min_cost) *min_cost = std::ldexp((double)(cost->minval + cost->fp.k_c), -cost->fp.s);
    if (prob_argmin) *prob_argmin = amp_min.x * amp_min.x + amp_min.y * amp_min.y;
    return QAOA_OK;
}

qaoa_status qaoa_grad(qaoa_ctx c, qaoa_cost cost, int p, const double *gamma, const double *beta, double *out_expect,
                      double *dgamma, double *dbeta, int k_top, uint64_t *top_idx, float *top_prob) {
    if (!c || !cost || !out_expect || (p > 0 && (!dgamma || !dbeta)))
        return fail(QAOA_ERR_INVALID_ARG, "null argument");
    QAOA_TRY(check_angles(p, gamma, beta));
    if (p < 1) return fail(QAOA_ERR_INVALID_ARG, "qaoa_grad needs p >= 1");
    if (k_top < 0 || k_top > 16) return fail(QAOA_ERR_INVALID_ARG, "k_top=%d not in [0, 16]", k_top);
    if (k_top > 0 && (!top_idx || !top_prob)) return fail(QAOA_ERR_INVALID_ARG, "top-K outputs are null");
    const int n = cost->n;
    if (((int64_t)1 << n) < k_top) return fail(QAOA_ERR_INVALID_ARG, "k_top exceeds 2^n");
    QAOA_TRY(set_device(c->device));
    const bool fp64 = c->opt.state_fp64 != 0;
    if (n <= SMALL_MAXN) {
        if (p > SMALL_MAXP) return fail(QAOA_ERR_INVALID_ARG, "p=%d > %d for n <= 12", p, SMALL_MAXP);
        std::vector<SmallItem> items(1);
        fill_small(items[0], cost, p, gamma, beta);
        QAOA_TRY(c->small_out.ensure(8 * (1 + 2 * (size_t)p) + 16 * 8 + 64, &c->held, c->opt.memory_budget));
        items[0].grad = 1;
        items[0].out = c->small_out.as<double>();
        items[0].ktop = k_top;
        items[0].topk = reinterpret_cast<unsigned long long *>(c->small_out.as<double>() + 1 + 2 * p);
        QAOA_TRY(run_small(c, items, fp64, true, n));
        std::vector<double> h(1 + 2 * p + 16);
        CUDA_TRY(cudaMemcpyAsync(h.data(), c->small_out.p, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        *out_expect = h[0];
        for (int l = 0; l < p; ++l) {
            dgamma[l] = h[1 + l];
            dbeta[l] = h[1 + p + l];
        }
        if (k_top > 0) decode_keys(reinterpret_cast<const unsigned long long *>(&h[1 + 2 * p]), k_top, top_idx, top_prob);
        return QAOA_OK;
    }
    if (fp64) return fail(QAOA_ERR_INVALID_ARG, "complex128 states are limited to n <= 12");
    QAOA_TRY(ensure_scratch(c, n, 1, k_top, true));
    return run_passes(c, cost, p, gamma, beta, c->work_psi.as<float2>(), true, out_expect, dgamma, dbeta, k_top,
                      top_idx, top_prob);
}

qaoa_status qaoa_grad_batch(qaoa_ctx c, int nq, const qaoa_cost *costs, const int32_t *item_cost, int B, int p,
                            const double *gamma, const double *beta, double *expect, double *dgamma, double *dbeta) {
    if (!c || !costs || nq < 1 || B < 1 || !gamma || !beta || !expect)
        return fail(QAOA_ERR_INVALID_ARG, "bad batch arguments");
    if ((dgamma == nullptr) != (dbeta == nullptr)) return fail(QAOA_ERR_INVALID_ARG, "dgamma and dbeta must both be set or both be null");
    if (p < 1 || p > SMALL_MAXP) return fail(QAOA_ERR_INVALID_ARG, "p=%d not in [1, %d]", p, SMALL_MAXP);
    for (int b = 0; b < B; ++b) {
        const int ci = item_cost ? item_cost[b] : 0;
        if (ci < 0 || ci >= nq || !costs[ci]) return fail(QAOA_ERR_INVALID_ARG, "item %d: bad cost index %d", b, ci);
    }
    QAOA_TRY(check_angles(p * B, gamma, beta));
    QAOA_TRY(set_device(c->device));
    const bool grad = dgamma != nullptr;
    // small items: one resident-kernel launch
    std::vector<SmallItem> small;
    std::vector<int> small_ids;
    int max_small_n = 1;
    for (int b = 0; b < B; ++b) {
        const qaoa_cost_s *cs = costs[item_cost ? item_cost[b] : 0];
        if (cs->n > SMALL_MAXN) continue;
        SmallItem it;
        fill_small(it, cs, p, gamma + (size_t)b * p, beta + (size_t)b * p);
        it.grad = grad ? 1 : 0;
        small.push_back(it);
        small_ids.push_back(b);
        max_small_n = std::max(max_small_n, cs->n);
    }
    if (!small.empty()) {
        const size_t per = 1 + 2 * (size_t)p;
        QAOA_TRY(c->small_out.ensure(small.size() * per * 8 + 64, &c->held, c->opt.memory_budget));
        for (size_t i = 0; i < small.size(); ++i) small[i].out = c->small_out.as<double>() + i * per;
        QAOA_TRY(run_small(c, small, false, grad, max_small_n));
        std::vector<double> h(small.size() * per);
        CUDA_TRY(cudaMemcpyAsync(h.data(), c->small_out.p, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < small.size(); ++i) {
            const int b = small_ids[i];
            expect[b] = h[i * per];
            if (grad)
                for (int l = 0; l < p; ++l) {
                    dgamma[(size_t)b * p + l] = h[i * per + 1 + l];
                    dbeta[(size_t)b * p + l] = h[i * per + 1 + p + l];
                }
        }
    }
    // large items: the pass schedule, one item at a time on the context stream
    for (int b = 0; b < B; ++b) {
        const qaoa_cost_s *cs = costs[item_cost ? item_cost[b] : 0];
        if (cs->n <= SMALL_MAXN) continue;
        if (grad) {
            QAOA_TRY(qaoa_grad(c, const_cast<qaoa_cost>(cs), p, gamma + (size_t)b * p, beta + (size_t)b * p, &expect[b],
                               dgamma + (size_t)b * p, dbeta + (size_t)b * p, 0, nullptr, nullptr));
        } else {
            QAOA_TRY(ensure_scratch(c, cs->n, 1, 0, false));
            QAOA_TRY(run_passes(c, cs, p, gamma + (size_t)b * p, beta + (size_t)b * p, c->work_psi.as<float2>(), false,
                                nullptr, nullptr, nullptr, 0, nullptr, nullptr));
            qaoa_state_s tmp;
            tmp.n = cs->n;
            tmp.amps = c->work_psi.p;
            tmp.device = c->device;
            qaoa_status st = qaoa_expect(c, const_cast<qaoa_cost>(cs), &tmp, &expect[b]);
            tmp.amps = nullptr;
            QAOA_TRY(st);
        }
    }
    return QAOA_OK;
}

qaoa_status qaoa_partition(int n, int M, const int32_t *caps, const int32_t *manual, int32_t *qpu_of) {
    return partition(n, M, caps, manual, qpu_of);
}

qaoa_status qaoa_classify(qaoa_cost cost, const int32_t *qpu_of, int p, int64_t *n_local, int64_t *n_cross,
                          int64_t *remote_cx_est, int64_t *n_cross_all_pairs) {
    if (!cost || !qpu_of || !n_local || !n_cross || !remote_cx_est || p < 0)
        return fail(QAOA_ERR_INVALID_ARG, "null argument or p < 0");
    classify(cost->can, qpu_of, n_local, n_cross, n_cross_all_pairs);
    *remote_cx_est = 2 * (*n_cross) * (int64_t)p;  // two remote CNOTs per cross term per layer
    return QAOA_OK;
}

qaoa_status qaoa_check_factorisation(qaoa_ctx c, qaoa_cost cost, const int32_t *qpu_of, double gamma_probe,
                                     int64_t *mismatches, double *max_phase_err) {
    if (!c || !cost || !qpu_of || !mismatches) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    const int n = cost->n;
    int M = 0;
    for (int i = 0; i < n; ++i) {
        if (qpu_of[i] < 0) return fail(QAOA_ERR_ALLOCATION, "variable %d has no QPU", i);
        M = std::max(M, qpu_of[i] + 1);
    }
    if (M > 16) return fail(QAOA_ERR_INVALID_ARG, "at most 16 QPUs are supported by the check");
    std::vector<std::vector<int>> vars(M);
    std::vector<int> pos(n);
    for (int i = 0; i < n; ++i) {
        pos[i] = (int)vars[qpu_of[i]].size();
        vars[qpu_of[i]].push_back(i);
    }
    for (int m = 0; m < M; ++m) {
        if (vars[m].empty()) return fail(QAOA_ERR_ALLOCATION, "QPU %d is not used", m);
        if (vars[m].size() > 16) return fail(QAOA_ERR_INVALID_ARG, "QPU %d holds %zu > 16 variables", m, vars[m].size());
    }
    const FixedPoint &fp = cost->fp;
    // local tables L_m[u] = sum_{a in m} l z_a + sum_{a<b in m} b z_a z_b (fixed point)
    std::vector<long long> L, Loff(M), V, Voff(256, 0);
    for (int m = 0; m < M; ++m) {
        Loff[m] = (long long)L.size();
        const int cm = (int)vars[m].size();
        for (uint32_t u = 0; u < (1u << cm); ++u) {
            long long v = 0;
            for (int a = 0; a < cm; ++a) {
                if (!((u >> a) & 1u)) continue;
                const int i = vars[m][a];
                v += fp.ell_q[i];
                for (int b2 = a + 1; b2 < cm; ++b2)
                    if ((u >> b2) & 1u) {
                        const int j = vars[m][b2];
                        v += fp.b_q[(size_t)std::min(i, j) * n + std::max(i, j)];
                    }
            }
            L.push_back(v);
        }
    }
    // pair tables V_{m,m'}[u'][a] = sum_{b in m'} b_{ia, jb} z_b
    for (int m = 0; m < M; ++m)
        for (int m2 = m + 1; m2 < M; ++m2) {
            Voff[m * 16 + m2] = (long long)V.size();
            const int c1 = (int)vars[m].size(), c2 = (int)vars[m2].size();
            for (uint32_t u2 = 0; u2 < (1u << c2); ++u2)
                for (int a = 0; a < c1; ++a) {
                    long long v = 0;
                    const int i = vars[m][a];
                    for (int b2 = 0; b2 < c2; ++b2)
                        if ((u2 >> b2) & 1u) {
                            const int j = vars[m2][b2];
                            v += fp.b_q[(size_t)std::min(i, j) * n + std::max(i, j)];
                        }
                    V.push_back(v);
                }
        }
    if (V.empty()) V.push_back(0);
    std::vector<int> qs(M + 1, 0);
    for (int m = 0; m < M; ++m) qs[m + 1] = qs[m] + (int)vars[m].size();
    QAOA_TRY(set_device(c->device));
    const size_t bytes = n * 4 * 2 + (M + 1) * 4 + L.size() * 8 + Loff.size() * 8 + V.size() * 8 + Voff.size() * 8 + 64 * 8;
    QAOA_TRY(c->misc.ensure(bytes + 1024, &c->held, c->opt.memory_budget));
    char *d = c->misc.as<char>();
    size_t o = 0;
    auto put = [&](const void *src, size_t nb) -> char * {
        char *dst = d + o;
        cudaMemcpyAsync(dst, src, nb, cudaMemcpyHostToDevice, c->stream);
        o += (nb + 15) & ~size_t(15);
        return dst;
    };
    std::vector<int> q32(qpu_of, qpu_of + n);
    FactArgs a{};
    a.T = cost->T;
    a.n = n;
    a.M = M;
    a.qpu_of = (const int *)put(q32.data(), n * 4);
    a.pos_in_q = (const int *)put(pos.data(), n * 4);
    a.q_start = (const int *)put(qs.data(), (M + 1) * 4);
    a.Ltab = (const long long *)put(L.data(), L.size() * 8);
    a.L_off = (const long long *)put(Loff.data(), Loff.size() * 8);
    a.V = (const long long *)put(V.data(), V.size() * 8);
    a.V_off = (const long long *)put(Voff.data(), Voff.size() * 8);
    unsigned long long zero[2] = {0, 0};
    char *res = put(zero, 16);
    a.mismatches = (unsigned long long *)res;
    a.max_err_bits = (unsigned int *)(res + 8);
    a.c_off = fp.c0_q - fp.k_c;
    a.k_c = fp.k_c;
    a.phi = phase_multiplier(gamma_probe, fp.s);
    // contiguous: QPU indices start at 0 and never decrease, stepping by 0 or 1
    a.contiguous = qpu_of[0] == 0 ? 1 : 0;
    for (int i = 1; i < n; ++i)
        if (qpu_of[i] != qpu_of[i - 1] && qpu_of[i] != qpu_of[i - 1] + 1) a.contiguous = 0;
    a.c0 = (int)vars[0].size();
    if (a.c0 > 12 || n - a.c0 > 31) a.contiguous = 0;
    CUDA_TRY(cudaGetLastError());
    {
        ProfScope ps(c, 4, std::ldexp(4.0, n));
        CUDA_TRY(launch_fact_check(a, c->stream));
        c->launches_total += 1;
    }
    unsigned long long hres[2];
    CUDA_TRY(cudaMemcpyAsync(hres, res, 16, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    *mismatches = (int64_t)hres[0];
    if (max_phase_err) {
        uint32_t bits = (uint32_t)hres[1];
        float f;
        std::memcpy(&f, &bits, 4);
        *max_phase_err = f;
    }
    return QAOA_OK;
}

qaoa_status qaoa_profile_read(qaoa_ctx c, int kind, int64_t *launches, double *ms, double *bytes, int reset) {
    if (!c || kind < 0 || kind > 5) return fail(QAOA_ERR_INVALID_ARG, "bad context or kind");
    QAOA_TRY(set_device(c->device));
    if (kind == 5) {
        if (launches) *launches = c->launches_total;
        if (ms) *ms = 0.0;
        if (bytes) *bytes = 0.0;
        if (reset) c->launches_total = 0;
        return QAOA_OK;
    }
    drain_profile(c);
    if (launches) *launches = c->prof_launches[kind];
    if (ms) *ms = c->prof_ms[kind];
    if (bytes) *bytes = c->prof_bytes[kind];
    if (reset) {
        c->prof_launches[kind] = 0;
        c->prof_ms[kind] = 0;
        c->prof_bytes[kind] = 0;
    }
    return QAOA_OK;
}

}  // extern "C"
