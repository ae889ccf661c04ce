// C ABI of the QAOA statevector library (include/qaoa.h): handles, execution
// of the layer-pass plan for one item or a batch, gradient assembly, the
// Adam loop captured in a CUDA graph, and the DQAOA entry points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels_misc.h"
#include "qaoa_internal.h"
#include "schedule.cuh"

using namespace qaoa;

#include "api_state.h"

using namespace qaoa::api;

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
    int kind, kind2;
    double bytes;
    bool on;
    cudaEvent_t a = nullptr;
    ProfScope(qaoa_ctx c_, int kind_, double bytes_, bool allow = true, int kind2_ = -1)
        : c(c_), kind(kind_), kind2(kind2_), bytes(bytes_), on(c_->opt.profile != 0 && allow) {
        if (on) {
            a = get_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~ProfScope() {
        if (on) {
            cudaEvent_t b = get_event(c);
            cudaEventRecord(b, c->stream);
            c->pending.push_back({kind, kind2, a, b, bytes});
        }
    }
};

void drain_profile(qaoa_ctx c) {
    if (c->pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto &r : c->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        for (int k : {r.kind, r.kind2}) {
            if (k < 0) continue;
            c->prof_launches[k] += 1;
            c->prof_ms[k] += ms;
            c->prof_bytes[k] += r.bytes;
        }
        c->ev_free.push_back(r.a);
        c->ev_free.push_back(r.b);
    }
    c->pending.clear();
}

qaoa_status set_device(int dev) {
    CUDA_TRY(cudaSetDevice(dev));
    return QAOA_OK;
}

qaoa_status check_angles(int p, const double *gamma, const double *beta) {
    if (p < 0) return fail(QAOA_ERR_INVALID_ARG, "p=%d < 0", p);
    if (p > 0 && (!gamma || !beta)) return fail(QAOA_ERR_INVALID_ARG, "gamma/beta is null");
    for (int l = 0; l < p; ++l)
        if (!std::isfinite(gamma[l]) || !std::isfinite(beta[l]))
            return fail(QAOA_ERR_INVALID_ARG, "non-finite angle at parameter %d", l);
    return QAOA_OK;
}

// Fusion width (qubits per mixer pass) for states of n qubits: the explicit
// option, else the autotuner's pick for n (options.autotune), else 10.
int maxq_for(qaoa_ctx c, int n) {
    if (c->opt.max_fused_qubits) return c->opt.max_fused_qubits;
    if (c->opt.autotune) {
        auto it = c->tuned_k.find(n);
        if (it != c->tuned_k.end()) return it->second;
    }
    return 10;
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

// ---- plan execution ---------------------------------------------------------------

struct PlanRun {
    int n, p, nitems, ntables;
    bool grad;
    int ktop;
    std::vector<PassPlan> plan;
    int rows;
    float2 *psi_ext = nullptr;  // forward-only: evolve in this caller buffer instead of b.psi
    bool stored = false;        // adjoint with stored forward states (all or some; else uncompute)
    int nslots = 0;             // stored states per item
    int kept = 0;               // mixer-only passes whose input is stored
};

// Build the pass plan of r (r.n, r.p, r.grad, r.nitems set): the adjoint
// keeps the forward states it needs when options.adjoint_mode asks for it, or
// (auto) when they fit in free device memory (and the memory budget) with a
// margin; when only some fit (auto), it keeps the inputs of as many of the
// last mixer-only passes as fit and uncomputes psi on the interleaved buffer
// for the rest; with none, the whole reverse sweep uncomputes.
qaoa_status make_run_plan(qaoa_ctx c, PlanRun &r, const PlanBufs &b, int keep_cap = -1) {
    const int maxq = maxq_for(c, r.n);
    r.stored = false;
    r.nslots = 0;
    r.kept = 0;
    bool tuned_unc = false;
    if (c->opt.autotune && c->opt.adjoint_mode == QAOA_ADJ_AUTO) {
        auto it = c->tuned_uncompute.find(r.n);
        tuned_unc = it != c->tuned_uncompute.end() && it->second;
    }
    if (r.grad && c->opt.adjoint_mode != QAOA_ADJ_UNCOMPUTE && !tuned_unc) {
        int ns = 0, nm = 0;
        std::vector<PassPlan> sp = make_plan(r.n, r.p, true, maxq, -1, &ns, &nm);
        const double N8 = std::ldexp(8.0 * r.nitems, r.n);
        // bytes that can hold lambda and the stored states: free memory less a margin,
        // plus what the context already holds for them (psi and the interleaved
        // buffer of the uncompute sweep are needed either way)
        size_t freeb = 0, total = 0;
        cudaMemGetInfo(&freeb, &total);
        const double margin = 4.0 * (1ull << 30);
        const double held = (double)(b.states.cap + b.lam.cap);
        double avail = (double)freeb - margin + held;
        if (c->opt.memory_budget > 0)
            avail = std::min(avail, (double)c->opt.memory_budget - (double)c->held + held);
        const bool all = c->opt.adjoint_mode == QAOA_ADJ_STORE || (ns + 1) * N8 <= avail;
        if (ns > 0 && all && (keep_cap < 0 || keep_cap >= nm)) {
            r.plan = std::move(sp);
            r.stored = true;
            r.nslots = ns;
            r.kept = nm;
        } else if (ns > 0) {
            int keep = all ? nm : (int)std::floor(avail / N8) - 1;  // one state for lambda
            if (keep_cap >= 0) keep = std::min(keep, keep_cap);
            if (keep >= 1) {
                r.plan = make_plan(r.n, r.p, true, maxq, keep, &ns);
                r.stored = true;
                r.nslots = ns;
                r.kept = keep;
            }
        }
    }
    if (!r.stored) r.plan = make_plan(r.n, r.p, r.grad, maxq);
    if (r.plan.empty()) return fail(QAOA_ERR_INVALID_ARG, "no pass layout for n=%d", r.n);
    if (c->opt.reverse_blocks == 2) use_half_block_counts(r.plan);
    r.rows = plan_rows(r.plan);
    return QAOA_OK;
}

qaoa_status ensure_plan_bufs(qaoa_ctx c, PlanBufs &b, const PlanRun &r);

// Plan and allocate.  When the allocation runs out of memory, the adjoint
// scratch of the context's other working sets is released and the plan made
// again (once); then, with the automatic adjoint choice, a plan that keeps
// stored states is retried with one kept state fewer, down to the uncompute
// sweep.
qaoa_status plan_and_allocate(qaoa_ctx c, PlanRun &r, PlanBufs &b) {
    int cap = -1;
    bool released = false;
    for (;;) {
        QAOA_TRY(make_run_plan(c, r, b, cap));
        const qaoa_status st = ensure_plan_bufs(c, b, r);
        if (st == QAOA_OK) return QAOA_OK;
        if (st != QAOA_ERR_OUT_OF_MEMORY) return st;
        if (!released) {
            released = true;
            if (release_adjoint_scratch(c, &b)) continue;
        }
        if (!r.stored || c->opt.adjoint_mode != QAOA_ADJ_AUTO) return st;
        cap = r.kept - 1;
        b.states.release(&c->held);
        b.lam.release(&c->held);
    }
}

// Allocate the working set of a plan for `nitems` items of size n.
qaoa_status ensure_plan_bufs(qaoa_ctx c, PlanBufs &b, const PlanRun &r) {
    const size_t N = (size_t)1 << r.n;
    const int nb = 1 << (r.n - BLOCK_BITS);
    const size_t B = (size_t)r.nitems;
    const int64_t bud = c->opt.memory_budget;
    int64_t *h = &c->held;
    if (!r.psi_ext) QAOA_TRY(b.psi.ensure(B * N * sizeof(float2), h, bud));
    if (r.grad) QAOA_TRY(b.pl.ensure(B * N * sizeof(float4), h, bud));
    if (r.grad && r.stored) {
        QAOA_TRY(b.states.ensure((size_t)r.nslots * B * N * sizeof(float2), h, bud));
        QAOA_TRY(b.lam.ensure(B * N * sizeof(float2), h, bud));
    } else if (r.grad) {
        b.states.release(h);
        b.lam.release(h);
    }
    // the half-block reverse passes write one partial-sum row per 2^12 amplitudes
    const int nunit = 2 * nb;
    QAOA_TRY(b.partials.ensure(B * nunit * NSLOT * sizeof(double), h, bud));
    QAOA_TRY(b.partials2.ensure(std::max<size_t>((size_t)B * reduce_chunk_count(nunit) * NSLOT * sizeof(double), 64), h, bud));
    QAOA_TRY(b.sums.ensure((size_t)std::max(r.rows, 1) * B * NSLOT * sizeof(double), h, bud));
    QAOA_TRY(b.scal.ensure(r.plan.size() * B * sizeof(PassScal), h, bud));
    QAOA_TRY(b.slot_scale.ensure(r.plan.size() * B * NSLOT * sizeof(double), h, bud));
    QAOA_TRY(b.plan.ensure(r.plan.size() * sizeof(PassPlan), h, bud));
    QAOA_TRY(b.gamma.ensure(B * std::max(r.p, 1) * sizeof(double), h, bud));
    QAOA_TRY(b.beta.ensure(B * std::max(r.p, 1) * sizeof(double), h, bud));
    QAOA_TRY(b.item_s.ensure(B * sizeof(int), h, bud));
    QAOA_TRY(b.item_kc.ensure(B * sizeof(long long), h, bud));
    QAOA_TRY(b.out_E.ensure(B * sizeof(double), h, bud));
    QAOA_TRY(b.out_dg.ensure(B * std::max(r.p, 1) * sizeof(double), h, bud));
    QAOA_TRY(b.out_db.ensure(B * std::max(r.p, 1) * sizeof(double), h, bud));
    const int kk = std::max(r.ktop, 1);
    const size_t nlists = (size_t)std::max(nb, c->num_sms * (PASS_THREADS / 32));  // final pass: one per warp
    QAOA_TRY(b.topk_a.ensure(nlists * kk * 8 + 64, h, bud));
    QAOA_TRY(b.topk_b.ensure((size_t)((nlists + 255) / 256 + 1) * kk * 8 + 64, h, bud));
    QAOA_TRY(c->status.ensure(16, h, bud));
    return QAOA_OK;
}

// Enqueue every pass of the plan (and the partial-sum reductions) on the
// context stream.  Device-side scalars (b.scal) must be ready.
qaoa_status enqueue_plan(qaoa_ctx c, PlanBufs &b, const PlanRun &r, const int32_t *tables, const int *item_table,
                         bool profile) {
    const int n = r.n;
    const int nb = 1 << (n - BLOCK_BITS);
    PassScal *scal = b.scal.as<PassScal>();
    unsigned int *stw = c->status.as<unsigned int>();
    for (size_t i = 0; i < r.plan.size(); ++i) {
        const PassPlan &pl = r.plan[i];
        PassArgs a{};
        float2 *W = r.psi_ext ? r.psi_ext : b.psi.as<float2>();
        const size_t stride = (size_t)r.nitems << n;  // elements of one stored state (all items)
        auto slot_ptr = [&](int sl) -> float2 * {
            return sl >= 0 ? b.states.as<float2>() + (size_t)sl * stride : W;
        };
        a.psi = W;
        a.pl = b.pl.as<float4>();
        if (r.stored) {
            a.split = (pl.kind == 1 || pl.kind == 2) && pl.split_out;  // write lambda alone
            a.lam = b.lam.as<float2>();
            if (pl.kind == 0) {
                a.psi = slot_ptr(pl.in_slot);
                a.psi_out = slot_ptr(pl.out_slot);
            } else if (pl.kind == 1) {
                a.psi = slot_ptr(pl.in_slot);
            } else if (pl.kind == 3) {
                a.psi_src = slot_ptr(pl.psi_slot);
                a.pl_out = pl.pl_out;
            }
        }
        a.C = tables;
        a.item_table = item_table;
        a.scal = scal + i * r.nitems;
        a.partials = b.partials.as<double>();
        a.topk_keys = b.topk_a.as<unsigned long long>();
        a.n = n;
        a.loA = pl.loA;
        a.loB = pl.loB;
        a.mask = pl.mask;
        a.nitems = r.nitems;
        a.ntables = r.ntables;
        a.init = pl.init;
        a.has_pre = pl.la >= 0;
        a.has_cost = pl.lc >= 0;
        a.has_post = pl.lb >= 0;
        a.store = pl.kind >= 2 ? !pl.init : 1;
        a.precise_phase = 0;
        a.ktop = pl.kind == 1 ? r.ktop : 0;
        a.amp0 = (float)std::pow(2.0, -0.5 * n);
        const double bytes = pass_bytes_per_amp(pl) * std::ldexp((double)r.nitems, n);
        const bool fwd_tma = pl.kind == 0 && a.has_pre && a.has_cost && a.has_post && !a.init;
        // final and cost-layer reverse passes on half blocks (two CTAs per SM); by
        // default for the low group, where they are faster (n = 30: 9.4 against
        // 9.8 ms per reverse pass; n = 32, eight-qubit groups: 919 against 931 ms
        // per evaluation), not for the high groups (n = 30: 13.4 against 10.4 ms)
        const bool half = (pl.kind == 1 || pl.kind == 2) &&
                          ((c->opt.reverse_blocks == 0 && pl.type == 0) || c->opt.reverse_blocks == 2);
        // kernel-level profile kinds, one per kernel (see qaoa_profile_read)
        const int kernel_kind = pl.kind == 0   ? (fwd_tma ? 9 : 8)
                                : pl.kind == 1 ? (half ? 13 : 10)
                                : pl.kind == 2 ? (half ? 14 : 11)
                                               : 12;
        {
            ProfScope ps(c, pl.kind >= 2 ? 1 : 0, bytes, profile, kernel_kind);
            // a named range per pass for timeline tools (no cost when no tool is attached)
            static const char *const pass_names[4] = {"qaoa forward pass", "qaoa final pass",
                                                      "qaoa reverse pass (psi, lambda)", "qaoa reverse pass (lambda)"};
            nvtxRangePushA(pass_names[pl.kind & 3]);
            cudaError_t e = pl.kind == 0   ? (fwd_tma
                                                  ? launch_fwd_cost_tma(pl.type, a, 2 * c->num_sms, stw, c->stream)
                                                  : launch_fwd_pass(pl.type, a, c->stream))
                            : pl.kind == 1 ? (half ? launch_final_pass_half(pl.type, a, 2 * c->num_sms, stw, c->stream)
                                                   : launch_final_pass(pl.type, a, c->num_sms, stw, c->stream))
                            : pl.kind == 2 ? (half ? launch_rev_pass_half(pl.type, a, 2 * c->num_sms, stw, c->stream)
                                                   : launch_rev_pass(pl.type, a, c->num_sms, stw, c->stream))
                                           : launch_rev_mid(pl.type, a, c->num_sms, stw, c->stream);
            nvtxRangePop();
            if (e) return fail(QAOA_ERR_CUDA, "layer-pass launch failed: %s", cudaGetErrorString(e));
            c->launches_total += 1;
        }
        if (pl.sum_index >= 0) {
            int nl = 0;
            CUDA_TRY(launch_reduce_partials_chunked(a.partials, r.nitems, half ? 2 * nb : nb, b.partials2.as<double>(),
                                                    b.sums.as<double>() + (size_t)pl.sum_index * r.nitems * NSLOT,
                                                    &nl, c->stream));
            c->launches_total += nl;
        }
    }
    return QAOA_OK;
}

DevPlan dev_plan(PlanBufs &b, const PlanRun &r) {
    DevPlan d{};
    d.plan = b.plan.as<PassPlan>();
    d.npasses = (int)r.plan.size();
    d.p = r.p;
    d.nitems = r.nitems;
    d.gamma = b.gamma.as<double>();
    d.beta = b.beta.as<double>();
    d.item_s = b.item_s.as<int>();
    d.item_kc = b.item_kc.as<long long>();
    d.scal = b.scal.as<PassScal>();
    d.slot_scale = b.slot_scale.as<double>();
    return d;
}

// Fill the small-item block for one parameter set (n <= 12).
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

qaoa_status run_small(qaoa_ctx c, DevBuf &items_buf, const std::vector<SmallItem> &items, bool fp64, bool grad,
                      int max_n) {
    QAOA_TRY(items_buf.ensure(items.size() * sizeof(SmallItem), &c->held, c->opt.memory_budget));
    CUDA_TRY(cudaMemcpyAsync(items_buf.p, items.data(), items.size() * sizeof(SmallItem), cudaMemcpyHostToDevice,
                             c->stream));
    double bytes = 0;
    for (auto &it : items) bytes += std::ldexp(4.0, it.n);
    ProfScope ps(c, 3, bytes);
    CUDA_TRY(launch_small(items_buf.as<SmallItem>(), (int)items.size(), max_n, fp64, grad, c->stream));
    c->launches_total += 1;
    return QAOA_OK;
}

qaoa_status status_check(qaoa_ctx c) {
    unsigned int hs = 0;
    CUDA_TRY(cudaMemcpyAsync(&hs, c->status.p, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (hs) return fail(QAOA_ERR_TIMEOUT, "a bounded wait of a layer-pass kernel expired");
    return QAOA_OK;
}

// Single-item evaluation on the pass path (n >= 13): forward only (psi ends in
// b.psi) or forward + adjoint (E, gradient, optional top-K).
qaoa_status run_single(qaoa_ctx c, const qaoa_cost_s *cost, int p, const double *gamma, const double *beta,
                       bool grad, float2 *psi_out, double *E, double *dg, double *db, int ktop, uint64_t *top_idx,
                       float *top_prob) {
    PlanRun r;
    r.n = cost->n;
    r.p = p;
    r.nitems = 1;
    r.ntables = 1;
    r.grad = grad;
    r.ktop = grad ? ktop : 0;
    r.psi_ext = grad ? nullptr : psi_out;
    PlanBufs &b = c->single;
    QAOA_TRY(plan_and_allocate(c, r, b));
    // scalars on the host (one item)
    std::vector<PassScal> sc(r.plan.size());
    std::vector<double> ss(r.plan.size() * NSLOT);
    for (size_t i = 0; i < r.plan.size(); ++i)
        pass_scalars(r.plan[i], gamma, beta, cost->fp.s, cost->fp.k_c, &sc[i], &ss[i * NSLOT]);
    const int s_h = cost->fp.s;
    const long long kc_h = cost->fp.k_c;
    CUDA_TRY(cudaMemcpyAsync(b.scal.p, sc.data(), sc.size() * sizeof(PassScal), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(b.slot_scale.p, ss.data(), ss.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(b.plan.p, r.plan.data(), r.plan.size() * sizeof(PassPlan), cudaMemcpyHostToDevice,
                             c->stream));
    CUDA_TRY(cudaMemcpyAsync(b.item_s.p, &s_h, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(b.item_kc.p, &kc_h, sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->status.p, 0, 16, c->stream));
    QAOA_TRY(enqueue_plan(c, b, r, cost->T, nullptr, true));
    if (!grad) return status_check(c);
    DevPlan d = dev_plan(b, r);
    CUDA_TRY(launch_assemble(d, b.sums.as<double>(), b.out_E.as<double>(), b.out_dg.as<double>(),
                             b.out_db.as<double>(), c->stream));
    c->launches_total += 1;
    std::vector<unsigned long long> keys(std::max(ktop, 1));
    if (ktop > 0) {
        int which = 0, nl = 0;
        // the final pass leaves one list per warp of its persistent grid
        const int grid = std::min(c->num_sms, 1 << (r.n - BLOCK_BITS));
        CUDA_TRY(launch_topk_merge(b.topk_a.as<unsigned long long>(), grid * (PASS_THREADS / 32), ktop,
                                   b.topk_b.as<unsigned long long>(), &which, &nl, c->stream));
        c->launches_total += nl;
        const void *src = which ? b.topk_b.p : b.topk_a.p;
        CUDA_TRY(cudaMemcpyAsync(keys.data(), src, (size_t)ktop * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(E, b.out_E.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(dg, b.out_dg.p, p * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(db, b.out_db.p, p * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    QAOA_TRY(status_check(c));
    if (ktop > 0) decode_keys(keys.data(), ktop, top_idx, top_prob);
    return QAOA_OK;
}

}  // namespace

namespace {

// ---- batches -------------------------------------------------------------------------

// ---- autotuner -----------------------------------------------------------------------
// Candidate fusion widths, largest first (fewer passes, more work per pass).
constexpr int TUNE_K[] = {10, 9, 8, 7, 6, 5};

// Time one forward + adjoint evaluation (depth p, linear-ramp angles) of
// `cost` for every candidate width; the fastest is kept for cost->n.
// ms_by_k[k - 3] receives the time of width k (NaN where not timed).
qaoa_status tune_width(qaoa_ctx c, const qaoa_cost_s *cost, int p, int *best_k, double *ms_by_k) {
    const int n = cost->n;
    std::vector<double> g(p), b(p), dg(p), db(p);
    for (int l = 0; l < p; ++l) {
        const double t = (l + 0.5) / p;
        g[l] = 0.4 * t;
        b[l] = 0.4 * (1.0 - t);
    }
    for (int k = 0; k < 8; ++k)
        if (ms_by_k) ms_by_k[k] = std::nan("");
    const int saved = c->opt.max_fused_qubits, saved_prof = c->opt.profile;
    c->opt.profile = 0;
    double best = 1e300;
    int bk = 10;
    qaoa_status st = QAOA_OK;
    for (int k : TUNE_K) {
        if (k > n) continue;
        c->opt.max_fused_qubits = k;
        double E = 0.0;
        st = run_single(c, cost, p, g.data(), b.data(), true, nullptr, &E, dg.data(), db.data(), 0, nullptr, nullptr);
        if (st != QAOA_OK) break;
        cudaEvent_t e0 = get_event(c), e1 = get_event(c);
        cudaEventRecord(e0, c->stream);
        st = run_single(c, cost, p, g.data(), b.data(), true, nullptr, &E, dg.data(), db.data(), 0, nullptr, nullptr);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        c->ev_free.push_back(e0);
        c->ev_free.push_back(e1);
        if (st != QAOA_OK) break;
        if (ms_by_k) ms_by_k[k - 3] = ms;
        if (ms < best) {
            best = ms;
            bk = k;
        }
    }
    // at the chosen width, time the adjoint with stored forward states (when
    // they fit) against the uncompute sweep and keep the faster for this n
    double ms_mode[2] = {1e300, 1e300};
    const int saved_mode = c->opt.adjoint_mode;
    c->opt.max_fused_qubits = bk;
    for (int m = 0; m < 2 && st == QAOA_OK; ++m) {
        c->opt.adjoint_mode = m == 0 ? QAOA_ADJ_AUTO : QAOA_ADJ_UNCOMPUTE;
        double E = 0.0;
        st = run_single(c, cost, p, g.data(), b.data(), true, nullptr, &E, dg.data(), db.data(), 0, nullptr, nullptr);
        if (st != QAOA_OK) break;
        cudaEvent_t e0 = get_event(c), e1 = get_event(c);
        cudaEventRecord(e0, c->stream);
        st = run_single(c, cost, p, g.data(), b.data(), true, nullptr, &E, dg.data(), db.data(), 0, nullptr, nullptr);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        c->ev_free.push_back(e0);
        c->ev_free.push_back(e1);
        ms_mode[m] = ms;
    }
    c->opt.adjoint_mode = saved_mode;
    c->opt.max_fused_qubits = saved;
    c->opt.profile = saved_prof;
    QAOA_TRY(st);
    c->tuned_k[n] = bk;
    c->tuned_uncompute[n] = ms_mode[1] < ms_mode[0] ? 1 : 0;
    if (ms_by_k) {
        ms_by_k[0] = ms_mode[0];  // widths 3 and 4 are never timed: their slots carry the adjoint forms
        ms_by_k[1] = ms_mode[1];
    }
    if (best_k) *best_k = bk;
    return QAOA_OK;
}

// With options.autotune, tune each n >= 13 on first use (depth 2 is enough:
// every candidate's time is a sum of per-pass times).
qaoa_status maybe_tune(qaoa_ctx c, const qaoa_cost_s *cost) {
    if (!c->opt.autotune || c->opt.max_fused_qubits || cost->n <= SMALL_MAXN || c->tuned_k.count(cost->n))
        return QAOA_OK;
    return tune_width(c, cost, 2, nullptr, nullptr);
}

// Items of one n evaluated together on the pass path.
struct BatchGroup {
    int n = 0;
    std::vector<int> items;               // indices into the caller's batch
    std::vector<const qaoa_cost_s *> tabs;  // distinct tables
    std::vector<int> item_table;          // per item, index into tabs
    PlanRun r;
    PlanBufs *b = nullptr;
    const int32_t *tables = nullptr;      // contiguous tables (device)
    const int *item_table_dev = nullptr;
};

// Small items (n <= 12) evaluated by the shared-memory-resident kernel.
struct SmallSet {
    std::vector<int> items;
    std::vector<SmallItem> host;
    std::vector<int> item_s;
    std::vector<long long> item_kc;
    int max_n = 1;
    PlanBufs *b = nullptr;  // gamma/beta/item_s/item_kc/adam/history buffers
};

// Clears the in-use mark of a batch call's working sets when the call ends.
struct GroupsInUse {
    std::vector<BatchGroup> &gs;
    ~GroupsInUse() {
        for (BatchGroup &g : gs)
            if (g.b) g.b->in_use = false;
    }
};

qaoa_status build_groups(qaoa_ctx c, int nq, const qaoa_cost *costs, const int32_t *item_cost, int B, int p,
                         bool grad, std::vector<BatchGroup> &groups, SmallSet &small) {
    std::map<int, int> gi;
    for (int b = 0; b < B; ++b) {
        const int ci = item_cost ? item_cost[b] : 0;
        if (ci < 0 || ci >= nq || !costs[ci]) return fail(QAOA_ERR_INVALID_ARG, "item %d: bad cost index %d", b, ci);
        const qaoa_cost_s *cs = costs[ci];
        if (cs->n <= SMALL_MAXN) {
            small.items.push_back(b);
            small.max_n = std::max(small.max_n, cs->n);
            continue;
        }
        auto it = gi.find(cs->n);
        if (it == gi.end()) {
            it = gi.emplace(cs->n, (int)groups.size()).first;
            groups.emplace_back();
            groups.back().n = cs->n;
        }
        BatchGroup &g = groups[it->second];
        g.items.push_back(b);
        int t = -1;
        for (size_t k = 0; k < g.tabs.size(); ++k)
            if (g.tabs[k] == cs) t = (int)k;
        if (t < 0) {
            t = (int)g.tabs.size();
            g.tabs.push_back(cs);
        }
        g.item_table.push_back(t);
    }
    for (BatchGroup &g : groups) {
        g.r.n = g.n;
        g.r.p = p;
        g.r.nitems = (int)g.items.size();
        g.r.ntables = (int)g.tabs.size();
        g.r.grad = grad;
        g.r.ktop = 0;
        auto &slot = c->groups[g.n];
        if (!slot) slot.reset(new PlanBufs());
        g.b = slot.get();
        g.b->in_use = true;
        QAOA_TRY(plan_and_allocate(c, g.r, *g.b));
        const size_t N = (size_t)1 << g.n;
        if (g.tabs.size() == 1) {
            g.tables = g.tabs[0]->T;
            g.item_table_dev = nullptr;
        } else {
            qaoa_status st = g.b->tables.ensure(g.tabs.size() * N * 4, &c->held, c->opt.memory_budget);
            if (st == QAOA_ERR_OUT_OF_MEMORY && release_adjoint_scratch(c, nullptr))
                st = g.b->tables.ensure(g.tabs.size() * N * 4, &c->held, c->opt.memory_budget);
            QAOA_TRY(st);
            for (size_t k = 0; k < g.tabs.size(); ++k)
                CUDA_TRY(cudaMemcpyAsync(g.b->tables.as<int32_t>() + k * N, g.tabs[k]->T, N * 4,
                                         cudaMemcpyDeviceToDevice, c->stream));
            QAOA_TRY(g.b->item_table.ensure(g.items.size() * sizeof(int), &c->held, c->opt.memory_budget));
            CUDA_TRY(cudaMemcpyAsync(g.b->item_table.p, g.item_table.data(), g.items.size() * sizeof(int),
                                     cudaMemcpyHostToDevice, c->stream));
            g.tables = g.b->tables.as<int32_t>();
            g.item_table_dev = g.b->item_table.as<int>();
        }
        std::vector<int> s_h(g.items.size());
        std::vector<long long> kc_h(g.items.size());
        for (size_t i = 0; i < g.items.size(); ++i) {
            s_h[i] = g.tabs[g.item_table[i]]->fp.s;
            kc_h[i] = g.tabs[g.item_table[i]]->fp.k_c;
        }
        CUDA_TRY(cudaMemcpyAsync(g.b->item_s.p, s_h.data(), s_h.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 c->stream));
        CUDA_TRY(cudaMemcpyAsync(g.b->item_kc.p, kc_h.data(), kc_h.size() * sizeof(long long),
                                 cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemcpyAsync(g.b->plan.p, g.r.plan.data(), g.r.plan.size() * sizeof(PassPlan),
                                 cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));  // host vectors above are about to go out of scope
    }
    return QAOA_OK;
}

// Upload the angles of the group's items ([items][p], gathered from the batch).
qaoa_status upload_angles(qaoa_ctx c, const std::vector<int> &items, int p, const double *gamma, const double *beta,
                          DevBuf &dg, DevBuf &db) {
    std::vector<double> g((size_t)items.size() * p), b((size_t)items.size() * p);
    for (size_t i = 0; i < items.size(); ++i)
        for (int l = 0; l < p; ++l) {
            g[i * p + l] = gamma[(size_t)items[i] * p + l];
            b[i * p + l] = beta[(size_t)items[i] * p + l];
        }
    QAOA_TRY(dg.ensure(g.size() * sizeof(double), &c->held, c->opt.memory_budget));
    QAOA_TRY(db.ensure(b.size() * sizeof(double), &c->held, c->opt.memory_budget));
    CUDA_TRY(cudaMemcpyAsync(dg.p, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(db.p, b.data(), b.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return QAOA_OK;
}

// One evaluation of a group from its device angles: scalars, passes,
// reductions, and (grad) the assembled E and gradient in b.out_*.
qaoa_status enqueue_group(qaoa_ctx c, BatchGroup &g, bool profile) {
    DevPlan d = dev_plan(*g.b, g.r);
    CUDA_TRY(launch_prep_scalars(d, c->stream));
    c->launches_total += 1;
    QAOA_TRY(enqueue_plan(c, *g.b, g.r, g.tables, g.item_table_dev, profile));
    if (g.r.grad) {
        CUDA_TRY(launch_assemble(d, g.b->sums.as<double>(), g.b->out_E.as<double>(), g.b->out_dg.as<double>(),
                                 g.b->out_db.as<double>(), c->stream));
        c->launches_total += 1;
    }
    return QAOA_OK;
}

constexpr int POOL_STREAMS = 4;

qaoa_status ensure_pool(qaoa_ctx c) {
    if (!c->pool_fork) CUDA_TRY(cudaEventCreateWithFlags(&c->pool_fork, cudaEventDisableTiming));
    while ((int)c->pool.size() < POOL_STREAMS) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        c->pool.push_back(s);
        CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->pool_join.push_back(e);
    }
    return QAOA_OK;
}

// Enqueue `home_work` on the context's stream and fn(g) for every group of a
// batch, the groups on the streams of a small pool forked from and joined back
// into the context's stream: the passes of a small n fill a few SMs only, so
// groups of different n overlap on the GPU instead of running one after the
// other.  Largest n first (the longest chain starts at once).  Legal inside a
// stream capture (the fork and join are event waits).
template <class H, class F>
qaoa_status enqueue_groups(qaoa_ctx c, std::vector<BatchGroup> &groups, H &&home_work, F &&fn) {
    if (groups.size() <= 1) {
        QAOA_TRY(home_work());
        for (BatchGroup &g : groups) QAOA_TRY(fn(g));
        return QAOA_OK;
    }
    QAOA_TRY(ensure_pool(c));
    std::vector<int> order(groups.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return groups[a].n > groups[b].n; });
    const cudaStream_t home = c->stream;
    const int used = (int)std::min(groups.size(), c->pool.size());
    CUDA_TRY(cudaEventRecord(c->pool_fork, home));
    for (int k = 0; k < used; ++k) CUDA_TRY(cudaStreamWaitEvent(c->pool[k], c->pool_fork, 0));
    qaoa_status st = home_work();
    for (size_t i = 0; i < order.size() && st == QAOA_OK; ++i) {
        c->stream = c->pool[i % c->pool.size()];
        st = fn(groups[order[i]]);
        c->stream = home;
    }
    // join every forked stream, also after an error (a capture must end joined)
    for (int k = 0; k < used; ++k) {
        const cudaError_t e1 = cudaEventRecord(c->pool_join[k], c->pool[k]);
        const cudaError_t e2 = cudaStreamWaitEvent(home, c->pool_join[k], 0);
        if (st == QAOA_OK && (e1 || e2))
            st = fail(QAOA_ERR_CUDA, "stream join: %s", cudaGetErrorString(e1 ? e1 : e2));
    }
    return st;
}

// Small items: host blocks with device output pointers; the resident kernel
// reads angles from the blocks (refreshed on the device by small_prep).
qaoa_status build_small(qaoa_ctx c, SmallSet &s, const qaoa_cost *costs, const int32_t *item_cost, int p,
                        const double *gamma, const double *beta, bool grad) {
    if (s.items.empty()) return QAOA_OK;
    auto &slot = c->groups[0];
    if (!slot) slot.reset(new PlanBufs());
    s.b = slot.get();
    const size_t per = 1 + 2 * (size_t)p;
    const size_t K = s.items.size();
    QAOA_TRY(s.b->small_out.ensure(K * per * sizeof(double) + 64, &c->held, c->opt.memory_budget));
    s.host.resize(K);
    s.item_s.resize(K);
    s.item_kc.resize(K);
    for (size_t i = 0; i < K; ++i) {
        const int b = s.items[i];
        const qaoa_cost_s *cs = costs[item_cost ? item_cost[b] : 0];
        fill_small(s.host[i], cs, p, gamma + (size_t)b * p, beta + (size_t)b * p);
        s.host[i].grad = grad ? 1 : 0;
        s.host[i].out = s.b->small_out.as<double>() + i * per;
        s.item_s[i] = cs->fp.s;
        s.item_kc[i] = cs->fp.k_c;
    }
    QAOA_TRY(s.b->small_items.ensure(K * sizeof(SmallItem), &c->held, c->opt.memory_budget));
    CUDA_TRY(cudaMemcpyAsync(s.b->small_items.p, s.host.data(), K * sizeof(SmallItem), cudaMemcpyHostToDevice,
                             c->stream));
    QAOA_TRY(s.b->item_s.ensure(K * sizeof(int), &c->held, c->opt.memory_budget));
    QAOA_TRY(s.b->item_kc.ensure(K * sizeof(long long), &c->held, c->opt.memory_budget));
    CUDA_TRY(cudaMemcpyAsync(s.b->item_s.p, s.item_s.data(), K * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(s.b->item_kc.p, s.item_kc.data(), K * sizeof(long long), cudaMemcpyHostToDevice,
                             c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return QAOA_OK;
}

qaoa_status enqueue_small(qaoa_ctx c, SmallSet &s, int p, bool from_device_angles) {
    if (s.items.empty()) return QAOA_OK;
    const int K = (int)s.items.size();
    if (from_device_angles) {
        CUDA_TRY(launch_small_prep(s.b->small_items.as<SmallItem>(), K, s.b->gamma.as<double>(),
                                   s.b->beta.as<double>(), p, s.b->item_s.as<int>(), s.b->item_kc.as<long long>(),
                                   c->stream));
        c->launches_total += 1;
    }
    double bytes = 0;
    for (auto &it : s.host) bytes += std::ldexp(4.0, it.n);
    ProfScope ps(c, 3, bytes, !from_device_angles);
    CUDA_TRY(launch_small(s.b->small_items.as<SmallItem>(), K, s.max_n, false, s.host[0].grad != 0, c->stream));
    c->launches_total += 1;
    return QAOA_OK;
}

}  // namespace

extern "C" {

const char *qaoa_last_error(void) { return qaoa::last_error(); }

qaoa_status qaoa_ctx_create(int device, void *cuda_stream, const qaoa_options *opt, qaoa_ctx *out) {
    if (!out) return fail(QAOA_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    int count = 0;
    CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count)
        return fail(QAOA_ERR_INVALID_ARG, "device %d not present (%d devices)", device, count);
    QAOA_TRY(set_device(device));
    qaoa_options o{};
    if (opt) o = *opt;
    if (o.max_fused_qubits != 0 && (o.max_fused_qubits < 3 || o.max_fused_qubits > 10))
        return fail(QAOA_ERR_INVALID_ARG, "max_fused_qubits must be 0 or in [3, 10]");
    if (o.table_build < 0 || o.table_build > 1) return fail(QAOA_ERR_INVALID_ARG, "table_build must be 0 or 1");
    if (o.autotune < 0 || o.autotune > 1) return fail(QAOA_ERR_INVALID_ARG, "autotune must be 0 or 1");
    if (o.adjoint_mode < 0 || o.adjoint_mode > 2) return fail(QAOA_ERR_INVALID_ARG, "adjoint_mode must be 0, 1 or 2");
    if (o.reverse_blocks < 0 || o.reverse_blocks > 2) return fail(QAOA_ERR_INVALID_ARG, "reverse_blocks must be 0, 1 or 2");
    for (int k = 0; k < 3; ++k)
        if (o.reserved[k]) return fail(QAOA_ERR_INVALID_ARG, "options.reserved[%d] must be zero", k);
    auto *c = new qaoa_ctx_s();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->opt = o;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
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
    if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
    for (auto s : c->pool) cudaStreamDestroy(s);
    for (auto e : c->pool_join) cudaEventDestroy(e);
    if (c->pool_fork) cudaEventDestroy(c->pool_fork);
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
        cudaError_t e = ctx_malloc(c, reinterpret_cast<void **>(&h->T), N * sizeof(int32_t));
        if (e) {
            return fail(QAOA_ERR_OUT_OF_MEMORY, "objective table (%zu bytes): %s", N * 4, cudaGetErrorString(e));
        }
    }
    const size_t coef_bytes = (size_t)(n + n * n) * 8;
    std::vector<long long> coef(n + n * n);
    for (int i = 0; i < n; ++i) coef[i] = h->fp.ell_q[i];
    for (int k = 0; k < n * n; ++k) coef[n + k] = h->fp.b_q[k];
    // tensor-core build for n >= 14 unless disabled: the cross couplings between
    // the low n - n_hi and the high n_hi = min(16, n - 7) variables must fit
    // four base-2^11 digits (always true for tables that fit int32)
    int digits = -1;
    const int nhi = n - 7 < 16 ? n - 7 : 16, nlo = n - nhi;
    if (n >= 14 && c->opt.table_build == 0) {
        long long wmax = 0;
        for (int j = 0; j < nhi; ++j) {
            long long w = 0;
            for (int i = 0; i < nlo; ++i) w += std::llabs(h->fp.b_q[(size_t)i * n + nlo + j]);
            wmax = std::max(wmax, w);
        }
        digits = table_mma_digits(wmax);
    }
    long long *min_val = nullptr;
    unsigned long long *min_idx = nullptr;
    if (digits > 0) {
        const int grid = 2 * c->num_sms;  // two tile CTAs per SM
        const size_t alo_b = ((size_t)8 << nlo), ahi_b = ((size_t)8 << nhi), w_b = (size_t)digits * 32 << nlo;
        const size_t tot = coef_bytes + (size_t)grid * 16 + 64 + alo_b + ahi_b + w_b + 1024;
        QAOA_TRY(c->misc.ensure(tot, &c->held, c->opt.memory_budget));
        QAOA_TRY(c->status.ensure(16, &c->held, c->opt.memory_budget));
        char *m = c->misc.as<char>();
        CUDA_TRY(cudaMemcpyAsync(m, coef.data(), coef_bytes, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemsetAsync(c->status.p, 0, 16, c->stream));
        size_t o = (coef_bytes + 255) & ~size_t(255);
        TableMmaArgs a{};
        a.n = n;
        a.digits = digits;
        a.ell = reinterpret_cast<long long *>(m);
        a.b = reinterpret_cast<long long *>(m) + n;
        a.c_off = h->fp.c0_q - h->fp.k_c;
        a.T = h->T;
        a.blk_val = reinterpret_cast<long long *>(m + o);
        a.blk_idx = reinterpret_cast<unsigned long long *>(m + o + (size_t)grid * 8);
        o += (size_t)grid * 16;
        a.min_val = reinterpret_cast<long long *>(m + o);
        a.min_idx = reinterpret_cast<unsigned long long *>(m + o + 8);
        o = (o + 16 + 255) & ~size_t(255);
        a.alo = reinterpret_cast<long long *>(m + o);
        o += alo_b;
        a.ahi = reinterpret_cast<long long *>(m + o);
        o += ahi_b;
        a.wdig = reinterpret_cast<__half *>(m + o);
        a.status = c->status.as<unsigned int>();
        {
            ProfScope ps(c, 2, (double)N * 4.0);
            CUDA_TRY(launch_table_mma(a, grid, c->stream));
            c->launches_total += 3;
        }
        min_val = a.min_val;
        min_idx = a.min_idx;
        QAOA_TRY(status_check(c));
    } else {
        const int nblk = cost_build_blocks(n);
        QAOA_TRY(c->misc.ensure(coef_bytes + (size_t)nblk * 16 + 64, &c->held, c->opt.memory_budget));
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
        min_val = a.min_val;
        min_idx = a.min_idx;
    }
    long long mv = 0;
    unsigned long long mi = 0;
    CUDA_TRY(cudaMemcpyAsync(&mv, min_val, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(&mi, min_idx, 8, cudaMemcpyDeviceToHost, c->stream));
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

qaoa_status qaoa_cost_device_ptr(qaoa_cost cost, const int32_t **table, int64_t *count) {
    if (!cost) return fail(QAOA_ERR_INVALID_ARG, "cost is null");
    if (table) *table = cost->T;
    if (count) *count = (int64_t)1 << cost->n;
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
        cudaError_t e = ctx_malloc(c, &fresh->amps, bytes);
        if (e) {
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
        QAOA_TRY(run_small(c, c->small_items, items, fp64, false, n));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    } else {
        QAOA_TRY(maybe_tune(c, cost));
        QAOA_TRY(run_single(c, cost, p, gamma, beta, false, static_cast<float2 *>(st->amps), nullptr, nullptr,
                            nullptr, 0, nullptr, nullptr));
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

qaoa_status qaoa_state_gather(qaoa_ctx c, qaoa_state s, const uint64_t *idx, int count, void *out) {
    if (!c || !s || !idx || !out || count < 0) return fail(QAOA_ERR_INVALID_ARG, "null argument or count < 0");
    if (count == 0) return QAOA_OK;
    const uint64_t N = (uint64_t)1 << s->n;
    for (int i = 0; i < count; ++i)
        if (idx[i] >= N) return fail(QAOA_ERR_INVALID_ARG, "index %llu outside the 2^%d amplitudes", (unsigned long long)idx[i], s->n);
    QAOA_TRY(set_device(c->device));
    const int es = s->fp64 ? 16 : 8;
    const size_t ib = (size_t)count * 8, ob = (size_t)count * es;
    QAOA_TRY(c->misc.ensure(ib + ob + 64, &c->held, c->opt.memory_budget));
    char *m = c->misc.as<char>();
    unsigned int *bad = reinterpret_cast<unsigned int *>(m + ib + ob);
    CUDA_TRY(cudaMemcpyAsync(m, idx, ib, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemsetAsync(bad, 0, 4, c->stream));
    CUDA_TRY(launch_gather(s->amps, es, s->n, reinterpret_cast<const unsigned long long *>(m), count, m + ib, bad,
                           c->stream));
    c->launches_total += 1;
    unsigned int hb = 0;
    CUDA_TRY(cudaMemcpyAsync(out, m + ib, ob, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (hb) return fail(QAOA_ERR_INVALID_ARG, "gather index outside the state");
    return QAOA_OK;
}

qaoa_status qaoa_expect(qaoa_ctx c, qaoa_cost cost, qaoa_state s, double *out) {
    if (!c || !cost || !s || !out) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    if (s->n != cost->n) return fail(QAOA_ERR_INVALID_ARG, "state and cost differ in n");
    if (s->fp64)
        return fail(QAOA_ERR_INVALID_ARG,
                    "qaoa_expect takes complex64 states; complex128 states report E from qaoa_grad");
    QAOA_TRY(set_device(c->device));
    const int n = s->n;
    const int nb = (int)((((size_t)1 << n) + 8191) / 8192);
    QAOA_TRY(c->partials_e.ensure((size_t)nb * NSLOT * 8, &c->held, c->opt.memory_budget));
    QAOA_TRY(c->sums_e.ensure(NSLOT * 8, &c->held, c->opt.memory_budget));
    CUDA_TRY(launch_expect((const float2 *)s->amps, cost->T, n, c->partials_e.as<double>(), c->stream));
    CUDA_TRY(launch_reduce_partials(c->partials_e.as<double>(), 1, nb, c->sums_e.as<double>(), c->stream));
    c->launches_total += 2;
    double h[NSLOT];
    CUDA_TRY(cudaMemcpyAsync(h, c->sums_e.p, sizeof h, cudaMemcpyDeviceToHost, c->stream));
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
    float2 amp_min = make_float2(0, 0);
    CUDA_TRY(cudaMemcpyAsync(&amp_min, (const float2 *)s->amps + cost->argmin, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    decode_keys(keys.data(), k, idx, prob);
    if (cost_out) {
        std::vector<int32_t> tv(k);
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
        QAOA_TRY(run_small(c, c->small_items, items, fp64, true, n));
        std::vector<double> h(1 + 2 * p + 16);
        CUDA_TRY(cudaMemcpyAsync(h.data(), c->small_out.p, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        *out_expect = h[0];
        for (int l = 0; l < p; ++l) {
            dgamma[l] = h[1 + l];
            dbeta[l] = h[1 + p + l];
        }
        if (k_top > 0)
            decode_keys(reinterpret_cast<const unsigned long long *>(&h[1 + 2 * p]), k_top, top_idx, top_prob);
        return QAOA_OK;
    }
    if (fp64) return fail(QAOA_ERR_INVALID_ARG, "complex128 states are limited to n <= 12");
    QAOA_TRY(maybe_tune(c, cost));
    return run_single(c, cost, p, gamma, beta, true, nullptr, out_expect, dgamma, dbeta, k_top, top_idx, top_prob);
}

}  // extern "C"

qaoa_status qaoa::api::run_batch(qaoa_ctx c, int nq, const qaoa_cost *costs, const int32_t *item_cost, int B, int p,
                                 const double *gamma, const double *beta, double *expect, double *dgamma,
                                 double *dbeta, std::vector<ItemState> *states) {
    if (!c || !costs || nq < 1 || B < 1 || !gamma || !beta || !expect)
        return fail(QAOA_ERR_INVALID_ARG, "bad batch arguments");
    if ((dgamma == nullptr) != (dbeta == nullptr))
        return fail(QAOA_ERR_INVALID_ARG, "dgamma and dbeta must both be set or both be null");
    if (p < 1 || p > SMALL_MAXP) return fail(QAOA_ERR_INVALID_ARG, "p=%d not in [1, %d]", p, SMALL_MAXP);
    if (c->opt.state_fp64) return fail(QAOA_ERR_INVALID_ARG, "batched evaluation runs in complex64 only");
    QAOA_TRY(check_angles(p * B, gamma, beta));
    QAOA_TRY(set_device(c->device));
    const bool grad = dgamma != nullptr;
    for (int k = 0; k < nq; ++k)
        if (costs[k]) QAOA_TRY(maybe_tune(c, costs[k]));
    std::vector<BatchGroup> groups;
    GroupsInUse in_use{groups};
    SmallSet small;
    QAOA_TRY(build_groups(c, nq, costs, item_cost, B, p, grad, groups, small));
    QAOA_TRY(build_small(c, small, costs, item_cost, p, gamma, beta, grad));
    if (states) {
        if (grad) return fail(QAOA_ERR_INVALID_ARG, "final states are kept by forward-only batches");
        states->assign(B, ItemState{});
        // small items write their final state to a context buffer
        size_t off = 0;
        for (size_t i = 0; i < small.items.size(); ++i) off += (size_t)8 << small.host[i].n;
        QAOA_TRY(c->small_states.ensure(off + 16, &c->held, c->opt.memory_budget));
        off = 0;
        for (size_t i = 0; i < small.items.size(); ++i) {
            small.host[i].psi_out = c->small_states.as<char>() + off;
            const int b = small.items[i];
            (*states)[b] = ItemState{small.host[i].psi_out, small.host[i].n,
                                     costs[item_cost ? item_cost[b] : 0]};
            off += (size_t)8 << small.host[i].n;
        }
        if (!small.items.empty())
            CUDA_TRY(cudaMemcpyAsync(small.b->small_items.p, small.host.data(), small.host.size() * sizeof(SmallItem),
                                     cudaMemcpyHostToDevice, c->stream));
    }
    CUDA_TRY(cudaMemsetAsync(c->status.p, 0, 16, c->stream));
    // every group's angles before any launch: a copy from pageable host memory
    // waits for the work already on the stream
    for (BatchGroup &g : groups) QAOA_TRY(upload_angles(c, g.items, p, gamma, beta, g.b->gamma, g.b->beta));
    auto home = [&]() { return enqueue_small(c, small, p, false); };
    auto one = [&](BatchGroup &g) -> qaoa_status {
        QAOA_TRY(enqueue_group(c, g, true));
        if (!grad) {
            if (states)
                for (size_t i = 0; i < g.items.size(); ++i)
                    (*states)[g.items[i]] =
                        ItemState{g.b->psi.as<float2>() + i * ((size_t)1 << g.n), g.n, g.tabs[g.item_table[i]]};
            // forward only: <H_C> of every item's final state
            const int nb = 1 << (g.n - BLOCK_BITS);
            const size_t N = (size_t)1 << g.n;
            for (size_t i = 0; i < g.items.size(); ++i) {
                CUDA_TRY(launch_expect(g.b->psi.as<float2>() + i * N, g.tabs[g.item_table[i]]->T, g.n,
                                       g.b->partials.as<double>() + i * nb * NSLOT, c->stream));
                c->launches_total += 1;
            }
            CUDA_TRY(launch_reduce_partials(g.b->partials.as<double>(), (int)g.items.size(), nb,
                                            g.b->sums.as<double>(), c->stream));
            c->launches_total += 1;
        }
        return QAOA_OK;
    };
    QAOA_TRY(enqueue_groups(c, groups, home, one));
    QAOA_TRY(status_check(c));
    // results
    if (!small.items.empty()) {
        const size_t per = 1 + 2 * (size_t)p;
        std::vector<double> h(small.items.size() * per);
        CUDA_TRY(cudaMemcpyAsync(h.data(), small.b->small_out.p, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < small.items.size(); ++i) {
            const int b = small.items[i];
            expect[b] = h[i * per];
            if (grad)
                for (int l = 0; l < p; ++l) {
                    dgamma[(size_t)b * p + l] = h[i * per + 1 + l];
                    dbeta[(size_t)b * p + l] = h[i * per + 1 + p + l];
                }
        }
    }
    for (BatchGroup &g : groups) {
        const size_t K = g.items.size();
        if (grad) {
            std::vector<double> E(K), dg(K * p), db(K * p);
            CUDA_TRY(cudaMemcpyAsync(E.data(), g.b->out_E.p, K * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaMemcpyAsync(dg.data(), g.b->out_dg.p, K * p * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaMemcpyAsync(db.data(), g.b->out_db.p, K * p * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            for (size_t i = 0; i < K; ++i) {
                const int b = g.items[i];
                expect[b] = E[i];
                for (int l = 0; l < p; ++l) {
                    dgamma[(size_t)b * p + l] = dg[i * p + l];
                    dbeta[(size_t)b * p + l] = db[i * p + l];
                }
            }
        } else {
            std::vector<double> S(K * NSLOT);
            CUDA_TRY(cudaMemcpyAsync(S.data(), g.b->sums.p, S.size() * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            for (size_t i = 0; i < K; ++i) {
                const qaoa_cost_s *cs = g.tabs[g.item_table[i]];
                expect[g.items[i]] = std::ldexp(S[i * NSLOT] + (double)cs->fp.k_c * S[i * NSLOT + 1], -cs->fp.s);
            }
        }
    }
    return QAOA_OK;
}

extern "C" {

qaoa_status qaoa_grad_batch(qaoa_ctx c, int nq, const qaoa_cost *costs, const int32_t *item_cost, int B, int p,
                            const double *gamma, const double *beta, double *expect, double *dgamma, double *dbeta) {
    return run_batch(c, nq, costs, item_cost, B, p, gamma, beta, expect, dgamma, dbeta, nullptr);
}

}  // extern "C"

namespace {

// Adam state of a run that continues an earlier one (host, caller-owned):
// m, v as [B][2p] (gamma then beta of each item), step = steps already taken.
struct AdamResume {
    double *m = nullptr, *v = nullptr;
    int32_t *step = nullptr;
};

qaoa_status optimize_adam(qaoa_ctx c, int nq, const qaoa_cost *costs, const int32_t *item_cost, int B, int p,
                          double *gamma, double *beta, const qaoa_adam_options *aopt, double *history,
                          double *final_expect, const AdamResume &rs) {
    if (!c || !costs || nq < 1 || B < 1 || !gamma || !beta || !aopt)
        return fail(QAOA_ERR_INVALID_ARG, "bad optimiser arguments");
    const int step0 = rs.step ? *rs.step : 0;
    if (step0 < 0) return fail(QAOA_ERR_INVALID_ARG, "step=%d < 0", step0);
    if (p < 1 || p > SMALL_MAXP) return fail(QAOA_ERR_INVALID_ARG, "p=%d not in [1, %d]", p, SMALL_MAXP);
    if (aopt->iterations < 1) return fail(QAOA_ERR_INVALID_ARG, "iterations=%d < 1", aopt->iterations);
    if (c->opt.state_fp64) return fail(QAOA_ERR_INVALID_ARG, "the optimiser runs in complex64 only");
    QAOA_TRY(check_angles(p * B, gamma, beta));
    const double lr = aopt->lr > 0 ? aopt->lr : 0.01;
    const double b1 = aopt->beta1 > 0 ? aopt->beta1 : 0.9;
    const double b2 = aopt->beta2 > 0 ? aopt->beta2 : 0.999;
    const double eps = aopt->eps > 0 ? aopt->eps : 1e-8;
    if (!(lr < 1e6) || b1 >= 1.0 || b2 >= 1.0) return fail(QAOA_ERR_INVALID_ARG, "bad Adam hyper-parameters");
    const int iters = aopt->iterations;
    QAOA_TRY(set_device(c->device));
    if (!c->aux_stream) CUDA_TRY(cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
    for (int k = 0; k < nq; ++k)
        if (costs[k]) QAOA_TRY(maybe_tune(c, costs[k]));
    std::vector<BatchGroup> groups;
    GroupsInUse in_use{groups};
    SmallSet small;
    QAOA_TRY(build_groups(c, nq, costs, item_cost, B, p, true, groups, small));
    QAOA_TRY(build_small(c, small, costs, item_cost, p, gamma, beta, true));
    // every group (and the small set) keeps its angles, moments and history on the device
    struct Opt {
        PlanBufs *b;
        const std::vector<int> *items;
        AdamArgs a;
    };
    std::vector<Opt> opts;
    auto setup = [&](PlanBufs *b, const std::vector<int> &items, const double *dg, const double *db, int gstride,
                     const double *E, int estride) -> qaoa_status {
        const size_t K = items.size();
        QAOA_TRY(upload_angles(c, items, p, gamma, beta, b->gamma, b->beta));
        QAOA_TRY(b->adam_m.ensure(2 * K * p * 8, &c->held, c->opt.memory_budget));
        QAOA_TRY(b->adam_v.ensure(2 * K * p * 8, &c->held, c->opt.memory_budget));
        QAOA_TRY(b->adam_step.ensure(16, &c->held, c->opt.memory_budget));
        QAOA_TRY(b->history.ensure((size_t)iters * K * 8, &c->held, c->opt.memory_budget));
        if (rs.m) {
            // device moments are [gamma | beta][item][l]
            std::vector<double> hm(2 * K * p), hv(2 * K * p);
            for (size_t i = 0; i < K; ++i)
                for (int l = 0; l < p; ++l)
                    for (int h = 0; h < 2; ++h) {
                        const size_t src = (size_t)items[i] * 2 * p + (size_t)h * p + l;
                        const size_t dst = (size_t)h * K * p + i * p + l;
                        hm[dst] = rs.m[src];
                        hv[dst] = rs.v[src];
                    }
            CUDA_TRY(cudaMemcpyAsync(b->adam_m.p, hm.data(), hm.size() * 8, cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(cudaMemcpyAsync(b->adam_v.p, hv.data(), hv.size() * 8, cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
        } else {
            CUDA_TRY(cudaMemsetAsync(b->adam_m.p, 0, 2 * K * p * 8, c->stream));
            CUDA_TRY(cudaMemsetAsync(b->adam_v.p, 0, 2 * K * p * 8, c->stream));
        }
        const int st0[4] = {step0, 0, 0, 0};
        CUDA_TRY(cudaMemcpyAsync(b->adam_step.p, st0, sizeof st0, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        AdamArgs a{};
        a.gamma = b->gamma.as<double>();
        a.beta = b->beta.as<double>();
        a.dgamma = dg;
        a.dbeta = db;
        a.gstride = gstride;
        a.m = b->adam_m.as<double>();
        a.v = b->adam_v.as<double>();
        a.step = b->adam_step.as<int>();
        a.E = E;
        a.estride = estride;
        a.history = b->history.as<double>();
        a.max_steps = iters;
        a.step0 = step0;
        a.nitems = (int)K;
        a.p = p;
        a.lr = lr;
        a.beta1 = b1;
        a.beta2 = b2;
        a.eps = eps;
        opts.push_back({b, &items, a});
        return QAOA_OK;
    };
    if (!small.items.empty()) {
        const int per = 1 + 2 * p;
        double *o = small.b->small_out.as<double>();
        QAOA_TRY(setup(small.b, small.items, o + 1, o + 1 + p, per, o, per));
    }
    for (BatchGroup &g : groups)
        QAOA_TRY(setup(g.b, g.items, g.b->out_dg.as<double>(), g.b->out_db.as<double>(), p, g.b->out_E.as<double>(), 1));
    CUDA_TRY(cudaMemsetAsync(c->status.p, 0, 16, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    // The loop runs on the context's own non-blocking stream (a capture cannot
    // use the legacy default stream); the caller's stream is joined at the end.
    cudaStream_t user = c->stream;
    c->stream = c->aux_stream;
    struct Restore {
        qaoa_ctx c;
        cudaStream_t s;
        ~Restore() { c->stream = s; }
    } restore{c, user};
    auto eval = [&](bool profile) -> qaoa_status {
        return enqueue_groups(
            c, groups, [&]() { return enqueue_small(c, small, p, true); },
            [&](BatchGroup &g) { return enqueue_group(c, g, profile); });
    };
    auto step = [&](bool profile) -> qaoa_status {
        QAOA_TRY(eval(profile));
        for (Opt &o : opts) {
            CUDA_TRY(launch_adam(o.a, c->stream));
            c->launches_total += 2;
        }
        return QAOA_OK;
    };
    const int64_t before = c->launches_total;
    QAOA_TRY(step(true));  // eager first step (also sets every kernel attribute before capture)
    const int64_t per_step = c->launches_total - before;
    if (iters > 1) {
        if (aopt->disable_graph) {
            for (int t = 1; t < iters; ++t) QAOA_TRY(step(true));
        } else {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
            qaoa_status st = step(false);
            cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
            if (st != QAOA_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            CUDA_TRY(ce);
            c->launches_total -= per_step;  // counted again per replay below
            cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
            if (ie != cudaSuccess) {
                cudaGraphDestroy(graph);
                CUDA_TRY(ie);
            }
            cudaError_t le = cudaSuccess;
            for (int t = 1; t < iters && le == cudaSuccess; ++t) le = cudaGraphLaunch(exec, c->stream);
            c->launches_total += per_step * (iters - 1);
            cudaError_t se = cudaStreamSynchronize(c->stream);
            cudaGraphExecDestroy(exec);
            cudaGraphDestroy(graph);
            CUDA_TRY(le);
            CUDA_TRY(se);
        }
    }
    // objective at the final parameters
    QAOA_TRY(eval(true));
    QAOA_TRY(status_check(c));
    for (Opt &o : opts) {
        const std::vector<int> &items = *o.items;
        const size_t K = items.size();
        std::vector<double> g(K * p), bt(K * p), hist((size_t)iters * K), E(K);
        CUDA_TRY(cudaMemcpyAsync(g.data(), o.a.gamma, K * p * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(bt.data(), o.a.beta, K * p * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(hist.data(), o.a.history, hist.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpy2DAsync(E.data(), 8, o.a.E, (size_t)o.a.estride * 8, 8, K, cudaMemcpyDeviceToHost,
                                   c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < K; ++i) {
            const int b = items[i];
            for (int l = 0; l < p; ++l) {
                gamma[(size_t)b * p + l] = g[i * p + l];
                beta[(size_t)b * p + l] = bt[i * p + l];
            }
            if (history)
                for (int t = 0; t < iters; ++t) history[(size_t)t * B + b] = hist[(size_t)t * K + i];
            if (final_expect) final_expect[b] = E[i];
        }
        if (rs.m) {
            std::vector<double> hm(2 * K * p), hv(2 * K * p);
            CUDA_TRY(cudaMemcpyAsync(hm.data(), o.a.m, hm.size() * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaMemcpyAsync(hv.data(), o.a.v, hv.size() * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            for (size_t i = 0; i < K; ++i)
                for (int l = 0; l < p; ++l)
                    for (int h = 0; h < 2; ++h) {
                        const size_t dst = (size_t)items[i] * 2 * p + (size_t)h * p + l;
                        const size_t src = (size_t)h * K * p + i * p + l;
                        rs.m[dst] = hm[src];
                        rs.v[dst] = hv[src];
                    }
        }
    }
    if (rs.step) *rs.step = step0 + iters;
    // order the caller's stream after the loop
    cudaEvent_t done = get_event(c);
    CUDA_TRY(cudaEventRecord(done, c->aux_stream));
    CUDA_TRY(cudaStreamWaitEvent(user, done, 0));
    c->ev_free.push_back(done);
    return QAOA_OK;
}

}  // namespace

extern "C" {

qaoa_status qaoa_optimize_adam(qaoa_ctx c, int nq, const qaoa_cost *costs, const int32_t *item_cost, int B, int p,
                               double *gamma, double *beta, const qaoa_adam_options *aopt, double *history,
                               double *final_expect) {
    return optimize_adam(c, nq, costs, item_cost, B, p, gamma, beta, aopt, history, final_expect, AdamResume{});
}

qaoa_status qaoa_optimize_adam_resume(qaoa_ctx c, int nq, const qaoa_cost *costs, const int32_t *item_cost, int B,
                                      int p, double *gamma, double *beta, const qaoa_adam_options *aopt,
                                      double *history, double *final_expect, double *m, double *v, int32_t *step) {
    if (!m || !v || !step) return fail(QAOA_ERR_INVALID_ARG, "m, v and step are required");
    AdamResume rs;
    rs.m = m;
    rs.v = v;
    rs.step = step;
    return optimize_adam(c, nq, costs, item_cost, B, p, gamma, beta, aopt, history, final_expect, rs);
}

qaoa_status qaoa_autotune(qaoa_ctx c, qaoa_cost cost, int p, int32_t *best_k, double *ms_by_k) {
    if (!c || !cost || !best_k) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    if (p < 1 || p > 64) return fail(QAOA_ERR_INVALID_ARG, "p=%d not in [1, 64]", p);
    if (cost->n <= SMALL_MAXN)
        return fail(QAOA_ERR_INVALID_ARG, "n=%d is evaluated by the shared-memory kernel; nothing to tune", cost->n);
    if (c->opt.state_fp64) return fail(QAOA_ERR_INVALID_ARG, "the layer-pass path runs in complex64 only");
    QAOA_TRY(set_device(c->device));
    int k = 10;
    QAOA_TRY(tune_width(c, cost, p, &k, ms_by_k));
    *best_k = k;
    return QAOA_OK;
}

qaoa_status qaoa_partition(int n, int M, const int32_t *caps, const int32_t *manual, int32_t *qpu_of) {
    return partition(n, M, caps, manual, qpu_of);
}

qaoa_status qaoa_plan_describe(int n, int p, int grad, int max_fused_qubits, int stored_mids, qaoa_pass_info *out,
                               int capacity, int32_t *count, int32_t *nslots, int32_t *nmids) {
    if (!count) return fail(QAOA_ERR_INVALID_ARG, "count is null");
    if (n < 13 || n > 33) return fail(QAOA_ERR_INVALID_ARG, "n=%d outside [13, 33] (the pass path)", n);
    if (p < 0 || p > SMALL_MAXP) return fail(QAOA_ERR_INVALID_ARG, "p=%d outside [0, %d]", p, SMALL_MAXP);
    if (max_fused_qubits < 3 || max_fused_qubits > 10)
        return fail(QAOA_ERR_INVALID_ARG, "max_fused_qubits=%d outside [3, 10]", max_fused_qubits);
    int ns = 0, nm = 0;
    const std::vector<PassPlan> plan = make_plan(n, p, grad != 0, max_fused_qubits, stored_mids, &ns, &nm);
    if (plan.empty()) return fail(QAOA_ERR_INVALID_ARG, "no layout for n=%d at width %d", n, max_fused_qubits);
    *count = (int32_t)plan.size();
    if (nslots) *nslots = ns;
    if (nmids) *nmids = nm;
    if (!out) return QAOA_OK;
    if (capacity < (int)plan.size()) return fail(QAOA_ERR_INVALID_ARG, "capacity %d < %zu passes", capacity, plan.size());
    for (size_t i = 0; i < plan.size(); ++i) {
        const PassPlan &pl = plan[i];
        qaoa_pass_info &o = out[i];
        o.kind = pl.kind;
        o.group_type = pl.type;
        o.loA = pl.loA;
        o.loB = pl.loB;
        o.mask = pl.mask;
        o.pre_layer = pl.la;
        o.cost_layer = pl.lc;
        o.post_layer = pl.lb;
        o.in_slot = pl.in_slot;
        o.out_slot = pl.out_slot;
        o.psi_slot = pl.psi_slot;
        o.lambda_alone_out = (pl.kind == 1 || pl.kind == 2) ? pl.split_out : 0;
        o.interleaved_out = pl.kind == 3 ? pl.pl_out : 0;
        for (int s = 0; s < 8; ++s) o.slot_param[s] = s < NSLOT ? pl.slot_param[s] : -1;
        o.bytes_per_amp = pass_bytes_per_amp(pl);
    }
    return QAOA_OK;
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
    // contiguous: QPU indices start at 0 and never decrease, stepping by 0 or 1
    bool contiguous = qpu_of[0] == 0;
    for (int i = 1; i < n; ++i)
        if (qpu_of[i] != qpu_of[i - 1] && qpu_of[i] != qpu_of[i - 1] + 1) contiguous = false;
    const int c0 = (int)vars[0].size();
    if (c0 > 16 || n - c0 > 31 || n - c0 < 1) contiguous = false;
    const size_t hhi_bytes = contiguous ? ((size_t)8 << (n - c0)) : 0;
    const size_t bytes = n * 4 * 2 + (M + 1) * 4 + L.size() * 8 + Loff.size() * 8 + V.size() * 8 + Voff.size() * 8 +
                         64 * 8 + hhi_bytes;
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
    a.contiguous = contiguous ? 1 : 0;
    a.c0 = c0;
    if (contiguous) {
        a.hhi = reinterpret_cast<long long *>(d + ((o + 255) & ~size_t(255)));
        o = ((o + 255) & ~size_t(255)) + hhi_bytes;
    }
    CUDA_TRY(cudaGetLastError());
    {
        ProfScope ps(c, 4, std::ldexp(4.0, n));
        CUDA_TRY(launch_fact_check(a, c->stream));
        c->launches_total += contiguous ? 2 : 1;
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
    if (!c || kind < 0 || kind >= QAOA_PROF_KINDS) return fail(QAOA_ERR_INVALID_ARG, "bad context or kind");
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
