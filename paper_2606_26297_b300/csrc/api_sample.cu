// C ABI of the measurement by shots (Sec. 3.4 shot objective, Sec. 3.6 final
// evaluation and its metrics) and of the SPSA-Adam optimiser (Sec. 3.4).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_state.h"
#include "philox.cuh"

using namespace qaoa;
using namespace qaoa::api;

namespace {

// One batch of shots on one measured state.
struct ShotSet {
    int state = 0;              // index into the measured states
    long long shots = 0;
    uint64_t seed = 0, stream = 0;
    const unsigned long long *rand = nullptr;  // device, or null (Philox)
    unsigned long long *idx = nullptr;         // device, or null
    int32_t *tval = nullptr;                   // device, or null
    long long *tsum = nullptr;                 // device, or null (zeroed here)
};

// CUDA-event timing of one launch group under options.profile (kind 6 =
// weights and scan, 7 = shots), read back by qaoa_profile_read.
struct SampleProf {
    qaoa_ctx c;
    int kind;
    double bytes;
    cudaEvent_t a = nullptr;
    static cudaEvent_t event(qaoa_ctx c) {
        if (!c->ev_free.empty()) {
            cudaEvent_t e = c->ev_free.back();
            c->ev_free.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    SampleProf(qaoa_ctx c_, int kind_, double bytes_) : c(c_), kind(kind_), bytes(bytes_) {
        if (c->opt.profile) {
            a = event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~SampleProf() {
        if (a) {
            cudaEvent_t b = event(c);
            cudaEventRecord(b, c->stream);
            c->pending.push_back({kind, -1, a, b, bytes});
        }
    }
};

// Measure: weights and prefix sums of every state once, then every shot set.
qaoa_status measure(qaoa_ctx c, const std::vector<ItemState> &st, bool fp64, const std::vector<ShotSet> &sets) {
    const size_t K = st.size();
    std::vector<size_t> off(K + 1, 0);
    int max_n = 1;
    for (size_t i = 0; i < K; ++i) {
        if (reinterpret_cast<uintptr_t>(st[i].amps) % 16)  // the weights pass reads 16-byte vectors
            return fail(QAOA_ERR_INVALID_ARG, "measure: state not 16-byte aligned");
        off[i + 1] = off[i] + (size_t)(sample_chunk_count(st[i].n) + sample_super_count(st[i].n) + 1);
        max_n = std::max(max_n, st[i].n);
    }
    QAOA_TRY(c->sample_scratch.ensure(off[K] * 8 + 64, &c->held, c->opt.memory_budget));
    unsigned long long *scr = c->sample_scratch.as<unsigned long long>();
    std::vector<SampleItem> items(K + sets.size());
    for (size_t i = 0; i < K; ++i) {
        SampleItem &it = items[i];
        std::memset(&it, 0, sizeof(it));
        it.amps = st[i].amps;
        it.n = st[i].n;
        it.chunk = scr + off[i];
        it.sup = it.chunk + sample_chunk_count(it.n);
        it.total = it.sup + sample_super_count(it.n);
    }
    long long max_shots = 0;
    for (size_t j = 0; j < sets.size(); ++j) {
        const ShotSet &s = sets[j];
        SampleItem &it = items[K + j];
        it = items[s.state];
        it.T = s.tval || s.tsum ? st[s.state].cost->T : nullptr;
        it.rand = s.rand;
        it.idx = s.idx;
        it.tval = s.tval;
        it.tsum = s.tsum;
        it.seed = s.seed;
        it.stream = s.stream;
        it.shots = s.shots;
        max_shots = std::max(max_shots, s.shots);
        if (s.tsum) CUDA_TRY(cudaMemsetAsync(s.tsum, 0, 8, c->stream));
    }
    QAOA_TRY(c->sample_items.ensure(items.size() * sizeof(SampleItem), &c->held, c->opt.memory_budget));
    SampleItem *dev = c->sample_items.as<SampleItem>();
    CUDA_TRY(cudaMemcpyAsync(dev, items.data(), items.size() * sizeof(SampleItem), cudaMemcpyHostToDevice, c->stream));
    {
        double wb = 0;
        for (size_t i = 0; i < K; ++i) wb += std::ldexp(fp64 ? 16.0 : 8.0, st[i].n);
        QAOA_TRY(c->status.ensure(16, &c->held, c->opt.memory_budget));
        CUDA_TRY(cudaMemsetAsync(c->status.p, 0, 4, c->stream));
        SampleProf prof(c, 6, wb);
        CUDA_TRY(launch_sample_weights(dev, (int)K, max_n, fp64, c->status.as<unsigned int>(), c->stream));
    }
    c->launches_total += 2;
    std::vector<unsigned long long> Q(K);
    unsigned int ws = 0;
    for (size_t i = 0; i < K; ++i)
        CUDA_TRY(cudaMemcpyAsync(&Q[i], items[i].total, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(&ws, c->status.p, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (ws & 4u) return fail(QAOA_ERR_RANGE, "a state holds a component of magnitude >= 2, infinite or NaN");
    for (size_t i = 0; i < K; ++i)
        if (Q[i] < (1ull << 58) || Q[i] > (1ull << 62))
            return fail(QAOA_ERR_RANGE, "state %zu: total probability %.6g outside [0.25, 4]", i,
                        std::ldexp((double)Q[i], -60));
    if (max_shots > 0) {
        QAOA_TRY(c->status.ensure(16, &c->held, c->opt.memory_budget));
        CUDA_TRY(cudaMemsetAsync(c->status.p, 0, 4, c->stream));
        double sb = 0;
        for (const ShotSet &x : sets)
            sb += (double)x.shots * std::ldexp(fp64 ? 16.0 : 8.0, std::min(st[x.state].n, 8));
        SampleProf prof(c, 7, sb);
        CUDA_TRY(launch_sample_shots(dev + K, (int)sets.size(), max_shots, fp64, c->status.as<unsigned int>(),
                                     c->stream));
        c->launches_total += 1;
        unsigned int hs = 0;
        CUDA_TRY(cudaMemcpyAsync(&hs, c->status.p, 4, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (hs) return fail(QAOA_ERR_CUDA, "shot search left its interval (status %u)", hs);
    }
    return QAOA_OK;
}

qaoa_status check_angles_host(int count, const double *gamma, const double *beta) {
    for (int i = 0; i < count; ++i)
        if (!std::isfinite(gamma[i]) || !std::isfinite(beta[i]))
            return fail(QAOA_ERR_INVALID_ARG, "non-finite angle at parameter %d", i);
    return QAOA_OK;
}

double fixed_to_cost(long long t, const qaoa_cost_s *cs) { return std::ldexp((double)t + (double)cs->fp.k_c, -cs->fp.s); }

// Mean cost of `shots` shots whose table values sum to tsum.
double mean_of(long long tsum, long long shots, const qaoa_cost_s *cs) {
    return std::ldexp((double)tsum + (double)shots * (double)cs->fp.k_c, -cs->fp.s) / (double)shots;
}

// ---- Algorithm 1 helpers ------------------------------------------------------

constexpr uint32_t TAG_RAND = 0x52414E44u, TAG_WARM = 0x57415250u;
constexpr uint64_t FINAL_STREAM = 0xF000000000000000ull;
constexpr uint64_t DEPTH_SEED_STEP = 0x9E3779B97F4A7C15ull;

double unit_of(uint32_t w0, uint32_t w1) {
    return (double)((((uint64_t)w1 << 32) | w0) >> 11) * 0x1p-53;
}

double start_uniform(uint64_t seed, uint32_t i, uint32_t j, uint32_t p) {
    const Philox4 o = philox4x32_10(i, j, p, TAG_RAND, (uint32_t)seed, (uint32_t)(seed >> 32));
    return unit_of(o.w[0], o.w[1]);
}

double start_normal(uint64_t seed, uint32_t i, uint32_t j, uint32_t p) {
    const Philox4 o = philox4x32_10(i, j, p, TAG_WARM, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = unit_of(o.w[0], o.w[1]), u2 = unit_of(o.w[2], o.w[3]);
    return std::sqrt(-2.0 * std::log(1.0 - u1)) * std::cos(2.0 * M_PI * u2);
}

// INTERP lifting of one angle sequence from depth p to p + 1.
std::vector<double> lift_interp(const std::vector<double> &v) {
    const int p = (int)v.size();
    std::vector<double> out(p + 1);
    for (int i = 1; i <= p + 1; ++i) {
        const double prev = i - 1 >= 1 ? v[i - 2] : 0.0, cur = i <= p ? v[i - 1] : 0.0;
        out[i - 1] = ((double)(i - 1) / p) * prev + ((double)(p - i + 1) / p) * cur;
    }
    return out;
}

// Lexicographic ranking key of a candidate (smaller is better).
std::vector<double> rank_key(const qaoa_sample_metrics &m, bool ref) {
    std::vector<double> k;
    if (ref) {
        k = {-(double)m.best_cost_matches_ref, -(double)m.best_index_matches_ref, -m.p_ref_cost, -m.p_ref_index};
    }
    k.insert(k.end(), {m.best_cost, -m.p_best_cost, -m.p_best_index, m.mean_cost});
    if (!ref) k.push_back(m.mean_cost - m.best_cost);
    return k;
}

int best_candidate(const std::vector<qaoa_sample_metrics> &ms, bool ref) {
    int best = 0;
    std::vector<double> kb = rank_key(ms[0], ref);
    for (size_t j = 1; j < ms.size(); ++j) {
        std::vector<double> kj = rank_key(ms[j], ref);
        if (kj < kb) {
            kb = kj;
            best = (int)j;
        }
    }
    return best;
}

// ---- distributed (TeleGate) circuit, Sec. 3.3 ------------------------------------

TgOp tg(int kind, int q0, int q1 = 0, double theta = 0.0) {
    TgOp o;
    o.kind = kind;
    o.q0 = q0;
    o.q1 = q1;
    o.midx = -1;
    o.c = (float)std::cos(theta);
    o.s = (float)std::sin(theta);
    return o;
}

// Remote CNOT (control a, target t) through the communication pair (cA = n,
// cB = n + 1): reset both, entangle them, couple cA to the control and
// measure it, couple cB to the target and measure it in the X basis, then
// X^m1 on the target and Z^m2 on the control.
void remote_cnot(std::vector<TgOp> &ops, int n, int a, int t, int *midx) {
    const int cA = n, cB = n + 1;
    ops.push_back(tg(TG_RESET, cA));
    ops.push_back(tg(TG_RESET, cB));
    ops.push_back(tg(TG_H, cA));
    ops.push_back(tg(TG_CNOT, cA, cB));
    ops.push_back(tg(TG_CNOT, a, cA));
    ops.push_back(tg(TG_MEASURE, cA, 0));
    ops.back().midx = (*midx)++;
    ops.push_back(tg(TG_CNOT, cB, t));
    ops.push_back(tg(TG_H, cB));
    ops.push_back(tg(TG_MEASURE, cB, 1));
    ops.back().midx = (*midx)++;
    ops.push_back(tg(TG_XIF, t, 0));
    ops.push_back(tg(TG_ZIF, a, 1));
}

// The distributed circuit in the 0/1 form of the objective, so that it equals
// exp(-i g F) exactly: each qubit's phase -g (l_i + sum_j b_ij / 2), each
// coupling CNOT(i, j), phase +g b_ij / 2 on j, CNOT(i, j) (remote when i and j
// sit on different QPUs), the constant as the global phase -g c0, then
// RX(2 beta) on every data qubit.
std::vector<TgOp> telegate_circuit(const Canonical &c, const int32_t *qpu_of, int p, const double *gamma,
                                   const double *beta, qaoa_telegate_counts *cnt) {
    const int n = c.n;
    std::vector<TgOp> ops;
    int midx = 0;
    int64_t loc = 0, cross = 0;
    for (int q = 0; q < n; ++q) ops.push_back(tg(TG_H, q));
    for (int l = 0; l < p; ++l) {
        const double g = gamma[l];
        ops.push_back(tg(TG_GPHASE, 0, 0, -g * c.c0));
        for (int i = 0; i < n; ++i) {
            double lin = 0.0;
            for (int j = 0; j < n; ++j)
                if (j != i) lin += c.b[(size_t)std::min(i, j) * n + std::max(i, j)];
            ops.push_back(tg(TG_PHASE, i, 0, -g * (c.ell[i] + 0.5 * lin)));
        }
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                const double bij = c.b[(size_t)i * n + j];
                if (bij == 0.0) continue;
                const bool local = qpu_of[i] == qpu_of[j];
                for (int rep = 0; rep < 2; ++rep) {
                    if (local)
                        ops.push_back(tg(TG_CNOT, i, j));
                    else
                        remote_cnot(ops, n, i, j, &midx);
                    if (rep == 0) ops.push_back(tg(TG_PHASE, j, 0, 0.5 * g * bij));
                }
                if (local) ++loc; else ++cross;
            }
        for (int q = 0; q < n; ++q) ops.push_back(tg(TG_RX, q, 0, beta[l]));
    }
    if (cnt) {
        cnt->ops = (int64_t)ops.size();
        cnt->local_zz = loc;
        cnt->cross_zz = cross;
        cnt->remote_cx = 2 * cross;
        cnt->measurements = 4 * cross;
        cnt->resets = 4 * cross;
        cnt->feedforward = 4 * cross;
    }
    return ops;
}

}  // namespace

extern "C" {

qaoa_status qaoa_state_from_host(qaoa_ctx c, int n, int fp64, const void *amps, qaoa_state *out) {
    if (!c || !amps || !out) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    if (n < 1 || n > 33) return fail(QAOA_ERR_INVALID_ARG, "n=%d out of range [1, 33]", n);
    if (fp64 && n > SMALL_MAXN) return fail(QAOA_ERR_INVALID_ARG, "complex128 states are limited to n <= 12");
    CUDA_TRY(cudaSetDevice(c->device));
    std::unique_ptr<qaoa_state_s> s(new qaoa_state_s());
    s->n = n;
    s->fp64 = fp64 != 0;
    s->device = c->device;
    const size_t bytes = ((size_t)1 << n) * (fp64 ? 16 : 8);
    cudaError_t e = ctx_malloc(c, &s->amps, bytes);
    if (e) {
        return fail(QAOA_ERR_OUT_OF_MEMORY, "state (%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    CUDA_TRY(cudaMemcpyAsync(s->amps, amps, bytes, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    *out = s.release();
    return QAOA_OK;
}

qaoa_status qaoa_sample(qaoa_ctx c, qaoa_cost cost, qaoa_state s, int64_t shots, uint64_t seed, uint64_t stream,
                        const uint64_t *rand, uint64_t *idx, double *cost_out, double *mean_cost) {
    if (!c || !s) return fail(QAOA_ERR_INVALID_ARG, "null context or state");
    if (shots < 1 || shots > (int64_t)1 << 34) return fail(QAOA_ERR_INVALID_ARG, "shots=%lld not in [1, 2^34]", (long long)shots);
    const bool want_cost = cost_out || mean_cost;
    if (want_cost && !cost) return fail(QAOA_ERR_INVALID_ARG, "costs of the shots need a cost handle");
    if (cost && cost->n != s->n) return fail(QAOA_ERR_INVALID_ARG, "state and cost differ in n");
    CUDA_TRY(cudaSetDevice(c->device));
    const size_t S = (size_t)shots;
    const size_t b_rand = rand ? S * 8 : 0, b_idx = idx ? S * 8 : 0, b_tv = cost_out ? S * 4 : 0;
    QAOA_TRY(c->sample_out.ensure(b_rand + b_idx + b_tv + 64, &c->held, c->opt.memory_budget));
    char *m = c->sample_out.as<char>();
    ShotSet set;
    set.shots = shots;
    set.seed = seed;
    set.stream = stream;
    if (rand) {
        CUDA_TRY(cudaMemcpyAsync(m, rand, b_rand, cudaMemcpyHostToDevice, c->stream));
        set.rand = reinterpret_cast<const unsigned long long *>(m);
    }
    if (idx) set.idx = reinterpret_cast<unsigned long long *>(m + b_rand);
    if (cost_out) set.tval = reinterpret_cast<int32_t *>(m + b_rand + b_idx);
    long long *tsum = reinterpret_cast<long long *>(m + ((b_rand + b_idx + b_tv + 15) & ~(size_t)15));
    if (mean_cost) set.tsum = tsum;
    std::vector<ItemState> st{ItemState{s->amps, s->n, cost}};
    QAOA_TRY(measure(c, st, s->fp64, {set}));
    std::vector<int32_t> tv(cost_out ? S : 0);
    long long hsum = 0;
    if (idx) CUDA_TRY(cudaMemcpyAsync(idx, set.idx, b_idx, cudaMemcpyDeviceToHost, c->stream));
    if (cost_out) CUDA_TRY(cudaMemcpyAsync(tv.data(), set.tval, b_tv, cudaMemcpyDeviceToHost, c->stream));
    if (mean_cost) CUDA_TRY(cudaMemcpyAsync(&hsum, tsum, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (cost_out)
        for (size_t i = 0; i < S; ++i) cost_out[i] = fixed_to_cost(tv[i], cost);
    if (mean_cost) *mean_cost = mean_of(hsum, shots, cost);
    return QAOA_OK;
}

qaoa_status qaoa_sample_stats(int64_t shots, const uint64_t *idx, const double *cost, double margin, int elite,
                              uint64_t *elite_idx, double *elite_cost, int64_t *elite_count, int has_ref,
                              double ref_cost, uint64_t ref_index, double tol, qaoa_sample_metrics *out) {
    if (shots < 1 || !idx || !cost || !out) return fail(QAOA_ERR_INVALID_ARG, "null argument or shots < 1");
    if (elite < 0 || (elite > 0 && (!elite_idx || !elite_cost || !elite_count)))
        return fail(QAOA_ERR_INVALID_ARG, "elite=%d needs elite_idx, elite_cost and elite_count", elite);
    if (!(margin >= 0.0) || !(tol >= 0.0)) return fail(QAOA_ERR_INVALID_ARG, "margin and tol must be >= 0");
    // decoded distribution: distinct indices with their counts and costs
    std::vector<std::pair<uint64_t, int64_t>> order((size_t)shots);
    for (int64_t s = 0; s < shots; ++s) order[s] = {idx[s], s};
    std::sort(order.begin(), order.end());
    struct Entry {
        uint64_t x;
        double c;
        int64_t count;
    };
    std::vector<Entry> d;
    for (size_t i = 0; i < order.size(); ++i) {
        if (d.empty() || d.back().x != order[i].first) d.push_back({order[i].first, cost[order[i].second], 0});
        d.back().count += 1;
    }
    const double S = (double)shots;
    qaoa_sample_metrics m;
    std::memset(&m, 0, sizeof(m));
    m.shots = shots;
    m.distinct = (int64_t)d.size();
    double sum = 0.0;
    m.best_cost = d[0].c;
    m.best_index = d[0].x;
    for (const Entry &e : d) {
        sum += e.c * (double)e.count;
        if (e.c < m.best_cost) {
            m.best_cost = e.c;
            m.best_index = e.x;
        }
    }
    m.mean_cost = sum / S;
    int64_t n_best_cost = 0, n_low = 0, n_best_idx = 0, n_ref_cost = 0, n_ref_idx = 0;
    for (const Entry &e : d) {
        if (e.c == m.best_cost) n_best_cost += e.count;
        if (e.c <= m.best_cost + margin) n_low += e.count;
        if (e.x == m.best_index) n_best_idx = e.count;
        if (has_ref && std::fabs(e.c - ref_cost) <= tol) n_ref_cost += e.count;
        if (has_ref && e.x == ref_index) n_ref_idx = e.count;
    }
    m.p_best_index = (double)n_best_idx / S;
    m.p_best_cost = (double)n_best_cost / S;
    m.low_cost_mass = (double)n_low / S;
    if (has_ref) {
        m.p_ref_cost = (double)n_ref_cost / S;
        m.p_ref_index = (double)n_ref_idx / S;
        m.best_cost_matches_ref = std::fabs(m.best_cost - ref_cost) <= tol ? 1 : 0;
        m.best_index_matches_ref = m.best_index == ref_index ? 1 : 0;
    } else {
        m.p_ref_cost = m.p_ref_index = std::nan("");
        m.best_cost_matches_ref = m.best_index_matches_ref = -1;
    }
    // elite set: count descending, cost ascending, index ascending
    const size_t ne = std::min((size_t)elite, d.size());
    std::partial_sort(d.begin(), d.begin() + ne, d.end(), [](const Entry &a, const Entry &b) {
        if (a.count != b.count) return a.count > b.count;
        if (a.c != b.c) return a.c < b.c;
        return a.x < b.x;
    });
    for (int i = 0; i < elite; ++i) {
        const bool have = (size_t)i < ne;
        elite_idx[i] = have ? d[i].x : ~0ull;
        elite_cost[i] = have ? d[i].c : std::nan("");
        elite_count[i] = have ? d[i].count : 0;
    }
    *out = m;
    return QAOA_OK;
}

qaoa_status qaoa_optimize_spsa(qaoa_ctx c, int nq, const qaoa_cost *costs, const int32_t *item_cost, int B, int p,
                               double *gamma, double *beta, const qaoa_spsa_options *sopt, double *history,
                               double *final_expect) {
    if (!c || !costs || nq < 1 || B < 1 || !gamma || !beta || !sopt)
        return fail(QAOA_ERR_INVALID_ARG, "bad SPSA arguments");
    if (p < 1 || p > SMALL_MAXP) return fail(QAOA_ERR_INVALID_ARG, "p=%d not in [1, %d]", p, SMALL_MAXP);
    if (B >= (1 << 22)) return fail(QAOA_ERR_INVALID_ARG, "B=%d >= 2^22", B);
    qaoa_spsa_options o = *sopt;
    for (int k = 0; k < 6; ++k)
        if (o.reserved[k]) return fail(QAOA_ERR_INVALID_ARG, "reserved SPSA option field %d is not zero", k);
    if (o.lr == 0) o.lr = 0.01;
    if (o.beta1 == 0) o.beta1 = 0.9;
    if (o.beta2 == 0) o.beta2 = 0.999;
    if (o.eps == 0) o.eps = 1e-8;
    if (o.c == 0) o.c = 0.1;
    if (o.averaging == 0) o.averaging = 1;
    if (o.iterations < 1 || o.shots < 0 || o.averaging < 1 || o.averaging > 512 || !(o.c > 0) ||
        !(o.c_decay >= 0) || !(o.lr > 0) || !(o.eps > 0) || !(o.beta1 >= 0 && o.beta1 < 1) ||
        !(o.beta2 >= 0 && o.beta2 < 1))
        return fail(QAOA_ERR_INVALID_ARG, "SPSA options out of range");
    QAOA_TRY(check_angles_host(p * B, gamma, beta));
    CUDA_TRY(cudaSetDevice(c->device));
    const int P2 = 2 * p;
    std::vector<double> x((size_t)B * P2), m((size_t)B * P2, 0.0), v((size_t)B * P2, 0.0);
    for (int b = 0; b < B; ++b)
        for (int l = 0; l < p; ++l) {
            x[(size_t)b * P2 + 2 * l] = gamma[(size_t)b * p + l];
            x[(size_t)b * P2 + 2 * l + 1] = beta[(size_t)b * p + l];
        }
    std::vector<int32_t> ic2(2 * (size_t)B);
    for (int b = 0; b < B; ++b) ic2[2 * b] = ic2[2 * b + 1] = item_cost ? item_cost[b] : 0;
    std::vector<double> g2((size_t)2 * B * p), b2((size_t)2 * B * p), J(2 * (size_t)B), D((size_t)B * P2);
    const int A = o.averaging;
    QAOA_TRY(c->sample_out.ensure((size_t)2 * B * A * 8 + 64, &c->held, c->opt.memory_budget));
    long long *tsum = c->sample_out.as<long long>();
    std::vector<long long> hsum((size_t)2 * B * A);
    for (int k = 0; k < o.iterations; ++k) {
        const double ck = o.c / std::pow((double)(k + 1), o.c_decay);
        for (int b = 0; b < B; ++b)
            for (int i = 0; i < P2; ++i) {
                const double d = spsa_sign(o.seed, (uint32_t)k, (uint32_t)b, (uint32_t)i);
                D[(size_t)b * P2 + i] = d;
                const double xi = x[(size_t)b * P2 + i];
                const int l = i / 2;
                double *dst0 = (i & 1) ? b2.data() : g2.data();
                dst0[(size_t)(2 * b) * p + l] = xi + ck * d;
                dst0[(size_t)(2 * b + 1) * p + l] = xi - ck * d;
            }
        if (o.shots == 0) {
            QAOA_TRY(run_batch(c, nq, costs, ic2.data(), 2 * B, p, g2.data(), b2.data(), J.data(), nullptr, nullptr,
                               nullptr));
        } else {
            std::vector<ItemState> st;
            QAOA_TRY(run_batch(c, nq, costs, ic2.data(), 2 * B, p, g2.data(), b2.data(), J.data(), nullptr, nullptr,
                               &st));
            std::vector<ShotSet> sets((size_t)2 * B * A);
            for (int b = 0; b < B; ++b)
                for (int w = 0; w < 2; ++w)
                    for (int a = 0; a < A; ++a) {
                        ShotSet &s = sets[((size_t)(2 * b + w)) * A + a];
                        s.state = 2 * b + w;
                        s.shots = o.shots;
                        s.seed = o.seed;
                        s.stream = ((uint64_t)k << 32) | ((uint64_t)b << 10) | ((uint64_t)w << 9) | (uint64_t)a;
                        s.tsum = tsum + ((size_t)(2 * b + w)) * A + a;
                    }
            QAOA_TRY(measure(c, st, false, sets));
            CUDA_TRY(cudaMemcpyAsync(hsum.data(), tsum, hsum.size() * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            for (int j = 0; j < 2 * B; ++j) {
                long long t = 0;
                for (int a = 0; a < A; ++a) t += hsum[(size_t)j * A + a];
                J[j] = mean_of(t, (long long)o.shots * A, st[j].cost);
            }
        }
        const double t1 = (double)(k + 1);
        const double bc1 = 1.0 - std::pow(o.beta1, t1), bc2 = 1.0 - std::pow(o.beta2, t1);
        for (int b = 0; b < B; ++b) {
            const double jp = J[2 * b], jm = J[2 * b + 1];
            if (history) {
                history[((size_t)k * B + b) * 2] = jp;
                history[((size_t)k * B + b) * 2 + 1] = jm;
            }
            for (int i = 0; i < P2; ++i) {
                const size_t q = (size_t)b * P2 + i;
                const double g = (jp - jm) / (2.0 * ck * D[q]);
                m[q] = o.beta1 * m[q] + (1.0 - o.beta1) * g;
                v[q] = o.beta2 * v[q] + (1.0 - o.beta2) * g * g;
                x[q] = x[q] - o.lr * (m[q] / bc1) / (std::sqrt(v[q] / bc2) + o.eps);
            }
        }
    }
    for (int b = 0; b < B; ++b)
        for (int l = 0; l < p; ++l) {
            gamma[(size_t)b * p + l] = x[(size_t)b * P2 + 2 * l];
            beta[(size_t)b * p + l] = x[(size_t)b * P2 + 2 * l + 1];
        }
    if (final_expect)
        QAOA_TRY(run_batch(c, nq, costs, item_cost, B, p, gamma, beta, final_expect, nullptr, nullptr, nullptr));
    return QAOA_OK;
}

qaoa_status qaoa_solve(qaoa_ctx c, qaoa_cost cost, const qaoa_solve_options *sopt, double *gamma, double *beta,
                       int elite, uint64_t *elite_idx, double *elite_cost, int64_t *elite_count,
                       qaoa_sample_metrics *depth_metrics, qaoa_solve_result *out) {
    if (!c || !cost || !sopt || !gamma || !beta || !out) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    qaoa_solve_options o = *sopt;
    for (int k = 0; k < 8; ++k)
        if (o.reserved[k]) return fail(QAOA_ERR_INVALID_ARG, "reserved solve option field %d is not zero", k);
    if (o.lr == 0) o.lr = 0.01;
    if (o.beta1 == 0) o.beta1 = 0.9;
    if (o.beta2 == 0) o.beta2 = 0.999;
    if (o.eps == 0) o.eps = 1e-8;
    if (o.c == 0) o.c = 0.1;
    if (o.averaging == 0) o.averaging = 1;
    if (o.p_max < 1 || o.p_max > SMALL_MAXP || (o.optimizer != 0 && o.optimizer != 1) || o.iterations < 1 ||
        o.shots < 0 || o.averaging < 1 || o.random_starts < 1 || o.warm_perturb < 0 || o.final_shots < 1 ||
        (o.include_warm != 0 && o.include_warm != 1) || !(o.warm_sigma >= 0) || !std::isfinite(o.gamma_range) ||
        !std::isfinite(o.beta_range) || !(o.margin >= 0) || !(o.tol >= 0))
        return fail(QAOA_ERR_INVALID_ARG, "solve options out of range");
    if (elite < 0 || (elite > 0 && (!elite_idx || !elite_cost || !elite_count)))
        return fail(QAOA_ERR_INVALID_ARG, "elite=%d needs elite_idx, elite_cost and elite_count", elite);
    if (c->opt.state_fp64) return fail(QAOA_ERR_INVALID_ARG, "the search runs in complex64 only");
    CUDA_TRY(cudaSetDevice(c->device));
    const bool ref = o.use_reference != 0;
    const double ref_cost = fixed_to_cost(cost->minval, cost);
    const uint64_t ref_index = cost->argmin;
    const long long S = o.final_shots;
    struct Rep {
        int p;
        std::vector<double> g, b;
        qaoa_sample_metrics m;
        std::vector<uint64_t> idx;
        std::vector<double> cst;
        double E;
    };
    std::vector<Rep> reps;
    std::vector<double> prev_g, prev_b;
    int runs = 0;
    for (int p = 1; p <= o.p_max; ++p) {
        // initial points: lifted best, its perturbations, random points
        std::vector<std::vector<double>> X;
        uint32_t j = 0;
        if (!prev_g.empty()) {
            const std::vector<double> lg = lift_interp(prev_g), lb = lift_interp(prev_b);
            std::vector<double> lifted(2 * p);
            for (int l = 0; l < p; ++l) {
                lifted[2 * l] = lg[l];
                lifted[2 * l + 1] = lb[l];
            }
            if (o.include_warm) {
                X.push_back(lifted);
                ++j;
            }
            for (int r = 0; r < o.warm_perturb; ++r, ++j) {
                std::vector<double> x = lifted;
                for (int i = 0; i < 2 * p; ++i) x[i] += o.warm_sigma * start_normal(o.seed, (uint32_t)i, j, (uint32_t)p);
                X.push_back(x);
            }
        }
        for (int r = 0; r < o.random_starts; ++r, ++j) {
            std::vector<double> x(2 * p);
            for (int i = 0; i < 2 * p; ++i)
                x[i] = ((i & 1) ? o.beta_range : o.gamma_range) * start_uniform(o.seed, (uint32_t)i, j, (uint32_t)p);
            X.push_back(x);
        }
        const int B = (int)X.size();
        std::vector<double> g((size_t)B * p), b((size_t)B * p);
        for (int k = 0; k < B; ++k)
            for (int l = 0; l < p; ++l) {
                g[(size_t)k * p + l] = X[k][2 * l];
                b[(size_t)k * p + l] = X[k][2 * l + 1];
            }
        // optimise every start of this depth as one batch
        if (o.optimizer == 0) {
            qaoa_spsa_options so;
            std::memset(&so, 0, sizeof(so));
            so.lr = o.lr;
            so.beta1 = o.beta1;
            so.beta2 = o.beta2;
            so.eps = o.eps;
            so.c = o.c;
            so.c_decay = o.c_decay;
            so.iterations = o.iterations;
            so.shots = o.shots;
            so.averaging = o.averaging;
            so.seed = o.seed + (uint64_t)p * DEPTH_SEED_STEP;
            QAOA_TRY(qaoa_optimize_spsa(c, 1, &cost, nullptr, B, p, g.data(), b.data(), &so, nullptr, nullptr));
        } else {
            qaoa_adam_options ao;
            std::memset(&ao, 0, sizeof(ao));
            ao.lr = o.lr;
            ao.beta1 = o.beta1;
            ao.beta2 = o.beta2;
            ao.eps = o.eps;
            ao.iterations = o.iterations;
            QAOA_TRY(qaoa_optimize_adam(c, 1, &cost, nullptr, B, p, g.data(), b.data(), &ao, nullptr, nullptr));
        }
        runs += B;
        // final shot-based evaluation of every candidate
        std::vector<ItemState> st;
        std::vector<double> E(B);
        QAOA_TRY(run_batch(c, 1, &cost, nullptr, B, p, g.data(), b.data(), E.data(), nullptr, nullptr, &st));
        QAOA_TRY(c->sample_out.ensure((size_t)B * S * 12 + 64, &c->held, c->opt.memory_budget));
        unsigned long long *didx = c->sample_out.as<unsigned long long>();
        int32_t *dtv = reinterpret_cast<int32_t *>(didx + (size_t)B * S);
        std::vector<ShotSet> sets(B);
        for (int k = 0; k < B; ++k) {
            sets[k].state = k;
            sets[k].shots = S;
            sets[k].seed = o.seed;
            sets[k].stream = FINAL_STREAM + ((uint64_t)p << 32) + (uint64_t)k;
            sets[k].idx = didx + (size_t)k * S;
            sets[k].tval = dtv + (size_t)k * S;
        }
        QAOA_TRY(measure(c, st, false, sets));
        std::vector<uint64_t> hidx((size_t)B * S);
        std::vector<int32_t> htv((size_t)B * S);
        CUDA_TRY(cudaMemcpyAsync(hidx.data(), didx, hidx.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(htv.data(), dtv, htv.size() * 4, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        std::vector<qaoa_sample_metrics> ms(B);
        std::vector<double> hc((size_t)B * S);
        for (size_t t = 0; t < hc.size(); ++t) hc[t] = fixed_to_cost(htv[t], cost);
        for (int k = 0; k < B; ++k)
            QAOA_TRY(qaoa_sample_stats(S, hidx.data() + (size_t)k * S, hc.data() + (size_t)k * S, o.margin, 0,
                                       nullptr, nullptr, nullptr, ref ? 1 : 0, ref_cost, ref_index, o.tol, &ms[k]));
        const int kb = best_candidate(ms, ref);
        Rep r;
        r.p = p;
        r.g.assign(g.begin() + (size_t)kb * p, g.begin() + (size_t)(kb + 1) * p);
        r.b.assign(b.begin() + (size_t)kb * p, b.begin() + (size_t)(kb + 1) * p);
        r.m = ms[kb];
        r.idx.assign(hidx.begin() + (size_t)kb * S, hidx.begin() + (size_t)(kb + 1) * S);
        r.cst.assign(hc.begin() + (size_t)kb * S, hc.begin() + (size_t)(kb + 1) * S);
        r.E = E[kb];
        prev_g = r.g;
        prev_b = r.b;
        if (depth_metrics) depth_metrics[p - 1] = r.m;
        reps.push_back(std::move(r));
    }
    std::vector<qaoa_sample_metrics> rm;
    for (const Rep &r : reps) rm.push_back(r.m);
    const Rep &best = reps[best_candidate(rm, ref)];
    for (int l = 0; l < o.p_max; ++l) {
        gamma[l] = l < best.p ? best.g[l] : 0.0;
        beta[l] = l < best.p ? best.b[l] : 0.0;
    }
    qaoa_sample_metrics m;
    QAOA_TRY(qaoa_sample_stats(S, best.idx.data(), best.cst.data(), o.margin, elite, elite_idx, elite_cost,
                               elite_count, ref ? 1 : 0, ref_cost, ref_index, o.tol, &m));
    out->best_p = best.p;
    out->runs = runs;
    out->expect = best.E;
    out->metrics = m;
    return QAOA_OK;
}

qaoa_status qaoa_telegate_simulate(qaoa_ctx c, qaoa_cost cost, const int32_t *qpu_of, int p, const double *gamma,
                                   const double *beta, int trajectories, uint64_t seed, double *fidelity,
                                   float *amps, qaoa_telegate_counts *counts) {
    if (!c || !cost || !qpu_of || !fidelity) return fail(QAOA_ERR_INVALID_ARG, "null argument");
    const int n = cost->n;
    if (n > SMALL_MAXN) return fail(QAOA_ERR_INVALID_ARG, "n=%d: the circuit simulation holds n + 2 <= 14 qubits", n);
    if (p < 1 || p > SMALL_MAXP) return fail(QAOA_ERR_INVALID_ARG, "p=%d not in [1, %d]", p, SMALL_MAXP);
    if (trajectories < 1 || trajectories > (1 << 20))
        return fail(QAOA_ERR_INVALID_ARG, "trajectories=%d not in [1, 2^20]", trajectories);
    if (c->opt.state_fp64) return fail(QAOA_ERR_INVALID_ARG, "the circuit simulation runs in complex64");
    QAOA_TRY(check_angles_host(p, gamma, beta));
    for (int i = 0; i < n; ++i)
        if (qpu_of[i] < 0) return fail(QAOA_ERR_INVALID_ARG, "variable %d has no QPU", i);
    CUDA_TRY(cudaSetDevice(c->device));
    qaoa_telegate_counts cnt;
    std::memset(&cnt, 0, sizeof(cnt));
    const std::vector<TgOp> ops = telegate_circuit(cost->can, qpu_of, p, gamma, beta, &cnt);
    // the monolithic state of the same angles, from the fused path
    qaoa_state mono = nullptr;
    QAOA_TRY(qaoa_forward(c, cost, p, gamma, beta, &mono));
    std::unique_ptr<qaoa_state_s> mono_guard(mono);
    const size_t D = (size_t)1 << n, T = (size_t)trajectories;
    const size_t b_ops = ops.size() * sizeof(TgOp), b_fid = T * 8, b_amp = amps ? T * D * 8 : 0;
    QAOA_TRY(c->sample_out.ensure(b_ops + b_fid + b_amp + 64, &c->held, c->opt.memory_budget));
    char *m = c->sample_out.as<char>();
    TgOp *dops = reinterpret_cast<TgOp *>(m);
    double *dfid = reinterpret_cast<double *>(m + ((b_ops + 15) & ~(size_t)15));
    float2 *damp = amps ? reinterpret_cast<float2 *>(reinterpret_cast<char *>(dfid) + b_fid) : nullptr;
    CUDA_TRY(cudaMemcpyAsync(dops, ops.data(), b_ops, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(launch_telegate(dops, (int)ops.size(), n, seed, 0, trajectories, damp,
                             static_cast<const float2 *>(mono->amps), dfid, c->stream));
    c->launches_total += 1;
    CUDA_TRY(cudaMemcpyAsync(fidelity, dfid, b_fid, cudaMemcpyDeviceToHost, c->stream));
    if (amps) CUDA_TRY(cudaMemcpyAsync(amps, damp, b_amp, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (counts) *counts = cnt;
    return QAOA_OK;
}

qaoa_status qaoa_peak_probe(qaoa_ctx c, int kind, double *ops_per_s, double *flops_per_s) {
    if (!c || kind < 0 || kind > 3) return fail(QAOA_ERR_INVALID_ARG, "bad context or kind %d", kind);
    CUDA_TRY(cudaSetDevice(c->device));
    QAOA_TRY(c->misc.ensure(4096, &c->held, c->opt.memory_budget));
    const int blocks = c->num_sms * 8;
    const int iters = kind == 2 ? 2048 : kind == 3 ? 8192 : 32768;
    float *out = c->misc.as<float>();
    CUDA_TRY(launch_peak(kind, blocks, iters, out, c->stream));  // warm-up
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const int reps = 3;
    cudaError_t err = cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && !err; ++r) err = launch_peak(kind, blocks, iters, out, c->stream);
    if (!err) err = cudaEventRecord(e1, c->stream);
    if (!err) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (!err) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_TRY(err);
    c->launches_total += 1 + reps;
    const double ops = peak_ops_per_launch(blocks, iters) * reps / (ms / 1e3);
    if (ops_per_s) *ops_per_s = ops;
    if (flops_per_s) *flops_per_s = kind == 1 ? 4.0 * ops : kind == 3 ? ops : 2.0 * ops;
    return QAOA_OK;
}

qaoa_status qaoa_wait_probe(qaoa_ctx c) {
    if (!c) return fail(QAOA_ERR_INVALID_ARG, "null context");
    CUDA_TRY(cudaSetDevice(c->device));
    QAOA_TRY(c->status.ensure(16, &c->held, c->opt.memory_budget));
    CUDA_TRY(cudaMemsetAsync(c->status.p, 0, 4, c->stream));
    CUDA_TRY(launch_wait_probe(c->status.as<unsigned int>(), c->stream));
    c->launches_total += 1;
    unsigned int hs = 0;
    CUDA_TRY(cudaMemcpyAsync(&hs, c->status.p, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(cudaMemsetAsync(c->status.p, 0, 4, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (hs) return fail(QAOA_ERR_TIMEOUT, "the probe's bounded wait expired, as it must");
    return QAOA_OK;
}

}  // extern "C"
