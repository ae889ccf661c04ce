// Host-side logic of the QAOA library: errors, canonical QUBO (Sec. 2.1),
// fixed-point objective, exact phase constants, and the DQAOA allocation and
// coupling classification (Sec. 3.1, Sec. 3.2).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "qaoa_internal.h"

namespace qaoa {

static thread_local char g_err[512] = "no error";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

qaoa_status fail(qaoa_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

const char *last_error() { return g_err; }

// ---- Sec. 2.1 -----------------------------------------------------------------

static double coef(const void *p, qaoa_dtype dt, size_t k) {
    switch (dt) {
        case QAOA_I32: return (double)((const int32_t *)p)[k];
        case QAOA_F32: return (double)((const float *)p)[k];
        default: return ((const double *)p)[k];
    }
}

qaoa_status canonicalize(const qaoa_qubo *q, Canonical *out) {
    if (!q || !out) return fail(QAOA_ERR_INVALID_ARG, "null qubo");
    const int n = q->n;
    if (n < 1 || n > 33) return fail(QAOA_ERR_INVALID_ARG, "n=%d out of range [1,33]", n);
    if (!q->H) return fail(QAOA_ERR_INVALID_ARG, "H is null");
    if (q->dtype != QAOA_I32 && q->dtype != QAOA_F32 && q->dtype != QAOA_F64)
        return fail(QAOA_ERR_INVALID_ARG, "unknown dtype %d", (int)q->dtype);
    if (!std::isfinite(q->c0)) return fail(QAOA_ERR_INVALID_ARG, "c0 is not finite");
    out->n = n;
    out->c0 = q->c0;
    out->ell.assign(n, 0.0);
    out->b.assign((size_t)n * n, 0.0);
    bool integer = (q->c0 == std::floor(q->c0));
    for (int i = 0; i < n; ++i) {
        double fi = q->f ? coef(q->f, q->dtype, i) : 0.0;
        double v = fi + coef(q->H, q->dtype, (size_t)i * n + i);  // l_i = f_i + H_ii
        if (!std::isfinite(v)) return fail(QAOA_ERR_INVALID_ARG, "non-finite coefficient l_%d", i);
        out->ell[i] = v;
        integer = integer && v == std::floor(v);
    }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double v = coef(q->H, q->dtype, (size_t)i * n + j) + coef(q->H, q->dtype, (size_t)j * n + i);
            if (!std::isfinite(v)) return fail(QAOA_ERR_INVALID_ARG, "non-finite coupling b_%d%d", i, j);
            out->b[(size_t)i * n + j] = v;  // b_ij = H_ij + H_ji
            integer = integer && v == std::floor(v);
        }
    out->integer = (q->dtype == QAOA_I32) || integer;
    return QAOA_OK;
}

// Integer bounds of F 2^s = c0_q + sum ell_q z + sum b_q z z over all z.
static void int_bounds(const FixedPoint &fp, int n, int64_t *lo, int64_t *hi) {
    __int128 L = fp.c0_q, H = fp.c0_q;
    for (int i = 0; i < n; ++i) {
        if (fp.ell_q[i] > 0) H += fp.ell_q[i]; else L += fp.ell_q[i];
        for (int j = i + 1; j < n; ++j) {
            int64_t v = fp.b_q[(size_t)i * n + j];
            if (v > 0) H += v; else L += v;
        }
    }
    const __int128 cap = (__int128)1 << 62;
    if (L < -cap) L = -cap;
    if (H > cap) H = cap;
    *lo = (int64_t)L;
    *hi = (int64_t)H;
}

static bool quantize_at(const Canonical &c, int s, FixedPoint *fp) {
    const int n = c.n;
    const double sc = std::ldexp(1.0, s);
    auto q = [&](double v, int64_t *o) {
        double r = std::nearbyint(v * sc);
        if (!(std::fabs(r) < 4.0e18)) return false;
        *o = (int64_t)r;
        return true;
    };
    fp->s = s;
    fp->ell_q.assign(n, 0);
    fp->b_q.assign((size_t)n * n, 0);
    if (!q(c.c0, &fp->c0_q)) return false;
    for (int i = 0; i < n; ++i) {
        if (!q(c.ell[i], &fp->ell_q[i])) return false;
        for (int j = i + 1; j < n; ++j)
            if (!q(c.b[(size_t)i * n + j], &fp->b_q[(size_t)i * n + j])) return false;
    }
    int64_t lo, hi;
    int_bounds(*fp, n, &lo, &hi);
    fp->lo_bound = lo;
    fp->hi_bound = hi;
    // centre the table: T = F 2^s - k_c must satisfy -2^31 <= T <= 2^31 - 1
    int64_t k = (int64_t)(((__int128)lo + hi) / 2);
    fp->k_c = k;
    return (__int128)hi - k <= 2147483647 && (__int128)lo - k >= -2147483648LL;
}

qaoa_status make_fixed_point(const Canonical &c, FixedPoint *out) {
    if (c.integer) {
        if (!quantize_at(c, 0, out))
            return fail(QAOA_ERR_RANGE, "integer objective range exceeds the 32-bit table (|F| span >= 2^32)");
        return QAOA_OK;
    }
    double R = 0.0;  // the constant term only shifts k_c
    for (int i = 0; i < c.n; ++i) {
        R += std::fabs(c.ell[i]);
        for (int j = i + 1; j < c.n; ++j) R += std::fabs(c.b[(size_t)i * c.n + j]);
    }
    int s = 40;
    if (R > 0) {
        s = (int)std::floor(std::log2(2147483647.0 / (R / 2.0 + c.n * c.n + 4.0)));
        if (s > 40) s = 40;
    }
    for (int tries = 0; tries < 200; ++tries, --s) {
        if (s < -60) break;
        if (quantize_at(c, s, out)) return QAOA_OK;
    }
    return fail(QAOA_ERR_RANGE, "could not fit the real objective into a 32-bit fixed-point table");
}

// ---- Sec. 3.1, Sec. 3.2 -----------------------------------------------------------

qaoa_status partition(int n, int M, const int32_t *caps, const int32_t *manual, int32_t *qpu_of) {
    if (n < 1 || M < 1 || M > n || !qpu_of)
        return fail(QAOA_ERR_INVALID_ARG, "partition: bad n=%d or M=%d", n, M);
    std::vector<int32_t> c(M);
    for (int m = 0; m < M; ++m) c[m] = caps ? caps[m] : (n / M + (m < n % M ? 1 : 0));
    for (int m = 0; m < M; ++m)
        if (c[m] < 0) return fail(QAOA_ERR_ALLOCATION, "negative capacity on QPU %d", m);
    if (manual) {
        for (int i = 0; i < n; ++i) qpu_of[i] = manual[i];
    } else {
        // contiguous: QPU 0 takes the first c_0 variables, then QPU 1, ...
        int m = 0, used = 0;
        for (int i = 0; i < n; ++i) {
            while (m < M && used >= c[m]) { ++m; used = 0; }
            if (m >= M) return fail(QAOA_ERR_ALLOCATION, "total capacity %d < n=%d", i, n);
            qpu_of[i] = m;
            ++used;
        }
    }
    // validate_allocation: each variable once (by construction of qpu_of), in range,
    // no capacity exceeded, every QPU used
    std::vector<int> cnt(M, 0);
    for (int i = 0; i < n; ++i) {
        if (qpu_of[i] < 0 || qpu_of[i] >= M)
            return fail(QAOA_ERR_ALLOCATION, "variable %d assigned to unknown QPU %d", i, qpu_of[i]);
        ++cnt[qpu_of[i]];
    }
    for (int m = 0; m < M; ++m) {
        if (cnt[m] > c[m]) return fail(QAOA_ERR_ALLOCATION, "QPU %d holds %d > capacity %d", m, cnt[m], c[m]);
        if (cnt[m] == 0) return fail(QAOA_ERR_ALLOCATION, "QPU %d is not used", m);
    }
    return QAOA_OK;
}

void classify(const Canonical &c, const int32_t *qpu_of, int64_t *n_local, int64_t *n_cross,
              int64_t *n_cross_all) {
    int64_t loc = 0, cr = 0, cra = 0;
    for (int i = 0; i < c.n; ++i)
        for (int j = i + 1; j < c.n; ++j) {
            const bool same = qpu_of[i] == qpu_of[j];  // Eq. local_cross_rule
            if (!same) ++cra;
            if (c.b[(size_t)i * c.n + j] == 0.0) continue;
            if (same) ++loc; else ++cr;
        }
    *n_local = loc;
    *n_cross = cr;
    if (n_cross_all) *n_cross_all = cra;
}

// Graph-aware greedy allocation (Sec. 3.1): edge weight |b_ij|; QPU m opens
// with the free variable of largest weighted degree towards the free
// variables, then takes the free variable with the largest total weight to
// its members (ties: larger weighted degree to the free variables, then the
// smaller index) until it holds min(c_m, free - QPUs still to open).
qaoa_status graph_aware(const Canonical &c, int M, const std::vector<int32_t> &caps, int32_t *qpu_of) {
    const int n = c.n;
    auto w = [&](int i, int j) {
        return i == j ? 0.0 : std::fabs(i < j ? c.b[(size_t)i * n + j] : c.b[(size_t)j * n + i]);
    };
    std::vector<char> freev(n, 1);
    int nfree = n;
    for (int i = 0; i < n; ++i) qpu_of[i] = -1;
    auto free_degree = [&](int v) {
        double d = 0.0;
        for (int u = 0; u < n; ++u)
            if (freev[u] && u != v) d += w(v, u);
        return d;
    };
    for (int m = 0; m < M && nfree > 0; ++m) {
        const int take = std::min<int>(caps[m], nfree - (M - m - 1));
        if (take <= 0) continue;
        std::vector<int> members;
        int seed = -1;
        double sd = 0.0;
        for (int v = 0; v < n; ++v) {
            if (!freev[v]) continue;
            const double d = free_degree(v);
            if (seed < 0 || d > sd) {
                seed = v;
                sd = d;
            }
        }
        members.push_back(seed);
        freev[seed] = 0;
        --nfree;
        while ((int)members.size() < take && nfree > 0) {
            int best = -1;
            double bw = 0.0, bd = 0.0;
            for (int v = 0; v < n; ++v) {
                if (!freev[v]) continue;
                double tw = 0.0;
                for (int u : members) tw += w(v, u);
                const double d = free_degree(v);
                if (best < 0 || tw > bw || (tw == bw && d > bd)) {
                    best = v;
                    bw = tw;
                    bd = d;
                }
            }
            members.push_back(best);
            freev[best] = 0;
            --nfree;
        }
        for (int v : members) qpu_of[v] = m;
    }
    return QAOA_OK;
}

}  // namespace qaoa

namespace {

qaoa_status capacities(int n, int M, const int32_t *caps, std::vector<int32_t> *out) {
    if (n < 1 || M < 1 || M > n) return qaoa::fail(QAOA_ERR_INVALID_ARG, "bad n=%d or M=%d", n, M);
    out->resize(M);
    int64_t tot = 0;
    for (int m = 0; m < M; ++m) {
        (*out)[m] = caps ? caps[m] : (n / M + (m < n % M ? 1 : 0));
        if ((*out)[m] < 1) return qaoa::fail(QAOA_ERR_ALLOCATION, "capacity of QPU %d is %d < 1", m, (*out)[m]);
        tot += (*out)[m];
    }
    if (tot < n) return qaoa::fail(QAOA_ERR_ALLOCATION, "total capacity %lld < n=%d", (long long)tot, n);
    return QAOA_OK;
}

}  // namespace

extern "C" {

qaoa_status qaoa_partition_graph(const qaoa_qubo *q, int M, const int32_t *caps, int32_t *qpu_of) {
    if (!q || !qpu_of) return qaoa::fail(QAOA_ERR_INVALID_ARG, "null argument");
    qaoa::Canonical c;
    qaoa_status st = qaoa::canonicalize(q, &c);
    if (st) return st;
    std::vector<int32_t> cp;
    if ((st = capacities(c.n, M, caps, &cp))) return st;
    if ((st = qaoa::graph_aware(c, M, cp, qpu_of))) return st;
    return qaoa::partition(c.n, M, cp.data(), qpu_of, qpu_of);  // validate_allocation
}

qaoa_status qaoa_allocation_candidates(const qaoa_qubo *q, int M, const int32_t *caps, const int32_t *manual, int p,
                                       int32_t *qpu_of, int32_t *kind, int64_t *cross, int64_t *remote_cx) {
    if (!q || !qpu_of || !kind || p < 0) return qaoa::fail(QAOA_ERR_INVALID_ARG, "null argument or p < 0");
    qaoa::Canonical c;
    qaoa_status st = qaoa::canonicalize(q, &c);
    if (st) return st;
    const int n = c.n;
    std::vector<int32_t> cp;
    if ((st = capacities(n, M, caps, &cp))) return st;
    std::vector<std::vector<int32_t>> cand(3, std::vector<int32_t>(n));
    if ((st = qaoa::partition(n, M, cp.data(), nullptr, cand[0].data()))) return st;
    if ((st = qaoa::graph_aware(c, M, cp, cand[1].data()))) return st;
    if ((st = qaoa::partition(n, M, cp.data(), cand[1].data(), cand[1].data()))) return st;
    const int nc = manual ? 3 : 2;
    if (manual && (st = qaoa::partition(n, M, cp.data(), manual, cand[2].data()))) return st;
    const int prio[3] = {2, 1, 0};  // on equal cross counts: manual, graph-aware, contiguous
    int best = -1;
    int64_t bc = 0;
    for (int k = 0; k < 3; ++k) {
        int64_t loc = 0, cr = -1;
        if (k < nc) qaoa::classify(c, cand[k].data(), &loc, &cr, nullptr);
        if (cross) cross[k] = cr;
        if (remote_cx) remote_cx[k] = cr < 0 ? -1 : 2 * cr * p;
        if (k < nc && (best < 0 || cr < bc || (cr == bc && prio[k] < prio[best]))) {
            best = k;
            bc = cr;
        }
    }
    for (int i = 0; i < n; ++i) qpu_of[i] = cand[best][i];
    *kind = best;
    return QAOA_OK;
}

}  // extern "C"
