// Internal state of the C ABI shared by its translation units (api.cu,
// api_sample.cu): device buffers, the context, cost and state handles.
#pragma once

#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include "kernels_misc.h"
#include "qaoa_internal.h"
#include "schedule.cuh"

namespace qaoa {
const char *last_error();
}

#define CUDA_TRY(expr)                                                                             \
    do {                                                                                           \
        cudaError_t e__ = (expr);                                                                  \
        if (e__ != cudaSuccess)                                                                    \
            return qaoa::fail(e__ == cudaErrorMemoryAllocation ? QAOA_ERR_OUT_OF_MEMORY : QAOA_ERR_CUDA, \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e__), __FILE__, __LINE__);     \
    } while (0)

#define QAOA_TRY(expr)                  \
    do {                                \
        qaoa_status s__ = (expr);       \
        if (s__ != QAOA_OK) return s__; \
    } while (0)

constexpr int QAOA_PROF_KINDS = 15;

namespace qaoa {
namespace api {

// growable device buffer
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
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
    void release(int64_t *held) {
        if (p) cudaFree(p);
        p = nullptr;
        *held -= (int64_t)cap;
        cap = 0;
    }
    template <typename T>
    T *as() const {
        return reinterpret_cast<T *>(p);
    }
};

struct ProfRec {
    int kind, kind2;  // kind2: the kernel-level kind of a layer pass, or -1
    cudaEvent_t a, b;
    double bytes;
};

// Device buffers of one plan execution (one n, a batch of items).
struct PlanBufs {
    DevBuf psi, pl, states, lam, partials, partials2, sums, scal, slot_scale, plan, gamma, beta, item_s, item_kc, item_table, tables,
        out_E, out_dg, out_db, topk_a, topk_b, adam_m, adam_v, adam_step, history, small_items, small_out;
    bool in_use = false;  // planned for the batch call that is running
};

}  // namespace api
}  // namespace qaoa

using qaoa::api::DevBuf;
using qaoa::api::PlanBufs;
using qaoa::api::ProfRec;

struct qaoa_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    qaoa_options opt{};
    int64_t held = 0;
    int num_sms = 148;
    PlanBufs single;                  // qaoa_grad / qaoa_forward working set
    std::map<int, std::unique_ptr<PlanBufs>> groups;  // batched working sets, by n
    DevBuf partials_e, sums_e, topk_a, topk_b, small_items, small_out, misc, status;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> ev_free;
    // by profile kind (QAOA_PROF_KINDS of them; 5 is unused: it reads the launch count)
    int64_t prof_launches[QAOA_PROF_KINDS] = {};
    double prof_ms[QAOA_PROF_KINDS] = {};
    double prof_bytes[QAOA_PROF_KINDS] = {};
    int64_t launches_total = 0;  // every kernel launched by this context
    cudaStream_t aux_stream = nullptr;  // owned; runs captured optimisation loops
    std::vector<cudaStream_t> pool;     // owned; groups of a batch of several n run side by side
    std::vector<cudaEvent_t> pool_join; // owned; one per pool stream
    cudaEvent_t pool_fork = nullptr;    // owned
    std::map<int, int> tuned_k;         // fusion width picked by the autotuner, by n
    std::map<int, int> tuned_uncompute; // 1: the autotuner found the uncompute sweep faster, by n
    DevBuf sample_items, sample_scratch, sample_out, small_states;  // measurement by shots
};

// The stored forward states of the adjoint (and its lambda buffer) are
// scratch that a context re-creates on its next gradient call of that size.
// Releases them in every working set but `keep`; returns whether anything was
// released.
inline bool release_adjoint_scratch(qaoa_ctx_s *c, const PlanBufs *keep) {
    bool any = false;
    auto drop = [&](PlanBufs &b) {
        if (&b == keep || b.in_use) return;
        any = any || b.states.cap > 0 || b.lam.cap > 0;
        b.states.release(&c->held);
        b.lam.release(&c->held);
    };
    drop(c->single);
    for (auto &kv : c->groups) drop(*kv.second);
    return any;
}

// cudaMalloc for a caller-visible object (a state, an objective table): when
// device memory is short, the adjoint scratch is released and the allocation
// tried once more.
inline cudaError_t ctx_malloc(qaoa_ctx_s *c, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) return e;
    cudaGetLastError();
    *p = nullptr;
    if (!release_adjoint_scratch(c, nullptr)) return e;
    e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
    }
    return e;
}

struct qaoa_cost_s {
    int device = 0;
    int n = 0;
    qaoa::Canonical can;
    qaoa::FixedPoint fp;
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

namespace qaoa {
namespace api {

// Final state of one item of a forward-only batch (device memory owned by the
// context; valid until the next evaluation on the context).
struct ItemState {
    const void *amps = nullptr;
    int n = 0;
    const qaoa_cost_s *cost = nullptr;
};

// Batched evaluation behind qaoa_grad_batch; with states != null (forward
// only) it also returns where each item's final state lives.
qaoa_status run_batch(qaoa_ctx c, int nq, const qaoa_cost *costs, const int32_t *item_cost, int B, int p,
                      const double *gamma, const double *beta, double *expect, double *dgamma, double *dbeta,
                      std::vector<ItemState> *states);

}  // namespace api
}  // namespace qaoa
