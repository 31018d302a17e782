// prof.cuh -- optional per-kernel timing with CUDA events on the launching
// stream, plus a process-wide count of kernel launches.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <vector>

namespace amg {

enum KernelId : int {
    // solve phase, one scope per launch
    K_PRE = 0,        // fused pre-smoothing + residual, levels >= 1
    K_PRE_L0,         // same on level 0
    K_PRE_STEP,       // extra pre-smoothing sweeps
    K_RESTRICT,       // P^T r
    K_COARSE,         // dense coarsest solve
    K_POST,           // fused prolongation + post-smoothing, levels >= 1
    K_POST_L0,        // same on level 0 (writes z, r.z)
    K_SMOOTH,         // extra post-smoothing sweeps
    K_SPMV_DOT,       // q = A p, p.q
    K_UPDATE_XR,      // x += alpha p, r -= alpha q, ||r||^2
    K_UPDATE_P,       // p = z + beta p
    K_RESIDUAL,       // r = b - A x, norms
    K_DOT,            // stand-alone dot product
    K_CONVERT,        // FP64 -> FP32 copy of the level-0 residual (FP32 V-cycle)
    K_KFCG,           // K-cycle: the flexible CG steps of a coarse correction
    // setup phase, one scope per phase call
    S_VALIDATE,
    S_WEIGHTS,
    S_MATCH,
    S_MATCH_SORT,
    S_AGGREGATE,
    S_GALERKIN,
    S_COMPOSE,
    S_SMOOTHER,
    S_FORMAT,
    S_COARSE,
    S_SMOOTH_P,
    K_COUNT
};

inline const char* kernel_name(int id) {
    static const char* names[K_COUNT] = {
        "pre_residual",   "pre_residual_l0", "pre_step",     "restrict",  "coarse_solve", "post_smooth",
        "post_smooth_l0", "smooth",          "spmv_dot",     "update_xr", "update_p",     "residual",
        "dot",            "convert_l0",      "kcycle_fcg",   "setup_validate",  "setup_weights", "setup_match", "setup_match_sort", "setup_aggregate", "setup_galerkin",
        "setup_compose",  "setup_smoother",  "setup_format", "setup_coarse", "setup_smooth_p"};
    return (id >= 0 && id < K_COUNT) ? names[id] : "";
}

std::atomic<long long>& launch_counter();

struct KStat {
    long long launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
};

struct Profiler {
    bool on = false;
    KStat st[K_COUNT];
    struct Pending {
        int id;
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Pending> pending;

    cudaEvent_t get() {
        if (pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    // Accumulates every finished scope; call after a stream synchronisation.
    void flush() {
        for (auto& p : pending) {
            float ms = 0.f;
            cudaEventSynchronize(p.b);
            cudaEventElapsedTime(&ms, p.a, p.b);
            st[p.id].launches += 1;
            st[p.id].ms += ms;
            st[p.id].bytes += p.bytes;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
    void reset() {
        flush();
        for (auto& s : st) s = KStat{};
    }
    ~Profiler() {
        for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Records events around the work enqueued during its lifetime.
struct Scope {
    Profiler* p;
    cudaStream_t s;
    int id;
    double bytes;
    cudaEvent_t a = nullptr;
    Scope(Profiler* prof, cudaStream_t st, int kid, double by) : p(prof), s(st), id(kid), bytes(by) {
        if (p && p->on) {
            a = p->get();
            cudaEventRecord(a, s);
        }
    }
    ~Scope() {
        if (p && p->on) {
            cudaEvent_t b = p->get();
            cudaEventRecord(b, s);
            p->pending.push_back({id, a, b, bytes});
        }
    }
};

}  // namespace amg
