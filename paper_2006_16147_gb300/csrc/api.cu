// api.cu -- the extern "C" boundary declared in include/amg.h. Every entry
// point catches the library's internal errors and returns an amg_status; no
// exception crosses the ABI.
#include <chrono>
#include <cstring>

#include "amg_internal.cuh"

namespace amg {
const char* last_error_cstr();
}

using amg::Error;

namespace {

amg_status fail(amg_status s, const std::string& m) {
    amg::set_last_error(m);
    return s;
}

template <typename F>
amg_status guarded(F&& f) {
    try {
        amg::set_last_error("");
        return f();
    } catch (const Error& e) {
        return fail(e.status, e.msg);
    } catch (const std::bad_alloc&) {
        return fail(AMG_ERR_OOM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(AMG_ERR_CUDA, e.what());
    } catch (...) {
        return fail(AMG_ERR_CUDA, "unknown error");
    }
}

void bind_device(amg_hierarchy* h) { CUDA_CHECK(cudaSetDevice(h->device)); }

amg_status check_csr(const amg_csr* A, const double* w) {
    if (!A || !w || !A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))
        return fail(AMG_ERR_ARG, "null argument");
    if (A->n <= 0 || A->nnz <= 0) return fail(AMG_ERR_ARG, "empty matrix");
    if (A->n > 0x7ffffffe) return fail(AMG_ERR_TOO_LARGE, "n exceeds int32");
    return AMG_OK;
}

amg_status setup_common(const amg_csr* A, const double* w, const amg_options* opt, amg_hierarchy** out,
                        int many = 0, const double* const* ws = nullptr) {
    if (!out) return fail(AMG_ERR_ARG, "out is null");
    *out = nullptr;
    amg_status s = AMG_OK;
    if (many) {
        if (!A || !ws) return fail(AMG_ERR_ARG, "null argument");
        for (int i = 0; i < many && s == AMG_OK; ++i) s = check_csr(&A[i], ws[i]);
    } else {
        s = check_csr(A, w);
    }
    if (s != AMG_OK) return s;
    amg_options o;
    if (opt) o = *opt;
    else amg_options_default(&o);
    if (o.sweeps < 1 || o.sweeps > AMG_MAX_SWEEPS || o.max_levels < 1 || o.max_coarse < 1 || o.pre < 0 ||
        o.post < 0 || !(o.omega > 0.0) || (o.precision != AMG_FP64 && o.precision != AMG_FP32_VCYCLE) ||
        o.max_dense < 1 || o.krylov < 0 || o.krylov > 1 || !(o.min_ratio >= 1.0) || o.autotune < 0 ||
        o.autotune > 1 || o.cycle < 0 || o.cycle > AMG_KCYCLE_FULL || (o.cycle > 0 && (o.pre != 1 || o.post != 1)) ||
        o.smooth_p < 0 || o.smooth_p > 1 || (o.smooth_p && o.cycle != 0) || o.omega_rule < 0 || o.omega_rule > 1)
        return fail(AMG_ERR_ARG, "invalid options");
    if (many && (o.cycle != 0 || o.smooth_p)) return fail(AMG_ERR_ARG, "batches of systems use the unsmoothed V-cycle");
    amg_hierarchy* h = new amg_hierarchy;
    h->opt = o;
    h->stream = static_cast<cudaStream_t>(o.stream);
    h->mem.stream = h->stream;
    h->prof.on = o.profile != 0;
    s = guarded([&]() -> amg_status {
        CUDA_CHECK(cudaGetDevice(&h->device));
        CUDA_CHECK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
        if (many) amg::setup_many(h, many, A, ws);
        else amg::setup_hierarchy(h, A, w);
        amg::prepare_solve(h);
        if (o.autotune) amg::autotune_vcycle(h);
        return AMG_OK;
    });
    if (s != AMG_OK) {
        if (h->sc_host) cudaFreeHost(h->sc_host);
        delete h;
        return s;
    }
    *out = h;
    return AMG_OK;
}

}  // namespace

extern "C" {

void amg_options_default(amg_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->sweeps = 3;
    o->max_coarse = 200;
    o->max_levels = AMG_MAX_LEVELS;
    o->pre = 1;
    o->post = 1;
    o->omega = 1.0;
    o->precision = AMG_FP64;
    o->max_dense = 4096;
    o->keep_sweeps = 0;
    o->profile = 0;
    o->match_kernel = 0;
    o->krylov = 0;
    o->min_ratio = 1.5;
    o->stream = nullptr;
}

amg_status amg_setup(const amg_csr* A, const double* w, const amg_options* opt, amg_hierarchy** out) {
    return setup_common(A, w, opt, out);
}

amg_status amg_setup_host(const amg_csr* A, const double* w, const amg_options* opt, amg_hierarchy** out) {
    // The ingest copies use cudaMemcpyDefault, which takes host or device sources.
    return setup_common(A, w, opt, out);
}

amg_status amg_solve(amg_hierarchy* h, const double* b, double* x, double rtol, int maxit, amg_solve_info* info) {
    if (!h || !b || !x) return fail(AMG_ERR_ARG, "null argument");
    if (!(rtol > 0.0) || maxit < 0) return fail(AMG_ERR_ARG, "rtol must be > 0 and maxit >= 0");
    std::lock_guard<std::mutex> g(h->lock);
    return guarded([&]() -> amg_status {
        bind_device(h);
        amg_status s = amg::solve(h, b, x, rtol, maxit, info);
        if (s == AMG_ERR_BREAKDOWN) amg::set_last_error("CG breakdown: p^T A p <= 0 or non-finite scalar");
        return s;
    });
}

amg_status amg_solve_host(amg_hierarchy* h, const double* b, double* x, double rtol, int maxit,
                          amg_solve_info* info) {
    if (!h || !b || !x) return fail(AMG_ERR_ARG, "null argument");
    if (!(rtol > 0.0) || maxit < 0) return fail(AMG_ERR_ARG, "rtol must be > 0 and maxit >= 0");
    std::lock_guard<std::mutex> g(h->lock);
    return guarded([&]() -> amg_status {
        bind_device(h);
        auto t0 = std::chrono::steady_clock::now();
        const size_t bytes = sizeof(double) * (size_t)h->lev[0].A.n;
        double *db = nullptr, *dx = nullptr;
        CUDA_CHECK(cudaMallocAsync(&db, bytes, h->stream));
        CUDA_CHECK(cudaMallocAsync(&dx, bytes, h->stream));
        amg_status s = AMG_ERR_CUDA;
        try {
            CUDA_CHECK(cudaMemcpyAsync(db, b, bytes, cudaMemcpyHostToDevice, h->stream));
            CUDA_CHECK(cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, h->stream));
            s = amg::solve(h, db, dx, rtol, maxit, info);
            CUDA_CHECK(cudaMemcpyAsync(x, dx, bytes, cudaMemcpyDeviceToHost, h->stream));
            CUDA_CHECK(cudaStreamSynchronize(h->stream));
        } catch (...) {
            cudaFreeAsync(db, h->stream);
            cudaFreeAsync(dx, h->stream);
            throw;
        }
        CUDA_CHECK(cudaFreeAsync(db, h->stream));
        CUDA_CHECK(cudaFreeAsync(dx, h->stream));
        if (info) info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return s;
    });
}

amg_status amg_setup_many(int m, const amg_csr* As, const double* const* ws, const amg_options* opt,
                          amg_hierarchy** out) {
    if (m < 1) return fail(AMG_ERR_ARG, "m must be >= 1");
    return setup_common(As, nullptr, opt, out, m, ws);
}

amg_status amg_solve_many(amg_hierarchy* h, const double* b, double* x, double rtol, int maxit,
                          amg_solve_info* infos) {
    if (!h || !b || !x) return fail(AMG_ERR_ARG, "null argument");
    if (!(rtol > 0.0) || maxit < 0) return fail(AMG_ERR_ARG, "rtol must be > 0 and maxit >= 0");
    std::lock_guard<std::mutex> g(h->lock);
    return guarded([&]() -> amg_status {
        bind_device(h);
        amg_status s = amg::solve_many(h, b, x, rtol, maxit, infos);
        if (s == AMG_ERR_BREAKDOWN) amg::set_last_error("CG breakdown in at least one system");
        return s;
    });
}

amg_status amg_system_offsets(const amg_hierarchy* h, int32_t* offsets) {
    if (!h || !offsets) return fail(AMG_ERR_ARG, "null argument");
    if (h->seg0.empty()) {
        offsets[0] = 0;
        offsets[1] = h->lev[0].A.n;
        return AMG_OK;
    }
    for (size_t i = 0; i < h->seg0.size(); ++i) offsets[i] = h->seg0[i];
    return AMG_OK;
}

amg_status amg_solve_batch(amg_hierarchy* h, int k, const double* B, double* X, double rtol, int maxit,
                           amg_solve_info* infos) {
    if (!h || !B || !X) return fail(AMG_ERR_ARG, "null argument");
    if (!(rtol > 0.0) || maxit < 0 || k < 1) return fail(AMG_ERR_ARG, "bad k, rtol or maxit");
    std::lock_guard<std::mutex> g(h->lock);
    return guarded([&]() -> amg_status {
        bind_device(h);
        amg_status s = amg::solve_batch(h, k, B, X, rtol, maxit, infos);
        if (s == AMG_ERR_BREAKDOWN) amg::set_last_error("CG breakdown in at least one column");
        return s;
    });
}

amg_status amg_vcycle(amg_hierarchy* h, const double* r, double* z) {
    if (!h || !r || !z) return fail(AMG_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> g(h->lock);
    return guarded([&]() -> amg_status {
        bind_device(h);
        amg::vcycle_apply(h, r, z);
        return AMG_OK;
    });
}

amg_status amg_hierarchy_info(const amg_hierarchy* h, amg_hier_info* out) {
    if (!h || !out) return fail(AMG_ERR_ARG, "null argument");
    std::memset(out, 0, sizeof(*out));
    const int nl = (int)h->lev.size();
    out->num_levels = nl;
    double sum = 0.0, cr = 0.0;
    for (int l = 0; l < nl; ++l) {
        out->n[l] = h->lev[l].A.n;
        out->nnz[l] = h->lev[l].A.nnz;
        out->sweeps_done[l] = h->lev[l].sweeps_done;
        for (int s = 0; s < AMG_MAX_SWEEPS; ++s) out->rounds[l][s] = h->lev[l].rounds[s];
        sum += (double)h->lev[l].A.nnz;
        if (l + 1 < nl) cr += (double)h->lev[l].A.n / (double)h->lev[l + 1].A.n;
    }
    out->opc = sum / (double)h->lev[0].A.nnz;
    out->avg_coarsening_ratio = nl > 1 ? cr / (nl - 1) : 0.0;
    out->setup_ms = h->setup_ms;
    out->coarse_solver = h->coarse_cg;
    out->device_bytes = h->mem.bytes;
    return AMG_OK;
}

amg_status amg_export_level(const amg_hierarchy* h, int level, int32_t* row_ptr, int32_t* col, double* val, double* w,
                            double* minv, int32_t* agg, double* p) {
    if (!h || level < 0 || level >= (int)h->lev.size()) return fail(AMG_ERR_ARG, "bad level");
    amg_hierarchy* hh = const_cast<amg_hierarchy*>(h);
    std::lock_guard<std::mutex> g(hh->lock);
    return guarded([&]() -> amg_status {
        bind_device(hh);
        const amg::Level& L = h->lev[level];
        const size_t n = L.A.n, nnz = L.A.nnz;
        const bool last = level == (int)h->lev.size() - 1;
        if ((agg || p) && last) AMG_THROW(AMG_ERR_ARG, "the coarsest level has no prolongator");
        if (row_ptr) CUDA_CHECK(cudaMemcpy(row_ptr, L.A.ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
        if (col) CUDA_CHECK(cudaMemcpy(col, L.A.col, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
        if (val) CUDA_CHECK(cudaMemcpy(val, L.A.val, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
        if (w) CUDA_CHECK(cudaMemcpy(w, L.w, sizeof(double) * n, cudaMemcpyDeviceToHost));
        if (minv) CUDA_CHECK(cudaMemcpy(minv, L.minv, sizeof(double) * n, cudaMemcpyDeviceToHost));
        if (agg) CUDA_CHECK(cudaMemcpy(agg, L.agg, sizeof(int) * n, cudaMemcpyDeviceToHost));
        if (p) CUDA_CHECK(cudaMemcpy(p, L.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
        return AMG_OK;
    });
}

amg_status amg_sweep_dims(const amg_hierarchy* h, int level, int sweep, int32_t* n, int32_t* nc, int64_t* nnz_c) {
    if (!h || level < 0 || level >= (int)h->lev.size()) return fail(AMG_ERR_ARG, "bad level");
    const amg::Level& L = h->lev[level];
    if (sweep < 0 || sweep >= (int)L.sweeps.size()) return fail(AMG_ERR_ARG, "sweep not recorded (keep_sweeps?)");
    const amg::SweepRecord& R = L.sweeps[sweep];
    if (n) *n = R.n;
    if (nc) *nc = R.nc;
    if (nnz_c) *nnz_c = R.nnz_c;
    return AMG_OK;
}

amg_status amg_export_sweep(const amg_hierarchy* h, int level, int sweep, int32_t* mate, int32_t* agg, double* p,
                            double* wc) {
    if (!h || level < 0 || level >= (int)h->lev.size()) return fail(AMG_ERR_ARG, "bad level");
    const amg::Level& L = h->lev[level];
    if (sweep < 0 || sweep >= (int)L.sweeps.size()) return fail(AMG_ERR_ARG, "sweep not recorded (keep_sweeps?)");
    amg_hierarchy* hh = const_cast<amg_hierarchy*>(h);
    std::lock_guard<std::mutex> g(hh->lock);
    return guarded([&]() -> amg_status {
        bind_device(hh);
        const amg::SweepRecord& R = L.sweeps[sweep];
        if (mate) CUDA_CHECK(cudaMemcpy(mate, R.mate, sizeof(int) * R.n, cudaMemcpyDeviceToHost));
        if (agg) CUDA_CHECK(cudaMemcpy(agg, R.agg, sizeof(int) * R.n, cudaMemcpyDeviceToHost));
        if (p) CUDA_CHECK(cudaMemcpy(p, R.p, sizeof(double) * R.n, cudaMemcpyDeviceToHost));
        if (wc) CUDA_CHECK(cudaMemcpy(wc, R.wc, sizeof(double) * R.nc, cudaMemcpyDeviceToHost));
        return AMG_OK;
    });
}

amg_status amg_coarse_factor(const amg_hierarchy* h, double* L) {
    if (!h || !L) return fail(AMG_ERR_ARG, "null argument");
    if (h->coarse_cg) return fail(AMG_ERR_ARG, "the coarsest level is solved by CG; there is no dense factor");
    amg_hierarchy* hh = const_cast<amg_hierarchy*>(h);
    std::lock_guard<std::mutex> g(hh->lock);
    return guarded([&]() -> amg_status {
        bind_device(hh);
        CUDA_CHECK(cudaMemcpy(L, h->coarse_L, sizeof(double) * (size_t)h->nc * h->nc, cudaMemcpyDeviceToHost));
        return AMG_OK;
    });
}

void amg_free(amg_hierarchy* h) {
    if (!h) return;
    {
        std::lock_guard<std::mutex> g(h->lock);
        cudaSetDevice(h->device);
        if (h->stream) cudaStreamSynchronize(h->stream);
        else cudaDeviceSynchronize();
        amg::block_free(h);
        h->mem.free_all();
        if (h->sc_host) cudaFreeHost(h->sc_host);
        h->sc_host = nullptr;
    }
    delete h;
}

const char* amg_last_error(void) { return amg::last_error_cstr(); }

int amg_kernel_stats_count(void) { return amg::K_COUNT; }

amg_status amg_kernel_stats(amg_hierarchy* h, int idx, const char** name, int64_t* scopes, double* total_ms,
                            double* bytes) {
    if (!h || idx < 0 || idx >= amg::K_COUNT) return fail(AMG_ERR_ARG, "bad argument");
    std::lock_guard<std::mutex> g(h->lock);
    return guarded([&]() -> amg_status {
        bind_device(h);
        h->prof.flush();
        const amg::KStat& k = h->prof.st[idx];
        if (name) *name = amg::kernel_name(idx);
        if (scopes) *scopes = k.launches;
        if (total_ms) *total_ms = k.ms;
        if (bytes) *bytes = k.bytes;
        return AMG_OK;
    });
}

amg_status amg_kernel_stats_reset(amg_hierarchy* h) {
    if (!h) return fail(AMG_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> g(h->lock);
    return guarded([&]() -> amg_status {
        bind_device(h);
        h->prof.reset();
        return AMG_OK;
    });
}

int64_t amg_launch_count(void) { return amg::launch_counter().load(); }

amg_status amg_serve_create(int nh, amg_hierarchy* const* hs, int slots, size_t budget_bytes, double rtol, int maxit,
                            amg_server** out) {
    if (!out || nh < 1 || !hs || slots < 1 || slots > 256 || !(rtol > 0.0) || maxit < 1)
        return fail(AMG_ERR_ARG, "bad server arguments");
    *out = nullptr;
    for (int i = 0; i < nh; ++i)
        if (!hs[i]) return fail(AMG_ERR_ARG, "null hierarchy");
    return guarded([&]() -> amg_status {
        *out = amg::serve_create(nh, hs, slots, budget_bytes, rtol, maxit);
        return AMG_OK;
    });
}

amg_status amg_serve_submit(amg_server* s, int hid, int k, const double* B, double* X, int64_t* id) {
    if (!s || !B || !X) return fail(AMG_ERR_ARG, "null argument");
    return guarded([&]() -> amg_status {
        const int64_t v = amg::serve_submit(s, hid, k, B, X);
        if (id) *id = v;
        return AMG_OK;
    });
}

amg_status amg_serve_step(amg_server* s, int64_t* pending) {
    if (!s) return fail(AMG_ERR_ARG, "null server");
    return guarded([&]() -> amg_status {
        const int64_t p = amg::serve_step(s);
        if (pending) *pending = p;
        return AMG_OK;
    });
}

int amg_serve_poll(amg_server* s, int64_t* ids, int* statuses, double* latency_ms, int* iterations, double* relres,
                   int max) {
    if (!s || max < 1) return 0;
    return amg::serve_poll(s, ids, statuses, latency_ms, iterations, relres, max);
}

amg_status amg_serve_stats_get(amg_server* s, amg_serve_stats* out) {
    if (!s || !out) return fail(AMG_ERR_ARG, "null argument");
    amg::serve_stats(s, out);
    return AMG_OK;
}

void amg_serve_free(amg_server* s) {
    if (s) amg::serve_free(s);
}

amg_status amg_pbar_nnz(const amg_hierarchy* h, int level, int64_t* nnz) {
    if (!h || !nnz) return fail(AMG_ERR_ARG, "null argument");
    if (level < 0 || level + 1 >= (int)h->lev.size() || !h->lev[level].pbar.ptr)
        return fail(AMG_ERR_ARG, "no smoothed prolongator on this level");
    *nnz = h->lev[level].pbar.nnz;
    return AMG_OK;
}

amg_status amg_export_pbar(const amg_hierarchy* h, int level, int32_t* row_ptr, int32_t* col, double* val,
                           double* omega) {
    if (!h) return fail(AMG_ERR_ARG, "null argument");
    if (level < 0 || level + 1 >= (int)h->lev.size() || !h->lev[level].pbar.ptr)
        return fail(AMG_ERR_ARG, "no smoothed prolongator on this level");
    const amg::DevCsr& P = h->lev[level].pbar;
    return guarded([&]() -> amg_status {
        CUDA_CHECK(cudaSetDevice(h->device));
        if (row_ptr) CUDA_CHECK(cudaMemcpy(row_ptr, P.ptr, sizeof(int) * (P.n + 1), cudaMemcpyDeviceToHost));
        if (col) CUDA_CHECK(cudaMemcpy(col, P.col, sizeof(int) * (size_t)P.nnz, cudaMemcpyDeviceToHost));
        if (val) CUDA_CHECK(cudaMemcpy(val, P.val, sizeof(double) * (size_t)P.nnz, cudaMemcpyDeviceToHost));
        if (omega) *omega = h->lev[level].omega_p;
        return AMG_OK;
    });
}

amg_status amg_smooth_vector(const amg_csr* A, const double* w0, double* w, int sweeps, double omega, void* stream) {
    if (!w) return fail(AMG_ERR_ARG, "w is null");
    if (sweeps < 0 || !(omega > 0.0)) return fail(AMG_ERR_ARG, "sweeps must be >= 0 and omega > 0");
    amg_status s = check_csr(A, w0);
    if (s != AMG_OK) return s;
    if (w0 == w && sweeps % 2 == 1)
        return fail(AMG_ERR_ARG, "w0 and w must differ for an odd number of sweeps");
    return guarded([&]() -> amg_status {
        amg::smooth_vector(A, w0, w, sweeps, omega, static_cast<cudaStream_t>(stream));
        return AMG_OK;
    });
}

amg_status amg_match_noalloc(const amg_csr* A, const double* w, int32_t* mate, void* stream, int32_t* rounds) {
    if (!mate) return fail(AMG_ERR_ARG, "mate is null");
    amg_status s = check_csr(A, w);
    if (s != AMG_OK) return s;
    return guarded([&]() -> amg_status { return amg::match_noalloc(A, w, mate, stream, rounds); });
}

}  // extern "C"
