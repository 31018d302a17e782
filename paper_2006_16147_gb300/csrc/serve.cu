// serve.cu -- continuous-batching solve server over cached hierarchies.
//
// The preconditioner is built once per matrix and reused for every solve
// (the reuse that makes an AMG setup worth its cost, Sections 1 and 5). Each
// cached hierarchy gets a block of K column slots (block.cu). Requests (1..K
// right-hand sides of one hierarchy) wait in a per-hierarchy FIFO; between
// steps, the head request is admitted when it finds enough free slots and the
// device-memory budget allows its columns. Every step advances every
// hierarchy with live columns by one CG iteration, each on its own stream so
// the work of different hierarchies overlaps on the GPU; a converged column is
// copied to its request's output and its slot is freed for the next request
// at once (iteration-level continuous batching). Columns use a fixed group
// width, so a column's arithmetic does not depend on what else is in flight.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <unordered_map>

#include "amg_internal.cuh"

namespace {

using clock_type = std::chrono::steady_clock;

double now_ms() {
    return std::chrono::duration<double, std::milli>(clock_type::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    int hid = 0;
    int k = 0;
    const double* B = nullptr;   // host, row-major n x k
    double* X = nullptr;         // host, row-major n x k
    double t_submit = 0.0, t_done = 0.0;
    int cols_done = 0;
    int status = AMG_OK;
    int iters = 0;
    double worst_relres = 0.0;
    std::vector<int> slots;
    double* dX = nullptr;        // device n x k result block, copied to X at completion
};

struct Served {
    amg_hierarchy* h = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t old_stream = nullptr;
    int K = 0;
    int n = 0;
    double* B = nullptr;          // device n x K
    double* X = nullptr;          // device n x K
    double* rtol_host = nullptr;  // pinned K
    std::vector<int64_t> owner;   // slot -> request id, -1 free
    std::deque<int64_t> queue;
    size_t bytes_per_col = 0;
};

}  // namespace

struct amg_server {
    std::vector<Served> hs;
    std::unordered_map<int64_t, Request> reqs;
    std::deque<int64_t> completed;
    size_t budget = 0, used = 0, peak = 0;
    double rtol = 1e-6;
    int maxit = 1000;
    int64_t next_id = 1;
    int64_t submitted = 0, done = 0, steps = 0, cols_done = 0;
    std::vector<double> latencies;
    double t_first = -1.0, t_last = 0.0;
    std::mutex mu;
};

namespace amg {

amg_server* serve_create(int nh, amg_hierarchy* const* hs, int K, size_t budget, double rtol, int maxit) {
    auto* S = new amg_server;
    S->budget = budget;
    S->rtol = rtol;
    S->maxit = maxit;
    try {
        for (int i = 0; i < nh; ++i) {
            Served sv;
            sv.h = hs[i];
            sv.K = K;
            sv.n = hs[i]->lev[0].A.n;
            CUDA_CHECK(cudaSetDevice(hs[i]->device));
            CUDA_CHECK(cudaStreamSynchronize(hs[i]->stream));
            sv.old_stream = hs[i]->stream;
            CUDA_CHECK(cudaStreamCreateWithFlags(&sv.stream, cudaStreamNonBlocking));
            hs[i]->stream = sv.stream;
            S->hs.push_back(sv);
            Served& cur = S->hs.back();
            block_ensure(hs[i], K, true);
            cur.B = hs[i]->blk->mem.alloc<double>((size_t)cur.n * K);
            cur.X = hs[i]->blk->mem.alloc<double>((size_t)cur.n * K);
            CUDA_CHECK(cudaHostAlloc(&cur.rtol_host, sizeof(double) * K, cudaHostAllocDefault));
            for (int c = 0; c < K; ++c) cur.rtol_host[c] = rtol;
            cur.owner.assign(K, -1);
            cur.bytes_per_col = block_bytes_per_column(hs[i]);
            CUDA_CHECK(cudaStreamSynchronize(cur.stream));
        }
    } catch (...) {
        for (auto& sv : S->hs) {
            cudaStreamSynchronize(sv.stream);
            block_free(sv.h);           // its memory is ordered on sv.stream: release before that stream goes
            sv.h->stream = sv.old_stream;
            if (sv.rtol_host) cudaFreeHost(sv.rtol_host);
            if (sv.stream) cudaStreamDestroy(sv.stream);
        }
        delete S;
        throw;
    }
    return S;
}

void serve_free(amg_server* S) {
    for (auto& sv : S->hs) {
        cudaStreamSynchronize(sv.stream);
        block_free(sv.h);
        sv.h->stream = sv.old_stream;
        cudaFreeHost(sv.rtol_host);
        cudaStreamDestroy(sv.stream);
    }
    delete S;
}

int64_t serve_submit(amg_server* S, int hid, int k, const double* B, double* X) {
    std::lock_guard<std::mutex> g(S->mu);
    if (hid < 0 || hid >= (int)S->hs.size()) AMG_THROW(AMG_ERR_ARG, "no hierarchy %d", hid);
    Served& sv = S->hs[hid];
    if (k < 1 || k > sv.K) AMG_THROW(AMG_ERR_TOO_LARGE, "a request takes 1..%d right-hand sides", sv.K);
    const size_t need = (size_t)k * (sv.bytes_per_col + 2 * sizeof(double) * sv.n);
    if (need > S->budget)
        AMG_THROW(AMG_ERR_BUDGET, "request needs %zu bytes, above the %zu-byte budget", need, S->budget);
    Request r;
    r.id = S->next_id++;
    r.hid = hid;
    r.k = k;
    r.B = B;
    r.X = X;
    r.t_submit = now_ms();
    if (S->t_first < 0.0) S->t_first = r.t_submit;
    S->reqs[r.id] = r;
    sv.queue.push_back(r.id);
    ++S->submitted;
    return r.id;
}

namespace {

// Device bytes a request holds while in flight: its columns' share of the
// block workspace plus its staging and result blocks.
size_t request_bytes(const Served& sv, int k) { return (size_t)k * (sv.bytes_per_col + 2 * sizeof(double) * sv.n); }

// Admits queue heads of one hierarchy while slots and budget allow (FIFO,
// no overtaking). Returns whether columns were admitted.
bool admit(amg_server* S, Served& sv) {
    BlockWork& W = *sv.h->blk;
    bool any = false;
    while (!sv.queue.empty()) {
        Request& r = S->reqs[sv.queue.front()];
        std::vector<int> free_slots;
        for (int c = 0; c < sv.K && (int)free_slots.size() < r.k; ++c)
            if (sv.owner[c] < 0) free_slots.push_back(c);
        const size_t need = request_bytes(sv, r.k);
        if ((int)free_slots.size() < r.k || S->used + need > S->budget) break;
        S->used += need;
        S->peak = std::max(S->peak, S->used);
        r.slots = free_slots;
        // one contiguous copy of the request's right-hand sides, then a
        // scatter into the slot columns; the initial guesses are zero
        double* dB = nullptr;
        const size_t blk = sizeof(double) * (size_t)sv.n * r.k;
        CUDA_CHECK(cudaMallocAsync(&dB, blk, sv.stream));
        CUDA_CHECK(cudaMallocAsync(&r.dX, blk, sv.stream));
        CUDA_CHECK(cudaMemcpyAsync(dB, r.B, blk, cudaMemcpyHostToDevice, sv.stream));
        block_scatter_request(sv.h, dB, r.k, free_slots.data(), sv.B);
        block_scatter_request(sv.h, nullptr, r.k, free_slots.data(), sv.X);
        CUDA_CHECK(cudaFreeAsync(dB, sv.stream));
        for (int j = 0; j < r.k; ++j) {
            const int c = free_slots[j];
            sv.owner[c] = r.id;
            W.mode_host[c] = COL_INIT;
            W.iters_host[c] = 0;
        }
        sv.queue.pop_front();
        any = true;
    }
    return any;
}

int active_width(const Served& sv) {
    int k = 0;
    for (int c = 0; c < sv.K; ++c)
        if (sv.owner[c] >= 0) k = c + 1;
    return k;
}

void push_states(Served& sv) {
    BlockWork& W = *sv.h->blk;
    CUDA_CHECK(cudaMemcpyAsync(W.sc.mode, W.mode_host, sizeof(int) * sv.K, cudaMemcpyHostToDevice, sv.stream));
    CUDA_CHECK(cudaMemcpyAsync(W.sc.iters, W.iters_host, sizeof(int) * sv.K, cudaMemcpyHostToDevice, sv.stream));
    CUDA_CHECK(cudaMemcpyAsync(W.sc.rtol, sv.rtol_host, sizeof(double) * sv.K, cudaMemcpyHostToDevice, sv.stream));
}

// Finished columns: copy out, free the slot; a request whose last column
// finished has its copy to the host queued and is listed in `finished` (its
// completion time is taken once that copy is done).
void retire(amg_server* S, Served& sv, int maxit, std::vector<int64_t>& finished) {
    BlockWork& W = *sv.h->blk;
    for (int c = 0; c < sv.K; ++c) {
        const int64_t id = sv.owner[c];
        if (id < 0) continue;
        const int md = W.mode_host[c];
        const bool fin = md == COL_DONE || md == COL_FAILED || W.iters_host[c] >= maxit;
        if (!fin) continue;
        Request& r = S->reqs[id];
        int j = 0;
        while (r.slots[j] != c) ++j;
        block_gather_column(sv.h, sv.X, c, r.dX, r.k, j);
        const double nb = std::sqrt(W.bb_host[c]);
        const double rel = nb > 0.0 ? std::sqrt(W.rr_host[c]) / nb : 0.0;
        r.worst_relres = std::max(r.worst_relres, rel);
        r.iters = std::max(r.iters, W.iters_host[c]);
        if (md == COL_FAILED) r.status = AMG_ERR_BREAKDOWN;
        else if (md != COL_DONE && r.status == AMG_OK) r.status = AMG_NOT_CONVERGED;
        sv.owner[c] = -1;
        W.mode_host[c] = COL_IDLE;
        ++S->cols_done;
        if (++r.cols_done == r.k) {
            CUDA_CHECK(cudaMemcpyAsync(r.X, r.dX, sizeof(double) * (size_t)sv.n * r.k, cudaMemcpyDeviceToHost,
                                       sv.stream));
            CUDA_CHECK(cudaFreeAsync(r.dX, sv.stream));
            r.dX = nullptr;
            S->used -= request_bytes(sv, r.k);
            finished.push_back(id);
        }
    }
}

}  // namespace

// One scheduling step over every hierarchy. Returns the number of columns
// still in flight or queued.
int64_t serve_step(amg_server* S) {
    std::lock_guard<std::mutex> g(S->mu);
    ++S->steps;
    std::vector<int> width(S->hs.size(), 0);
    for (size_t i = 0; i < S->hs.size(); ++i) {
        Served& sv = S->hs[i];
        const bool fresh = admit(S, sv);
        width[i] = active_width(sv);
        if (width[i] == 0) continue;
        push_states(sv);
        if (fresh) block_init_launch(sv.h, sv.B, sv.X, width[i]);
        block_step_launch(sv.h, sv.B, sv.X, width[i]);
    }
    for (size_t i = 0; i < S->hs.size(); ++i)
        if (width[i]) CUDA_CHECK(cudaStreamSynchronize(S->hs[i].stream));
    bool again = false;
    for (size_t i = 0; i < S->hs.size(); ++i)
        if (width[i]) again |= block_check_launch(S->hs[i].h, S->hs[i].B, S->hs[i].X, width[i]);
    if (again)
        for (size_t i = 0; i < S->hs.size(); ++i)
            if (width[i]) CUDA_CHECK(cudaStreamSynchronize(S->hs[i].stream));
    std::vector<int64_t> finished;
    for (size_t i = 0; i < S->hs.size(); ++i)
        if (width[i]) retire(S, S->hs[i], S->maxit, finished);
    for (size_t i = 0; i < S->hs.size(); ++i)
        if (width[i]) CUDA_CHECK(cudaStreamSynchronize(S->hs[i].stream));
    // latency = submission to result in the caller's host buffer
    const double t = now_ms();
    for (int64_t id : finished) {
        Request& r = S->reqs[id];
        r.t_done = t;
        S->latencies.push_back(r.t_done - r.t_submit);
        S->completed.push_back(id);
        ++S->done;
        S->t_last = t;
    }
    int64_t pending = 0;
    for (auto& sv : S->hs) {
        for (int c = 0; c < sv.K; ++c) pending += sv.owner[c] >= 0;
        for (int64_t id : sv.queue) pending += S->reqs[id].k;
    }
    return pending;
}

int serve_poll(amg_server* S, int64_t* ids, int* statuses, double* latency_ms, int* iters, double* relres, int max) {
    std::lock_guard<std::mutex> g(S->mu);
    int n = 0;
    while (n < max && !S->completed.empty()) {
        const int64_t id = S->completed.front();
        S->completed.pop_front();
        const Request& r = S->reqs[id];
        if (ids) ids[n] = id;
        if (statuses) statuses[n] = r.status;
        if (latency_ms) latency_ms[n] = r.t_done - r.t_submit;
        if (iters) iters[n] = r.iters;
        if (relres) relres[n] = r.worst_relres;
        S->reqs.erase(id);
        ++n;
    }
    return n;
}

void serve_stats(amg_server* S, amg_serve_stats* o) {
    std::lock_guard<std::mutex> g(S->mu);
    std::memset(o, 0, sizeof(*o));
    o->submitted = S->submitted;
    o->completed = S->done;
    o->steps = S->steps;
    o->columns_completed = S->cols_done;
    o->budget_bytes = S->budget;
    o->peak_bytes = S->peak;
    std::vector<double> l = S->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)std::floor(f * (l.size() - 1) + 0.5))]; };
        o->p50_ms = q(0.50);
        o->p99_ms = q(0.99);
        double s = 0.0;
        for (double v : l) s += v;
        o->mean_ms = s / l.size();
    }
    if (S->t_first >= 0.0 && S->t_last > S->t_first) {
        o->elapsed_s = (S->t_last - S->t_first) * 1e-3;
        o->columns_per_s = S->cols_done / o->elapsed_s;
    }
}

}  // namespace amg
