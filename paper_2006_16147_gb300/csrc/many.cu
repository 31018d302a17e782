// many.cu -- many independent systems in one hierarchy and one solve.
//
// The systems are set up as one block-diagonal matrix (setup.cu keeps their
// row offsets on every level: a matching never crosses systems, so every
// system is coarsened exactly as it would be on its own, and its aggregates
// stay contiguous). The V-cycle of the union is then the V-cycle of each
// system at once, and each CG step runs the same kernels over all systems,
// with every system's own alpha, beta, rho and convergence from segmented
// sums (one block per system, fixed order). The step is captured once into a
// CUDA graph and replayed, so a CG step of all systems is one graph launch.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "amg_internal.cuh"
#include "device_util.cuh"

namespace amg {

void vcycle_plain(amg_hierarchy* h, const double* r, double* z);

namespace {

constexpr int TPB = 256;
constexpr int WARPS = TPB / 32;

struct SellM {
    int n, nslices;
    const int* __restrict__ sptr;
    const int* __restrict__ col;
    const int* __restrict__ perm;
};

// y = A x over SELL-32 (rows may be permuted), no reduction.
__global__ void __launch_bounds__(TPB) m_spmv(SellM S, const double* __restrict__ val, const double* __restrict__ x,
                                              const double* __restrict__ bsub, double* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * WARPS;
    for (int s = blockIdx.x * WARPS + (threadIdx.x >> 5); s < S.nslices; s += nw) {
        const int w = S.sptr[s + 1] - S.sptr[s];
        long long base = (long long)S.sptr[s] * 32 + lane;
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
        for (; k + 2 <= w; k += 2, base += 64) {
            a0 = fma(__ldg(val + base), __ldg(x + __ldg(S.col + base)), a0);
            a1 = fma(__ldg(val + base + 32), __ldg(x + __ldg(S.col + base + 32)), a1);
        }
        for (; k < w; ++k, base += 32) a0 = fma(__ldg(val + base), __ldg(x + __ldg(S.col + base)), a0);
        const int ip = s * 32 + lane;
        if (ip < S.n) {
            const int i = S.perm ? __ldg(S.perm + ip) : ip;
            y[i] = bsub ? bsub[i] - (a0 + a1) : a0 + a1;
        }
    }
}

enum SegMode : int { SEG_NORMS = 0, SEG_PQ = 1, SEG_RR = 2, SEG_RZ = 3, SEG_CHECK = 4 };

// Per-system sums in two passes. The rows are cut into chunks of at most
// CHUNK rows that never cross a system boundary; pass 1 sums every chunk
// (all SMs, one CTA per chunk, a fixed tree order), pass 2 adds each system's
// chunk sums in ascending chunk order and applies the system's scalar update.
// The order depends only on the system sizes, so results are reproducible.
constexpr int CHUNK = 4096;

__global__ void __launch_bounds__(TPB) m_chunk_sums(const int* __restrict__ ch_row, const double* __restrict__ u,
                                                    const double* __restrict__ v, const double* __restrict__ w,
                                                    int mode, double* __restrict__ part_a, double* __restrict__ part_b) {
    const int c = blockIdx.x;
    const int r0 = ch_row[c], r1 = ch_row[c + 1];
    double a = 0.0, b = 0.0;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double ui = __ldg(u + i);
        if (mode == SEG_NORMS || mode == SEG_CHECK) {
            const double vi = __ldg(v + i);
            a = fma(ui, ui, a);
            b = fma(vi, vi, b);
        } else if (mode == SEG_RR) {
            a = fma(ui, ui, a);
        } else {
            const double vi = __ldg(v + i);
            a = fma(ui, vi, a);
            if (w) b = fma(__ldg(w + i), vi, b);
        }
    }
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        part_a[c] = a;
        part_b[c] = b;
    }
}

// One thread per system: the system's sums, then its scalar update.
__global__ void m_seg_update(int m, const int* __restrict__ sys_ch, const double* __restrict__ part_a,
                             const double* __restrict__ part_b, BlockScalars sc, int mode, int flexible) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m) return;
    double a = 0.0, b = 0.0;
    for (int c = sys_ch[s]; c < sys_ch[s + 1]; ++c) {
        a += part_a[c];
        b += part_b[c];
    }
    const int md = sc.mode[s];
    switch (mode) {
        case SEG_NORMS:   // u = r = b - A x0, v = b
            if (md != COL_INIT) break;
            sc.rr[s] = a;
            sc.bb[s] = b;
            sc.iters[s] = 0;
            sc.mode[s] = b == 0.0 ? COL_DONE : (a <= sc.rtol[s] * sc.rtol[s] * b ? COL_DONE : COL_START);
            break;
        case SEG_PQ: {    // u = p, v = q
            sc.pq[s] = a;
            if (md == COL_ACTIVE) {
                const double alpha = sc.rho[s] / a;
                if (!(a > 0.0) || !isfinite(alpha)) {
                    sc.mode[s] = COL_FAILED;
                    sc.alpha[s] = 0.0;
                } else {
                    sc.alpha[s] = alpha;
                }
            } else {
                sc.alpha[s] = 0.0;
            }
            break;
        }
        case SEG_RR:      // u = r
            if (md != COL_ACTIVE) break;
            sc.rr[s] = a;
            sc.iters[s] += 1;
            if (a <= sc.rtol[s] * sc.rtol[s] * sc.bb[s]) sc.mode[s] = COL_CHECK;
            break;
        case SEG_RZ:      // u = r, v = z, w = q (flexible)
            if (md == COL_START) {
                sc.rho[s] = a;
                sc.beta[s] = 0.0;
                sc.mode[s] = isfinite(a) ? COL_ACTIVE : COL_FAILED;
            } else if (md == COL_ACTIVE) {
                const double beta = flexible ? -sc.alpha[s] * b / sc.rho[s] : a / sc.rho[s];
                sc.beta[s] = beta;
                sc.rho[s] = a;
                if (!isfinite(beta)) sc.mode[s] = COL_FAILED;
            }
            break;
        case SEG_CHECK:   // u = true residual, v = b
            if (md != COL_CHECK) break;
            sc.rr[s] = a;
            sc.mode[s] = a <= sc.rtol[s] * sc.rtol[s] * sc.bb[s] ? COL_DONE : COL_START;
            break;
        default: break;
    }
}

// The chunk table of a batch and the two passes over it.
struct SegSums {
    int m = 0, nch = 0;
    int* ch_row = nullptr;      // nch + 1 row offsets
    int* sys_ch = nullptr;      // m + 1 chunk offsets
    double *part_a = nullptr, *part_b = nullptr;
    void run(cudaStream_t st, const double* u, const double* v, const double* w, BlockScalars sc, int mode,
             int flexible) const {
        if (nch > 0) {
            m_chunk_sums<<<nch, TPB, 0, st>>>(ch_row, u, v, w, mode, part_a, part_b);
            KERNEL_CHECK();
        }
        m_seg_update<<<(m + 127) / 128, 128, 0, st>>>(m, sys_ch, part_a, part_b, sc, mode, flexible);
        KERNEL_CHECK();
    }
};

// x += alpha_s p, r -= alpha_s q for rows of ACTIVE systems.
__global__ void __launch_bounds__(TPB) m_update_xr(int n, const int* __restrict__ seg_row,
                                                   const double* __restrict__ p, const double* __restrict__ q,
                                                   double* __restrict__ x, double* __restrict__ r, BlockScalars sc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = __ldg(seg_row + i);
        if (sc.mode[s] != COL_ACTIVE) continue;
        const double a = sc.alpha[s];
        x[i] = fma(a, p[i], x[i]);
        r[i] = fma(-a, q[i], r[i]);
    }
}

// p = z + beta_s p for rows of ACTIVE systems (p = z when beta_s = 0).
__global__ void __launch_bounds__(TPB) m_update_p(int n, const int* __restrict__ seg_row,
                                                  const double* __restrict__ z, double* __restrict__ p,
                                                  BlockScalars sc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = __ldg(seg_row + i);
        if (sc.mode[s] != COL_ACTIVE) continue;
        const double be = sc.beta[s];
        p[i] = be == 0.0 ? z[i] : fma(be, p[i], z[i]);
    }
}

// Rows of restarted systems continue from the true residual t.
__global__ void m_copy_restart(int n, const int* __restrict__ seg_row, const double* __restrict__ t,
                               double* __restrict__ r, BlockScalars sc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (sc.mode[__ldg(seg_row + i)] == COL_START) r[i] = t[i];
}

// Rows of systems that converge with b = 0: x = 0.
__global__ void m_zero_done(int n, const int* __restrict__ seg_row, double* __restrict__ x, BlockScalars sc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = __ldg(seg_row + i);
        if (sc.mode[s] == COL_DONE && sc.bb[s] == 0.0) x[i] = 0.0;
    }
}

struct ManyWork {
    DevArena mem;
    BlockScalars sc{};
    int* mode_host = nullptr;
    int* iters_host = nullptr;
    double* rr_host = nullptr;
    double* bb_host = nullptr;
    cudaGraphExec_t step = nullptr;
    long long step_kernels = 0;         // kernels in the step graph (added to the launch count per replay)
    const double* b = nullptr;
    double* x = nullptr;
    ~ManyWork() {
        if (step) cudaGraphExecDestroy(step);
        if (mode_host) cudaFreeHost(mode_host);
        if (iters_host) cudaFreeHost(iters_host);
        if (rr_host) cudaFreeHost(rr_host);
        if (bb_host) cudaFreeHost(bb_host);
    }
};

void copy_state(amg_hierarchy* h, ManyWork& M, int m) {
    cudaStream_t st = h->stream;
    CUDA_CHECK(cudaMemcpyAsync(M.mode_host, M.sc.mode, sizeof(int) * m, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(M.iters_host, M.sc.iters, sizeof(int) * m, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(M.rr_host, M.sc.rr, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(M.bb_host, M.sc.bb, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
}

}  // namespace

amg_status solve_many(amg_hierarchy* h, const double* b, double* x, double rtol, int maxit, amg_solve_info* infos) {
    auto t0 = std::chrono::steady_clock::now();
    const int m = (int)h->seg0.size() - 1;
    if (m < 1) AMG_THROW(AMG_ERR_ARG, "the hierarchy was not built from a batch of systems");
    cudaStream_t st = h->stream;
    Level& L0 = h->lev[0];
    const int n = L0.A.n;
    const SellM S{L0.S.n, L0.S.nslices, L0.S.sptr, L0.S.col, L0.S.perm};
    ManyWork M;
    M.mem.stream = h->stream;
    M.sc.mode = M.mem.alloc<int>(m);
    M.sc.iters = M.mem.alloc<int>(m);
    M.sc.rho = M.mem.alloc<double>(m);
    M.sc.alpha = M.mem.alloc<double>(m);
    M.sc.beta = M.mem.alloc<double>(m);
    M.sc.pq = M.mem.alloc<double>(m);
    M.sc.rr = M.mem.alloc<double>(m);
    M.sc.bb = M.mem.alloc<double>(m);
    M.sc.rtol = M.mem.alloc<double>(m);
    CUDA_CHECK(cudaHostAlloc(&M.mode_host, sizeof(int) * m, cudaHostAllocDefault));
    CUDA_CHECK(cudaHostAlloc(&M.iters_host, sizeof(int) * m, cudaHostAllocDefault));
    CUDA_CHECK(cudaHostAlloc(&M.rr_host, sizeof(double) * m, cudaHostAllocDefault));
    CUDA_CHECK(cudaHostAlloc(&M.bb_host, sizeof(double) * m, cudaHostAllocDefault));
    {
        std::vector<int> md(m, COL_INIT);
        std::vector<double> rt(m, rtol);
        CUDA_CHECK(cudaMemcpyAsync(M.sc.mode, md.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
        CUDA_CHECK(cudaMemcpyAsync(M.sc.rtol, rt.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
        CUDA_CHECK(cudaMemsetAsync(M.sc.iters, 0, sizeof(int) * m, st));
        CUDA_CHECK(cudaStreamSynchronize(st));
    }
    SegSums R;
    {
        std::vector<int> ch_row{0}, sys_ch{0};
        for (int s2 = 0; s2 < m; ++s2) {
            for (int r0 = h->seg0[s2]; r0 < h->seg0[s2 + 1]; r0 += CHUNK)
                ch_row.push_back(std::min(r0 + CHUNK, h->seg0[s2 + 1]));
            sys_ch.push_back((int)ch_row.size() - 1);
        }
        R.m = m;
        R.nch = (int)ch_row.size() - 1;
        R.ch_row = M.mem.alloc<int>(R.nch + 1);
        R.sys_ch = M.mem.alloc<int>(m + 1);
        R.part_a = M.mem.alloc<double>(std::max(R.nch, 1));
        R.part_b = M.mem.alloc<double>(std::max(R.nch, 1));
        CUDA_CHECK(cudaMemcpyAsync(R.ch_row, ch_row.data(), sizeof(int) * (R.nch + 1), cudaMemcpyHostToDevice, st));
        CUDA_CHECK(cudaMemcpyAsync(R.sys_ch, sys_ch.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, st));
        CUDA_CHECK(cudaStreamSynchronize(st));
    }
    const int flexible = h->opt.krylov == 1;
    const int sgrid = std::max(1, std::min((L0.S.nslices + WARPS - 1) / WARPS, h->num_sms * 8));
    const int vgrid = blocks_for(n, TPB, h->num_sms * 8);
    double *r = h->r, *z = h->z, *p = h->p, *q = h->q, *t = h->t;

    // r = b - A x0, per-system norms
    m_spmv<<<sgrid, TPB, 0, st>>>(S, L0.S.val, x, b, r);
    KERNEL_CHECK();
    R.run(st, r, b, nullptr, M.sc, SEG_NORMS, flexible);
    m_zero_done<<<vgrid, TPB, 0, st>>>(n, h->seg_row0, x, M.sc);
    KERNEL_CHECK();

    // one CG step of every system, captured once on a private stream (the
    // caller's stream may be the legacy default stream, which cannot capture)
    // and replayed on the caller's stream
    const bool prof_on = h->prof.on;
    h->prof.on = false;
    cudaStream_t cs = nullptr;
    CUDA_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    h->stream = cs;
    cudaGraph_t graph = nullptr;
    auto restore = [&]() {
        h->stream = st;
        h->prof.on = prof_on;
    };
    try {
        CUDA_CHECK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        const long long before = launch_counter().load();
        try {
            m_spmv<<<sgrid, TPB, 0, cs>>>(S, L0.S.val, p, nullptr, q);
            KERNEL_CHECK();
            R.run(cs, p, q, nullptr, M.sc, SEG_PQ, flexible);
            m_update_xr<<<vgrid, TPB, 0, cs>>>(n, h->seg_row0, p, q, x, r, M.sc);
            KERNEL_CHECK();
            R.run(cs, r, nullptr, nullptr, M.sc, SEG_RR, flexible);
            vcycle_plain(h, r, z);
            R.run(cs, r, z, flexible ? q : nullptr, M.sc, SEG_RZ, flexible);
            m_update_p<<<vgrid, TPB, 0, cs>>>(n, h->seg_row0, z, p, M.sc);
            KERNEL_CHECK();
            M.step_kernels = launch_counter().load() - before;
        } catch (...) {
            cudaStreamEndCapture(cs, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        CUDA_CHECK(cudaStreamEndCapture(cs, &graph));
        CUDA_CHECK(cudaGraphInstantiate(&M.step, graph, 0));
        CUDA_CHECK(cudaGraphDestroy(graph));
    } catch (...) {
        restore();
        cudaStreamDestroy(cs);
        throw;
    }
    restore();
    CUDA_CHECK(cudaStreamDestroy(cs));

    copy_state(h, M, m);
    int steps = 0;
    for (;;) {
        bool live = false;
        int maxi = 0;
        for (int s = 0; s < m; ++s) {
            live |= M.mode_host[s] == COL_START || M.mode_host[s] == COL_ACTIVE;
            maxi = std::max(maxi, M.iters_host[s]);
        }
        if (!live || maxi >= maxit || ++steps > 4 * maxit + 16) break;
        CUDA_CHECK(cudaGraphLaunch(M.step, st));
        launch_counter().fetch_add(M.step_kernels, std::memory_order_relaxed);
        copy_state(h, M, m);
        bool check = false;
        for (int s = 0; s < m; ++s) check |= M.mode_host[s] == COL_CHECK;
        if (check) {
            m_spmv<<<sgrid, TPB, 0, st>>>(S, L0.S.val, x, b, t);
            KERNEL_CHECK();
            R.run(st, t, b, nullptr, M.sc, SEG_CHECK, flexible);
            m_copy_restart<<<vgrid, TPB, 0, st>>>(n, h->seg_row0, t, r, M.sc);
            KERNEL_CHECK();
            copy_state(h, M, m);
        }
    }
    // true residual of every system for the report
    m_spmv<<<sgrid, TPB, 0, st>>>(S, L0.S.val, x, b, t);
    KERNEL_CHECK();
    {
        std::vector<int> md(m, COL_CHECK);
        std::vector<int> keep(M.mode_host, M.mode_host + m);
        CUDA_CHECK(cudaMemcpyAsync(M.sc.mode, md.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
        R.run(st, t, b, nullptr, M.sc, SEG_CHECK, flexible);
        copy_state(h, M, m);
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        amg_status status = AMG_OK;
        for (int s = 0; s < m; ++s) {
            const double nb = std::sqrt(M.bb_host[s]);
            const double tr = nb > 0.0 ? std::sqrt(M.rr_host[s]) / nb : 0.0;
            if (keep[s] == COL_FAILED) status = AMG_ERR_BREAKDOWN;
            else if (keep[s] != COL_DONE && status == AMG_OK) status = AMG_NOT_CONVERGED;
            if (infos) {
                infos[s].iterations = M.iters_host[s];
                infos[s].restarts = 0;
                infos[s].relres = tr;
                infos[s].true_relres = tr;
                infos[s].solve_ms = ms;
            }
        }
        return status;
    }
}

}  // namespace amg
