// amg_internal.cuh -- types and helpers shared by the library's translation
// units (setup, solve, api). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/amg.h"
#include "prof.cuh"

namespace amg {

// ------------------------------------------------------------ errors -------
struct Error {
    amg_status status;
    std::string msg;
};

void set_last_error(const std::string& m);

#define AMG_THROW(st, ...)                                                  \
    do {                                                                    \
        char _b[512];                                                       \
        snprintf(_b, sizeof(_b), __VA_ARGS__);                              \
        throw ::amg::Error{(st), std::string(_b)};                          \
    } while (0)

#define CUDA_CHECK(expr)                                                                  \
    do {                                                                                  \
        cudaError_t _e = (expr);                                                          \
        if (_e != cudaSuccess) {                                                          \
            amg_status _s = (_e == cudaErrorMemoryAllocation) ? AMG_ERR_OOM : AMG_ERR_CUDA; \
            AMG_THROW(_s, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__); \
        }                                                                                 \
    } while (0)

#define KERNEL_CHECK()                                     \
    do {                                                   \
        ::amg::launch_counter().fetch_add(1, std::memory_order_relaxed); \
        CUDA_CHECK(cudaGetLastError());                    \
    } while (0)

// ------------------------------------------------------ device memory ------
// Owner of a set of device allocations, released together.
// Keeps memory freed to the device's default stream-ordered pool reserved for
// the process (release threshold at its maximum), so a later setup reuses it
// without new page mappings. Once per device; a process-local setting.
void keep_pool_reserved();

// Device allocations of one owner, stream-ordered on `stream` (cudaMallocAsync
// / cudaFreeAsync from the device's default pool): allocation and release cost
// no device synchronisation. Work that uses an allocation on another stream
// must be ordered after the allocating stream (a synchronisation or event),
// and `stream` must stay valid until the arena releases its memory.
struct DevArena {
    cudaStream_t stream = nullptr;
    std::vector<void*> ptrs;
    size_t bytes = 0;
    template <typename T>
    T* alloc(size_t count) {
        if (count == 0) count = 1;
        keep_pool_reserved();
        void* p = nullptr;
        CUDA_CHECK(cudaMallocAsync(&p, count * sizeof(T), stream));
        ptrs.push_back(p);
        bytes += count * sizeof(T);
        return static_cast<T*>(p);
    }
    void release(void* p) {
        for (size_t i = 0; i < ptrs.size(); ++i)
            if (ptrs[i] == p) {
                cudaFreeAsync(p, stream);
                ptrs[i] = ptrs.back();
                ptrs.pop_back();
                return;
            }
    }
    void free_all() {
        for (void* p : ptrs) cudaFreeAsync(p, stream);
        ptrs.clear();
        bytes = 0;
    }
    ~DevArena() { free_all(); }
};

// ------------------------------------------------------------ formats ------
struct DevCsr {
    int n = 0;
    int nnz = 0;
    int* ptr = nullptr;
    int* col = nullptr;
    double* val = nullptr;
    int max_row = 0;   // entries of the longest row (0: not known)
};

// SELL-32 (sliced ELLPACK, slice height 32, no row sorting): slice s holds
// rows 32s..32s+31; its entries start at sptr[s] and are stored column-major
// inside the slice (entry k of lane r at sptr[s] + 32k + r). Short rows are
// padded with (col = the row's last column, val = 0). When identity slicing
// would pad more than 30%, rows are sorted by length inside windows of 256
// (SELL-C-sigma) and perm maps slice positions to rows.
constexpr int SELL_C = 32;
struct DevSell {
    int n = 0;
    int nslices = 0;
    int64_t padded = 0;
    int* sptr = nullptr;   // nslices + 1, in units of 32 entries
    int* perm = nullptr;   // row held by each slice position (SELL-C-sigma); null: identity
    int nlong = 0;         // hybrid layout only: rows kept out of the slices (read from the CSR)
    int* long_rows = nullptr;
    int* col = nullptr;
    double* val = nullptr;
    float* val32 = nullptr;
};

struct SweepRecord {
    int n = 0, nc = 0;
    int64_t nnz_c = 0;
    int rounds = 0;
    int* mate = nullptr;
    int* agg = nullptr;
    double* p = nullptr;
    double* wc = nullptr;
};

struct Level {
    DevCsr A;
    DevSell S;                  // A_l in SELL-32 (PCG product, extra smoothing sweeps)
    double* valm = nullptr;     // A_l M_l^{-1} values in S's layout (first pre-smoothing sweep)
    float* valm32 = nullptr;
    DevSell AP;                 // omega M_l^{-1} A_l P_l in SELL-32 (coarse-correction residual update)
    int64_t ap_nnz = 0;
    double* w = nullptr;        // smooth vector on this level
    double* minv = nullptr;     // l1-Jacobi inverse diagonal
    float* minv32 = nullptr;
    double* wminv = nullptr;    // omega M_l^{-1} (the same array as minv when omega = 1)
    float* wminv32 = nullptr;
    // prolongator to the next level (one nonzero per row) and its transpose
    int* agg = nullptr;
    double* p = nullptr;
    float* p32 = nullptr;
    int* pt_ptr = nullptr;      // n_{l+1} + 1
    int* pt_idx = nullptr;      // n_l, members of each aggregate ascending
    int sweeps_done = 0;
    int rounds[AMG_MAX_SWEEPS] = {0};
    std::vector<SweepRecord> sweeps;
    // smoothed prolongator Pbar = (I - omega D^-1 A) P to the next level and
    // its transpose (options.smooth_p): CSR (kept for export) and SELL
    DevCsr pbar, pbar_t;
    DevSell PB, PBT;
    double omega_p = 0.0;
    // K-cycle work vectors of this level as the coarse level of an FCG(2)
    // correction (d1, q1, r2, z2, d2, e), in the V-cycle's value type
    void* kv[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // launch shapes chosen by the autotuner, indexed by value type (0 FP64,
    // 1 FP32); 0 = the fixed heuristic
    int grid_pre[2] = {0, 0}, grid_post[2] = {0, 0}, grid_restrict[2] = {0, 0};
    // V-cycle work vectors (FP64 and FP32 copies)
    double *b = nullptr, *x = nullptr, *r = nullptr, *y = nullptr, *t = nullptr, *u = nullptr;
    float *b32 = nullptr, *x32 = nullptr, *r32 = nullptr, *y32 = nullptr, *t32 = nullptr, *u32 = nullptr;
};

// Device-resident scalars of one PCG solve.
struct PcgScalars {
    double rho;       // r . z
    double rho_new;
    double alpha, beta;
    double pq;        // p . A p
    double rr;        // ||r||^2
    double bb;        // ||b||^2
    int breakdown;
    int pad;
};

// Device scalars of the two FCG iterations of the K-cycle on one level.
struct KcScalars {
    double rho1;     // d1 . A d1
    double alpha1;   // d1 . b / rho1
    double beta;     // z2 . A d1 / rho1
    double alpha2;   // d2 . r2 / d2 . A d2
};

// Workspace of the iterative coarsest solve (coarsest level above max_dense).
struct CoarseCg {
    int blocks = 0;
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    double* part = nullptr;   // 2 buffers x 2 slots x blocks
    int* ctl = nullptr;       // [0] barrier arrivals, [1] error
};

// Column states of a block (multi right-hand side) solve.
enum ColMode : int {
    COL_IDLE = 0, COL_START = 1, COL_ACTIVE = 2, COL_CHECK = 3, COL_DONE = 4, COL_FAILED = 5, COL_INIT = 6
};

// Per-column scalars of a block solve, device arrays of length K.
struct BlockScalars {
    int* mode;
    int* iters;
    double *rho, *alpha, *beta, *pq, *rr, *bb, *rtol;
};

// Workspace of a block solve with K column slots (all arrays row-major n x K).
struct BlockWork {
    int K = 0;
    bool fixed_width = false;           // lanes per row set by K, whatever the column count in flight
    int vec_cols = 1;                   // columns per vector load: 4 (float) or 2 (double)
    int tuned_G = 0;                    // lanes per row chosen by the autotuner (0: heuristic)
    DevArena mem;
    std::vector<void*> b, x, r, y;      // per level V-cycle vectors (float or double)
    double *R = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr, *T = nullptr;   // level 0, FP64
    BlockScalars sc{};
    int* mode_host = nullptr;           // pinned mirrors
    int* iters_host = nullptr;
    double* rr_host = nullptr;
    double* bb_host = nullptr;
    double* partial = nullptr;          // grid x K x 2
    unsigned* ticket = nullptr;
    int grid = 0;
    double* cw[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // coarsest CG x, r, z, p, q (n_c x K)
    double* cpart = nullptr;            // coarsest CG block partials
    int* cctl = nullptr;                // [0] barrier arrivals, [1] error
    cudaGraphExec_t gstep[2] = {nullptr, nullptr};   // captured steps without / with active columns
    long long gkernels[2] = {0, 0};     // kernels in each graph (added to the launch count per replay)
    int gk = -1;                        // column count and output the graphs were captured for
    const double* gX = nullptr;
    ~BlockWork();
};

struct Reducer {
    double* partial = nullptr;   // one slot per block
    unsigned* ticket = nullptr;  // last-block counter
    int blocks = 0;
};

}  // namespace amg

struct amg_hierarchy {
    amg_options opt;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    int coop_blocks = 0;        // grid of the cooperative matching kernel (0: not available)
    amg::DevArena mem;
    std::vector<amg::Level> lev;
    int nc = 0;                 // coarsest size
    int coarse_cg = 0;          // 1: coarsest solved by CG (above max_dense)
    bool r32_ready = false;     // the CG update wrote level 0's float r for the next V-cycle call
    amg::CoarseCg ccg;
    double* coarse_L = nullptr;  // dense Cholesky factor (column-major)
    double* coarse_inv = nullptr;// dense inverse A_L^{-1} (row-major)
    // PCG workspace (level 0 sized)
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *t = nullptr;
    amg::PcgScalars* sc = nullptr;      // device
    amg::PcgScalars* sc_host = nullptr; // pinned mirror
    amg::Reducer red;
    amg::KcScalars* ks = nullptr;       // K-cycle scalars, one per level (device)
    amg::BlockWork* blk = nullptr;      // block-solve workspace, created on first use
    // batch of independent systems (block-diagonal union): system offsets
    std::vector<int> seg0;               // level 0, m + 1 entries (empty: one system)
    std::vector<std::vector<int>> segs;  // per level
    int* seg_row0 = nullptr;             // device: system of each level-0 row
    int* segL_ptr = nullptr;             // device: coarsest-level system offsets
    long long* segL_blk = nullptr;       // device: offsets of the per-system dense inverses
    double setup_ms = 0.0;
    amg::Profiler prof;
    std::mutex lock;
};

namespace amg {

// ------------------------------------------------------- launch sizes ------
inline int blocks_for(long long n, int threads, int cap) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// Exclusive prefix sum of int32 counts (out may alias in). Returns the total
// through *total_dev (device) and, if total_host is non-null, synchronously
// to the host.
void scan_exclusive(const int* in, int* out, int n, int* total_dev, cudaStream_t st, int* scratch_blocks);
size_t scan_scratch_ints(int n);

// Setup and solve entry points used by the api translation unit.
void setup_hierarchy(amg_hierarchy* h, const amg_csr* A, const double* w);
void prepare_solve(amg_hierarchy* h);

// Autotuner (tune.cu holds the cache): choose the V-cycle launch shapes of
// every level by timing candidates (solve.cu).
bool tune_get(const std::string& key, int* value);
void tune_put(const std::string& key, int value);
std::string tune_key(const char* kind, int vbytes, long long n, long long nnz, long long slices, int k, int sms);
void autotune_vcycle(amg_hierarchy* h);

// Mean time in ms of `reps` launches issued by `launch` on stream st, after
// one untimed launch.
template <typename F>
double time_launches(cudaStream_t st, F&& launch, int reps) {
    launch();
    cudaEvent_t e0, e1;
    CUDA_CHECK(cudaEventCreate(&e0));
    CUDA_CHECK(cudaEventCreate(&e1));
    CUDA_CHECK(cudaEventRecord(e0, st));
    for (int i = 0; i < reps; ++i) launch();
    CUDA_CHECK(cudaEventRecord(e1, st));
    CUDA_CHECK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (double)ms / reps;
}
amg_status solve(amg_hierarchy* h, const double* b, double* x, double rtol, int maxit, amg_solve_info* info);
void vcycle_apply(amg_hierarchy* h, const double* r, double* z);
// Single-column coarsest CG solve on contiguous FP64 vectors (coarse_cg hierarchies).
void coarse_cg_solve(amg_hierarchy* h, const double* b, double* x);
// Block (multi right-hand side) solve.
amg_status solve_batch(amg_hierarchy* h, int k, const double* B, double* X, double rtol, int maxit,
                       amg_solve_info* infos);
void block_free(amg_hierarchy* h);
// Batch of independent systems (many.cu, setup_many in setup.cu).
void setup_many(amg_hierarchy* h, int m, const amg_csr* As, const double* const* ws);
amg_status solve_many(amg_hierarchy* h, const double* b, double* x, double rtol, int maxit, amg_solve_info* infos);
// Solve server (serve.cu).
amg_server* serve_create(int nh, amg_hierarchy* const* hs, int K, size_t budget, double rtol, int maxit);
void serve_free(amg_server* S);
int64_t serve_submit(amg_server* S, int hid, int k, const double* B, double* X);
int64_t serve_step(amg_server* S);
int serve_poll(amg_server* S, int64_t* ids, int* statuses, double* latency_ms, int* iters, double* relres, int max);
void serve_stats(amg_server* S, amg_serve_stats* o);
// Pieces of a block solve for a scheduler (all launch-only on h->stream).
BlockWork& block_ensure(amg_hierarchy* h, int K, bool fixed_width);
size_t block_bytes_per_column(const amg_hierarchy* h);
void block_set_columns(amg_hierarchy* h, int c0, int cnt, int mode, double rtol);
void block_init_launch(amg_hierarchy* h, const double* B, double* X, int k);
void block_step_launch(amg_hierarchy* h, const double* B, double* X, int k);
bool block_check_launch(amg_hierarchy* h, const double* B, double* X, int k);
// Request staging for the server: scatter a contiguous n x k block into slot
// columns (src null: zero them) / gather one slot column into column j of n x k.
void block_scatter_request(amg_hierarchy* h, const double* src, int k, const int* slots, double* dst);
void block_gather_column(amg_hierarchy* h, const double* src, int slot, double* dst, int k, int j);
amg_status match_noalloc(const amg_csr* A, const double* w, int32_t* mate, void* stream, int32_t* rounds_out);
void smooth_vector(const amg_csr* A, const double* w0, double* w, int sweeps, double omega, cudaStream_t st);

}  // namespace amg
