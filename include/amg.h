/*
 * amg.h -- C ABI of the GB300 matching-aggregation AMG + PCG library.
 *
 * Method: D'Ambra, Durastante, Filippone, "AMG preconditioners for linear
 * solvers towards extreme scale". The library solves A x = b (Eq. 1) for a
 * symmetric positive definite sparse A (Section 3.1) with conjugate gradients
 * preconditioned by one V-cycle (Eq. 2) over a hierarchy built by coarsening
 * based on compatible weighted matching (Section 3.2): edge weights from A and
 * a smooth vector w (Eq. 3), a locally-dominant half-approximate matching with
 * an index tiebreak, pairwise aggregates and the tentative prolongator (Eq. 4)
 * repeated `sweeps` times per level, Galerkin products A_{l+1} = P^T A_l P,
 * l1-Jacobi smoothing (Eq. 5-6 with blocks of one row) and a dense Cholesky
 * solve on the coarsest level.
 *
 * Conventions shared by every call:
 *  - Indices are int32, values float64. CSR: row_ptr[n+1], col[nnz] strictly
 *    ascending within each row, val[nnz]. The pattern must be structurally
 *    symmetric with a stored, positive diagonal.
 *  - Array arguments of amg_setup / amg_solve / amg_vcycle are DEVICE pointers
 *    (cudaMalloc'd or torch tensors on the current device) read and written in
 *    stream order on the stream given in amg_options. The *_host variants take
 *    host pointers and copy through device memory inside the call.
 *  - The caller owns every array it passes; the library copies what it keeps
 *    and never retains a caller pointer after a call returns.
 *  - A hierarchy owns all of its device memory and is released by amg_free.
 *    One call at a time per hierarchy (calls on one handle are serialised).
 *  - No exception or abort crosses the ABI: every failure is an amg_status;
 *    amg_last_error() returns a message for the calling thread. Partial
 *    allocations are freed on failure.
 */
#ifndef AMG_H
#define AMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amg_hierarchy amg_hierarchy;

typedef enum {
    AMG_OK = 0,
    AMG_NOT_CONVERGED = 1,   /* maxit reached; x holds the last iterate, info filled */
    AMG_ERR_ARG = -1,        /* null pointer, bad size, malformed CSR */
    AMG_ERR_NOT_SPD = -2,    /* diagonal missing or <= 0, non-finite value, failed Cholesky pivot */
    AMG_ERR_BAD_W = -3,      /* smooth vector entry zero or non-finite */
    AMG_ERR_OOM = -4,        /* device allocation failed */
    AMG_ERR_CUDA = -5,       /* any other CUDA runtime error */
    AMG_ERR_BREAKDOWN = -6,  /* CG breakdown: p^T A p <= 0 or non-finite scalar */
    AMG_ERR_TIMEOUT = -7,    /* a bounded device-side loop gave up */
    AMG_ERR_TOO_LARGE = -8,  /* coarsest level too large for the dense solve, or size limits */
    AMG_ERR_BUDGET = -9      /* request exceeds the configured device-memory budget */
} amg_status;

enum { AMG_FP64 = 0, AMG_FP32_VCYCLE = 1 };

/* Sparse matrix in CSR form (see conventions). */
typedef struct {
    int32_t n;
    int32_t nnz;
    const int32_t* row_ptr;
    const int32_t* col;
    const double* val;
} amg_csr;

/* amg_options.cycle value for the K-cycle on every intermediate level. */
#define AMG_KCYCLE_FULL 32

/* Options; amg_options_default fills the defaults noted in brackets. */
typedef struct {
    int sweeps;        /* [3] pairwise matching steps per level; aggregates up to 2^sweeps (Section 3.2) */
    int max_coarse;    /* [200] stop when a level has at most this many rows (Section 5) */
    int max_levels;    /* [32] hierarchy depth limit, including the coarsest level */
    int pre, post;     /* [1, 1] l1-Jacobi sweeps before and after the coarse correction (Eq. 2) */
    double omega;      /* [1.0] smoother damping */
    int precision;     /* [AMG_FP64] or AMG_FP32_VCYCLE: V-cycle in float inside FP64 CG */
    int max_dense;     /* [4096] largest coarsest level solved by dense Cholesky; a larger coarsest level is
                          solved by CG with l1-Jacobi to rel-res 1e-4 or 30 iterations (the coarsest-solver
                          setting of Section 5); use krylov = 1 then, as that solve is not a fixed operator */
    int keep_sweeps;   /* [0] keep every sweep's matching and aggregates for amg_export_sweep */
    int profile;       /* [0] time every kernel / setup phase with CUDA events (amg_kernel_stats) */
    int match_kernel;  /* [0] how the locally-dominant matching of each sweep is computed (the same matching
                          every way): 0 = proposals without rounds (Suitor method; hierarchy rounds report
                          0); 1 = locally-dominant rounds, a launch pair per round; 2 = the same rounds in one
                          cooperative launch when the device allows it (else as 1) */
    int krylov;        /* [0] 0 = PCG; 1 = flexible CG keeping one direction (FCG(1), the paper's outer
                          solver, Section 5), robust to a V-cycle that is not exactly linear (FP32) */
    int cycle;         /* [0] 0: V-cycle (Eq. 2). c >= 1: K-cycle on the first c coarse levels: on levels
                          1..c (those that are not the coarsest) the coarse correction is two flexible CG
                          iterations preconditioned by the cycle starting on that level; deeper levels use
                          the V-cycle. AMG_KCYCLE_FULL is the paper's K-cycle on every intermediate level
                          (Section 3.2, the cycle it uses with this unsmoothed aggregation). The
                          preconditioner is then not linear, so the outer solver is flexible CG whatever
                          `krylov` says. Requires pre = post = 1; single right-hand-side solves only */
    int smooth_p;      /* [0] 1: smoothed prolongator Pbar = (I - omega D^-1 A) P on every level, omega =
                          4 / (3 ||D^-1 A||_inf) (see omega_rule), coarse matrices Pbar^T A Pbar (Section 3.2;
                          the paper's VA3 setting; its GPU runs use l1-Jacobi with pre = post = 4). V-cycle
                          (cycle = 0), any pre/post, single right-hand-side solves only. When the next
                          level has more than 12288 rows, a row of A Pbar or of Pbar^T A Pbar may hold up to
                          8192 entries (else AMG_ERR_TOO_LARGE); narrower products have no row limit. The
                          environment variable AMG_SPGEMM_CAP_SHIFT = k (0..3) divides that limit and the
                          product's internal capacity tiers by 2^k (a tier of a warp per row keeps at least
                          64 slots) and turns the narrow-product path off, so small tests reach every tier */
    int autotune;      /* [0] 1: choose the launch shapes of the V-cycle kernels (grid per level and kernel; lanes
                          per row and columns per lane of block solves) by timing candidates once per shape;
                          results are cached per process (see amg_tune_save). 0: fixed heuristics */
    int omega_rule;    /* [0] prolongator smoothing weight of smooth_p: 0 = 4 / (3 ||D^-1 A||_inf), the weight
                          that reproduces the paper's smoothed-aggregation convergence constants; 1 =
                          1 / ||D^-1 A||_inf, the weight the text of Section 3.2 states */
    double min_ratio;  /* [1.5] stop coarsening after a level with n_l / n_{l+1} below this (stalled matching) */
    void* stream;      /* [NULL] cudaStream_t for every device operation and for the hierarchy's stream-ordered
                          allocations; NULL = legacy default. Must stay valid until amg_free */
} amg_options;

/* Per-solve report. */
typedef struct {
    int iterations;      /* products A p (PCG iterations) */
    int restarts;        /* restarts after a failed true-residual check */
    double relres;       /* recursive ||r|| / ||b|| at exit */
    double true_relres;  /* ||b - A x|| / ||b|| at exit, computed in FP64 */
    double solve_ms;     /* wall time of the call on its stream */
} amg_solve_info;

#define AMG_MAX_LEVELS 32
#define AMG_MAX_SWEEPS 8

/* Hierarchy report (Section 5: operator complexity, coarsening ratio). */
typedef struct {
    int num_levels;                                  /* nl, including the coarsest */
    int64_t n[AMG_MAX_LEVELS];                       /* rows per level */
    int64_t nnz[AMG_MAX_LEVELS];                     /* stored entries per level */
    int sweeps_done[AMG_MAX_LEVELS];                 /* matching sweeps applied on each level */
    int rounds[AMG_MAX_LEVELS][AMG_MAX_SWEEPS];      /* locally-dominant rounds per sweep */
    double opc;                                      /* sum nnz(A_l) / nnz(A_0) */
    double avg_coarsening_ratio;                     /* mean of n_l / n_{l+1} over the nl-1 steps */
    double setup_ms;                                 /* wall time of amg_setup */
    int coarse_solver;                               /* 0: dense Cholesky, 1: CG (coarsest above max_dense) */
    size_t device_bytes;                             /* device memory held by the hierarchy */
} amg_hier_info;

void amg_options_default(amg_options* opt);

/*
 * Builds the hierarchy (Sections 3.1-3.3) from A and the smooth vector w
 * (length n; the paper's experiments use w = 1). Device pointers.
 * Errors: AMG_ERR_ARG (null/malformed), AMG_ERR_NOT_SPD, AMG_ERR_BAD_W,
 * AMG_ERR_OOM, AMG_ERR_TOO_LARGE (coarsest level above max_dense),
 * AMG_ERR_TIMEOUT, AMG_ERR_CUDA. *out is NULL on failure.
 */
amg_status amg_setup(const amg_csr* A, const double* w, const amg_options* opt, amg_hierarchy** out);

/* As amg_setup with host arrays (A's three arrays and w). */
amg_status amg_setup_host(const amg_csr* A, const double* w, const amg_options* opt, amg_hierarchy** out);

/*
 * PCG on A x = b preconditioned by one V-cycle (Eq. 2) per iteration, to
 * ||b - A x|| <= rtol ||b|| (Section 5: rtol = 1e-6). Device pointers of
 * length n: b is read, x holds the initial guess on entry and the solution on
 * return. b = 0 returns x = 0 after zero iterations. Returns AMG_OK,
 * AMG_NOT_CONVERGED (x and info still filled) or an error. info may be NULL.
 */
amg_status amg_solve(amg_hierarchy* h, const double* b, double* x, double rtol, int maxit, amg_solve_info* info);

/* As amg_solve with host arrays b and x (copies inside the call). */
amg_status amg_solve_host(amg_hierarchy* h, const double* b, double* x, double rtol, int maxit,
                          amg_solve_info* info);

/*
 * Several right-hand sides at once: B and X are DEVICE arrays, row-major n x k
 * (entry (i, c) at i*k + c), 1 <= k <= 256. Every column runs its own PCG
 * (or flexible CG) with the V-cycle of Eq. 2 to ||b_c - A x_c|| <= rtol ||b_c||;
 * the sparse products and the V-cycle serve all columns in one pass over the
 * matrices. X holds the initial guesses on entry. infos (host, k entries, may
 * be NULL) receives each column's iterations and true relative residual.
 * Needs a hierarchy with at least two levels and pre = post = 1.
 * Returns AMG_OK when every column converged, AMG_NOT_CONVERGED otherwise,
 * AMG_ERR_BREAKDOWN if a column broke down.
 */
amg_status amg_solve_batch(amg_hierarchy* h, int k, const double* B, double* X, double rtol, int maxit,
                           amg_solve_info* infos);

/*
 * Many independent systems at once. amg_setup_many builds one hierarchy for
 * the block-diagonal union of m systems (As[s], ws[s]: DEVICE arrays as for
 * amg_setup). No edge joins two systems, so every system is matched and
 * aggregated exactly as on its own; coarsening stops when the largest system
 * has at most max_coarse rows, and the coarsest level is solved by a dense
 * inverse per system. amg_solve_many runs one CG per system (its own
 * scalars and convergence, all systems in each kernel, each step replayed
 * as one CUDA graph); b and x are the systems' vectors concatenated in order
 * (DEVICE, length = total rows), infos (host, m entries, may be NULL).
 * amg_system_offsets copies the m + 1 row offsets of the systems (host).
 */
amg_status amg_setup_many(int m, const amg_csr* As, const double* const* ws, const amg_options* opt,
                          amg_hierarchy** out);
amg_status amg_solve_many(amg_hierarchy* h, const double* b, double* x, double rtol, int maxit,
                          amg_solve_info* infos);
amg_status amg_system_offsets(const amg_hierarchy* h, int32_t* offsets);

/* One application of the preconditioner, z = B r (Eq. 2), device pointers of length n. */
amg_status amg_vcycle(amg_hierarchy* h, const double* r, double* z);

/* Fills *out (see amg_hier_info). */
amg_status amg_hierarchy_info(const amg_hierarchy* h, amg_hier_info* out);

/*
 * Copies level `level` to HOST arrays; any pointer may be NULL to skip it.
 * row_ptr[n+1], col[nnz], val[nnz]: A_l. w[n]: smooth vector on level l.
 * minv[n]: l1-Jacobi inverse diagonal. agg[n], p[n]: the level prolongator
 * (one nonzero p[i] in column agg[i] of row i; not available on the coarsest).
 */
amg_status amg_export_level(const amg_hierarchy* h, int level, int32_t* row_ptr, int32_t* col, double* val,
                            double* w, double* minv, int32_t* agg, double* p);

/*
 * Smoothed prolongator of level `level` (hierarchies built with smooth_p):
 * amg_pbar_nnz gives its number of stored entries; amg_export_pbar copies the
 * n_l x n_{l+1} CSR to HOST arrays row_ptr[n_l+1], col[nnz], val[nnz]
 * (ascending columns) and its smoothing weight to *omega. Any pointer may be
 * NULL to skip it. AMG_ERR_ARG for a hierarchy without it or a bad level.
 */
amg_status amg_pbar_nnz(const amg_hierarchy* h, int level, int64_t* nnz);
amg_status amg_export_pbar(const amg_hierarchy* h, int level, int32_t* row_ptr, int32_t* col, double* val,
                           double* omega);

/*
 * Copies matching sweep `sweep` of level `level` to HOST arrays (requires
 * keep_sweeps). n = rows of the matrix the sweep matched; mate[n] (partner or
 * -1), agg[n], p[n] (Eq. 4), wc[nc] (coarse smooth vector). Any may be NULL.
 */
amg_status amg_sweep_dims(const amg_hierarchy* h, int level, int sweep, int32_t* n, int32_t* nc, int64_t* nnz_c);
amg_status amg_export_sweep(const amg_hierarchy* h, int level, int sweep, int32_t* mate, int32_t* agg, double* p,
                            double* wc);

/* Dense Cholesky factor L (lower, column-major nc x nc, HOST) of the coarsest level
 * (AMG_ERR_ARG when the coarsest level is solved by CG). */
amg_status amg_coarse_factor(const amg_hierarchy* h, double* L);

/*
 * Per-kernel timing of hierarchy h (requires options.profile): entry `idx`
 * (0 <= idx < count returned by amg_kernel_stats_count) gives the kernel or
 * setup-phase name, the number of timed scopes, their summed CUDA-event time
 * on the hierarchy's stream in ms, and the summed algorithmic bytes (every
 * array the kernel must read or write, counted once). Host outputs; any may
 * be NULL. amg_kernel_stats_reset zeroes the counters.
 */
int amg_kernel_stats_count(void);
amg_status amg_kernel_stats(amg_hierarchy* h, int idx, const char** name, int64_t* scopes, double* total_ms,
                            double* bytes);
amg_status amg_kernel_stats_reset(amg_hierarchy* h);

/* Number of CUDA kernels this library has launched in the process so far. */
int64_t amg_launch_count(void);

/*
 * Algebraically smooth vector for amg_setup (Section 3.2: a few iterations of
 * an A-convergent smoother on a sample vector). Writes to w (DEVICE, length
 * n) the result of `sweeps` l1-Jacobi iterations on A w = 0 from the sample
 * w0 (DEVICE, length n, no zero entries): w <- w - omega M^{-1} A w with
 * M_ii = a_ii + sum_{j != i} |a_ij|. A as for amg_setup; `stream` is a
 * cudaStream_t (NULL = legacy default); returns after the stream work has
 * finished. w may equal w0 for an even number of sweeps. Errors as amg_setup
 * (validation codes on A and w0), AMG_ERR_ARG for sweeps < 0 or omega <= 0.
 */
amg_status amg_smooth_vector(const amg_csr* A, const double* w0, double* w, int sweeps, double omega, void* stream);

/*
 * Matching without allocation. The paper has no counterpart: this is a
 * service for callers that may not allocate device memory at the point where
 * they need a matching -- applications that reserve all device memory at
 * start-up and hand it out from their own pool or budget (a cudaMalloc there
 * would fail or push another tenant out of memory), and latency-bound hosts
 * that forbid allocation after start-up (cudaMalloc and cudaFree can
 * synchronise the device and take an unbounded time).
 *
 * Computes the same edge weights and the same locally-dominant matching with
 * the index tiebreak as the first sweep of amg_setup, and writes mate[i]
 * (partner index, or -1 for an unmatched row) to the caller's DEVICE array
 * of length n. A and w are device arrays as for amg_setup; `stream` is a
 * cudaStream_t (NULL = legacy default stream); *rounds (host, may be NULL)
 * receives the number of matching rounds. The call reads counters back to
 * the host and returns after the stream work has finished.
 *
 * The only working memory is a fixed array inside the library image
 * (about 5.5 MB of device memory on every GPU that loads the library, held
 * until the process exits). Limits: n <= AMG_NOALLOC_MAX_N and
 * nnz <= AMG_NOALLOC_MAX_NNZ; larger inputs return AMG_ERR_TOO_LARGE before
 * any device work. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress), so make that first call before any stream
 * capture begins. All calls share the one array and every call clears the
 * counters it needs: calls that overlap on the GPU (other threads, other
 * streams) race and must be serialised by the caller. No cudaMalloc, cudaFree
 * or other allocating routine is called.
 * Errors as amg_setup (validation codes), AMG_ERR_TIMEOUT, AMG_ERR_CUDA.
 */
#define AMG_NOALLOC_MAX_N 65536
#define AMG_NOALLOC_MAX_NNZ 524288
amg_status amg_match_noalloc(const amg_csr* A, const double* w, int32_t* mate, void* stream, int32_t* rounds);

/*
 * Solve server with continuous batching over cached hierarchies. The paper
 * reuses one preconditioner for many solves (Sections 1 and 5); the server
 * keeps several hierarchies resident and serves right-hand sides for them.
 *
 * amg_serve_create takes nh hierarchies (they must outlive the server, which
 * runs each on a stream of its own until amg_serve_free), `slots` column
 * slots per hierarchy (1..256; the largest request), a device-memory budget
 * in bytes for the columns in flight, and the tolerance / iteration limit of
 * every solve. A hierarchy's workspace for `slots` columns is allocated here.
 *
 * amg_serve_submit queues a request of k right-hand sides for hierarchy hid:
 * B and X are HOST arrays, row-major n x k, that must stay valid until the
 * request completes (X receives the solutions, started from 0). Requests of
 * one hierarchy are admitted in arrival order when enough slots are free and
 * the budget allows; larger requests than the budget return AMG_ERR_BUDGET.
 *
 * amg_serve_step admits what fits, advances every hierarchy with columns in
 * flight by one CG iteration (hierarchies overlap on their own streams),
 * copies finished columns to their X and frees their slots; *pending gets the
 * number of columns still in flight or queued. A column's arithmetic does not
 * depend on the other columns in flight, so a request's result is the same
 * whether it was served alone or in a mix.
 *
 * amg_serve_poll returns up to max completed requests (id, status, latency
 * in ms from submit until the result is in the request's host X, iterations,
 * worst true relative residual);
 * any output pointer may be NULL. amg_serve_stats fills latency percentiles
 * and throughput over all completed requests.
 */
typedef struct amg_server amg_server;
typedef struct {
    int64_t submitted, completed, steps, columns_completed;
    double p50_ms, p99_ms, mean_ms;
    double columns_per_s;   /* right-hand sides completed per second, first submit to last completion */
    double elapsed_s;
    size_t budget_bytes, peak_bytes;
} amg_serve_stats;

amg_status amg_serve_create(int nh, amg_hierarchy* const* hs, int slots, size_t budget_bytes, double rtol, int maxit,
                            amg_server** out);
amg_status amg_serve_submit(amg_server* s, int hid, int k, const double* B, double* X, int64_t* id);
amg_status amg_serve_step(amg_server* s, int64_t* pending);
int amg_serve_poll(amg_server* s, int64_t* ids, int* statuses, double* latency_ms, int* iterations, double* relres,
                   int max);
amg_status amg_serve_stats_get(amg_server* s, amg_serve_stats* out);
void amg_serve_free(amg_server* s);

/*
 * Launch-shape cache of the autotuner (options.autotune). Each entry maps a
 * problem shape (kernel, value type, rows, nonzeros, SELL slices, column
 * count, SM count) to the launch shape that timed fastest. The paper has no
 * counterpart; the GPU kernels' shapes are tuned, not the method.
 * amg_tune_save writes the cache as text (one "key value" per line) to a host
 * file; amg_tune_load merges such a file into the cache (entries with the
 * same key are replaced; malformed lines give AMG_ERR_ARG after the valid
 * ones are read); amg_tune_clear empties it; amg_tune_size counts entries.
 * File errors return AMG_ERR_ARG. Thread-safe.
 */
amg_status amg_tune_save(const char* path);
amg_status amg_tune_load(const char* path);
void amg_tune_clear(void);
int amg_tune_size(void);

/* Releases every device allocation of h. NULL is accepted. */
void amg_free(amg_hierarchy* h);

/* Message of the last failing call on this thread ("" if none). */
const char* amg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AMG_H */
