// setup.cu -- hierarchy construction on the device: coarsening based on
// compatible weighted matching (Section 3.2), Galerkin products (Section 3.1),
// l1-Jacobi smoother setup (Section 3.3, Eq. 5-6 with one-row blocks) and the
// dense Cholesky factor of the coarsest level.
//
// The matching and the operators it produces must not depend on rounding
// choices: weights (Eq. 3), the pair normalisation (Eq. 4) and the Galerkin
// sums use explicitly rounded operations (__dmul_rn, __dadd_rn, ...), never a
// fused multiply-add, in a fixed order that is part of the definition.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstring>

#include "amg_internal.cuh"
#include "device_util.cuh"

namespace amg {

namespace {

constexpr int TPB = 256;

// ------------------------------------------------------------- checks ------
enum : int { F_SHAPE = 1, F_NOT_SPD = 2, F_BAD_W = 4 };

__device__ __forceinline__ int find_in_row(const int* __restrict__ ptr, const int* __restrict__ col, int row, int j) {
    int lo = ptr[row], hi = ptr[row + 1];
    if (hi - lo <= 8) {
        // a short row: its (at most 8) columns are loaded together, one
        // memory latency instead of one per bisection step
        int c[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) c[t] = lo + t < hi ? col[lo + t] : -1;
        int at = -1;
#pragma unroll
        for (int t = 0; t < 8; ++t) at = c[t] == j ? lo + t : at;
        return at;
    }
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (col[mid] < j) lo = mid + 1; else hi = mid;
    }
    return (lo < ptr[row + 1] && col[lo] == j) ? lo : -1;
}

// Edge weights mark non-edges with -inf. Tested on the bits: a double
// compare issues on this GPU's FP64 pipe (1/64 of the FP32 rate), an integer
// compare does not.
constexpr long long NEG_INF_BITS = (long long)0xfff0000000000000ULL;
__device__ __forceinline__ bool is_edge(double cw) { return __double_as_longlong(cw) != NEG_INF_BITS; }

// Row pointers first: monotone, starting at 0, ending at nnz.
__global__ void k_check_ptr(int n, int nnz, const int* __restrict__ ptr, int* flags) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i <= n; i += (long long)gridDim.x * blockDim.x) {
        int a = ptr[i];
        bool bad = (a < 0 || a > nnz) || (i == 0 && a != 0) || (i == n && a != nnz) || (i < n && ptr[i + 1] < a);
        if (bad) atomicOr(flags, F_SHAPE);
    }
}

// Columns sorted and in range, finite values, positive stored diagonal,
// symmetric pattern; w finite and nonzero. Writes the diagonal.
__global__ void k_check_rows(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ w, double* __restrict__ diag,
                             int* flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int f = 0;
        double d = 0.0;
        int prev = -1;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
            int j = col[k];
            if (j < 0 || j >= n || j <= prev) { f |= F_SHAPE; break; }
            prev = j;
            double v = val[k];
            if (!isfinite(v)) f |= F_NOT_SPD;
            if (j == i) d = v;
            else if (find_in_row(ptr, col, j, i) < 0) f |= F_SHAPE;
        }
        if (!(d > 0.0)) f |= F_NOT_SPD;
        double wi = w[i];
        if (!isfinite(wi) || wi == 0.0) f |= F_BAD_W;
        diag[i] = d;
        if (f) atomicOr(flags, f);
    }
}

// *mx = max(*mx, longest row): a block maximum, then one atomic per block.
__global__ void k_max_row(int n, const int* __restrict__ ptr, int* mx) {
    int m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, ptr[i + 1] - ptr[i]);
    m = block_max_int(m);
    if (threadIdx.x == 0 && m > 0) atomicMax(mx, m);
}

// dww[i] = (a_ii w_i) w_i, the per-vertex half of the weight denominator
// (the same rounded value in every edge of i).
__global__ void k_diag(int n, const int* __restrict__ ptr, const int* __restrict__ col, const double* __restrict__ val,
                       const double* __restrict__ w, double* __restrict__ dww) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int k = find_in_row(ptr, col, i, i);
        const double d = k >= 0 ? val[k] : 0.0;
        dww[i] = __dmul_rn(__dmul_rn(d, w[i]), w[i]);
    }
}

// In place: diag[i] <- (diag[i] w_i) w_i.
__global__ void k_dww(int n, double* __restrict__ diag, const double* __restrict__ w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        diag[i] = __dmul_rn(__dmul_rn(diag[i], w[i]), w[i]);
}

// --------------------------------------------------- Eq. 3 edge weights ----
// c_ij = 1 - 2 a_ij w_i w_j / (a_ii w_i^2 + a_jj w_j^2) for the pair {lo, hi}
// from the upper entry a_{lo,hi}; written at both stored positions of the
// pair. Diagonal entries and pairs whose upper entry is 0 are not edges and
// get -inf.
// dww = (a_ii w_i) w_i per vertex (k_diag / k_dww): the denominator is
// dww_i + dww_j, the same rounded terms as evaluated per edge; the numerator
// (2 a) w_i w_j is formed as (a (2 w_i)) w_j, the same single rounding of
// the same exact product. FP64 work per edge: one add, two multiplies, the
// division and the subtraction (this GPU's FP64 pipe bounds this kernel).
// A group of G lanes per row (G = 1, 8, 16 or 32 by the mean row length),
// the row's entries strided over the group, so long rows are shared out.
template <int G>
__global__ void __launch_bounds__(TPB) k_weights(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                                                 const double* __restrict__ val, const double* __restrict__ dww,
                                                 const double* __restrict__ w, double* __restrict__ c) {
    const double NEG_INF = -__longlong_as_double(0x7ff0000000000000LL);
    const int gl = threadIdx.x & (G - 1);
    const int ng = (gridDim.x * blockDim.x) / G;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / G; i < n; i += ng) {
        const double wi = w[i], si = dww[i];
        const double w2i = wi + wi;
        const int e = ptr[i + 1];
        for (int k = ptr[i] + gl; k < e; k += G) {
            const int j = col[k];
            if (j < i) continue;                 // written by the group of row j
            if (j == i) { c[k] = NEG_INF; continue; }
            const double a = val[k];
            double cw = NEG_INF;
            if (a != 0.0) {
                const double den = __dadd_rn(si, dww[j]);
                const double num = __dmul_rn(__dmul_rn(a, w2i), w[j]);
                cw = __dsub_rn(1.0, __ddiv_rn(num, den));
            }
            c[k] = cw;
            const int mirror = find_in_row(ptr, col, j, i);
            if (mirror >= 0) c[mirror] = cw;
        }
    }
}

// ------------------------------------- locally-dominant matching rounds ----
// mate[v]: -1 free, -2 free without free neighbours, >= 0 partner.
// cand[v]: best free neighbour of a free v under the strict edge order
// (weight descending, lower end ascending, upper end ascending).
// The weight comparison runs on integers: the bits of a non-NaN double,
// with the magnitude bits flipped when the sign is set (and -0 taken as +0),
// order like the double itself. On this GPU a double compare issues on the
// FP64 pipe, which runs at 1/64 of the FP32 rate; integer compares do not.
__device__ __forceinline__ long long weight_order(double c) {
    const long long b = __double_as_longlong(c);
    if (b == (long long)0x8000000000000000ULL) return 0;
    return b < 0 ? (b ^ 0x7fffffffffffffffLL) : b;
}

__device__ __forceinline__ bool key_better(double c1, int lo1, int hi1, double c2, int lo2, int hi2) {
    const long long k1 = weight_order(c1), k2 = weight_order(c2);
    if (k1 != k2) return k1 > k2;
    if (lo1 != lo2) return lo1 < lo2;
    return hi1 < hi2;
}

__device__ __forceinline__ int best_free(int v, const int* __restrict__ ptr, const int* __restrict__ col,
                                         const double* __restrict__ c, const int* mate) {
    int best = -1, blo = 0, bhi = 0;
    double bc = 0.0;
    const double NEG_INF = -__longlong_as_double(0x7ff0000000000000LL);
    for (int k = ptr[v]; k < ptr[v + 1]; ++k) {
        const double cw = c[k];
        if (!is_edge(cw)) continue;
        const int u = col[k];
        if (mate[u] != -1) continue;
        const int lo = min(u, v), hi = max(u, v);
        if (best < 0 || key_better(cw, lo, hi, bc, blo, bhi)) {
            best = u; bc = cw; blo = lo; bhi = hi;
        }
    }
    return best;
}

__global__ void k_ld_init(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                          const double* __restrict__ c, int* cand, int* mate) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int b = best_free(v, ptr, col, c, mate);
        cand[v] = b;
        if (b < 0) mate[v] = -2;   // isolated: nobody reads it
    }
}

// Round, part 1: mutual candidates are locally dominant edges; match them.
// list == nullptr means every vertex. Zeroes the next round's list counter.
__global__ void k_ld_match(int n, const int* __restrict__ list, const int* __restrict__ list_cnt, const int* cand,
                           int* mate, int* mlist, int* mcnt, int* zero_next, int* rounds) {
    const int cnt = list ? min(*list_cnt, n) : n;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *zero_next = 0;
        if (cnt > 0) *rounds += 1;
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int v = list ? list[t] : t;
        bool take = false;
        int lo = 0, hi = 0;
        if (mate[v] == -1) {
            const int u = cand[v];
            if (u >= 0 && cand[u] == v) {
                lo = min(u, v); hi = max(u, v);
                if (atomicCAS(&mate[lo], -1, hi) == -1) {
                    mate[hi] = lo;
                    take = true;
                }
            }
        }
        warp_append(take, lo, mlist, mcnt, n);
        warp_append(take, hi, mlist, mcnt, n);
    }
}

// Round, part 2: free vertices whose candidate was just matched pick a new
// one; they form the next round's list. Zeroes the next round's match counter.
__global__ void k_ld_update(int n, const int* __restrict__ ptr, const int* __restrict__ col, const double* __restrict__ c,
                            int* cand, int* mate, const int* __restrict__ mlist, const int* __restrict__ mcnt,
                            int* next_list, int* next_cnt, int* zero_next_m) {
    const int cnt = min(*mcnt, n);
    if (blockIdx.x == 0 && threadIdx.x == 0) *zero_next_m = 0;
    const double NEG_INF = -__longlong_as_double(0x7ff0000000000000LL);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int m = mlist[t];
        for (int k = ptr[m]; k < ptr[m + 1]; ++k) {
            bool take = false;
            int x = col[k];
            if (is_edge(c[k]) && mate[x] == -1 && cand[x] == m) {
                const int b = best_free(x, ptr, col, c, mate);
                cand[x] = b;
                if (b < 0) mate[x] = -2;
                else take = true;
            }
            warp_append(take, x, next_list, next_cnt, n);
        }
    }
}


// ------------------------------- all matching rounds in one cooperative launch
// The same rounds as k_ld_match / k_ld_update, separated by a software grid
// barrier instead of kernel boundaries. Each vertex's edges are sorted once
// by the strict edge order, so its best free neighbour is found by moving a
// forward-only pointer past neighbours that are no longer free (vertices only
// ever stop being free). Values that other blocks change during the launch
// (mate, cand, pos, lists, counters) are read with ld.cg so the per-SM L1
// cannot serve a stale copy. Every wait is bounded by a 2 s timer: a block
// that waits longer sets *err and all blocks leave the round loop.
constexpr unsigned long long BAR_TIMEOUT_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier number `epoch` (1, 2, ...): every block adds one to *count and
// waits until it reaches epoch * gridDim.x. *count starts at 0 per launch.
__device__ __forceinline__ void grid_sync(unsigned* count, unsigned epoch, int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        const unsigned target = epoch * gridDim.x;
        if (ld_acquire_u32(count) < target) {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u32(count) < target) {
                if (global_ns() - t0 > BAR_TIMEOUT_NS) {
                    atomicExch(err, 1);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Sorts row v's edges by the strict order into (sc, nbr) at the row's own
// CSR segment; entries that are not edges go last with nbr = -1.
// With `list` set, only the rows list[0 .. *nlist) (those the group kernel
// below leaves out).
__global__ void k_sort_edges(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                             const double* __restrict__ c, double* __restrict__ sc, int* __restrict__ nbr,
                             int* __restrict__ pos, int* __restrict__ cand, int* mate, const int* __restrict__ list,
                             const int* __restrict__ nlist, int* __restrict__ spos) {
    const double NEG_INF = -__longlong_as_double(0x7ff0000000000000LL);
    const int nr = list ? *nlist : n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nr; t += gridDim.x * blockDim.x) {
        const int v = list ? list[t] : t;
        const int b = ptr[v], e = ptr[v + 1];
        int m = b;
        for (int k = b; k < e; ++k) {
            const double cw = c[k];
            if (!is_edge(cw)) continue;
            const int u = col[k];
            int d = m - 1;
            // insert (cw, u) keeping the order: larger weight, then smaller (lo, hi)
            while (d >= b && key_better(cw, min(u, v), max(u, v), sc[d], min(nbr[d], v), max(nbr[d], v))) {
                sc[d + 1] = sc[d];
                nbr[d + 1] = nbr[d];
                --d;
            }
            sc[d + 1] = cw;
            nbr[d + 1] = u;
            ++m;
        }
        for (int k = m; k < e; ++k) nbr[k] = -1;
        if (spos)
            for (int k = b; k < m; ++k) spos[find_in_row(ptr, col, v, nbr[k])] = k;
        pos[v] = b;
        cand[v] = m > b ? nbr[b] : -1;
        if (m == b) mate[v] = -2;
    }
}

// The same for rows of at most G entries, one group of G lanes per row: lane
// t holds entry t, its rank among the row's edges under the strict order comes
// from a shuffle sweep (edges have distinct keys), non-edges follow the edges
// in position order; entries are written to their ranks. With `list` set,
// only the listed rows. Longer rows are listed in long_list for a pass with
// more lanes or the block-per-row kernels.
template <int G>
__global__ void __launch_bounds__(TPB) k_sort_edges_group(int n, const int* __restrict__ list,
                                                         const int* __restrict__ nlist, const int* __restrict__ ptr,
                                                         const int* __restrict__ col, const double* __restrict__ c,
                                                         int* __restrict__ nbr, int* __restrict__ pos,
                                                         int* __restrict__ cand, int* mate, int* __restrict__ long_list,
                                                         int* __restrict__ nlong, int* __restrict__ spos) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int ng = (gridDim.x * blockDim.x) / G;
    const int v0 = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int warp_first = v0 - (lane - gl) / G;     // every lane of a warp runs the same iterations
    const int nr = list ? min(*nlist, n) : n;        // with a list, only the rows list[0 .. *nlist)
    for (int it = 0; warp_first + it * ng < nr; ++it) {
        const int t = v0 + it * ng;
        const int v = t < nr ? (list ? list[t] : t) : n;
        int b = 0, len = 0;
        if (v < n) {
            b = ptr[v];
            len = ptr[v + 1] - b;
            if (len > G) {
                if (gl == 0) long_list[atomicAdd(nlong, 1)] = v;
                len = -1;
            }
        }
        // key of this lane's entry: (weight order, neighbour); within one row
        // the strict order's (lo, hi) tiebreak is the neighbour's index order.
        // Non-edges carry neighbour INT_MAX.
        long long wk = (long long)0x8000000000000000ULL;
        int u = -1, uk = 0x7fffffff;
        bool edge = false;
        if (gl < len) {
            const double cw = c[b + gl];
            u = col[b + gl];
            edge = is_edge(cw);
            if (edge) {
                wk = weight_order(cw);
                uk = u;
            }
        }
        int better = 0, nedge = 0, nonedge_before = 0;
#pragma unroll
        for (int t = 0; t < G; ++t) {
            const long long wt = __shfl_sync(FULL_MASK, wk, t, G);
            const int ut = __shfl_sync(FULL_MASK, uk, t, G);
            const bool et = ut != 0x7fffffff;
            nedge += et;
            better += et && (wt > wk || (wt == wk && ut < uk));
            nonedge_before += (t < gl && t < len && !et);
        }
        if (gl < len) {
            const int rank = edge ? better : nedge + nonedge_before;
            nbr[b + rank] = edge ? u : -1;
            if (spos) spos[b + gl] = b + rank;
            if (edge && rank == 0) cand[v] = u;
        }
        if (gl == 0 && len >= 0 && v < n) {
            pos[v] = b;
            if (nedge == 0) {
                cand[v] = -1;
                mate[v] = -2;
            }
        }
    }
}

// Rows longer than the group kernel's G but at most CAP entries, one
// block per listed row: (edge, weight order, neighbour) keys bitonic-sorted in
// shared memory, edges first by the strict order (larger weight, then smaller
// (lo, hi), which for a fixed row is the smaller neighbour), non-edges last.
// Longer rows are appended to `longer` for a launch of larger CAP or for
// k_sort_edges.
constexpr int EDGE_CAPS[2] = {4096, 16384};
constexpr int LONG_TPB = 256;
__global__ void __launch_bounds__(LONG_TPB) k_sort_edges_long(const int* __restrict__ list,
                                                              const int* __restrict__ nlist, int CAP,
                                                              const int* __restrict__ ptr,
                                                              const int* __restrict__ col,
                                                              const double* __restrict__ c, int* __restrict__ nbr,
                                                              int* __restrict__ pos, int* __restrict__ cand, int* mate,
                                                              int* __restrict__ longer, int* __restrict__ nlonger,
                                                              int* __restrict__ spos) {
    extern __shared__ long long esm[];
    long long* WK = esm;
    int* U = reinterpret_cast<int*>(esm + CAP);
    const double NEG_INF = -__longlong_as_double(0x7ff0000000000000LL);
    const int tid = threadIdx.x;
    const int nr = *nlist;
    for (int t = blockIdx.x; t < nr; t += gridDim.x) {
        const int v = list[t];
        const int b = ptr[v], len = ptr[v + 1] - b;
        if (len > CAP) {
            if (tid == 0) longer[atomicAdd(nlonger, 1)] = v;
            continue;
        }
        int m2 = 1;
        while (m2 < len) m2 <<= 1;
        for (int s = tid; s < m2; s += LONG_TPB) {
            const double cw = s < len ? c[b + s] : NEG_INF;
            const bool edge = is_edge(cw);
            WK[s] = edge ? weight_order(cw) : (long long)0x8000000000000000ULL;
            U[s] = edge ? col[b + s] : 0x7fffffff;
        }
        __syncthreads();
        // x before y: edges first, then larger weight order, then smaller neighbour
        auto before = [](long long wx, int ux, long long wy, int uy) {
            const bool ex = ux != 0x7fffffff, ey = uy != 0x7fffffff;
            if (ex != ey) return ex;
            if (wx != wy) return wx > wy;
            return ux < uy;
        };
        for (int size = 2; size <= m2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int u = tid; u < m2 / 2; u += LONG_TPB) {
                    const int lo = 2 * u - (u & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const long long wl = WK[lo], wh = WK[hi];
                    const int ul = U[lo], uh = U[hi];
                    if (up ? before(wh, uh, wl, ul) : before(wl, ul, wh, uh)) {
                        WK[lo] = wh;
                        WK[hi] = wl;
                        U[lo] = uh;
                        U[hi] = ul;
                    }
                }
                __syncthreads();
            }
        for (int s = tid; s < len; s += LONG_TPB) {
            nbr[b + s] = U[s] != 0x7fffffff ? U[s] : -1;
            if (spos && U[s] != 0x7fffffff) spos[find_in_row(ptr, col, v, U[s])] = b + s;
        }
        if (tid == 0) {
            pos[v] = b;
            const bool any = len > 0 && U[0] != 0x7fffffff;
            cand[v] = any ? U[0] : -1;
            if (!any) mate[v] = -2;
        }
        __syncthreads();
    }
}

// The same as k_sort_edges_long for rows of up to WROW entries, one warp per
// listed row: the warp sorts its row in its own slice of shared memory with
// warp barriers between the bitonic stages (a block and its barriers would
// be spent on a few hundred entries). Longer rows go to `longer`.
constexpr int WROW = 256;
constexpr int WPB = TPB / 32;
__global__ void __launch_bounds__(TPB) k_sort_edges_warp(const int* __restrict__ list, const int* __restrict__ nlist,
                                                         const int* __restrict__ ptr, const int* __restrict__ col,
                                                         const double* __restrict__ c, int* __restrict__ nbr,
                                                         int* __restrict__ pos, int* __restrict__ cand, int* mate,
                                                         int* __restrict__ longer, int* __restrict__ nlonger,
                                                         int* __restrict__ spos) {
    __shared__ long long WKs[WPB][WROW];
    __shared__ int Us[WPB][WROW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long* WK = WKs[w];
    int* U = Us[w];
    const int nr = *nlist;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nr; t += nwarps) {
        const int v = list[t];
        const int b = ptr[v], len = ptr[v + 1] - b;
        if (len > WROW) {
            if (lane == 0) longer[atomicAdd(nlonger, 1)] = v;
            continue;
        }
        int m2 = 1;
        while (m2 < len) m2 <<= 1;
        for (int s = lane; s < m2; s += 32) {
            const double cw = s < len ? c[b + s] : -__longlong_as_double(0x7ff0000000000000LL);
            const bool edge = is_edge(cw);
            WK[s] = edge ? weight_order(cw) : (long long)0x8000000000000000ULL;
            U[s] = edge ? col[b + s] : 0x7fffffff;
        }
        __syncwarp();
        // x before y: edges first, then larger weight order, then smaller neighbour
        auto before = [](long long wx, int ux, long long wy, int uy) {
            const bool ex = ux != 0x7fffffff, ey = uy != 0x7fffffff;
            if (ex != ey) return ex;
            if (wx != wy) return wx > wy;
            return ux < uy;
        };
        for (int size = 2; size <= m2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int u = lane; u < m2 / 2; u += 32) {
                    const int lo = 2 * u - (u & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const long long wl = WK[lo], wh = WK[hi];
                    const int ul = U[lo], uh = U[hi];
                    if (up ? before(wh, uh, wl, ul) : before(wl, ul, wh, uh)) {
                        WK[lo] = wh;
                        WK[hi] = wl;
                        U[lo] = uh;
                        U[hi] = ul;
                    }
                }
                __syncwarp();
            }
        for (int s = lane; s < len; s += 32) {
            nbr[b + s] = U[s] != 0x7fffffff ? U[s] : -1;
            if (spos && U[s] != 0x7fffffff) spos[find_in_row(ptr, col, v, U[s])] = b + s;
        }
        if (lane == 0) {
            pos[v] = b;
            const bool any = len > 0 && U[0] != 0x7fffffff;
            cand[v] = any ? U[0] : -1;
            if (!any) mate[v] = -2;
        }
        __syncwarp();
    }
}

// Best free neighbour of v from its sorted list starting at k = pos[v]
// (e = end of v's row); advances pos[v]. Four list entries and their mate
// words are loaded together, so skipping matched neighbours costs two memory
// latencies per four entries rather than two per entry.
__device__ __forceinline__ int best_free_sorted(int v, int k, int e, const int* __restrict__ nbr, int* pos,
                                                const int* mate) {
    int found = -1;
    while (k < e) {
        int u[4], ms[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) u[t] = k + t < e ? __ldg(nbr + k + t) : -1;
#pragma unroll
        for (int t = 0; t < 4; ++t) ms[t] = u[t] >= 0 ? __ldcg(mate + u[t]) : 0;
        int t = 0;
        for (; t < 4; ++t) {
            if (u[t] < 0) {          // past the row or into its non-edges: nothing free
                k = e;
                break;
            }
            if (ms[t] == -1) {
                found = u[t];
                break;
            }
            ++k;
        }
        if (t < 4) break;
    }
    pos[v] = k;
    return k < e ? found : -1;
}

// Appends each thread's k items (k <= BA_MAX) to list[*cnt...] with one
// atomic per block. Every thread of the block must call it.
constexpr int BA_MAX = 8;
__device__ __forceinline__ void block_append(int k, const int* items, int* list, int* cnt, int cap) {
    __shared__ int s_base;
    const int off = block_exclusive_scan_int(k);
    if (threadIdx.x == blockDim.x - 1) {
        const int total = off + k;
        s_base = total > 0 ? atomicAdd(cnt, total) : 0;
    }
    __syncthreads();
    const int b = s_base + off;
    for (int i = 0; i < k; ++i)
        if (b + i < cap) list[b + i] = items[i];
    __syncthreads();
}

__device__ __forceinline__ void fence_sc_gpu() { asm volatile("fence.sc.gpu;" ::: "memory"); }

// Round r >= 1 of the persistent matching over work items first, first +
// stride, ...: 2^ngl consecutive items per vertex matched in round r - 1,
// item gl taking its neighbours gl, gl + 2^ngl, ...; no block-wide
// synchronisation inside the round, so the work items of a thread overlap.
// Pairs are collected per thread (beyond BA_MAX straight into the list) and
// appended once per block. Every thread of the block must call it.
constexpr int LD_SOLO_ITEMS = 1024;   // rounds with at most this many items run in one block
__device__ __forceinline__ void ld_round(long long r, long long first, long long stride, int ngl,
                                         const int* __restrict__ ptr,
                                         const int* __restrict__ col, const int* __restrict__ nbr, int* pos,
                                         int* cand, int* mate, int* const* lists, int* cnt, int n, bool leader) {
    const int* M = lists[(r - 1) & 1];
    const int m_cnt = min(__ldcg(cnt + (int)((r - 1) % 3)), n);
    int* nl = lists[r & 1];
    int* nc = cnt + (int)(r % 3);
    // slot (r+1) % 3 was last read at the start of round r-1; it collects round r+1's pairs
    if (leader) cnt[(int)((r + 1) % 3)] = 0;
    int items[BA_MAX];
    int k = 0;
    const int ng = 1 << ngl;
    const long long total = (long long)m_cnt << ngl;
    for (long long u = first; u < total; u += stride) {
        const int t = (int)(u >> ngl), gl = (int)(u & (ng - 1));
        const int m = __ldcg(M + t);
        const int ke = __ldg(ptr + m + 1);
        for (int q = __ldg(ptr + m) + gl; q < ke; q += ng) {
            const int x = __ldg(col + q);
            // x's state and its list position together (one latency)
            const int mx = __ldcg(mate + x), cx = __ldcg(cand + x);
            const int kx = __ldcg(pos + x), ex = __ldg(ptr + x + 1);
            if (x == m || mx != -1 || cx != m) continue;
            const int b = best_free_sorted(x, kx, ex, nbr, pos, mate);
            cand[x] = b;
            if (b < 0) {
                mate[x] = -2;
                continue;
            }
            fence_sc_gpu();
            if (__ldcg(cand + b) != x) continue;
            const int lo = min(x, b), hi = max(x, b);
            if (atomicCAS(&mate[lo], -1, hi) != -1) continue;
            mate[hi] = lo;
            if (k + 2 <= BA_MAX) {
                items[k++] = lo;
                items[k++] = hi;
            } else {
                const int at = atomicAdd(nc, 2);
                if (at < n) nl[at] = lo;
                if (at + 1 < n) nl[at + 1] = hi;
            }
        }
    }
    block_append(k, items, nl, nc, n);
}

// One round per grid barrier. Round 0 matches the mutual pairs of the initial
// candidates. Round r >= 1 takes the vertices matched in round r-1; each of
// their free neighbours whose candidate was one of them picks its next best
// free neighbour b, publishes cand[x] = b, and (after a sequentially
// consistent fence) checks cand[b] == x. When x and b recompute in the same
// round, the store-fence-load on both sides guarantees that at least one of
// them sees the pair; the CAS on mate[min] matches it once. A vertex
// recomputes only because its old candidate was matched, so a stale read of
// cand never names a free vertex; a pick that is matched concurrently is
// redone in the next round, when that vertex's neighbours are revisited.
// The set of pairs matched in each round equals one round of the
// locally-dominant algorithm.
//
// cnt: [0..2] match-list counters (ring of three rounds), [7] error, [8]
// rounds that matched at least one pair, [15] round number handed over after
// a one-block phase, [32] barrier arrivals (a cache line of its own, away
// from the counters the rounds update).
__global__ void __launch_bounds__(1024) k_ld_persistent(int n, const int* __restrict__ ptr,
                                                        const int* __restrict__ col, const int* __restrict__ nbr,
                                                        int* pos, int* cand, int* mate, int* list0, int* list1,
                                                        int ngl, int* cnt, long long max_rounds) {
    int* lists[2] = {list0, list1};
    unsigned* bar = reinterpret_cast<unsigned*>(cnt + 32);
    int* err = cnt + 7;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned epoch = 0;
    int items[BA_MAX];
    // round 0: mutual initial candidates
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int v = base + threadIdx.x;
        int k = 0;
        if (v < n && __ldcg(mate + v) == -1) {
            const int u = __ldcg(cand + v);
            if (u > v && __ldcg(cand + u) == v && atomicCAS(&mate[v], -1, u) == -1) {
                mate[u] = v;
                items[0] = v;
                items[1] = u;
                k = 2;
            }
        }
        block_append(k, items, lists[0], cnt + 0, n);
    }
    grid_sync(bar, ++epoch, err);
    if (__ldcg(err)) return;
    if (leader && __ldcg(cnt + 0) > 0) cnt[8] += 1;
    long long r = 1;
    for (;;) {
        const int m_cnt = min(__ldcg(cnt + (int)((r - 1) % 3)), n);
        if (m_cnt == 0) return;
        if (r > max_rounds) {
            if (leader) atomicExch(err, 2);
            return;
        }
        if (((long long)m_cnt << ngl) <= LD_SOLO_ITEMS) {
            // a small frontier: block 0 runs the rounds alone, separated by
            // block barriers, until the frontier grows or ends; the other
            // blocks wait at the grid barrier and then take up its round number
            if (blockIdx.x == 0) {
                for (;;) {
                    ld_round(r, threadIdx.x, blockDim.x, ngl, ptr, col, nbr, pos, cand, mate, lists, cnt, n, leader);
                    __syncthreads();
                    const int mc = min(__ldcg(cnt + (int)(r % 3)), n);
                    if (leader && mc > 0) cnt[8] += 1;
                    ++r;
                    if (mc == 0 || ((long long)mc << ngl) > LD_SOLO_ITEMS || r > max_rounds) break;
                }
                if (threadIdx.x == 0) cnt[15] = (int)r;
            }
            grid_sync(bar, ++epoch, err);
            if (__ldcg(err)) return;
            r = __ldcg(cnt + 15);
            continue;
        }
        ld_round(r, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, ngl, ptr, col, nbr, pos, cand,
                 mate, lists, cnt, n, leader);
        grid_sync(bar, ++epoch, err);
        if (__ldcg(err)) return;
        if (leader && __ldcg(cnt + (int)(r % 3)) > 0) cnt[8] += 1;
        ++r;
    }
}

// ------------------------------------------------ matching by proposals ---
// The same matching without rounds: every vertex proposes to its best
// neighbour (first in its sorted list) that would take it, displacing that
// neighbour's current suitor if the new proposal ranks higher; a displaced
// vertex proposes again further down its own list. With a strict order on
// the edges this ends in the greedy matching on that order, which is the
// locally-dominant matching the rounds compute (each vertex is matched to
// its suitor exactly when they are each other's suitor). The algorithm is
// the Suitor method of Manne and Halappanavar (IPDPS 2014).
//
// A proposal of cur, from sorted position k of its own row, to v is the
// position q of cur in v's sorted row: for a fixed v, positions order v's
// edges exactly as the strict order does. suitor[v] holds q << 32 | k of the
// best proposal not yet displaced (all ones for none), so one 64-bit
// atomicMin decides a proposal and returns, on a displacement, where the
// displaced vertex resumes: right after v in its own row (suitor values only
// decrease, so a vertex never has to look back up its list). No thread waits
// on another, and each vertex's list position only moves forward, so the
// work is bounded by the entry count.
//
// nq[s] for every sorted position s of row v: (u, position of v in u's
// sorted row) for an edge to u, (-1, -1) for the non-edges after the edges.
// Every row holds its diagonal, a non-edge, so every row ends in (-1, -1)
// and a scan never leaves its row (checked here: err |= 8 otherwise).
// spos[k] maps an original CSR position to its sorted position (written by
// the edge sorts for every edge). Also resets suitor[].
constexpr unsigned long long NO_SUITOR = ~0ull;

template <int G>
__global__ void __launch_bounds__(TPB) k_mirror_pos(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                                                    const double* __restrict__ c, const int* __restrict__ spos,
                                                    int2* __restrict__ nq, unsigned long long* __restrict__ suitor,
                                                    int* err) {
    const double NEG_INF = -__longlong_as_double(0x7ff0000000000000LL);
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int ng = (gridDim.x * blockDim.x) / G;
    const int v0 = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int warp_first = v0 - (lane - gl) / G;     // every lane of a warp runs the same iterations
    for (int it = 0; warp_first + it * ng < n; ++it) {
        const int v = v0 + it * ng;
        int b = 0, e = 0;
        if (v < n) {
            b = ptr[v];
            e = ptr[v + 1];
            if (gl == 0) suitor[v] = NO_SUITOR;
        }
        int edges = 0;
        for (int k = b + gl; k < e; k += G) {
            if (!is_edge(c[k])) continue;           // not an edge (diagonal, zero pair)
            ++edges;
            const int u = col[k];
            const int km = find_in_row(ptr, col, u, v);
            if (km < 0) {                            // no mirror entry: pattern not symmetric
                nq[spos[k]] = make_int2(-1, -1);
                atomicOr(err, 1);
                continue;
            }
            nq[spos[k]] = make_int2(u, spos[km]);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) edges += __shfl_xor_sync(FULL_MASK, edges, o, G);
        if (v < n) {
            if (gl == 0 && edges == e - b) atomicOr(err, 8);   // no non-edge ends the row
            for (int k = b + edges + gl; k < e; k += G) nq[k] = make_int2(-1, -1);
        }
    }
}

// One thread per vertex: its chain of proposals, and those of the vertices
// it displaces. err |= 2 if a thread takes more steps than there are
// entries (impossible for a valid mirror map; a guard, not a wait).
__global__ void __launch_bounds__(256) k_suitor(int n, long long nnz, const int* __restrict__ ptr,
                                                const int2* __restrict__ nq, unsigned long long* suitor, int* err) {
    const int u0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (u0 >= n || *err) return;
    int k = __ldg(ptr + u0);
    int2 cur = __ldg(nq + k);
    long long steps = 0;
    for (;;) {
        if (cur.x < 0) return;                       // the row's edges are exhausted: no partner so far
        const int2 nxt = __ldg(nq + k + 1);          // in the row: its (-1, -1) end follows every edge
        if (++steps > nnz) {
            atomicOr(err, 2);
            return;
        }
        const unsigned long long mine = ((unsigned long long)(unsigned)cur.y << 32) | (unsigned)k;
        const unsigned long long old = atomicMin(suitor + cur.x, mine);
        if (old > mine) {
            if (old == NO_SUITOR) return;            // first suitor of v: this chain ends
            k = (int)(unsigned)(old & 0xffffffffu) + 1;   // the displaced vertex, after v in its own row
            cur = __ldg(nq + k);
        } else {                                     // v holds a better proposal: next candidate
            ++k;
            cur = nxt;
        }
    }
}

// mate[v] = the vertex at v's suitor position, -1 without a suitor; the
// relation must be mutual (err |= 4 otherwise).
__global__ void k_suitor_mate(int n, const int2* __restrict__ nq, const unsigned long long* __restrict__ suitor,
                              int* __restrict__ mate, int* err) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const unsigned long long s = suitor[v];
        if (s == NO_SUITOR) {
            mate[v] = -1;
            continue;
        }
        const int2 e = nq[(int)(s >> 32)];           // v's edge to its suitor u: (u, position of v in u's row)
        mate[v] = e.x;
        if ((int)(suitor[e.x] >> 32) != e.y) atomicOr(err, 4);
    }
}

// ------------------------------------------ aggregates + Eq. 4 prolongator --
__global__ void k_head_flags(int n, const int* __restrict__ mate, int* __restrict__ flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int m = mate[i];
        flag[i] = (m < 0 || m > i) ? 1 : 0;
    }
}

// Aggregate q = number of heads (smallest members) before it. Pair columns
// are w restricted to the pair and normalised; singletons sign(w_s).
// Heads: the smallest member of each aggregate, heads[qid[i]] = i (and the
// kept copy of the matching with -1 for every unmatched vertex).
__global__ void k_heads(int n, const int* __restrict__ mate, const int* __restrict__ qid, int* __restrict__ heads,
                        int* __restrict__ mate_out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = mate[i];
        if (mate_out) mate_out[i] = j < 0 ? -1 : j;
        if (j < 0 || j > i) heads[qid[i]] = i;
    }
}

// One thread per aggregate q (all lanes busy on the FP64 square root and
// divisions, which bound this step): agg, the Eq. 4 column p and wc[q].
__global__ void k_aggregate(int nc, const int* __restrict__ heads, const int* __restrict__ mate,
                            const double* __restrict__ w, int* __restrict__ agg, double* __restrict__ p,
                            double* __restrict__ wc) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
        const int i = heads[q];
        const int j = mate[i];
        const double wi = w[i];
        agg[i] = q;
        if (j < 0) {
            p[i] = wi > 0.0 ? 1.0 : -1.0;
            wc[q] = fabs(wi);
        } else {
            const double wj = w[j];
            const double s = __dsqrt_rn(__dadd_rn(__dmul_rn(wi, wi), __dmul_rn(wj, wj)));
            agg[j] = q;
            p[i] = __ddiv_rn(wi, s);
            p[j] = __ddiv_rn(wj, s);
            wc[q] = s;
        }
    }
}

// --------------------------------------- pairwise Galerkin product ---------
// Coarse row q has members h = heads[q] and, for a pair, mate[h] > h.
__global__ void k_rap_bound(int nc, const int* __restrict__ heads, const int* __restrict__ mate,
                            const int* __restrict__ ptr, int* __restrict__ ub) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
        const int h = heads[q];
        const int m = mate[h];
        int u = ptr[h + 1] - ptr[h];
        if (m > h) u += ptr[m + 1] - ptr[m];
        ub[q] = u;
    }
}

// Expands coarse row q into scratch (coarse column, term) in member order
// then column order, sorts the segment stably by coarse column and sums each
// run left to right starting from its first term. cnt[q] = distinct columns.
// With `list` set, only the rows list[0 .. *nlist) are done (the rows the
// warp-cooperative kernel below leaves out).
__global__ void k_rap_rows(int nc, const int* __restrict__ heads, const int* __restrict__ mate,
                           const int* __restrict__ ptr, const int* __restrict__ col, const double* __restrict__ val,
                           const int* __restrict__ agg, const double* __restrict__ p, const int* __restrict__ off,
                           int* __restrict__ skey, double* __restrict__ sval, int* __restrict__ cnt,
                           const int* __restrict__ list, const int* __restrict__ nlist) {
    const int nr = list ? *nlist : nc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nr; t += gridDim.x * blockDim.x) {
        const int q = list ? list[t] : t;
        const int h = heads[q];
        const int m = mate[h];
        int* K = skey + off[q];
        double* V = sval + off[q];
        int len = 0;
        for (int s = 0; s < 2; ++s) {
            const int i = s == 0 ? h : m;
            if (s == 1 && m <= h) break;
            const double pi = p[i];
            for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
                const int j = col[k];
                K[len] = agg[j];
                V[len] = __dmul_rn(__dmul_rn(pi, val[k]), p[j]);
                ++len;
            }
        }
        for (int a = 1; a < len; ++a) {              // stable insertion sort by key
            const int key = K[a];
            const double v = V[a];
            int b = a - 1;
            while (b >= 0 && K[b] > key) {
                K[b + 1] = K[b];
                V[b + 1] = V[b];
                --b;
            }
            K[b + 1] = key;
            V[b + 1] = v;
        }
        int u = 0;
        for (int a = 0; a < len;) {
            const int key = K[a];
            double s = V[a];
            int e = a + 1;
            while (e < len && K[e] == key) { s = __dadd_rn(s, V[e]); ++e; }
            K[u] = key;
            V[u] = s;
            ++u;
            a = e;
        }
        cnt[q] = u;
    }
}

// The rows the group kernel below leaves out, up to CAP terms, one block per
// listed row: the terms (member order, then column order) are keyed by
// (coarse column, position), bitonic-sorted in shared memory (a stable sort
// by column), and the first thread of every run of equal columns sums the run
// left to right from its first term: the canonical order of k_rap_rows and
// k_ap_rows, bit for bit. Longer rows are appended to `longer` for a launch
// of larger CAP or for those kernels.
constexpr int ROW_CAPS[2] = {4096, 8192};
template <bool RAP>
__global__ void __launch_bounds__(LONG_TPB) k_rows_long(const int* __restrict__ list, const int* __restrict__ nlist,
                                                        int CAP,
                                                        const int* __restrict__ heads, const int* __restrict__ mate,
                                                        const int* __restrict__ ptr, const int* __restrict__ col,
                                                        const double* __restrict__ val, const int* __restrict__ agg,
                                                        const double* __restrict__ p, const int* __restrict__ off,
                                                        int* __restrict__ skey, double* __restrict__ sval,
                                                        int* __restrict__ cnt, int* __restrict__ longer,
                                                        int* __restrict__ nlonger, const double* __restrict__ rowscale) {
    extern __shared__ unsigned long long rsm[];
    unsigned long long* KS = rsm;
    double* VS = reinterpret_cast<double*>(rsm + CAP);
    __shared__ int wsum[LONG_TPB / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nr = *nlist;
    for (int t = blockIdx.x; t < nr; t += gridDim.x) {
        const int q = list[t];
        int h = q, m = -1;
        if (RAP) {
            h = heads[q];
            m = mate[h];
        }
        const int b0 = ptr[h], l0 = ptr[h + 1] - b0;
        int b1 = 0, l1 = 0;
        if (RAP && m > h) {
            b1 = ptr[m];
            l1 = ptr[m + 1] - b1;
        }
        const int len = l0 + l1;
        if (len > CAP) {
            if (tid == 0) longer[atomicAdd(nlonger, 1)] = q;
            continue;
        }
        int m2 = 1;
        while (m2 < len) m2 <<= 1;
        for (int s = tid; s < m2; s += LONG_TPB) {
            if (s < len) {
                const bool first = s < l0;
                const int k = first ? b0 + s : b1 + s - l0;
                const int j = col[k];
                KS[s] = ((unsigned long long)(unsigned)agg[j] << 32) | (unsigned)s;
                VS[s] = RAP ? __dmul_rn(__dmul_rn(p[first ? h : m], val[k]), p[j]) : __dmul_rn(val[k], p[j]);
            } else {
                KS[s] = ~0ull;
            }
        }
        __syncthreads();
        for (int size = 2; size <= m2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int u = tid; u < m2 / 2; u += LONG_TPB) {
                    const int lo = 2 * u - (u & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const unsigned long long a = KS[lo], bb = KS[hi];
                    if ((a > bb) == up) {
                        KS[lo] = bb;
                        KS[hi] = a;
                    }
                }
                __syncthreads();
            }
        int base = 0;
        for (int c0 = 0; c0 < len; c0 += LONG_TPB) {
            const int r = c0 + tid;
            const bool head = r < len && (r == 0 || (KS[r] >> 32) != (KS[r - 1] >> 32));
            const unsigned bal = __ballot_sync(FULL_MASK, head);
            if (lane == 0) wsum[wid] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
#pragma unroll
            for (int w2 = 0; w2 < LONG_TPB / 32; ++w2) {
                const int cw = wsum[w2];
                before += w2 < wid ? cw : 0;
                total += cw;
            }
            if (head) {
                const unsigned key = (unsigned)(KS[r] >> 32);
                double sum = VS[(unsigned)KS[r]];
                for (int e = r + 1; e < len && (unsigned)(KS[e] >> 32) == key; ++e)
                    sum = __dadd_rn(sum, VS[(unsigned)KS[e]]);
                if (rowscale) sum = __dmul_rn(rowscale[q], sum);
                const int u = base + before + __popc(bal & ((1u << lane) - 1u));
                skey[off[q] + u] = (int)key;
                sval[off[q] + u] = sum;
            }
            base += total;
            __syncthreads();
        }
        if (tid == 0) cnt[q] = base;
        __syncthreads();
    }
}

// The same as k_rows_long for rows of up to WROW terms, one warp per listed
// row in its own slice of shared memory (warp barriers between the bitonic
// stages); the same keys (coarse column, term position) and run sums, so the
// results are the same bits. Longer rows go to `longer`.
template <bool RAP>
__global__ void __launch_bounds__(TPB) k_rows_warp_sm(const int* __restrict__ list, const int* __restrict__ nlist,
                                                      const int* __restrict__ heads, const int* __restrict__ mate,
                                                      const int* __restrict__ ptr, const int* __restrict__ col,
                                                      const double* __restrict__ val, const int* __restrict__ agg,
                                                      const double* __restrict__ p, const int* __restrict__ off,
                                                      int* __restrict__ skey, double* __restrict__ sval,
                                                      int* __restrict__ cnt, int* __restrict__ longer,
                                                      int* __restrict__ nlonger, const double* __restrict__ rowscale) {
    __shared__ unsigned long long KSs[WPB][WROW];
    __shared__ double VSs[WPB][WROW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long* KS = KSs[w];
    double* VS = VSs[w];
    const int nr = *nlist;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nr; t += nwarps) {
        const int q = list[t];
        int h = q, m = -1;
        if (RAP) {
            h = heads[q];
            m = mate[h];
        }
        const int b0 = ptr[h], l0 = ptr[h + 1] - b0;
        int b1 = 0, l1 = 0;
        if (RAP && m > h) {
            b1 = ptr[m];
            l1 = ptr[m + 1] - b1;
        }
        const int len = l0 + l1;
        if (len > WROW) {
            if (lane == 0) longer[atomicAdd(nlonger, 1)] = q;
            continue;
        }
        int m2 = 1;
        while (m2 < len) m2 <<= 1;
        for (int s = lane; s < m2; s += 32) {
            if (s < len) {
                const bool first = s < l0;
                const int k = first ? b0 + s : b1 + s - l0;
                const int j = col[k];
                KS[s] = ((unsigned long long)(unsigned)agg[j] << 32) | (unsigned)s;
                VS[s] = RAP ? __dmul_rn(__dmul_rn(p[first ? h : m], val[k]), p[j]) : __dmul_rn(val[k], p[j]);
            } else {
                KS[s] = ~0ull;
            }
        }
        __syncwarp();
        for (int size = 2; size <= m2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int u = lane; u < m2 / 2; u += 32) {
                    const int lo = 2 * u - (u & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const unsigned long long a = KS[lo], bb = KS[hi];
                    if ((a > bb) == up) {
                        KS[lo] = bb;
                        KS[hi] = a;
                    }
                }
                __syncwarp();
            }
        int base = 0;
        for (int c0 = 0; c0 < len; c0 += 32) {
            const int r = c0 + lane;
            const bool head = r < len && (r == 0 || (KS[r] >> 32) != (KS[r - 1] >> 32));
            const unsigned bal = __ballot_sync(FULL_MASK, head);
            if (head) {
                const unsigned key = (unsigned)(KS[r] >> 32);
                double sum = VS[(unsigned)KS[r]];
                for (int e = r + 1; e < len && (unsigned)(KS[e] >> 32) == key; ++e)
                    sum = __dadd_rn(sum, VS[(unsigned)KS[e]]);
                if (rowscale) sum = __dmul_rn(rowscale[q], sum);
                const int u = base + __popc(bal & ((1u << lane) - 1u));
                skey[off[q] + u] = (int)key;
                sval[off[q] + u] = sum;
            }
            base += __popc(bal);
        }
        if (lane == 0) cnt[q] = base;
        __syncwarp();
    }
}

// Compacts the per-row results from scratch (row q at off[q]) into the CSR
// arrays; a group of G lanes per row, lanes over the row's entries. With dww
// set (zeroed by the caller), also dww[q] = (c_qq w_q) w_q, the value k_diag
// would compute for the new matrix and smooth vector w.
template <int G>
__global__ void __launch_bounds__(TPB) k_rap_copy(int nc, const int* __restrict__ off, const int* __restrict__ cptr,
                                                 const int* __restrict__ skey, const double* __restrict__ sval,
                                                 int* __restrict__ ccol, double* __restrict__ cval,
                                                 const double* __restrict__ w, double* __restrict__ dww) {
    const int gl = threadIdx.x & (G - 1);
    const int ng = (gridDim.x * blockDim.x) / G;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) / G; q < nc; q += ng) {
        const int s = off[q], d = cptr[q], e = cptr[q + 1];
        for (int k = gl; k < e - d; k += G) {
            const int c = skey[s + k];
            const double v = sval[s + k];
            ccol[d + k] = c;
            cval[d + k] = v;
            if (dww && c == q) dww[q] = __dmul_rn(__dmul_rn(v, w[q]), w[q]);
        }
    }
}

// Pairwise Galerkin rows (RAP = true: row q of P^T A P from the members h, m
// of aggregate q, term (p_i a_ij) p_j) or rows of A P (RAP = false: row i,
// term a_ij p_j), one group of G lanes per row (32 / G rows per warp at a
// time): lane t of the group holds term t in member order then column order,
// its stable rank by coarse column comes from a shuffle sweep, the terms are
// placed in rank order in shared memory, and the first lane of every run of
// equal columns sums the run left to right from its first term. This is the
// canonical order of the thread-per-row kernels, bit for bit. Rows with more
// than G terms are listed in long_list for those kernels.
template <bool RAP, int G>
__global__ void __launch_bounds__(TPB) k_rows_warp(int nrows, const int* __restrict__ list,
                                                  const int* __restrict__ nlist, const int* __restrict__ heads,
                                                  const int* __restrict__ mate, const int* __restrict__ ptr,
                                                  const int* __restrict__ col, const double* __restrict__ val,
                                                  const int* __restrict__ agg, const double* __restrict__ p,
                                                  const int* __restrict__ off, int* __restrict__ skey,
                                                  double* __restrict__ sval, int* __restrict__ cnt,
                                                  int* __restrict__ long_list, int* __restrict__ nlong,
                                                  const double* __restrict__ rowscale) {
    __shared__ int sk[TPB];
    __shared__ double sv[TPB];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);                 // lane in the group
    const int gbase = threadIdx.x - gl;            // group's first slot in shared memory
    const int gshift = lane - gl;                  // group's first lane in the warp
    const unsigned gmask = G == 32 ? FULL_MASK : (((1u << G) - 1u) << gshift);
    const int ng = (gridDim.x * blockDim.x) / G;
    const int q0 = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    // every lane of a warp runs the same number of iterations (shuffles)
    const int warp_first = q0 - (gshift / G);
    const int nr = list ? min(*nlist, nrows) : nrows;   // with a list, only the rows list[0 .. *nlist)
    for (int it = 0; warp_first + it * ng < nr; ++it) {
        const int t = q0 + it * ng;
        const int q = t < nr ? (list ? list[t] : t) : nrows;
        int len = 0, l0 = 0, b0 = 0, b1 = 0, h = q, m = -1;
        if (q < nrows) {
            if (RAP) {
                h = heads[q];
                m = mate[h];
            }
            b0 = ptr[h];
            l0 = ptr[h + 1] - b0;
            int l1 = 0;
            if (RAP && m > h) {
                b1 = ptr[m];
                l1 = ptr[m + 1] - b1;
            }
            len = l0 + l1;
            if (len > G) {
                if (gl == 0) long_list[atomicAdd(nlong, 1)] = q;
                len = -1;                           // left to the thread-per-row kernel
            }
        }
        int key = 0x7fffffff;
        double v = 0.0;
        if (gl < len) {
            const bool first = gl < l0;
            const int k = first ? b0 + gl : b1 + gl - l0;
            const int j = col[k];
            key = agg[j];
            if (RAP) v = __dmul_rn(__dmul_rn(p[first ? h : m], val[k]), p[j]);
            else v = __dmul_rn(val[k], p[j]);
        }
        int rank = 0;
#pragma unroll 8
        for (int t = 0; t < G; ++t) {
            const int kt = __shfl_sync(FULL_MASK, key, t, G);
            rank += (kt < key) || (kt == key && t < gl);
        }
        if (gl < len) {
            sk[gbase + rank] = key;
            sv[gbase + rank] = v;
        }
        __syncwarp();
        const bool head = gl < len && (gl == 0 || sk[threadIdx.x - 1] != sk[threadIdx.x]);
        const unsigned hm = __ballot_sync(FULL_MASK, head) & gmask;
        if (head) {
            const int kk = sk[threadIdx.x];
            double sum = sv[threadIdx.x];
            for (int e = gl + 1; e < len && sk[gbase + e] == kk; ++e) sum = __dadd_rn(sum, sv[gbase + e]);
            if (rowscale) sum = __dmul_rn(rowscale[q], sum);
            const int u = __popc(hm & ((1u << lane) - 1u));
            skey[off[q] + u] = kk;
            sval[off[q] + u] = sum;
        }
        if (gl == 0 && len >= 0 && q < nrows) cnt[q] = __popc(hm);
        __syncwarp();
    }
}

// Lanes per row for the warp-cooperative row products: the power of two that
// covers the typical row (longer rows go to the thread-per-row kernels).
int rows_group(long long terms, long long rows) {
    const double avg = rows > 0 ? (double)terms / (double)rows : 0.0;
    return avg <= 7.0 ? 8 : (avg <= 14.0 ? 16 : 32);
}

// Eq. 3 weights of every stored pair. The kernel is bound by the FP64
// division of each upper entry: with short rows one thread per row keeps
// every lane dividing (rows of a stencil have their upper entries at the
// same positions); long rows take a group of lanes each.
int weights_group(long long nnz, long long n) {
    const double mean = n > 0 ? (double)nnz / (double)n : 0.0;
    return mean < 24.0 ? 1 : (mean < 48.0 ? 8 : (mean < 96.0 ? 16 : 32));
}

void launch_weights(int G, int grid_cap, cudaStream_t st, int n, const int* ptr, const int* col, const double* val,
                    const double* dww, const double* w, double* c) {
    const int blocks = blocks_for((long long)n * G, TPB, grid_cap);
    if (G == 1) k_weights<1><<<blocks, TPB, 0, st>>>(n, ptr, col, val, dww, w, c);
    else if (G == 8) k_weights<8><<<blocks, TPB, 0, st>>>(n, ptr, col, val, dww, w, c);
    else if (G == 16) k_weights<16><<<blocks, TPB, 0, st>>>(n, ptr, col, val, dww, w, c);
    else k_weights<32><<<blocks, TPB, 0, st>>>(n, ptr, col, val, dww, w, c);
    KERNEL_CHECK();
}

// Row products with G lanes per row (rows of more than G terms are listed in
// long_list); with `list` set, only the rows list[0 .. *nlist).
template <bool RAP>
void launch_rows(amg_hierarchy* h, int G, int nrows, const int* heads, const int* mate, const int* ptr,
                 const int* col, const double* val, const int* agg, const double* p, const int* off, int* skey,
                 double* sval, int* cnt, int* long_list, int* nlong, const double* rowscale, cudaStream_t st,
                 const int* list = nullptr, const int* nlist = nullptr) {
    const int blocks = list ? h->num_sms * 16 : blocks_for((long long)nrows * G, TPB, h->num_sms * 16);
    if (G == 8)
        k_rows_warp<RAP, 8><<<blocks, TPB, 0, st>>>(nrows, list, nlist, heads, mate, ptr, col, val, agg, p, off, skey,
                                                    sval, cnt, long_list, nlong, rowscale);
    else if (G == 16)
        k_rows_warp<RAP, 16><<<blocks, TPB, 0, st>>>(nrows, list, nlist, heads, mate, ptr, col, val, agg, p, off,
                                                     skey, sval, cnt, long_list, nlong, rowscale);
    else
        k_rows_warp<RAP, 32><<<blocks, TPB, 0, st>>>(nrows, list, nlist, heads, mate, ptr, col, val, agg, p, off,
                                                     skey, sval, cnt, long_list, nlong, rowscale);
    KERNEL_CHECK();
}

void launch_copy(amg_hierarchy* h, long long nnz, int nrows, const int* off, const int* cptr, const int* skey,
                 const double* sval, int* ccol, double* cval, cudaStream_t st, const double* w = nullptr,
                 double* dww = nullptr) {
    const int G = rows_group(nnz, nrows);
    const int blocks = blocks_for((long long)nrows * G, TPB, h->num_sms * 16);
    if (dww) CUDA_CHECK(cudaMemsetAsync(dww, 0, sizeof(double) * nrows, st));
    if (G == 8) k_rap_copy<8><<<blocks, TPB, 0, st>>>(nrows, off, cptr, skey, sval, ccol, cval, w, dww);
    else if (G == 16) k_rap_copy<16><<<blocks, TPB, 0, st>>>(nrows, off, cptr, skey, sval, ccol, cval, w, dww);
    else k_rap_copy<32><<<blocks, TPB, 0, st>>>(nrows, off, cptr, skey, sval, ccol, cval, w, dww);
    KERNEL_CHECK();
}

// P_l <- P_l P_s: agg_l = agg_s o agg_l, p_l = p_l * p_s(agg_l).
__global__ void k_compose(int n, int* __restrict__ agg_l, double* __restrict__ p_l, const int* __restrict__ agg_s,
                          const double* __restrict__ p_s) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int a = agg_l[i];
        p_l[i] = __dmul_rn(p_l[i], p_s[a]);
        agg_l[i] = agg_s[a];
    }
}

// ------------------------------------------------------- P^T member lists --
__global__ void k_member_count(int n, const int* __restrict__ agg, int* __restrict__ cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) atomicAdd(&cnt[agg[i]], 1);
}

__global__ void k_member_fill(int n, const int* __restrict__ agg, const int* __restrict__ pt_ptr, int* cursor,
                              int* __restrict__ idx) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int q = agg[i];
        idx[pt_ptr[q] + atomicAdd(&cursor[q], 1)] = i;
    }
}

__global__ void k_member_sort(int nc, const int* __restrict__ pt_ptr, int* __restrict__ idx) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
        const int b = pt_ptr[q], e = pt_ptr[q + 1];
        for (int a = b + 1; a < e; ++a) {
            const int v = idx[a];
            int c = a - 1;
            while (c >= b && idx[c] > v) { idx[c + 1] = idx[c]; --c; }
            idx[c + 1] = v;
        }
    }
}

// ----------------------------------------------- l1-Jacobi (Eq. 5-6) -------
// M_ii = a_ii + sum_{j != i} |a_ij| (row order), stored as its inverse.
__global__ void k_l1_jacobi(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                            const double* __restrict__ val, double* __restrict__ minv, float* __restrict__ minv32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0, d = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
            if (col[k] == i) d = val[k];
            else s = __dadd_rn(s, fabs(val[k]));
        }
        const double m = __ddiv_rn(1.0, __dadd_rn(d, s));
        minv[i] = m;
        if (minv32) minv32[i] = (float)m;
    }
}

__global__ void k_to_float(long long n, const double* __restrict__ a, float* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// ------------------------------------------------------------ SELL-32 ------
// width[s] = longest row of slice s.
// Row i of the source starts at ptr[i]; it has len[i] entries when len is
// set (rows written in place by a row product), else ptr[i + 1] - ptr[i].
__device__ __forceinline__ int src_len(const int* __restrict__ ptr, const int* __restrict__ len, int i) {
    return len ? len[i] : ptr[i + 1] - ptr[i];
}

// Slice widths; with nnz_out set, also the entry count (one atomic per block).
__global__ void k_sell_width(int n, int nslices, const int* __restrict__ ptr, const int* __restrict__ len,
                             const int* __restrict__ perm, int* __restrict__ width, int* __restrict__ nnz_out) {
    const int lane = threadIdx.x & 31;
    int sum = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nslices * 32;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t >> 5);
        const int ip = (int)t;
        const int i = ip < n ? (perm ? perm[ip] : ip) : 0;
        const int l = ip < n ? src_len(ptr, len, i) : 0;
        sum += l;
        const int m = warp_max_int(l);
        if (lane == 0) width[s] = m;
    }
    if (nnz_out) {
        sum = block_sum_int(sum);
        if (threadIdx.x == 0 && sum) atomicAdd(nnz_out, sum);
    }
}

__global__ void k_sell_fill(int n, int nslices, const int* __restrict__ ptr, const int* __restrict__ rlen,
                            const int* __restrict__ col, const double* __restrict__ val,
                            const int* __restrict__ sptr, const int* __restrict__ perm, int* __restrict__ scol,
                            double* __restrict__ sval) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nslices * 32;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t >> 5), lane = (int)(t & 31);
        const int ip = (int)t;
        const int width = sptr[s + 1] - sptr[s];
        long long pos = (long long)sptr[s] * 32 + lane;
        int len = 0, b = 0;
        if (ip < n) {
            const int i = perm ? perm[ip] : ip;
            b = ptr[i];
            len = src_len(ptr, rlen, i);
        }
        // padding repeats the row's last column (a valid index of this
        // matrix's column space, also for rectangular A P) with value 0
        const int pad = len > 0 ? col[b + len - 1] : 0;
        for (int k = 0; k < width; ++k, pos += 32) {
            if (k < len) { scol[pos] = col[b + k]; sval[pos] = val[b + k]; }
            else { scol[pos] = pad; sval[pos] = 0.0; }
        }
    }
}

// SELL-C-sigma row order: inside each window of SIGMA consecutive rows, rows
// by decreasing length (ties by index), so a slice holds rows of similar
// length. One block of SIGMA threads per window, bitonic sort in shared memory.
constexpr int SIGMA = 256;
__global__ void __launch_bounds__(SIGMA) k_sort_window(int n, const int* __restrict__ rows, const int* __restrict__ ptr,
                                                      const int* __restrict__ len, int* __restrict__ perm) {
    __shared__ long long key[SIGMA];
    const int t = threadIdx.x;
    const int it = blockIdx.x * SIGMA + t;
    const int i = it < n ? (rows ? rows[it] : it) : 0;
    // key: larger length first, then smaller row index; items past n sort last
    key[t] = it < n ? ((long long)(0x7fffffff - src_len(ptr, len, i)) << 32) | (unsigned)i : 0x7fffffffffffffffLL;
    __syncthreads();
    for (int k = 2; k <= SIGMA; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int o = t ^ j;
            if (o > t) {
                const bool up = (t & k) == 0;
                const long long a = key[t], b = key[o];
                if ((a > b) == up) { key[t] = b; key[o] = a; }
            }
            __syncthreads();
        }
    }
    if (it < n) perm[it] = (int)(key[t] & 0xffffffffLL);
}

// Rows longer than lmax are listed in long_rows (kept rows in short_rows).
__global__ void k_long_flags(int n, const int* __restrict__ ptr, int lmax, int* __restrict__ flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = (ptr[i + 1] - ptr[i]) > lmax ? 1 : 0;
}
__global__ void k_split_rows(int n, const int* __restrict__ flag, const int* __restrict__ pos,
                             int* __restrict__ long_rows, int* __restrict__ short_rows) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (flag[i]) long_rows[pos[i]] = i;
        else short_rows[i - pos[i]] = i;
    }
}

// Segment boundaries of the next level: aggregates are numbered by their
// smallest member and never cross systems, so system s starts at the number
// of aggregates whose head precedes its first row.
__global__ void k_seg_map(int m, const int* __restrict__ seg, const int* __restrict__ qid, int n, int nc,
                          int* __restrict__ out) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= m; s += gridDim.x * blockDim.x)
        out[s] = seg[s] < n ? qid[seg[s]] : nc;
}

__global__ void k_seg_rows(int m, const int* __restrict__ seg, int* __restrict__ seg_row) {
    const int s = blockIdx.x;
    if (s >= m) return;
    for (int i = seg[s] + threadIdx.x; i < seg[s + 1]; i += blockDim.x) seg_row[i] = s;
}

// Dense lower triangle of the diagonal block [r0, r0 + n) (block-diagonal matrix).
__global__ void k_dense_lower_block(int n, int r0, const int* __restrict__ ptr, const int* __restrict__ col,
                                    const double* __restrict__ val, double* __restrict__ D) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int k = ptr[r0 + i]; k < ptr[r0 + i + 1]; ++k) {
            const int j = col[k] - r0;
            if (j >= 0 && j <= i) D[(size_t)j * n + i] = val[k];
        }
}

// ----------------------------------------------- coarsest: dense Cholesky --
__global__ void k_dense_lower(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                              const double* __restrict__ val, double* __restrict__ D) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int k = ptr[i]; k < ptr[i + 1]; ++k)
            if (col[k] <= i) D[(size_t)col[k] * n + i] = val[k];
}

// Left-looking column Cholesky A = L L^T in one block; column-major,
// sequential sums in k (the textbook order). flag = 1 on a non-positive pivot.
__global__ void k_cholesky(int n, const double* __restrict__ D, double* __restrict__ L, int* flag) {
    __shared__ double ljj_s;
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            double s = D[(size_t)j * n + j];
            for (int k = 0; k < j; ++k) {
                const double l = L[(size_t)k * n + j];
                s = __dsub_rn(s, __dmul_rn(l, l));
            }
            if (!(s > 0.0)) { *flag = 1; s = 1.0; }
            ljj_s = __dsqrt_rn(s);
            L[(size_t)j * n + j] = ljj_s;
        }
        __syncthreads();
        const double ljj = ljj_s;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double t = D[(size_t)j * n + i];
            for (int k = 0; k < j; ++k) t = __dsub_rn(t, __dmul_rn(L[(size_t)k * n + i], L[(size_t)k * n + j]));
            L[(size_t)j * n + i] = __ddiv_rn(t, ljj);
        }
        __syncthreads();
    }
}

// The whole coarsest-level inverse of one diagonal block per CTA: the dense
// lower triangle from the block's CSR rows, the factor L, Y = L^{-1} and
// A^{-1} = Y^T Y (row-major, at Ainv + blk[s]); L is also written when Lout
// is set. Factor and inverse are right-looking: as soon as column j of L (or
// row k of Y) is final, every entry it touches takes its update at once. Each
// entry still sees the same operations in the same order as in k_cholesky /
// k_lower_inverse / k_gram (updates in ascending k, the same roundings), so
// the bits are the same; the dependent chain is O(n) barrier steps instead of
// O(n^2) serial operations. A block of n <= SM_DENSE rows works in shared
// memory, a larger one in gwork + gofs[s] (2 n^2 doubles). segp == nullptr
// means a single block of rows [0, n0).
constexpr int SM_DENSE = 96;
constexpr int CTA_DENSE = 256;      // largest block one CTA factors (its n^3 FP64 work runs on one SM)
__global__ void k_coarse_inverse_blocks(int n0, const int* __restrict__ segp, const long long* __restrict__ blk,
                                        const long long* __restrict__ gofs, const int* __restrict__ ptr,
                                        const int* __restrict__ col, const double* __restrict__ val,
                                        double* __restrict__ gwork, double* __restrict__ Ainv,
                                        double* __restrict__ Lout, int* flag) {
    const int sg = blockIdx.x;
    const int r0 = segp ? segp[sg] : 0;
    const int n = segp ? segp[sg + 1] - r0 : n0;
    if (n <= 0) return;
    extern __shared__ double sm_dense[];
    __shared__ double dg[SM_DENSE];
    double* M;                            // n x n column-major: D, then L in place
    double* Ys;                           // n x n column-major: partial sums, then L^{-1}
    double* diag;                         // L_jj
    if (n <= SM_DENSE) { M = sm_dense; Ys = sm_dense + n * n; diag = dg; }
    else { M = gwork + gofs[sg]; Ys = M + (size_t)n * n; diag = Ys + (size_t)n * n; }
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) { M[t] = 0.0; Ys[t] = 0.0; }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int k = ptr[r0 + i]; k < ptr[r0 + i + 1]; ++k) {
            const int j = col[k] - r0;
            if (j >= 0 && j <= i) M[j * n + i] = val[k];
        }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        double s = M[j * n + j];          // D_jj less l_jk^2 for every k < j
        if (!(s > 0.0)) { if (threadIdx.x == 0) *flag = 1; s = 1.0; }
        const double ljj = __dsqrt_rn(s);
        if (threadIdx.x == 0) diag[j] = ljj;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) M[j * n + i] = __ddiv_rn(M[j * n + i], ljj);
        __syncthreads();
        const int m = n - j - 1;          // trailing lower triangle, columns j+1..n-1
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            const int c = j + 1 + t / m, i = j + 1 + t % m;
            if (i >= c) M[c * n + i] = __dsub_rn(M[c * n + i], __dmul_rn(M[j * n + i], M[j * n + c]));
        }
        __syncthreads();
    }
    for (int k = 0; k < n; ++k) {
        for (int c = threadIdx.x; c <= k; c += blockDim.x)   // row k of every column c <= k is final
            Ys[c * n + k] = c == k ? 1.0 / diag[k] : -Ys[c * n + k] / diag[k];
        __syncthreads();
        const int m = n - k - 1;
        for (int t = threadIdx.x; t < (k + 1) * m; t += blockDim.x) {
            const int c = t / m, i = k + 1 + t % m;
            Ys[c * n + i] = fma(M[k * n + i], Ys[c * n + k], Ys[c * n + i]);
        }
        __syncthreads();
    }
    double* Ai = Ainv + (segp ? blk[sg] : 0);
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        double s = 0.0;
        for (int k = max(i, j); k < n; ++k) s = fma(Ys[i * n + k], Ys[j * n + k], s);
        Ai[t] = s;
        if (Lout) Lout[t] = j > i ? M[t] : (j == i ? diag[i] : 0.0);   // t = column i, row j
    }
}

// Y = L^{-1} (column-major, lower), one column per thread.
__global__ void k_lower_inverse(int n, const double* __restrict__ L, double* __restrict__ Y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    for (int i = 0; i < c; ++i) Y[(size_t)c * n + i] = 0.0;
    Y[(size_t)c * n + c] = 1.0 / L[(size_t)c * n + c];
    for (int i = c + 1; i < n; ++i) {
        double t = 0.0;
        for (int k = c; k < i; ++k) t = fma(L[(size_t)k * n + i], Y[(size_t)c * n + k], t);
        Y[(size_t)c * n + i] = -t / L[(size_t)i * n + i];
    }
}

// Ainv = Y^T Y (row-major).
__global__ void k_gram(int n, const double* __restrict__ Y, double* __restrict__ Ainv) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    double s = 0.0;
    for (int k = max(i, j); k < n; ++k) s = fma(Y[(size_t)i * n + k], Y[(size_t)j * n + k], s);
    Ainv[(size_t)i * n + j] = s;
}

// Column scaling for the pre-smoother: valm_k = val_k * minv[col_k].
// omega M^{-1} when omega != 1.
__global__ void k_scale_vec(int n, double omega, const double* __restrict__ a, double* __restrict__ b,
                            float* __restrict__ b32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = omega * a[i];
        b[i] = v;
        if (b32) b32[i] = (float)v;
    }
}

__global__ void k_scale_cols(long long m, const int* __restrict__ col, const double* __restrict__ val,
                             const double* __restrict__ minv, double* __restrict__ valm, float* __restrict__ valm32) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += (long long)gridDim.x * blockDim.x) {
        const double v = val[k] * minv[col[k]];
        valm[k] = v;
        if (valm32) valm32[k] = (float)v;
    }
}

// Row i of A P: terms a_ij p_j keyed by agg(j), stably sorted by key and
// summed per key in column order, in scratch at row i's own CSR segment.
__global__ void k_ap_rows(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                          const double* __restrict__ val, const int* __restrict__ agg, const double* __restrict__ p,
                          int* __restrict__ skey, double* __restrict__ sval, int* __restrict__ cnt,
                          const int* __restrict__ list, const int* __restrict__ nlist,
                          const double* __restrict__ rowscale) {
    const int nr = list ? *nlist : n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nr; t += gridDim.x * blockDim.x) {
        const int i = list ? list[t] : t;
        const int b = ptr[i], len = ptr[i + 1] - b;
        int* K = skey + b;
        double* V = sval + b;
        for (int k = 0; k < len; ++k) {
            const int j = col[b + k];
            K[k] = agg[j];
            V[k] = __dmul_rn(val[b + k], p[j]);
        }
        for (int a = 1; a < len; ++a) {
            const int key = K[a];
            const double v = V[a];
            int c = a - 1;
            while (c >= 0 && K[c] > key) { K[c + 1] = K[c]; V[c + 1] = V[c]; --c; }
            K[c + 1] = key;
            V[c + 1] = v;
        }
        int u = 0;
        for (int a = 0; a < len;) {
            const int key = K[a];
            double sum = V[a];
            int e = a + 1;
            while (e < len && K[e] == key) { sum = __dadd_rn(sum, V[e]); ++e; }
            K[u] = key;
            V[u] = rowscale ? __dmul_rn(rowscale[i], sum) : sum;
            ++u;
            a = e;
        }
        cnt[i] = u;
    }
}

// ------------------------------- smoothed prolongator (Section 3.2) -------
// eta = max_i sum_j |a_ij| / a_ii (row sums in column order); positive, so the
// double's bit pattern orders like an unsigned integer and atomicMax is exact.
__global__ void k_eta_max(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                          const double* __restrict__ val, unsigned long long* __restrict__ maxbits) {
    unsigned long long best = 0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0, d = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
            s = __dadd_rn(s, fabs(val[k]));
            if (col[k] == i) d = val[k];
        }
        const unsigned long long b = (unsigned long long)__double_as_longlong(__ddiv_rn(s, d));
        best = b > best ? b : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(FULL_MASK, best, o);
        best = t > best ? t : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(maxbits, best);
}

// Rows of A P (in place) become rows of Pbar: with t_i = omega / a_ii, the
// entry in column agg_i is p_i - t_i (A P)_iq, every other one -(t_i (A P)_iq).
__global__ void k_pbar_from_ap(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                               double* __restrict__ val, const int* __restrict__ aptr, const int* __restrict__ acol,
                               const double* __restrict__ aval, const int* __restrict__ agg,
                               const double* __restrict__ p, double omega) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int kd = find_in_row(aptr, acol, i, i);
        const double t = __ddiv_rn(omega, aval[kd]);
        const int ai = agg[i];
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
            const double u = __dmul_rn(t, val[k]);
            val[k] = col[k] == ai ? __dsub_rn(p[i], u) : -u;
        }
    }
}

// Transpose of an n x nc CSR: counts per column, then entries placed with a
// per-column cursor (any order), then each column's entries sorted by row.
__global__ void k_col_count(int n, const int* __restrict__ ptr, const int* __restrict__ col, int* __restrict__ cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) atomicAdd(&cnt[col[k]], 1);
}

__global__ void k_col_fill(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                           const double* __restrict__ val, const int* __restrict__ tptr, int* cursor,
                           int* __restrict__ tcol, double* __restrict__ tval) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) {
            const int q = col[k];
            const int at = tptr[q] + atomicAdd(&cursor[q], 1);
            tcol[at] = i;
            tval[at] = val[k];
        }
}

// Sort the (key, value) pairs of every row by key (keys distinct within a
// row): one warp per row (BLOCK = false, rows of at most CAP pairs) or one
// block per listed row (BLOCK = true), bitonic sort in shared memory. A row
// longer than CAP is appended to `longs` for the block launch, or flags
// `overflow` when there is no such list.
// Rows of at most 32 (key, value) pairs sorted by key in registers, a warp
// each (a bitonic network over the lanes; the keys of a row are distinct row
// indices); longer rows are appended to longs for k_sort_pairs.
__global__ void __launch_bounds__(TPB) k_sort_pairs_warp(int nrows, const int* __restrict__ ptr,
                                                         int* __restrict__ key, double* __restrict__ val,
                                                         int* __restrict__ longs, int* __restrict__ nlongs) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nw) {   // uniform in the warp
        const int b = ptr[r], m = ptr[r + 1] - b;
        if (m <= 1) continue;
        if (m > 32) {
            if (lane == 0) longs[atomicAdd(nlongs, 1)] = r;
            continue;
        }
        int k = lane < m ? key[b + lane] : 0x7fffffff;
        double v = lane < m ? val[b + lane] : 0.0;
#pragma unroll
        for (int size = 2; size <= 32; size <<= 1)
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                const int pk = __shfl_xor_sync(FULL_MASK, k, stride);
                const double pv = __shfl_xor_sync(FULL_MASK, v, stride);
                const bool up = (lane & size) == 0;              // ascending run (size 32: the whole warp)
                const bool lower = (lane & stride) == 0;
                if ((pk < k) == (lower == up) && pk != k) {     // lower lane of an ascending pair keeps the min
                    k = pk;
                    v = pv;
                }
            }
        if (lane < m) {
            key[b + lane] = k;
            val[b + lane] = v;
        }
    }
}

template <bool BLOCK>
__global__ void k_sort_pairs(int nrows, const int* __restrict__ list, const int* __restrict__ nlist, int CAP,
                             const int* __restrict__ ptr, int* __restrict__ key, double* __restrict__ val,
                             int* __restrict__ longs, int* __restrict__ nlongs, int* __restrict__ overflow) {
    extern __shared__ double ssm[];
    const int U = BLOCK ? blockDim.x : 32;                 // threads per row
    const int lane = BLOCK ? threadIdx.x : (threadIdx.x & 31);
    const int w = BLOCK ? 0 : (threadIdx.x >> 5);
    const int units = BLOCK ? 1 : (blockDim.x >> 5);
    double* V = ssm + (size_t)w * CAP;
    int* K = reinterpret_cast<int*>(ssm + (size_t)units * CAP) + (size_t)w * CAP;
    const int nunits = BLOCK ? gridDim.x : (gridDim.x * blockDim.x) >> 5;
    const int nr = list ? *nlist : nrows;
    auto sync = [] {
        if (BLOCK) __syncthreads();
        else __syncwarp();
    };
    for (int t = BLOCK ? blockIdx.x : ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < nr; t += nunits) {
        const int r = list ? list[t] : t;
        const int b = ptr[r], m = ptr[r + 1] - b;
        if (m <= 1) continue;
        if (m > CAP) {
            if (lane == 0) {
                if (longs) longs[atomicAdd(nlongs, 1)] = r;
                else atomicExch(overflow, 1);
            }
            continue;
        }
        int m2 = 1;
        while (m2 < m) m2 <<= 1;
        for (int s = lane; s < m2; s += U) {
            K[s] = s < m ? key[b + s] : 0x7fffffff;
            V[s] = s < m ? val[b + s] : 0.0;
        }
        sync();
        for (int size = 2; size <= m2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int u = lane; u < m2 / 2; u += U) {
                    const int lo = 2 * u - (u & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const int a = K[lo], c = K[hi];
                    if ((a > c) == up) {
                        K[lo] = c;
                        K[hi] = a;
                        const double tv = V[lo];
                        V[lo] = V[hi];
                        V[hi] = tv;
                    }
                }
                sync();
            }
        for (int s = lane; s < m; s += U) {
            key[b + s] = K[s];
            val[b + s] = V[s];
        }
        sync();
    }
}

// Sparse product X = Y Z, one unit per row p of X (a warp, or with BLOCK the
// whole block): for every entry y of row p of Y (column order) and every
// entry z of row j of Z, the term y z is added to the running sum of column
// q. Within one (p, j) step the threads hold distinct columns q, so the sums
// of a hash table in shared memory are updated without races and in the step
// order (steps are separated by a warp or block barrier), the first term of a
// column starting its sum: the oracle's order. The table has CAP slots per
// unit in dynamic shared memory and takes at most CAP / 2 columns, which
// keeps linear probing short; with `list` only the rows list[0 .. *nlist)
// are done. Modes:
//   SPG_COUNT  count the distinct columns (cnt[p]);
//   SPG_FILL   write the row, columns ascending (bitonic sort in shared
//              memory), at xoff[p] of (xcol, xval); rows whose count is above
//              the capacity are left to a launch of larger capacity;
//   SPG_ONE    one pass: write the sorted row into a scratch slot (at
//              xoff[p] * stride, or without xoff t * stride for the t-th
//              listed row) and its count to cnt[p].
// In SPG_COUNT and SPG_ONE a row with more columns stops at once and is
// appended to `longs` for a launch of larger capacity (its count set to
// INT_MAX until then), or flags `overflow` when there is no such list.
enum SpgMode : int { SPG_COUNT = 0, SPG_FILL = 1, SPG_ONE = 2 };
constexpr int SPG_TIERS = 5;
constexpr int SPG_CAP[SPG_TIERS] = {128, 512, 2048, 8192, 16384};   // hash slots per row; at most half are used
constexpr int SPG_UNITS[SPG_TIERS] = {4, 4, 1, 1, 1};               // rows per block (warps, or one block)
constexpr int SPG_THREADS[SPG_TIERS] = {128, 128, 128, 256, 512};   // threads per block
constexpr int SPG_WARP_MIN_CAP = 64;   // a warp tier's capacity stays >= 64 slots when divided for tests
// a unit's threads per step (32, or the block) never exceed half the capacity,
// also with the capacities divided by 8 for tests
static_assert(32 <= SPG_WARP_MIN_CAP / 2 && SPG_UNITS[0] > 1 && SPG_UNITS[1] > 1 &&
                  SPG_THREADS[2] <= (SPG_CAP[2] >> 3) / 2 && SPG_THREADS[3] <= (SPG_CAP[3] >> 3) / 2 &&
                  SPG_THREADS[4] <= (SPG_CAP[4] >> 3) / 2,
              "probe loop needs a free slot");
template <int MODE, bool BLOCK>
__global__ void k_spgemm_hash(int nrows, const int* __restrict__ list, const int* __restrict__ nlist, int CAP,
                              const int* __restrict__ yptr, const int* __restrict__ ycol,
                              const double* __restrict__ yval, const int* __restrict__ zptr,
                              const int* __restrict__ zcol, const double* __restrict__ zval, int* __restrict__ cnt,
                              const int* __restrict__ xoff, long long stride, int* __restrict__ xcol,
                              double* __restrict__ xval, int* __restrict__ longs, int* __restrict__ nlongs,
                              int* __restrict__ overflow) {
    constexpr bool FILL = MODE != SPG_COUNT;               // the values are summed
    extern __shared__ double gsm[];
    __shared__ int wsum[32];
    const int U = BLOCK ? blockDim.x : 32;                  // threads per row
    const int tid = BLOCK ? threadIdx.x : (threadIdx.x & 31);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int unit = BLOCK ? 0 : wid;
    const int upb = BLOCK ? 1 : (blockDim.x >> 5);
    double* V = gsm + (size_t)unit * CAP;
    int* K = reinterpret_cast<int*>(gsm + (size_t)upb * CAP) + (size_t)unit * CAP;
    const int nunits = BLOCK ? gridDim.x : (gridDim.x * blockDim.x) >> 5;
    const int nr = list ? *nlist : nrows;
    const int hshift = 32 - (31 - __clz(CAP));             // Fibonacci hashing: the top log2(CAP) bits
    auto sync = [] {
        if (BLOCK) __syncthreads();
        else __syncwarp();
    };
    // number of threads of the unit with `pred` (also a barrier)
    auto count = [](bool pred) {
        if (BLOCK) return __syncthreads_count(pred);
        return __popc(__ballot_sync(FULL_MASK, pred));
    };
    // exclusive rank of `pred` among the unit's threads and their total
    auto rank = [&](bool pred, int& total) {
        const unsigned bal = __ballot_sync(FULL_MASK, pred);
        const int in_warp = __popc(bal & ((1u << lane) - 1u));
        if (!BLOCK) {
            total = __popc(bal);
            return in_warp;
        }
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int before = 0;
        total = 0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) {
            const int c = wsum[w2];
            before += w2 < wid ? c : 0;
            total += c;
        }
        __syncthreads();
        return before + in_warp;
    };
    for (int t = BLOCK ? blockIdx.x : ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < nr; t += nunits) {
        const int p = list ? list[t] : t;
        if (MODE == SPG_FILL && cnt[p] > (CAP >> 1)) continue;   // done by a launch of larger capacity
        for (int s = tid; s < CAP; s += U) K[s] = -1;
        sync();
        bool full = false;
        int used = 0;                                     // distinct columns so far (uniform in the unit)
        const int eb = yptr[p], ee = yptr[p + 1];
        int jn = eb < ee ? ycol[eb] : 0;
        double yn = eb < ee ? yval[eb] : 0.0;
        int fbn = eb < ee ? zptr[jn] : 0, fen = eb < ee ? zptr[jn + 1] : 0;
        // a block's steps wait on the Z rows (DRAM-resident on large levels):
        // the first chunk of the next step is loaded during the current one
        int qn = BLOCK && fbn + tid < fen ? zcol[fbn + tid] : 0;
        double zn = BLOCK && fbn + tid < fen ? zval[fbn + tid] : 0.0;
        for (int e = eb; e < ee && !full; ++e) {
            const double y = yn;
            const int fb = fbn, fe = fen;
            const int q0 = qn;
            const double z0 = zn;
            if (e + 1 < ee) {                              // the next step's row, loaded ahead
                jn = ycol[e + 1];
                yn = yval[e + 1];
                fbn = zptr[jn];
                fen = zptr[jn + 1];
                if (BLOCK) {
                    qn = fbn + tid < fen ? zcol[fbn + tid] : 0;
                    zn = fbn + tid < fen ? zval[fbn + tid] : 0.0;
                }
            }
            for (int f0 = fb; f0 < fe && !full; f0 += U) {
                const int f = f0 + tid;
                bool added = false;
                if (f < fe) {
                    const bool pre = BLOCK && f0 == fb;
                    const int q = pre ? q0 : zcol[f];
                    const double term = __dmul_rn(y, pre ? z0 : zval[f]);
                    unsigned hs = ((unsigned)q * 2654435769u) >> hshift;
                    // ends: a step starts with at most CAP / 2 columns and adds at
                    // most U <= CAP / 2, so the key or a free slot is always found
                    for (;;) {
                        const int cur = K[hs];
                        if (cur == q) {
                            if (FILL) V[hs] = __dadd_rn(V[hs], term);
                            break;
                        }
                        if (cur == -1) {
                            const int prev = atomicCAS(&K[hs], -1, q);
                            if (prev == -1) {
                                if (FILL) V[hs] = term;
                                added = true;
                                break;
                            }
                            if (prev == q) {
                                if (FILL) V[hs] = __dadd_rn(V[hs], term);
                                break;
                            }
                        }
                        hs = (hs + 1) & (unsigned)(CAP - 1);
                    }
                }
                used += count(added);   // in a block also the barrier between steps (__syncthreads_count)
                full = used > (CAP >> 1);
            }
            if (!BLOCK) __syncwarp();   // a ballot does not order shared memory: the warp's step barrier
        }
        if (full) {
            if (tid == 0) {
                if (longs && MODE != SPG_FILL) {
                    longs[atomicAdd(nlongs, 1)] = p;
                    cnt[p] = 0x7fffffff;
                } else {
                    atomicExch(overflow, 1);
                }
            }
            sync();
            continue;
        }
        // gather the occupied slots to the front (slot order), then sort by column
        int m = 0;
        for (int s0 = 0; s0 < CAP; s0 += U) {
            const int kk = K[s0 + tid];
            const double vv = FILL ? V[s0 + tid] : 0.0;
            const bool occ = kk >= 0;
            int total;
            const int r = rank(occ, total);
            sync();
            if (occ) {
                K[m + r] = kk;
                if (FILL) V[m + r] = vv;
            }
            m += total;
            sync();
        }
        if (MODE == SPG_COUNT) {
            if (tid == 0) cnt[p] = m;
            continue;
        }
        int m2 = 1;
        while (m2 < m) m2 <<= 1;
        for (int s = m + tid; s < m2; s += U) K[s] = 0x7fffffff;
        sync();
        for (int size = 2; size <= m2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int u = tid; u < m2 / 2; u += U) {
                    const int lo = 2 * u - (u & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const int a = K[lo], b = K[hi];
                    if ((a > b) == up) {
                        K[lo] = b;
                        K[hi] = a;
                        const double tv = V[lo];
                        V[lo] = V[hi];
                        V[hi] = tv;
                    }
                }
                sync();
            }
        const long long c0 = MODE == SPG_FILL ? (long long)xoff[p]
                                              : (xoff ? (long long)xoff[p] * stride : (long long)t * stride);
        for (int s = tid; s < m; s += U) {
            xcol[c0 + s] = K[s];
            xval[c0 + s] = V[s];
        }
        if (MODE == SPG_ONE && tid == 0) cnt[p] = m;
        sync();
    }
}

// Rows of X = Y Z with at most 32 terms, a warp each (expand, sort,
// compress): lane t holds term t in the order of the hash kernel's steps
// (entries of row p of Y in column order, then the entries of the Z row each
// one reads), its stable rank by column comes from a shuffle sweep, the terms
// are placed in rank order in shared memory, and the first lane of every run
// of equal columns sums the run left to right from its first term: for every
// column the same products added in the same order as the hash kernel (and
// the oracle), bit for bit, without a table to clear and sweep. The sorted
// row goes to the first tier's scratch slot (xoff[p] * 8 entries, which
// holds min(terms, its capacity)) and its count to cnt[p]; a row of Y with
// more than 32 entries or a row with more than 32 terms is appended to
// longs for the hash kernel. The rows are list[0 .. *nlist).
__global__ void __launch_bounds__(TPB) k_spgemm_warp(const int* __restrict__ list, const int* __restrict__ nlist,
                                                     const int* __restrict__ yptr,
                                                     const int* __restrict__ ycol, const double* __restrict__ yval,
                                                     const int* __restrict__ zptr, const int* __restrict__ zcol,
                                                     const double* __restrict__ zval, int* __restrict__ cnt,
                                                     const int* __restrict__ xoff, int* __restrict__ xcol,
                                                     double* __restrict__ xval, int* __restrict__ longs,
                                                     int* __restrict__ nlongs) {
    __shared__ int Ks[TPB];
    __shared__ double Vs[TPB];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int* K = Ks + wid * 32;
    double* V = Vs + wid * 32;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int warp_first = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nr = *nlist;
    for (int t = warp_first; t < nr; t += nw) {                   // t is uniform in the warp
        const int p = list[t];
        const int eb = yptr[p], ly = yptr[p + 1] - eb;
        if (ly > 32) {
            if (lane == 0) longs[atomicAdd(nlongs, 1)] = p;
            continue;
        }
        int zb = 0, len = 0;
        double y = 0.0;
        if (lane < ly) {
            const int j = ycol[eb + lane];
            y = yval[eb + lane];
            zb = zptr[j];
            len = zptr[j + 1] - zb;
        }
        int incl = len;                                              // inclusive scan of the Z row lengths
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += v;
        }
        const int T = __shfl_sync(FULL_MASK, incl, 31);
        if (T > 32) {
            if (lane == 0) longs[atomicAdd(nlongs, 1)] = p;
            continue;
        }
        const int start = incl - len;
        for (int k = 0; k < len; ++k) K[start + k] = lane;          // owner entry of every term slot
        __syncwarp();
        const int e = lane < T ? K[lane] : 0;
        const double ye = __shfl_sync(FULL_MASK, y, e);
        const int zbe = __shfl_sync(FULL_MASK, zb, e);
        const int se = __shfl_sync(FULL_MASK, start, e);
        int q = 0x7fffffff;
        double term = 0.0;
        if (lane < T) {
            const int f = zbe + (lane - se);
            q = zcol[f];
            term = __dmul_rn(ye, zval[f]);
        }
        int rank = 0;                                                // stable rank by column
        for (int u = 0; u < T; ++u) {
            const int qu = __shfl_sync(FULL_MASK, q, u);
            rank += (qu < q || (qu == q && u < lane)) ? 1 : 0;
        }
        __syncwarp();
        if (lane < T) {
            K[rank] = q;
            V[rank] = term;
        }
        __syncwarp();
        const int kr = lane < T ? K[lane] : 0;
        const bool head = lane < T && (lane == 0 || K[lane - 1] != kr);
        const unsigned heads = __ballot_sync(FULL_MASK, head);
        const long long c0 = (long long)xoff[p] * 8;
        if (head) {
            double sum = V[lane];
            for (int k = lane + 1; k < T && K[k] == kr; ++k) sum = __dadd_rn(sum, V[k]);
            const int idx = __popc(heads & ((1u << lane) - 1u));
            xcol[c0 + idx] = kr;
            xval[c0 + idx] = sum;
        }
        if (lane == 0) cnt[p] = __popc(heads);
        __syncwarp();
    }
}

// Rows of X = Y Z whose columns lie in a window of at most dcap columns
// starting at base[p] (the listed rows list[0 .. *nlist)), a block each: a
// dense accumulator V[dcap] and an occupancy bitmap in shared memory. Step
// e (entry y of row p of Y) adds y z for every entry z of the Z row it reads;
// within a step the columns are distinct, a column's first term starts its
// sum and later steps add in step order (a barrier between steps): the hash
// kernel's and the oracle's order, bit for bit, with no probing and no sort
// (the bitmap is read in column order). The row goes to its scratch slot at
// xoff[p] * 8 (min(terms, window) entries) and its count to cnt[p].
constexpr int SPG_DENSE_MAX = 12288;
constexpr int SPG_DENSE_MIN_TERMS = 8192;   // rows of a wider product that take the dense kernel
constexpr int SPG_DENSE_THREADS = 256;
constexpr int SPG_STAGE = 512;      // entries of a Y row staged at a time (value and Z row bounds)
constexpr int SPG_PF = 4;           // steps whose first Z chunk is loaded one group ahead
__host__ __device__ constexpr int spg_dense_smem(int dcap) {
    return (int)(sizeof(double) * dcap + sizeof(unsigned) * ((dcap + 31) / 32) +
                 SPG_STAGE * (sizeof(double) + 2 * sizeof(int)));
}
__global__ void __launch_bounds__(SPG_DENSE_THREADS) k_spgemm_dense(
    const int* __restrict__ list, const int* __restrict__ nlist, const int* __restrict__ base, int dcap,
    const int* __restrict__ yptr, const int* __restrict__ ycol,
    const double* __restrict__ yval, const int* __restrict__ zptr, const int* __restrict__ zcol,
    const double* __restrict__ zval, int* __restrict__ cnt, const int* __restrict__ xoff, int* __restrict__ xcol,
    double* __restrict__ xval) {
    extern __shared__ double dsm[];
    __shared__ int wtot[SPG_DENSE_THREADS / 32];
    const int nw = (dcap + 31) >> 5;
    double* V = dsm;
    double* sy = dsm + dcap;                                   // staged y values
    int* sb = reinterpret_cast<int*>(sy + SPG_STAGE);           // staged Z row starts
    int* se = sb + SPG_STAGE;                                   // staged Z row ends
    unsigned* F = reinterpret_cast<unsigned*>(se + SPG_STAGE);  // occupancy bitmap
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int U = SPG_DENSE_THREADS;
    const int per = (nw + U - 1) / U;                       // bitmap words per thread in the read-out
    const int nr = *nlist;
    for (int t = blockIdx.x; t < nr; t += gridDim.x) {
        const int p = list[t];
        const int b = base[p];                                  // first column of the window
        for (int w = tid; w < nw; w += U) F[w] = 0u;
        const int eb = yptr[p], ee = yptr[p + 1];
        for (int b0 = eb; b0 < ee; b0 += SPG_STAGE) {
            const int nb = min(SPG_STAGE, ee - b0);
            __syncthreads();                                    // the previous batch's staged entries are done
            for (int i = tid; i < nb; i += U) {
                const int j = ycol[b0 + i];
                sy[i] = yval[b0 + i];
                sb[i] = zptr[j];
                se[i] = zptr[j + 1];
            }
            __syncthreads();
            int qa[SPG_PF];
            double za[SPG_PF];
#pragma unroll
            for (int k = 0; k < SPG_PF; ++k) {
                const bool ok = k < nb && sb[k] + tid < se[k];
                qa[k] = ok ? zcol[sb[k] + tid] : 0;
                za[k] = ok ? zval[sb[k] + tid] : 0.0;
            }
            for (int g = 0; g < nb; g += SPG_PF) {
                int qb[SPG_PF];
                double zb[SPG_PF];
#pragma unroll
                for (int k = 0; k < SPG_PF; ++k) {              // the next group's first chunks
                    const int sn = g + SPG_PF + k;
                    const bool ok = sn < nb && sb[sn] + tid < se[sn];
                    qb[k] = ok ? zcol[sb[sn] + tid] : 0;
                    zb[k] = ok ? zval[sb[sn] + tid] : 0.0;
                }
#pragma unroll
                for (int k = 0; k < SPG_PF; ++k) {
                    const int sk = g + k;
                    if (sk >= nb) break;                        // uniform in the block
                    const double y = sy[sk];
                    const int fb = sb[sk], fe = se[sk];
                    for (int f = fb + tid; f < fe; f += U) {
                        const bool pre = f - fb < U;
                        const int q = (pre ? qa[k] : zcol[f]) - b;
                        const double term = __dmul_rn(y, pre ? za[k] : zval[f]);
                        const unsigned bit = 1u << (q & 31);
                        if (F[q >> 5] & bit) {
                            V[q] = __dadd_rn(V[q], term);
                        } else {
                            V[q] = term;
                            atomicOr(&F[q >> 5], bit);
                        }
                    }
                    __syncthreads();                            // the barrier between steps
                }
#pragma unroll
                for (int k = 0; k < SPG_PF; ++k) {
                    qa[k] = qb[k];
                    za[k] = zb[k];
                }
            }
        }
        __syncthreads();                                        // the bitmap is complete (also for an empty row)
        // read-out in column order: thread t takes words [t * per, (t + 1) * per)
        int mine = 0;
        for (int k = 0; k < per; ++k) {
            const int w = tid * per + k;
            if (w < nw) mine += __popc(F[w]);
        }
        int incl = mine;                                        // block exclusive scan of the counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wtot[wid] = incl;
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int w2 = 0; w2 < U / 32; ++w2) {
            before += w2 < wid ? wtot[w2] : 0;
            total += wtot[w2];
        }
        int pos = before + incl - mine;
        const long long c0 = (long long)xoff[p] * 8;
        for (int k = 0; k < per; ++k) {
            const int w = tid * per + k;
            if (w >= nw) break;
            unsigned bits = F[w];
            while (bits) {
                const int q = (w << 5) + __ffs(bits) - 1;
                bits &= bits - 1;
                xcol[c0 + pos] = b + q;
                xval[c0 + pos] = V[q];
                ++pos;
            }
        }
        if (tid == 0) cnt[p] = total;
        __syncthreads();                                        // wtot and F are reused by the next row
    }
}


// Per row p of X = Y Z: its terms T (the lengths of the Z rows it reads) and
// the window [lo, hi] between the first and the last column of those rows.
// A row whose window has at most dcap columns and that has at least dmin
// terms goes to the dense kernel (base[p] = lo, listed in dlist), any other
// to the warp pass and the hash tiers (base[p] = -1, listed in olist): a
// block with a dense window is the faster way for rows of many terms, warps
// with small hash tables for rows of few. units[p] = the scratch units (8
// entries) of its slot, min(T, window) or min(T, hcap). Lists are appended a
// warp at a time (their order does not matter: every row has its own slot).
__global__ void k_spgemm_classify(int n, const int* __restrict__ yptr, const int* __restrict__ ycol,
                                  const int* __restrict__ zptr, const int* __restrict__ zcol, int hcap, int dcap,
                                  int dmin, int* __restrict__ units, int* __restrict__ base, int* __restrict__ dlist,
                                  int* __restrict__ ndl, int* __restrict__ olist, int* __restrict__ nol) {
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int p0 = blockIdx.x * blockDim.x + threadIdx.x - lane; p0 < n; p0 += stride) {   // uniform in the warp
        const int p = p0 + lane;
        const bool valid = p < n;
        bool dense = false;
        if (valid) {
            int T = 0, lo = 0x7fffffff, hi = -1;
            for (int e = yptr[p]; e < yptr[p + 1]; ++e) {
                const int j = ycol[e];
                const int zb = zptr[j], ze = zptr[j + 1];
                if (ze > zb) {
                    T += ze - zb;
                    lo = min(lo, zcol[zb]);
                    hi = max(hi, zcol[ze - 1]);
                }
            }
            const int win = hi >= lo ? hi - lo + 1 : 0;
            dense = win > 0 && win <= dcap && T >= dmin;
            units[p] = ((dense ? min(T, win) : min(T, hcap)) + 7) >> 3;
            base[p] = dense ? lo : -1;
        }
        const unsigned bd = __ballot_sync(FULL_MASK, valid && dense);
        const unsigned bo = __ballot_sync(FULL_MASK, valid && !dense);
        int d0 = 0, o0 = 0;
        if (lane == 0) {
            if (bd) d0 = atomicAdd(ndl, __popc(bd));
            if (bo) o0 = atomicAdd(nol, __popc(bo));
        }
        d0 = __shfl_sync(FULL_MASK, d0, 0);
        o0 = __shfl_sync(FULL_MASK, o0, 0);
        const unsigned below = (1u << lane) - 1u;
        if (valid && dense) dlist[d0 + __popc(bd & below)] = p;
        else if (valid) olist[o0 + __popc(bo & below)] = p;
    }
}

// k_spgemm_classify with a warp per row, for long rows of Y (the lanes
// stride the row; one append per row).
__global__ void k_spgemm_classify_warp(int n, const int* __restrict__ yptr, const int* __restrict__ ycol,
                                       const int* __restrict__ zptr, const int* __restrict__ zcol, int hcap,
                                       int dcap, int dmin, int* __restrict__ units, int* __restrict__ base,
                                       int* __restrict__ dlist, int* __restrict__ ndl, int* __restrict__ olist,
                                       int* __restrict__ nol) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += nw) {   // uniform in the warp
        int T = 0, lo = 0x7fffffff, hi = -1;
        for (int e = yptr[p] + lane; e < yptr[p + 1]; e += 32) {
            const int j = ycol[e];
            const int zb = zptr[j], ze = zptr[j + 1];
            if (ze > zb) {
                T += ze - zb;
                lo = min(lo, zcol[zb]);
                hi = max(hi, zcol[ze - 1]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T += __shfl_xor_sync(FULL_MASK, T, o);
            lo = min(lo, __shfl_xor_sync(FULL_MASK, lo, o));
            hi = max(hi, __shfl_xor_sync(FULL_MASK, hi, o));
        }
        if (lane == 0) {
            const int win = hi >= lo ? hi - lo + 1 : 0;
            const bool dense = win > 0 && win <= dcap && T >= dmin;
            units[p] = ((dense ? min(T, win) : min(T, hcap)) + 7) >> 3;
            base[p] = dense ? lo : -1;
            if (dense) dlist[atomicAdd(ndl, 1)] = p;
            else olist[atomicAdd(nol, 1)] = p;
        }
    }
}

// Rows of a one-pass product from their scratch slots (as in SPG_ONE) to the
// CSR arrays, a warp per row; rows with more than `limit` columns went on to
// a launch of larger capacity and are copied from its slots, except the rows
// of the dense kernel (dense[p] >= 0), which are always in these slots.
__global__ void k_spgemm_copy(int nrows, const int* __restrict__ list, const int* __restrict__ nlist, int limit,
                              const int* __restrict__ dense, const int* __restrict__ cnt,
                              const int* __restrict__ xoff, long long stride,
                              const int* __restrict__ scol, const double* __restrict__ sval,
                              const int* __restrict__ xptr, int* __restrict__ xcol, double* __restrict__ xval) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int nr = list ? *nlist : nrows;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nr; t += nw) {
        const int p = list ? list[t] : t;
        const int m = cnt[p];
        if (m > limit && !(dense && dense[p] >= 0)) continue;   // left to a tier of larger capacity
        const long long src = xoff ? (long long)xoff[p] * stride : (long long)t * stride;
        const int dst = xptr[p];
        for (int s = lane; s < m; s += 32) {
            xcol[dst + s] = scol[src + s];
            xval[dst + s] = sval[src + s];
        }
    }
}

// ------------------------------------------------------------ host side ----
struct Scratch {
    DevArena mem;
    double* diag = nullptr;
    double* c = nullptr;
    int *mate = nullptr, *cand = nullptr, *list0 = nullptr, *list1 = nullptr, *mlist = nullptr;
    int* cnt = nullptr;       // [0,1] list counters, [2,3] match counters, [4] rounds, [5] flags, [6..7] totals,
                              // [8] rows left by the group row-product kernels, [9] by the group edge sort,
                              // [10..13] sparse-product and pair-sort overflow and list counters,
                              // [13, 14] also rows left by the long-row kernels
    int* flag = nullptr;      // n
    int* qid = nullptr;       // n
    int* heads = nullptr;     // n
    int* ub = nullptr;        // n + 1
    int* off = nullptr;       // n + 1
    int* skey = nullptr;      // nnz
    double* sval = nullptr;   // nnz
    int* spos = nullptr;      // nnz: sorted position of each entry (matching by proposals)
    int2* nq = nullptr;       // nnz: (neighbour, mirror's sorted position) per sorted entry
    int* rowbase = nullptr;   // n: a sparse product row's column window base (-1: the hash path)
    unsigned long long* suitor = nullptr;   // n
    long long cap_nnz = 0;    // entries c, skey and sval hold
    int* scan_tmp = nullptr;
    int* host = nullptr;      // pinned
    ~Scratch() {
        if (host) cudaFreeHost(host);
    }
};

int grid_for(const amg_hierarchy* h, long long n) { return blocks_for(n, TPB, h->num_sms * 16); }

int read_int(const int* dev, int* host, cudaStream_t st) {
    CUDA_CHECK(cudaMemcpyAsync(host, dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    return *host;
}

// C.nnz from C.ptr[n] and C.max_row from a row-length maximum, with one
// stream synchronisation.
void finish_csr(amg_hierarchy* h, Scratch& S, DevCsr& C) {
    cudaStream_t st = h->stream;
    CUDA_CHECK(cudaMemsetAsync(S.cnt + 19, 0, sizeof(int), st));
    if (C.n > 0) {
        k_max_row<<<grid_for(h, C.n), TPB, 0, st>>>(C.n, C.ptr, S.cnt + 19);
        KERNEL_CHECK();
    }
    CUDA_CHECK(cudaMemcpyAsync(S.host, C.ptr + C.n, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(S.host + 1, S.cnt + 19, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    C.nnz = S.host[0];
    C.max_row = S.host[1];
}

// The rows of a row product that the group kernel listed in (list, *nlist):
// a block each up to ROW_CAPS[0] terms (rows left listed in S.qid, counted in
// S.cnt[13]), then up to ROW_CAPS[1] (rows left in S.list0, S.cnt[14]), then
// the thread-per-row kernel for any longer ones.
template <bool RAP>
void launch_rows_long(amg_hierarchy* h, Scratch& S, int nrows, const int* list, const int* nlist, const int* heads,
                      const int* mate, const int* ptr, const int* col, const double* val, const int* agg,
                      const double* p, const int* off, int* cnt, const double* rowscale, cudaStream_t st, int G,
                      int max_terms) {
    // rows of G+1 .. 32 terms: a warp each, 32 lanes (a block per row would
    // spend a whole block and its barriers on a few dozen terms); then rows up
    // to WROW terms: a warp each, sorted in shared memory. The passes
    // alternate between the caller's list (list1 / cnt[8]) and flag / cnt[12].
    int* lists[2] = {S.list1, S.flag};
    int* counts[2] = {S.cnt + 8, S.cnt + 12};
    int cur = 0;
    if (G < 32) {
        CUDA_CHECK(cudaMemsetAsync(counts[1], 0, sizeof(int), st));
        launch_rows<RAP>(h, 32, nrows, heads, mate, ptr, col, val, agg, p, off, S.skey, S.sval, cnt, lists[1],
                         counts[1], rowscale, st, lists[0], counts[0]);
        if (max_terms > 0 && max_terms <= 32) return;
        cur = 1;
    }
    CUDA_CHECK(cudaMemsetAsync(counts[cur ^ 1], 0, sizeof(int), st));
    k_rows_warp_sm<RAP><<<h->num_sms * 8, TPB, 0, st>>>(lists[cur], counts[cur], heads, mate, ptr, col, val, agg, p,
                                                        off, S.skey, S.sval, cnt, lists[cur ^ 1], counts[cur ^ 1],
                                                        rowscale);
    KERNEL_CHECK();
    if (max_terms > 0 && max_terms <= WROW) return;
    cur ^= 1;
    list = lists[cur];
    nlist = counts[cur];
    constexpr int tb = (int)(sizeof(unsigned long long) + sizeof(double));
    CUDA_CHECK(cudaFuncSetAttribute(k_rows_long<RAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, ROW_CAPS[1] * tb));
    CUDA_CHECK(cudaMemsetAsync(S.cnt + 13, 0, 2 * sizeof(int), st));
    k_rows_long<RAP><<<h->num_sms * 3, LONG_TPB, ROW_CAPS[0] * tb, st>>>(
        list, nlist, ROW_CAPS[0], heads, mate, ptr, col, val, agg, p, off, S.skey, S.sval, cnt, S.qid, S.cnt + 13,
        rowscale);
    KERNEL_CHECK();
    k_rows_long<RAP><<<h->num_sms, LONG_TPB, ROW_CAPS[1] * tb, st>>>(S.qid, S.cnt + 13, ROW_CAPS[1], heads, mate, ptr,
                                                                     col, val, agg, p, off, S.skey, S.sval, cnt,
                                                                     S.list0, S.cnt + 14, rowscale);
    KERNEL_CHECK();
    if (RAP)
        k_rap_rows<<<grid_for(h, nrows), TPB, 0, st>>>(nrows, heads, mate, ptr, col, val, agg, p, off, S.skey, S.sval,
                                                      cnt, S.list0, S.cnt + 14);
    else
        k_ap_rows<<<grid_for(h, nrows), TPB, 0, st>>>(nrows, ptr, col, val, agg, p, S.skey, S.sval, cnt, S.list0,
                                                     S.cnt + 14, rowscale);
    KERNEL_CHECK();
}

// Each row's edges sorted by the strict edge order into nbr (S.skey), the
// position pointer pos (S.flag), first candidates and isolated vertices; with
// spos set, also the sorted position of every original entry.
void sort_edges(amg_hierarchy* h, Scratch& S, const DevCsr& A, int* spos) {
    cudaStream_t st = h->stream;
    const int n = A.n;
    int* nbr = S.skey;
    double* sc = S.sval;
    int* pos = S.flag;
    CUDA_CHECK(cudaMemsetAsync(S.cnt + 9, 0, sizeof(int), st));
    const int G = rows_group(A.nnz, n);
    const int gblocks = blocks_for((long long)n * G, TPB, h->num_sms * 16);
    if (G == 8)
        k_sort_edges_group<8><<<gblocks, TPB, 0, st>>>(n, nullptr, nullptr, A.ptr, A.col, S.c, nbr, pos, S.cand,
                                                       S.mate, S.list1, S.cnt + 9, spos);
    else if (G == 16)
        k_sort_edges_group<16><<<gblocks, TPB, 0, st>>>(n, nullptr, nullptr, A.ptr, A.col, S.c, nbr, pos, S.cand,
                                                        S.mate, S.list1, S.cnt + 9, spos);
    else
        k_sort_edges_group<32><<<gblocks, TPB, 0, st>>>(n, nullptr, nullptr, A.ptr, A.col, S.c, nbr, pos, S.cand,
                                                        S.mate, S.list1, S.cnt + 9, spos);
    KERNEL_CHECK();
    if (A.max_row > 0 && A.max_row <= G) return;       // no row left for the long-row kernels
    // rows of G+1 .. 32 entries: a warp each, 32 lanes (a block per row would
    // spend a whole block and its barriers on a few dozen entries); then rows
    // up to WROW entries: a warp each, sorted in shared memory. The passes
    // alternate between two row lists (list1 / cnt[9] and list0 / cnt[12]).
    int* lists[2] = {S.list1, S.list0};
    int* counts[2] = {S.cnt + 9, S.cnt + 12};
    int cur = 0;
    if (G < 32) {
        CUDA_CHECK(cudaMemsetAsync(counts[1], 0, sizeof(int), st));
        k_sort_edges_group<32><<<h->num_sms * 16, TPB, 0, st>>>(n, lists[0], counts[0], A.ptr, A.col, S.c, nbr, pos,
                                                                 S.cand, S.mate, lists[1], counts[1], spos);
        KERNEL_CHECK();
        if (A.max_row > 0 && A.max_row <= 32) return;
        cur = 1;
    }
    CUDA_CHECK(cudaMemsetAsync(counts[cur ^ 1], 0, sizeof(int), st));
    k_sort_edges_warp<<<h->num_sms * 8, TPB, 0, st>>>(lists[cur], counts[cur], A.ptr, A.col, S.c, nbr, pos, S.cand,
                                                      S.mate, lists[cur ^ 1], counts[cur ^ 1], spos);
    KERNEL_CHECK();
    if (A.max_row > 0 && A.max_row <= WROW) return;
    cur ^= 1;
    const int* lrows = lists[cur];
    const int* nlrows = counts[cur];
    // longer rows: a block each in two capacities, then a thread each
    constexpr int eb = (int)(sizeof(long long) + sizeof(int));
    CUDA_CHECK(cudaFuncSetAttribute(k_sort_edges_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    EDGE_CAPS[1] * eb));
    k_sort_edges_long<<<h->num_sms * 4, LONG_TPB, EDGE_CAPS[0] * eb, st>>>(
        lrows, nlrows, EDGE_CAPS[0], A.ptr, A.col, S.c, nbr, pos, S.cand, S.mate, S.qid, S.cnt + 13, spos);
    KERNEL_CHECK();
    k_sort_edges_long<<<h->num_sms, LONG_TPB, EDGE_CAPS[1] * eb, st>>>(
        S.qid, S.cnt + 13, EDGE_CAPS[1], A.ptr, A.col, S.c, nbr, pos, S.cand, S.mate, S.heads, S.cnt + 14, spos);
    KERNEL_CHECK();
    k_sort_edges<<<grid_for(h, n), TPB, 0, st>>>(n, A.ptr, A.col, S.c, sc, nbr, pos, S.cand, S.mate, S.heads,
                                                 S.cnt + 14, spos);
    KERNEL_CHECK();
}

// The error word of the proposal matching (read by the caller together with
// the aggregate count, one synchronisation).
void check_suitor_error(int e) {
    if (e & 1) AMG_THROW(AMG_ERR_ARG, "matching: an edge has no mirror entry (pattern not symmetric)");
    if (e & 8) AMG_THROW(AMG_ERR_ARG, "matching: a row without a diagonal entry");
    if (e & 6) AMG_THROW(AMG_ERR_CUDA, "matching by proposals did not settle (internal error %d)", e);
}

// Proposals over the sorted rows in S.nq (suitor words reset), then mate.
// Errors are left in *err for the caller.
void suitor_match(amg_hierarchy* h, Scratch& S, const DevCsr& A, int* err) {
    cudaStream_t st = h->stream;
    const int n = A.n;
    Scope sc_(&h->prof, st, S_MATCH, 0.0);
    if (n > 0) {
        k_suitor<<<(n + 255) / 256, 256, 0, st>>>(n, (long long)A.nnz, A.ptr, S.nq, S.suitor, err);
        KERNEL_CHECK();
    }
    k_suitor_mate<<<grid_for(h, n), TPB, 0, st>>>(n, S.nq, S.suitor, S.mate, err);
    KERNEL_CHECK();
}

// The matching of one sweep into S.mate (partner, or < 0 unmatched).
// Returns the number of locally-dominant rounds (0 for the proposal method,
// which has none). match_kernel 0: proposals (k_suitor); 1: one launch pair
// per round with a host check every 16 rounds; 2: all rounds in one
// cooperative launch when the device allows it (else as 1). For 0, *pending
// is set to the device error word, which the caller must read and pass to
// check_suitor_error before it uses the matching beyond a scan of it.
int ld_match(amg_hierarchy* h, Scratch& S, const DevCsr& A, int** pending) {
    *pending = nullptr;
    cudaStream_t st = h->stream;
    const int n = A.n;
    CUDA_CHECK(cudaMemsetAsync(S.mate, 0xff, sizeof(int) * n, st));   // all -1
    // algorithmic bytes of the edge sort (c, col in; nbr, spos out) and of
    // the mirror map (c, col, spos in, the mirror's spos gathered, nq out)
    const double sort_bytes = 20.0 * A.nnz + 8.0 * n, mirror_bytes = 28.0 * A.nnz + 16.0 * n;
    if (h->opt.match_kernel == 0) {
        int* err = S.cnt + 16;
        {
            Scope sc_(&h->prof, st, S_MATCH_SORT, sort_bytes + mirror_bytes);
            CUDA_CHECK(cudaMemsetAsync(S.cnt + 13, 0, 4 * sizeof(int), st));   // [13, 14] long-row lists, [16] error
            sort_edges(h, S, A, S.spos);
            const int G = rows_group(A.nnz, n);
            const int mblocks = blocks_for((long long)n * G, TPB, h->num_sms * 16);
            if (G == 8)
                k_mirror_pos<8><<<mblocks, TPB, 0, st>>>(n, A.ptr, A.col, S.c, S.spos, S.nq, S.suitor, err);
            else if (G == 16)
                k_mirror_pos<16><<<mblocks, TPB, 0, st>>>(n, A.ptr, A.col, S.c, S.spos, S.nq, S.suitor, err);
            else
                k_mirror_pos<32><<<mblocks, TPB, 0, st>>>(n, A.ptr, A.col, S.c, S.spos, S.nq, S.suitor, err);
            KERNEL_CHECK();
        }
        suitor_match(h, S, A, err);
        *pending = err;
        return 0;
    }
    if (h->opt.match_kernel == 2 && h->coop_blocks > 0) {
        int* nbr = S.skey;            // sorted neighbour lists (free until the Galerkin step)
        int* pos = S.flag;
        CUDA_CHECK(cudaMemsetAsync(S.cnt, 0, sizeof(int) * 64, st));
        {
            Scope sc_(&h->prof, st, S_MATCH_SORT, sort_bytes);
            sort_edges(h, S, A, nullptr);
        }
        Scope sc_(&h->prof, st, S_MATCH, 0.0);
        int nn = n;
        const int* ptr = A.ptr;
        const int* col = A.col;
        long long max_rounds = (long long)n + 4;
        // lanes per frontier vertex: 8, 16 or 32 by the mean row length
        const double mean = n > 0 ? (double)A.nnz / n : 0.0;
        int ngl = mean >= 48.0 ? 5 : (mean >= 16.0 ? 4 : 3);
        void* args[] = {&nn, &ptr, &col, &nbr, &pos, &S.cand, &S.mate, &S.list0, &S.list1, &ngl, &S.cnt,
                        &max_rounds};
        CUDA_CHECK(cudaLaunchCooperativeKernel((const void*)k_ld_persistent, dim3(h->coop_blocks), dim3(1024), args, 0,
                                               st));
        KERNEL_CHECK();
        int hc[16];
        CUDA_CHECK(cudaMemcpyAsync(hc, S.cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
        CUDA_CHECK(cudaStreamSynchronize(st));
        if (hc[7] == 1) AMG_THROW(AMG_ERR_TIMEOUT, "matching kernel: grid barrier wait exceeded 2 s");
        if (hc[7] == 2) AMG_THROW(AMG_ERR_TIMEOUT, "matching did not settle after n rounds");
        return hc[8];
    }
    Scope sc_(&h->prof, st, S_MATCH, 0.0);
    CUDA_CHECK(cudaMemsetAsync(S.cnt, 0, sizeof(int) * 5, st));
    k_ld_init<<<grid_for(h, n), TPB, 0, st>>>(n, A.ptr, A.col, S.c, S.cand, S.mate);
    KERNEL_CHECK();
    int* lists[2] = {S.list0, S.list1};
    int* lcnt = S.cnt;          // two slots
    int* mcnt = S.cnt + 2;      // two slots
    const int grid = h->num_sms * 8;
    const int batch = 16;
    const long long max_rounds = (long long)n + 4;
    long long r = 0;
    for (;;) {
        for (int b = 0; b < batch; ++b, ++r) {
            const int cur = (int)(r & 1), nxt = (int)((r + 1) & 1);
            k_ld_match<<<grid, TPB, 0, st>>>(n, r == 0 ? nullptr : lists[cur], &lcnt[cur], S.cand, S.mate, S.mlist,
                                             &mcnt[cur], &lcnt[nxt], S.cnt + 4);
            KERNEL_CHECK();
            k_ld_update<<<grid, TPB, 0, st>>>(n, A.ptr, A.col, S.c, S.cand, S.mate, S.mlist, &mcnt[cur], lists[nxt],
                                              &lcnt[nxt], &mcnt[nxt]);
            KERNEL_CHECK();
        }
        if (read_int(&lcnt[r & 1], S.host, st) == 0) break;
        if (r > max_rounds) AMG_THROW(AMG_ERR_TIMEOUT, "matching did not settle after %lld rounds", r);
    }
    return read_int(S.cnt + 4, S.host, st);
}

struct SweepOut {
    int nc;
    int* agg;
    double* p;
    double* wc;
};

// Pairwise Galerkin product C = P^T A P (one nonzero per row of P).
DevCsr galerkin_pairwise(amg_hierarchy* h, Scratch& S, const DevCsr& A, const SweepOut& sw, DevArena& owner) {
    cudaStream_t st = h->stream;
    const int nc = sw.nc;
    k_rap_bound<<<grid_for(h, nc), TPB, 0, st>>>(nc, S.heads, S.mate, A.ptr, S.ub);
    KERNEL_CHECK();
    scan_exclusive(S.ub, S.off, nc, S.cnt + 6, st, S.scan_tmp);
    CUDA_CHECK(cudaMemsetAsync(S.cnt + 8, 0, sizeof(int), st));
    const int G = rows_group(2LL * A.nnz, A.n);
    launch_rows<true>(h, G, nc, S.heads, S.mate, A.ptr, A.col, A.val, sw.agg, sw.p, S.off, S.skey, S.sval, S.ub,
                      S.list1, S.cnt + 8, nullptr, st);
    if (A.max_row == 0 || 2 * A.max_row > G)            // a coarse row gathers the rows of its (at most two) members
        launch_rows_long<true>(h, S, nc, S.list1, S.cnt + 8, S.heads, S.mate, A.ptr, A.col, A.val, sw.agg, sw.p,
                               S.off, S.ub, nullptr, st, G, 2 * A.max_row);
    DevCsr C;
    C.n = nc;
    C.ptr = owner.alloc<int>(nc + 1);
    scan_exclusive(S.ub, C.ptr, nc, C.ptr + nc, st, S.scan_tmp);
    finish_csr(h, S, C);
    C.col = owner.alloc<int>(C.nnz);
    C.val = owner.alloc<double>(C.nnz);
    // the weight denominators of the next sweep come with the copy
    launch_copy(h, C.nnz, nc, S.off, C.ptr, S.skey, S.sval, C.col, C.val, st, sw.wc, S.diag);
    return C;
}

// SELL of A. With len set, row i of the source starts at A.ptr[i] and has
// len[i] entries (A.nnz is then counted here); wtmp is the slice-width
// scratch (S.ub when null).
void build_sell(amg_hierarchy* h, DevCsr A, DevSell& E, Scratch& S, bool fp32, const int* len = nullptr,
                int* wtmp = nullptr, int64_t* nnz_out = nullptr) {
    cudaStream_t st = h->stream;
    int* width = wtmp ? wtmp : S.ub;
    E.n = A.n;
    E.nslices = (A.n + SELL_C - 1) / SELL_C;
    E.sptr = h->mem.alloc<int>(E.nslices + 1);
    const int wgrid = blocks_for((long long)E.nslices * 32, TPB, h->num_sms * 16);
    int* cnt = len ? S.cnt + 19 : nullptr;
    if (cnt) CUDA_CHECK(cudaMemsetAsync(cnt, 0, sizeof(int), st));
    k_sell_width<<<wgrid, TPB, 0, st>>>(A.n, E.nslices, A.ptr, len, nullptr, width, cnt);
    KERNEL_CHECK();
    scan_exclusive(width, E.sptr, E.nslices, E.sptr + E.nslices, st, S.scan_tmp);
    CUDA_CHECK(cudaMemcpyAsync(S.host, E.sptr + E.nslices, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (cnt) CUDA_CHECK(cudaMemcpyAsync(S.host + 1, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    E.padded = (int64_t)S.host[0] * SELL_C;
    if (cnt) A.nnz = S.host[1];
    if (nnz_out) *nnz_out = A.nnz;
    if ((double)E.padded > 1.3 * (double)A.nnz) {
        // uneven rows: sort by length inside windows (SELL-C-sigma)
        E.perm = h->mem.alloc<int>(A.n);
        k_sort_window<<<(A.n + SIGMA - 1) / SIGMA, SIGMA, 0, st>>>(A.n, nullptr, A.ptr, len, E.perm);
        KERNEL_CHECK();
        k_sell_width<<<wgrid, TPB, 0, st>>>(A.n, E.nslices, A.ptr, len, E.perm, width, nullptr);
        KERNEL_CHECK();
        scan_exclusive(width, E.sptr, E.nslices, E.sptr + E.nslices, st, S.scan_tmp);
        E.padded = (int64_t)read_int(E.sptr + E.nslices, S.host, st) * SELL_C;
    }
    E.col = h->mem.alloc<int>(E.padded);
    E.val = h->mem.alloc<double>(E.padded);
    k_sell_fill<<<blocks_for((long long)E.nslices * 32, TPB, h->num_sms * 16), TPB, 0, st>>>(
        A.n, E.nslices, A.ptr, len, A.col, A.val, E.sptr, E.perm, E.col, E.val);
    KERNEL_CHECK();
    if (fp32) {
        E.val32 = h->mem.alloc<float>(E.padded);
        k_to_float<<<blocks_for(E.padded, TPB, h->num_sms * 16), TPB, 0, st>>>(E.padded, E.val, E.val32);
        KERNEL_CHECK();
    }
}

// Hybrid layout for the iterative coarsest solve: rows with at most lmax
// entries in SELL-C-sigma (positions map to rows through perm), longer rows
// listed in long_rows and read straight from the CSR by one warp each, so a
// few long rows cannot hold up a whole slice.
void build_sell_hybrid(amg_hierarchy* h, const DevCsr& A, DevSell& E, Scratch& S, int lmax) {
    cudaStream_t st = h->stream;
    const int n = A.n;
    k_long_flags<<<grid_for(h, n), TPB, 0, st>>>(n, A.ptr, lmax, S.flag);
    KERNEL_CHECK();
    scan_exclusive(S.flag, S.qid, n, S.cnt + 6, st, S.scan_tmp);
    const int nlong = read_int(S.cnt + 6, S.host, st);
    const int nshort = n - nlong;
    E.nlong = nlong;
    E.long_rows = h->mem.alloc<int>(nlong > 0 ? nlong : 1);
    int* short_rows = S.mem.alloc<int>(nshort > 0 ? nshort : 1);
    k_split_rows<<<grid_for(h, n), TPB, 0, st>>>(n, S.flag, S.qid, E.long_rows, short_rows);
    KERNEL_CHECK();
    E.n = nshort;
    E.nslices = (nshort + SELL_C - 1) / SELL_C;
    E.sptr = h->mem.alloc<int>(E.nslices + 1);
    E.perm = h->mem.alloc<int>(nshort > 0 ? nshort : 1);
    k_sort_window<<<(nshort + SIGMA - 1) / SIGMA > 0 ? (nshort + SIGMA - 1) / SIGMA : 1, SIGMA, 0, st>>>(
        nshort, short_rows, A.ptr, nullptr, E.perm);
    KERNEL_CHECK();
    const int wgrid = blocks_for((long long)E.nslices * 32, TPB, h->num_sms * 16);
    k_sell_width<<<wgrid, TPB, 0, st>>>(nshort, E.nslices, A.ptr, nullptr, E.perm, S.ub, nullptr);
    KERNEL_CHECK();
    scan_exclusive(S.ub, E.sptr, E.nslices, E.sptr + E.nslices, st, S.scan_tmp);
    E.padded = (int64_t)read_int(E.sptr + E.nslices, S.host, st) * SELL_C;
    E.col = h->mem.alloc<int>(E.padded);
    E.val = h->mem.alloc<double>(E.padded);
    k_sell_fill<<<wgrid, TPB, 0, st>>>(nshort, E.nslices, A.ptr, nullptr, A.col, A.val, E.sptr, E.perm, E.col,
                                       E.val);
    KERNEL_CHECK();
    S.mem.release(short_rows);
}

// Column-scaled values of A M^{-1} in A's SELL layout (padding stays 0).
void build_scaled(amg_hierarchy* h, Level& L, bool fp32) {
    cudaStream_t st = h->stream;
    const long long m = L.S.padded;
    L.valm = h->mem.alloc<double>(m);
    if (fp32) L.valm32 = h->mem.alloc<float>(m);
    k_scale_cols<<<blocks_for(m, TPB, h->num_sms * 16), TPB, 0, st>>>(m, L.S.col, L.S.val, L.minv, L.valm, L.valm32);
    KERNEL_CHECK();
}

// omega M_l^{-1} A_l P_l in SELL (rows of A_l scaled by omega / M_ii, columns
// the aggregates of level l+1): the coarse-correction term of the fused
// post-smoother needs no per-row scaling in the solve.
void build_ap(amg_hierarchy* h, Level& L, int nc, Scratch& S, bool fp32) {
    cudaStream_t st = h->stream;
    const int n = L.A.n;
    CUDA_CHECK(cudaMemsetAsync(S.cnt + 8, 0, sizeof(int), st));
    const int G = rows_group(L.A.nnz, n);
    launch_rows<false>(h, G, n, nullptr, nullptr, L.A.ptr, L.A.col, L.A.val, L.agg, L.p, L.A.ptr, S.skey, S.sval,
                       S.ub, S.list1, S.cnt + 8, L.wminv, st);
    if (L.A.max_row == 0 || L.A.max_row > G)
        launch_rows_long<false>(h, S, n, S.list1, S.cnt + 8, nullptr, nullptr, L.A.ptr, L.A.col, L.A.val, L.agg,
                                L.p, L.A.ptr, S.ub, L.wminv, st, G, L.A.max_row);
    // SELL straight from the row products: row i at L.A.ptr[i] in (skey, sval),
    // S.ub[i] entries (S.off holds the slice widths meanwhile)
    DevCsr AP;
    AP.n = n;
    AP.ptr = L.A.ptr;
    AP.col = S.skey;
    AP.val = S.sval;
    build_sell(h, AP, L.AP, S, fp32, S.ub, S.off, &L.ap_nnz);
}

void build_members(amg_hierarchy* h, Level& L, int nc, Scratch& S) {
    cudaStream_t st = h->stream;
    const int n = L.A.n;
    L.pt_ptr = h->mem.alloc<int>(nc + 1);
    L.pt_idx = h->mem.alloc<int>(n);
    CUDA_CHECK(cudaMemsetAsync(S.ub, 0, sizeof(int) * (nc + 1), st));
    k_member_count<<<grid_for(h, n), TPB, 0, st>>>(n, L.agg, S.ub);
    KERNEL_CHECK();
    scan_exclusive(S.ub, L.pt_ptr, nc, L.pt_ptr + nc, st, S.scan_tmp);
    CUDA_CHECK(cudaMemsetAsync(S.ub, 0, sizeof(int) * (nc + 1), st));
    k_member_fill<<<grid_for(h, n), TPB, 0, st>>>(n, L.agg, L.pt_ptr, S.ub, L.pt_idx);
    KERNEL_CHECK();
    k_member_sort<<<grid_for(h, nc), TPB, 0, st>>>(nc, L.pt_ptr, L.pt_idx);
    KERNEL_CHECK();
}

// Per-entry scratch for a matrix of nnz entries: the smoothed Galerkin product
// can give a coarse matrix with more entries than the finest one.
void ensure_entry_scratch(Scratch& S, long long nnz, cudaStream_t st) {
    if (nnz <= S.cap_nnz) return;
    S.mem.release(S.c);                 // stream-ordered: no synchronisation
    S.mem.release(S.skey);
    S.mem.release(S.sval);
    S.mem.release(S.spos);
    S.mem.release(S.nq);
    S.c = S.mem.alloc<double>(nnz);
    S.skey = S.mem.alloc<int>(nnz);
    S.sval = S.mem.alloc<double>(nnz);
    S.spos = S.mem.alloc<int>(nnz);
    S.nq = S.mem.alloc<int2>(nnz);
    S.cap_nnz = nnz;
}

// X = Y Z with k_spgemm_hash: passes of growing capacity, each taking the
// rows that did not fit the one before. A pass writes its rows, sorted, into
// scratch slots (then the offsets and a copy into place), or, when the slots
// would be too large, counts them and fills them after the offsets. The
// result lives in the scratch arena when `scratch`, else in the hierarchy's.
// A product with at most SPG_DENSE_MAX columns (ncols) takes the dense
// accumulator kernel instead, a block per row, into the same kind of slots.
// AMG_SPGEMM_CAP_SHIFT = k (0..3) divides every hash capacity by 2^k and
// turns the dense path off, so that small test matrices reach every tier.
DevCsr spgemm_hash(amg_hierarchy* h, const DevCsr& Y, const DevCsr& Z, int ncols, Scratch& S, bool scratch) {
    cudaStream_t st = h->stream;
    const int n = Y.n;
    const char* shift_env = std::getenv("AMG_SPGEMM_CAP_SHIFT");
    int* over = S.cnt + 10;
    int* nl = S.cnt + 11;                               // rows listed for tiers 1 .. 4
    int* lists[SPG_TIERS] = {nullptr, S.list0, S.list1, S.qid, S.spos};   // spos: free once the sweeps are done
    CUDA_CHECK(cudaMemsetAsync(S.cnt + 10, 0, 5 * sizeof(int), st));
    int cshift = 0;
    if (shift_env) cshift = std::max(0, std::min(3, std::atoi(shift_env)));
    auto cap = [&](int t) {
        return SPG_UNITS[t] > 1 ? std::max(SPG_CAP[t] >> cshift, SPG_WARP_MIN_CAP) : SPG_CAP[t] >> cshift;
    };
    auto smem = [&](int t) { return (size_t)SPG_UNITS[t] * cap(t) * (sizeof(double) + sizeof(int)); };
    const int smax = (int)smem(SPG_TIERS - 1);
    for (const void* f : {(const void*)k_spgemm_hash<SPG_COUNT, true>, (const void*)k_spgemm_hash<SPG_FILL, true>,
                          (const void*)k_spgemm_hash<SPG_ONE, true>, (const void*)k_spgemm_hash<SPG_COUNT, false>,
                          (const void*)k_spgemm_hash<SPG_FILL, false>, (const void*)k_spgemm_hash<SPG_ONE, false>})
        CUDA_CHECK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
    int rows[SPG_TIERS] = {n, 0, 0, 0, 0};
    const int* first_list = nullptr;                    // rows the warp pass left to the first hash tier
    const int* first_count = nullptr;
    bool one[SPG_TIERS] = {};                           // tier done in one pass (scratch slots)
    int* scol[SPG_TIERS] = {};
    double* sval[SPG_TIERS] = {};
    auto blocks = [&](int t) {
        static constexpr int per_sm[SPG_TIERS] = {16, 8, 9, 2, 2};   // blocks per SM (threads, shared memory)
        const int cp = h->num_sms * per_sm[t];
        return std::max(1, std::min((rows[t] + SPG_UNITS[t] - 1) / SPG_UNITS[t], cp));
    };
    auto launch = [&](int mode, int t, const int* xoff, long long stride, int* xcol, double* xval) {
        const bool last = t == SPG_TIERS - 1;
        int* longs = (mode == SPG_FILL || last) ? nullptr : lists[t + 1];
        int* nlongs = (mode == SPG_FILL || last) ? nullptr : nl + t;
        const int* lst = t ? lists[t] : first_list;
        const int* nls = t ? nl + t - 1 : first_count;
        const dim3 g(blocks(t)), b(SPG_THREADS[t]);
        const size_t sm = smem(t);
#define SPG_ARGS n, lst, nls, cap(t), Y.ptr, Y.col, Y.val, Z.ptr, Z.col, Z.val, S.ub, xoff, stride, xcol, xval, longs, nlongs, over
        if (SPG_UNITS[t] > 1) {                         // a warp per row
            if (mode == SPG_COUNT) k_spgemm_hash<SPG_COUNT, false><<<g, b, sm, st>>>(SPG_ARGS);
            else if (mode == SPG_FILL) k_spgemm_hash<SPG_FILL, false><<<g, b, sm, st>>>(SPG_ARGS);
            else k_spgemm_hash<SPG_ONE, false><<<g, b, sm, st>>>(SPG_ARGS);
        } else {
            if (mode == SPG_COUNT) k_spgemm_hash<SPG_COUNT, true><<<g, b, sm, st>>>(SPG_ARGS);
            else if (mode == SPG_FILL) k_spgemm_hash<SPG_FILL, true><<<g, b, sm, st>>>(SPG_ARGS);
            else k_spgemm_hash<SPG_ONE, true><<<g, b, sm, st>>>(SPG_ARGS);
        }
#undef SPG_ARGS
        KERNEL_CHECK();
    };
    // first tier: one pass into scratch slots of min(terms, capacity) entries
    // when their total fits int32 units, else count now and fill later. Rows
    // whose columns lie in a window of at most dcap columns take the dense
    // kernel (when even its largest slots fit int32 units, and not when the
    // capacities are divided for tests). A product with more columns than
    // the dense kernel holds sends it only rows of SPG_DENSE_MIN_TERMS terms
    // or more.
    one[0] = (long long)n * ((cap(0) / 2 + 7) / 8) <= 0x7fffffffLL;
    const int dcap = shift_env ? 0 : std::min(ncols, SPG_DENSE_MAX);
    const bool dense_on = dcap > 0 && (long long)n * ((dcap + 7) / 8) <= 0x7fffffffLL;
    int* dense_base = nullptr;
    if (one[0]) {
        int* dlist = reinterpret_cast<int*>(S.nq);        // S.nq: free once the sweeps are done
        int* olist = reinterpret_cast<int*>(S.nq) + n;
        dense_base = S.rowbase;
        CUDA_CHECK(cudaMemsetAsync(S.cnt + 24, 0, 3 * sizeof(int), st));   // [24] long, [25] dense, [26] other
        const int dmin = ncols <= SPG_DENSE_MAX ? 0 : SPG_DENSE_MIN_TERMS;
        if (Y.nnz >= 64LL * n)                            // long rows of Y: a warp each
            k_spgemm_classify_warp<<<blocks_for((long long)n * 32, TPB, h->num_sms * 16), TPB, 0, st>>>(
                n, Y.ptr, Y.col, Z.ptr, Z.col, cap(0) / 2, dense_on ? dcap : 0, dmin, S.flag, dense_base, dlist,
                S.cnt + 25, olist, S.cnt + 26);
        else
            k_spgemm_classify<<<grid_for(h, n), TPB, 0, st>>>(n, Y.ptr, Y.col, Z.ptr, Z.col, cap(0) / 2,
                                                              dense_on ? dcap : 0, dmin, S.flag, dense_base, dlist,
                                                              S.cnt + 25, olist, S.cnt + 26);
        KERNEL_CHECK();
        scan_exclusive(S.flag, S.off, n, S.off + n, st, S.scan_tmp);
        const long long units = read_int(S.off + n, S.host, st);
        scol[0] = S.mem.alloc<int>(units * 8 + 1);
        sval[0] = S.mem.alloc<double>(units * 8 + 1);
        if (dense_on) {
            const int smd = spg_dense_smem(dcap);
            CUDA_CHECK(cudaFuncSetAttribute(k_spgemm_dense, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            spg_dense_smem(SPG_DENSE_MAX)));
            const int per_sm = std::max(1, std::min(8, (220 * 1024) / smd));
            k_spgemm_dense<<<h->num_sms * per_sm, SPG_DENSE_THREADS, smd, st>>>(
                dlist, S.cnt + 25, dense_base, dcap, Y.ptr, Y.col, Y.val, Z.ptr, Z.col, Z.val, S.ub, S.off, scol[0],
                sval[0]);
            KERNEL_CHECK();
        }
        // the other rows: at most 32 terms by the warp pass, the rest (listed
        // in S.heads, counted in S.cnt[24]) by the first hash tier
        k_spgemm_warp<<<blocks_for((long long)n * 32, TPB, h->num_sms * 16), TPB, 0, st>>>(
            olist, S.cnt + 26, Y.ptr, Y.col, Y.val, Z.ptr, Z.col, Z.val, S.ub, S.off, scol[0], sval[0], S.heads,
            S.cnt + 24);
        KERNEL_CHECK();
        first_list = S.heads;
        first_count = S.cnt + 24;
        launch(SPG_ONE, 0, S.off, 8, scol[0], sval[0]);
    } else {
        launch(SPG_COUNT, 0, nullptr, 0, nullptr, nullptr);
    }
    // larger tiers on the listed rows: one pass when the slots stay below 2^28 entries
    for (int t = 1; t < SPG_TIERS; ++t) {
        rows[t] = read_int(nl + t - 1, S.host, st);
        if (rows[t] == 0) break;
        const long long slots = (long long)rows[t] * (cap(t) / 2);
        one[t] = slots <= (1LL << 28);
        if (one[t]) {
            scol[t] = S.mem.alloc<int>(slots);
            sval[t] = S.mem.alloc<double>(slots);
            launch(SPG_ONE, t, nullptr, cap(t) / 2, scol[t], sval[t]);
        } else {
            launch(SPG_COUNT, t, nullptr, 0, nullptr, nullptr);
        }
    }
    if (read_int(over, S.host, st))
        AMG_THROW(AMG_ERR_TOO_LARGE, "a row of a sparse product has more than %d entries",
                  cap(SPG_TIERS - 1) / 2);
    DevCsr X;
    X.n = n;
    X.ptr = scratch ? S.mem.alloc<int>(n + 1) : h->mem.alloc<int>(n + 1);
    scan_exclusive(S.ub, X.ptr, n, X.ptr + n, st, S.scan_tmp);
    finish_csr(h, S, X);
    X.col = scratch ? S.mem.alloc<int>(X.nnz) : h->mem.alloc<int>(X.nnz);
    X.val = scratch ? S.mem.alloc<double>(X.nnz) : h->mem.alloc<double>(X.nnz);
    for (int t = 0; t < SPG_TIERS && rows[t] > 0; ++t) {
        if (!one[t]) {
            launch(SPG_FILL, t, X.ptr, 0, X.col, X.val);
            continue;
        }
        const int* lst = lists[t];
        const int* nls = t ? nl + t - 1 : nullptr;
        k_spgemm_copy<<<blocks_for((long long)rows[t] * 32, TPB, h->num_sms * 16), TPB, 0, st>>>(
            n, lst, nls, cap(t) / 2, t ? nullptr : dense_base, S.ub, t ? nullptr : S.off, t ? cap(t) / 2 : 8,
            scol[t], sval[t], X.ptr, X.col, X.val);
        KERNEL_CHECK();
    }
    for (int t = 0; t < SPG_TIERS; ++t)
        if (scol[t]) {
            S.mem.release(scol[t]);
            S.mem.release(sval[t]);
        }
    return X;
}

// Smoothed prolongator of level L (aggregates agg/p to nc coarse rows) and
// the coarse matrix Pbar^T A Pbar (Section 3.2), the oracle's operation
// order throughout: omega = 4 / (3 eta) (omega_rule 0) or 1 / eta (omega_rule
// 1, the text's weight) from eta = max_i sum_j |a_ij| / a_ii, Pbar rows from
// the rows of A P, the transpose with ascending rows, then the product.
DevCsr smooth_level(amg_hierarchy* h, Level& L, int nc, Scratch& S) {
    cudaStream_t st = h->stream;
    const DevCsr& A = L.A;
    const int n = A.n;
    unsigned long long* eta_bits = S.mem.alloc<unsigned long long>(1);
    CUDA_CHECK(cudaMemsetAsync(eta_bits, 0, sizeof(unsigned long long), st));
    k_eta_max<<<grid_for(h, n), TPB, 0, st>>>(n, A.ptr, A.col, A.val, eta_bits);
    KERNEL_CHECK();
    unsigned long long eb = 0;
    CUDA_CHECK(cudaMemcpyAsync(&eb, eta_bits, sizeof(eb), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    S.mem.release(eta_bits);
    double eta;
    std::memcpy(&eta, &eb, sizeof(eta));
    const double omega = h->opt.omega_rule == 1 ? 1.0 / eta : 4.0 / (3.0 * eta);
    L.omega_p = omega;

    // rows of A P (canonical), compacted, then turned into rows of Pbar
    CUDA_CHECK(cudaMemsetAsync(S.cnt + 8, 0, sizeof(int), st));
    const int G = rows_group(A.nnz, n);
    launch_rows<false>(h, G, n, nullptr, nullptr, A.ptr, A.col, A.val, L.agg, L.p, A.ptr, S.skey, S.sval, S.ub,
                       S.list1, S.cnt + 8, nullptr, st);
    if (A.max_row == 0 || A.max_row > G)
        launch_rows_long<false>(h, S, n, S.list1, S.cnt + 8, nullptr, nullptr, A.ptr, A.col, A.val, L.agg, L.p,
                                A.ptr, S.ub, nullptr, st, G, A.max_row);
    DevCsr& P = L.pbar;
    P.n = n;
    P.ptr = h->mem.alloc<int>(n + 1);
    scan_exclusive(S.ub, P.ptr, n, P.ptr + n, st, S.scan_tmp);
    P.nnz = read_int(P.ptr + n, S.host, st);
    P.col = h->mem.alloc<int>(P.nnz);
    P.val = h->mem.alloc<double>(P.nnz);
    launch_copy(h, P.nnz, n, A.ptr, P.ptr, S.skey, S.sval, P.col, P.val, st);
    k_pbar_from_ap<<<grid_for(h, n), TPB, 0, st>>>(n, P.ptr, P.col, P.val, A.ptr, A.col, A.val, L.agg, L.p, omega);
    KERNEL_CHECK();

    // transpose, rows ascending in every column
    DevCsr& T = L.pbar_t;
    T.n = nc;
    T.nnz = P.nnz;
    T.ptr = h->mem.alloc<int>(nc + 1);
    T.col = h->mem.alloc<int>(P.nnz);
    T.val = h->mem.alloc<double>(P.nnz);
    CUDA_CHECK(cudaMemsetAsync(S.ub, 0, sizeof(int) * (nc + 1), st));
    k_col_count<<<grid_for(h, n), TPB, 0, st>>>(n, P.ptr, P.col, S.ub);
    KERNEL_CHECK();
    scan_exclusive(S.ub, T.ptr, nc, T.ptr + nc, st, S.scan_tmp);
    CUDA_CHECK(cudaMemsetAsync(S.ub, 0, sizeof(int) * (nc + 1), st));
    k_col_fill<<<grid_for(h, n), TPB, 0, st>>>(n, P.ptr, P.col, P.val, T.ptr, S.ub, T.col, T.val);
    KERNEL_CHECK();
    {
        // rows of up to 32 pairs: a warp each in registers; up to 2048: a warp
        // each in shared memory; longer rows: a block each
        constexpr int WCAP = 2048, WPB = 4, BCAP = 16384;
        const size_t sm_w = (size_t)WPB * WCAP * (sizeof(double) + sizeof(int));
        const size_t sm_b = (size_t)BCAP * (sizeof(double) + sizeof(int));
        CUDA_CHECK(cudaFuncSetAttribute(k_sort_pairs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_w));
        CUDA_CHECK(cudaFuncSetAttribute(k_sort_pairs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_b));
        int* over = S.cnt + 10;
        int* nl = S.cnt + 11;
        int* nm = S.cnt + 12;
        CUDA_CHECK(cudaMemsetAsync(S.cnt + 10, 0, 3 * sizeof(int), st));
        k_sort_pairs_warp<<<blocks_for((long long)nc * 32, TPB, h->num_sms * 16), TPB, 0, st>>>(nc, T.ptr, T.col,
                                                                                              T.val, S.list1, nm);
        KERNEL_CHECK();
        k_sort_pairs<false><<<blocks_for((long long)nc * 32, WPB * 32, h->num_sms * 8), WPB * 32, sm_w, st>>>(
            nc, S.list1, nm, WCAP, T.ptr, T.col, T.val, S.list0, nl, over);
        KERNEL_CHECK();
        const int nlong = read_int(nl, S.host, st);
        if (nlong > 0) {
            k_sort_pairs<true><<<std::min(nlong, h->num_sms), 1024, sm_b, st>>>(nc, S.list0, nl, BCAP, T.ptr, T.col,
                                                                               T.val, nullptr, nullptr, over);
            KERNEL_CHECK();
        }
        if (read_int(over, S.host, st))
            AMG_THROW(AMG_ERR_TOO_LARGE, "a column of Pbar has more than %d entries", BCAP);
    }

    // C = Pbar^T (A Pbar): two sparse products in the oracle's order
    DevCsr W = spgemm_hash(h, A, P, nc, S, true);
    DevCsr C = spgemm_hash(h, T, W, nc, S, false);
    S.mem.release(W.val);
    S.mem.release(W.col);
    S.mem.release(W.ptr);
    CUDA_CHECK(cudaStreamSynchronize(st));
    return C;
}

}  // namespace

void setup_hierarchy(amg_hierarchy* h, const amg_csr* Ain, const double* w_in) {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = h->stream;
    const amg_options& o = h->opt;
    const int n0 = Ain->n, nnz0 = Ain->nnz;

    Scratch S;
    S.mem.stream = h->stream;
    CUDA_CHECK(cudaHostAlloc(&S.host, 64, cudaHostAllocDefault));
    {
        int coop = 0, per_sm = 0;
        CUDA_CHECK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
        CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ld_persistent, 1024, 0));
        h->coop_blocks = (coop && per_sm >= 1) ? h->num_sms : 0;
    }
    S.diag = S.mem.alloc<double>(n0);
    S.c = S.mem.alloc<double>(nnz0);
    S.mate = S.mem.alloc<int>(n0);
    S.cand = S.mem.alloc<int>(n0);
    S.list0 = S.mem.alloc<int>(n0);
    S.list1 = S.mem.alloc<int>(n0);
    S.mlist = S.mem.alloc<int>(n0);
    S.cnt = S.mem.alloc<int>(64);
    S.flag = S.mem.alloc<int>(n0 + 1);
    S.qid = S.mem.alloc<int>(n0 + 1);
    S.heads = S.mem.alloc<int>(n0 + 1);
    S.ub = S.mem.alloc<int>(n0 + 2);
    S.off = S.mem.alloc<int>(n0 + 2);
    S.skey = S.mem.alloc<int>(nnz0);
    S.sval = S.mem.alloc<double>(nnz0);
    S.spos = S.mem.alloc<int>(nnz0);
    S.nq = S.mem.alloc<int2>(nnz0);
    S.rowbase = S.mem.alloc<int>(n0 + 1);
    S.suitor = S.mem.alloc<unsigned long long>(n0);
    S.cap_nnz = nnz0;
    S.scan_tmp = S.mem.alloc<int>(scan_scratch_ints(n0 + 2) + 64);

    // ---- level 0: private copy of A and w, validated
    h->lev.clear();
    h->lev.emplace_back();
    {
        Level& L0 = h->lev[0];
        L0.A.n = n0;
        L0.A.nnz = nnz0;
        L0.A.ptr = h->mem.alloc<int>(n0 + 1);
        L0.A.col = h->mem.alloc<int>(nnz0);
        L0.A.val = h->mem.alloc<double>(nnz0);
        L0.w = h->mem.alloc<double>(n0);
        CUDA_CHECK(cudaMemcpyAsync(L0.A.ptr, Ain->row_ptr, sizeof(int) * (n0 + 1), cudaMemcpyDefault, st));
        CUDA_CHECK(cudaMemcpyAsync(L0.A.col, Ain->col, sizeof(int) * (size_t)nnz0, cudaMemcpyDefault, st));
        CUDA_CHECK(cudaMemcpyAsync(L0.A.val, Ain->val, sizeof(double) * (size_t)nnz0, cudaMemcpyDefault, st));
        CUDA_CHECK(cudaMemcpyAsync(L0.w, w_in, sizeof(double) * n0, cudaMemcpyDefault, st));
        Scope sc_(&h->prof, st, S_VALIDATE, 16.0 * nnz0 + 16.0 * n0);
        CUDA_CHECK(cudaMemsetAsync(S.cnt + 5, 0, sizeof(int), st));
        k_check_ptr<<<grid_for(h, n0 + 1), TPB, 0, st>>>(n0, nnz0, L0.A.ptr, S.cnt + 5);
        KERNEL_CHECK();
        int f = read_int(S.cnt + 5, S.host, st);
        if (f & F_SHAPE) AMG_THROW(AMG_ERR_ARG, "row_ptr is not a valid CSR row pointer");
        k_check_rows<<<grid_for(h, n0), TPB, 0, st>>>(n0, L0.A.ptr, L0.A.col, L0.A.val, L0.w, S.diag, S.cnt + 5);
        KERNEL_CHECK();
        // the flags and the longest row, one synchronisation
        CUDA_CHECK(cudaMemsetAsync(S.cnt + 19, 0, sizeof(int), st));
        if (n0 > 0) {
            k_max_row<<<grid_for(h, n0), TPB, 0, st>>>(n0, L0.A.ptr, S.cnt + 19);
            KERNEL_CHECK();
        }
        CUDA_CHECK(cudaMemcpyAsync(S.host, S.cnt + 5, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_CHECK(cudaMemcpyAsync(S.host + 1, S.cnt + 19, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_CHECK(cudaStreamSynchronize(st));
        f = S.host[0];
        L0.A.max_row = S.host[1];
        if (f & F_SHAPE) AMG_THROW(AMG_ERR_ARG, "CSR columns unsorted, out of range, or pattern not symmetric");
        if (f & F_NOT_SPD) AMG_THROW(AMG_ERR_NOT_SPD, "non-finite value or diagonal entry missing or <= 0");
        if (f & F_BAD_W) AMG_THROW(AMG_ERR_BAD_W, "smooth vector w has a zero or non-finite entry");
    }

    // ---- batch of systems: level-0 offsets on the device
    const int nseg = h->seg0.size() > 1 ? (int)h->seg0.size() - 1 : 0;
    int* seg_dev = nullptr;
    int* seg_next = nullptr;
    h->segs.clear();
    if (nseg) {
        if (h->seg0.front() != 0 || h->seg0.back() != n0) AMG_THROW(AMG_ERR_ARG, "system offsets do not cover A");
        seg_dev = S.mem.alloc<int>(nseg + 1);
        seg_next = S.mem.alloc<int>(nseg + 1);
        CUDA_CHECK(cudaMemcpyAsync(seg_dev, h->seg0.data(), sizeof(int) * (nseg + 1), cudaMemcpyHostToDevice, st));
        h->segs.push_back(h->seg0);
        h->seg_row0 = h->mem.alloc<int>(n0);
        k_seg_rows<<<nseg, TPB, 0, st>>>(nseg, seg_dev, h->seg_row0);
        KERNEL_CHECK();
    }
    auto largest_system = [&](int l) {
        int mx = 0;
        for (int s2 = 0; s2 < nseg; ++s2) mx = std::max(mx, h->segs[l][s2 + 1] - h->segs[l][s2]);
        return mx;
    };

    // ---- level loop (Section 3.2 coarsening, Section 5 stop rule; for a
    // batch of systems the rule applies to the largest system)
    for (;;) {
        const int l = (int)h->lev.size() - 1;
        const int size_rule = nseg ? largest_system(l) : h->lev[l].A.n;
        if (size_rule <= o.max_coarse || l + 1 >= o.max_levels || l + 1 >= AMG_MAX_LEVELS) break;
        const int nl = h->lev[l].A.n;
        DevCsr A = h->lev[l].A;
        ensure_entry_scratch(S, A.nnz, st);
        double* w = h->lev[l].w;
        int* agg_l = h->mem.alloc<int>(nl);
        double* p_l = h->mem.alloc<double>(nl);
        std::vector<SweepRecord> recs;
        int sweeps_done = 0;
        int rounds[AMG_MAX_SWEEPS] = {0};
        for (int s = 0; s < o.sweeps && s < AMG_MAX_SWEEPS; ++s) {
            const int n = A.n;
            {
                Scope sc_(&h->prof, st, S_WEIGHTS, 20.0 * A.nnz + 24.0 * n);
                // S.diag: (a_ii w_i) w_i of the current A. Level 0 starts from the
                // diagonal the validation wrote; after a pairwise sweep the
                // Galerkin copy has written it; a level's first sweep recomputes
                // it (the level's matrix may come from the smoothed product).
                if (s == 0 && l == 0) k_dww<<<grid_for(h, n), TPB, 0, st>>>(n, S.diag, w);
                else if (s == 0) k_diag<<<grid_for(h, n), TPB, 0, st>>>(n, A.ptr, A.col, A.val, w, S.diag);
                KERNEL_CHECK();
                launch_weights(weights_group(A.nnz, n), h->num_sms * 16, st, n, A.ptr, A.col, A.val, S.diag, w,
                               S.c);
            }
            int* pending = nullptr;
            const int rr = ld_match(h, S, A, &pending);
            int nc = 0;
            {
                // head flags and their scan only compare mate values, so they
                // may run before the matching's error word is checked
                Scope sc_(&h->prof, st, S_AGGREGATE, 0.0);
                k_head_flags<<<grid_for(h, n), TPB, 0, st>>>(n, S.mate, S.flag);
                KERNEL_CHECK();
                scan_exclusive(S.flag, S.qid, n, S.cnt + 6, st, S.scan_tmp);
                if (pending) {
                    CUDA_CHECK(cudaMemcpyAsync(S.host, S.cnt + 6, sizeof(int), cudaMemcpyDeviceToHost, st));
                    CUDA_CHECK(cudaMemcpyAsync(S.host + 1, pending, sizeof(int), cudaMemcpyDeviceToHost, st));
                    CUDA_CHECK(cudaStreamSynchronize(st));
                    check_suitor_error(S.host[1]);
                    nc = S.host[0];
                } else {
                    nc = read_int(S.cnt + 6, S.host, st);
                }
            }
            if (nc == n) break;                                   // nothing matched: end the level
            if (nseg) {
                k_seg_map<<<1, TPB, 0, st>>>(nseg, seg_dev, S.qid, n, nc, seg_next);
                KERNEL_CHECK();
                std::swap(seg_dev, seg_next);
            }
            SweepOut sw;
            sw.nc = nc;
            sw.agg = h->mem.alloc<int>(n);
            sw.p = h->mem.alloc<double>(n);
            sw.wc = h->mem.alloc<double>(nc);
            int* mate_keep = o.keep_sweeps ? h->mem.alloc<int>(n) : nullptr;
            {
                Scope sc_(&h->prof, st, S_AGGREGATE, 0.0);
                k_heads<<<grid_for(h, n), TPB, 0, st>>>(n, S.mate, S.qid, S.heads, mate_keep);
                KERNEL_CHECK();
                k_aggregate<<<grid_for(h, nc), TPB, 0, st>>>(nc, S.heads, S.mate, w, sw.agg, sw.p, sw.wc);
                KERNEL_CHECK();
            }
            DevCsr C;
            {
                Scope sc_(&h->prof, st, S_GALERKIN, 12.0 * A.nnz + 12.0 * n);
                C = galerkin_pairwise(h, S, A, sw, h->mem);
            }
            Scope sc_compose(&h->prof, st, S_COMPOSE, 24.0 * nl);
            if (s == 0) {
                CUDA_CHECK(cudaMemcpyAsync(agg_l, sw.agg, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
                CUDA_CHECK(cudaMemcpyAsync(p_l, sw.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            } else {
                k_compose<<<grid_for(h, nl), TPB, 0, st>>>(nl, agg_l, p_l, sw.agg, sw.p);
                KERNEL_CHECK();
            }
            rounds[s] = rr;
            if (o.keep_sweeps) {
                SweepRecord R;
                R.n = n; R.nc = nc; R.nnz_c = C.nnz; R.rounds = rr;
                R.mate = mate_keep; R.agg = sw.agg; R.p = sw.p; R.wc = sw.wc;
                recs.push_back(R);
            } else {
                h->mem.release(sw.agg);                   // stream-ordered frees: no synchronisation
                h->mem.release(sw.p);
            }
            // the previous intermediate matrix and smooth vector are no longer needed
            if (A.ptr != h->lev[l].A.ptr) {
                h->mem.release(A.ptr); h->mem.release(A.col); h->mem.release(A.val);
                if (!o.keep_sweeps) h->mem.release(w);
            }
            A = C;
            w = sw.wc;
            ++sweeps_done;
        }
        if (sweeps_done == 0 || A.n == nl) {          // no reduction: level l is the coarsest
            h->mem.release(agg_l);
            h->mem.release(p_l);
            break;
        }
        if (nseg) {
            std::vector<int> sp(nseg + 1);
            CUDA_CHECK(cudaMemcpyAsync(sp.data(), seg_dev, sizeof(int) * (nseg + 1), cudaMemcpyDeviceToHost, st));
            CUDA_CHECK(cudaStreamSynchronize(st));
            h->segs.push_back(sp);
        }
        Level& cur = h->lev[l];
        cur.agg = agg_l;
        cur.p = p_l;
        cur.sweeps_done = sweeps_done;
        for (int s = 0; s < AMG_MAX_SWEEPS; ++s) cur.rounds[s] = rounds[s];
        cur.sweeps = std::move(recs);
        if (o.smooth_p) {
            // the next level matrix is Pbar^T A Pbar; the last pairwise matrix goes
            DevCsr C;
            {
                Scope sc_(&h->prof, st, S_SMOOTH_P, 0.0);
                C = smooth_level(h, cur, A.n, S);
            }
            if (A.ptr != cur.A.ptr) {
                h->mem.release(A.ptr);
                h->mem.release(A.col);
                h->mem.release(A.val);
            }
            A = C;
        }
        Level next;
        next.A = A;
        next.w = w;
        h->lev.push_back(std::move(next));
        if ((double)nl / (double)A.n < o.min_ratio) break;   // coarsening has stalled: stop here
    }

    // ---- per-level solve data: smoother, SELL copies, member lists
    const bool fp32 = o.precision == AMG_FP32_VCYCLE;
    const int nlev = (int)h->lev.size();
    for (int l = 0; l < nlev; ++l) {
        Level& L = h->lev[l];
        const int n = L.A.n;
        L.minv = h->mem.alloc<double>(n);
        if (fp32) L.minv32 = h->mem.alloc<float>(n);
        {
            Scope sc_(&h->prof, st, S_SMOOTHER, 12.0 * L.A.nnz + 12.0 * n);
            k_l1_jacobi<<<grid_for(h, n), TPB, 0, st>>>(n, L.A.ptr, L.A.col, L.A.val, L.minv, L.minv32);
            KERNEL_CHECK();
            if (o.omega == 1.0) {
                L.wminv = L.minv;
                L.wminv32 = L.minv32;
            } else {
                L.wminv = h->mem.alloc<double>(n);
                if (fp32) L.wminv32 = h->mem.alloc<float>(n);
                k_scale_vec<<<grid_for(h, n), TPB, 0, st>>>(n, o.omega, L.minv, L.wminv, L.wminv32);
                KERNEL_CHECK();
            }
        }
        Scope sc_(&h->prof, st, S_FORMAT, 24.0 * L.A.nnz);
        const bool coarsest_cg = l == nlev - 1 && L.A.n > o.max_dense;
        if (coarsest_cg && l > 0) build_sell_hybrid(h, L.A, L.S, S, 32);
        else if (l == 0 || l < nlev - 1 || coarsest_cg) build_sell(h, L.A, L.S, S, fp32);
        if (l == nlev - 1) break;
        build_scaled(h, L, fp32);
        if (o.smooth_p) {
            build_sell(h, L.pbar, L.PB, S, fp32);
            build_sell(h, L.pbar_t, L.PBT, S, fp32);
        } else {
            build_members(h, L, h->lev[l + 1].A.n, S);
            build_ap(h, L, h->lev[l + 1].A.n, S, fp32);
        }
        if (fp32) {
            L.p32 = h->mem.alloc<float>(n);
            k_to_float<<<grid_for(h, n), TPB, 0, st>>>(n, L.p, L.p32);
            KERNEL_CHECK();
        }
    }

    // ---- coarsest level: dense Cholesky and explicit inverse (per system
    // for a batch of systems: the coarsest matrix is block diagonal)
    {
        Level& Lc = h->lev.back();
        const int nc = Lc.A.n;
        h->nc = nc;
        h->coarse_cg = (!nseg && nc > o.max_dense) ? 1 : 0;
    }
    if (nseg) {
        Level& Lc = h->lev.back();
        const std::vector<int>& sp = h->segs.back();
        std::vector<long long> boff(nseg + 1, 0);
        for (int s2 = 0; s2 < nseg; ++s2) {
            const long long ns = sp[s2 + 1] - sp[s2];
            if (ns > o.max_dense) AMG_THROW(AMG_ERR_TOO_LARGE, "coarsest block of system %d has %lld rows", s2, ns);
            boff[s2 + 1] = boff[s2] + ns * ns;
        }
        Scope sc_(&h->prof, st, S_COARSE, 0.0);
        h->coarse_inv = h->mem.alloc<double>(boff[nseg] > 0 ? boff[nseg] : 1);
        h->coarse_L = nullptr;
        h->segL_ptr = h->mem.alloc<int>(nseg + 1);
        h->segL_blk = h->mem.alloc<long long>(nseg + 1);
        CUDA_CHECK(cudaMemcpyAsync(h->segL_ptr, sp.data(), sizeof(int) * (nseg + 1), cudaMemcpyHostToDevice, st));
        CUDA_CHECK(cudaMemcpyAsync(h->segL_blk, boff.data(), sizeof(long long) * (nseg + 1), cudaMemcpyHostToDevice, st));
        // one CTA per block in a single launch (blocks above SM_DENSE rows work in
        // global scratch); with a block above CTA_DENSE rows, or scratch above
        // 1 GiB, the blocks are factored one after another by the multi-block
        // kernels instead
        int maxb = 0, maxsm = 0;
        std::vector<long long> gofs(nseg, 0);
        long long gw = 0;
        for (int s2 = 0; s2 < nseg; ++s2) {
            const int ns = sp[s2 + 1] - sp[s2];
            maxb = std::max(maxb, ns);
            if (ns <= SM_DENSE) maxsm = std::max(maxsm, ns);
            else { gofs[s2] = gw; gw += 2LL * ns * ns + ns; }
        }
        CUDA_CHECK(cudaMemsetAsync(S.cnt + 5, 0, sizeof(int), st));
        if (maxb <= CTA_DENSE && gw <= (1LL << 27)) {
            double* gwork = S.mem.alloc<double>(gw + 1);
            long long* d_gofs = S.mem.alloc<long long>(nseg);
            CUDA_CHECK(cudaMemcpyAsync(d_gofs, gofs.data(), sizeof(long long) * nseg, cudaMemcpyHostToDevice, st));
            const int smd = (int)(2 * sizeof(double) * (size_t)maxsm * maxsm);
            CUDA_CHECK(cudaFuncSetAttribute(k_coarse_inverse_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(2 * sizeof(double) * SM_DENSE * SM_DENSE)));
            k_coarse_inverse_blocks<<<nseg, 1024, smd, st>>>(0, h->segL_ptr, h->segL_blk, d_gofs, Lc.A.ptr,
                                                             Lc.A.col, Lc.A.val, gwork, h->coarse_inv, nullptr,
                                                             S.cnt + 5);
            KERNEL_CHECK();
        } else {
            double* D = S.mem.alloc<double>((size_t)maxb * maxb + 1);
            double* Lf = S.mem.alloc<double>((size_t)maxb * maxb + 1);
            double* Y = S.mem.alloc<double>((size_t)maxb * maxb + 1);
            for (int s2 = 0; s2 < nseg; ++s2) {
                const int ns = sp[s2 + 1] - sp[s2];
                if (ns == 0) continue;
                CUDA_CHECK(cudaMemsetAsync(D, 0, sizeof(double) * ns * ns, st));
                CUDA_CHECK(cudaMemsetAsync(Lf, 0, sizeof(double) * ns * ns, st));
                k_dense_lower_block<<<grid_for(h, ns), TPB, 0, st>>>(ns, sp[s2], Lc.A.ptr, Lc.A.col, Lc.A.val, D);
                KERNEL_CHECK();
                k_cholesky<<<1, 1024, 0, st>>>(ns, D, Lf, S.cnt + 5);
                KERNEL_CHECK();
                k_lower_inverse<<<(ns + 127) / 128, 128, 0, st>>>(ns, Lf, Y);
                KERNEL_CHECK();
                k_gram<<<(int)(((long long)ns * ns + 255) / 256), 256, 0, st>>>(ns, Y, h->coarse_inv + boff[s2]);
                KERNEL_CHECK();
            }
        }
        if (read_int(S.cnt + 5, S.host, st)) AMG_THROW(AMG_ERR_NOT_SPD, "a coarsest block hit a non-positive pivot");
    }
    if (!h->coarse_cg && !nseg) {
        Level& Lc = h->lev.back();
        const int nc = Lc.A.n;
        Scope sc_(&h->prof, st, S_COARSE, 0.0);
        h->coarse_L = h->mem.alloc<double>((size_t)nc * nc);
        h->coarse_inv = h->mem.alloc<double>((size_t)nc * nc);
        CUDA_CHECK(cudaMemsetAsync(S.cnt + 5, 0, sizeof(int), st));
        if (nc <= CTA_DENSE) {                            // one CTA: shared memory up to SM_DENSE rows
            const int smd = nc <= SM_DENSE ? (int)(2 * sizeof(double) * (size_t)nc * nc) : 0;
            double* gwork = nc <= SM_DENSE ? nullptr : S.mem.alloc<double>(2 * (size_t)nc * nc + nc);
            long long* gofs = S.mem.alloc<long long>(1);
            CUDA_CHECK(cudaMemsetAsync(gofs, 0, sizeof(long long), st));
            CUDA_CHECK(cudaFuncSetAttribute(k_coarse_inverse_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(2 * sizeof(double) * SM_DENSE * SM_DENSE)));
            k_coarse_inverse_blocks<<<1, 1024, smd, st>>>(nc, nullptr, nullptr, gofs, Lc.A.ptr, Lc.A.col,
                                                          Lc.A.val, gwork, h->coarse_inv, h->coarse_L, S.cnt + 5);
            KERNEL_CHECK();
            if (read_int(S.cnt + 5, S.host, st))
                AMG_THROW(AMG_ERR_NOT_SPD, "coarsest-level Cholesky hit a non-positive pivot");
        } else {
            double* D = S.mem.alloc<double>((size_t)nc * nc);
            double* Y = S.mem.alloc<double>((size_t)nc * nc);
            CUDA_CHECK(cudaMemsetAsync(D, 0, sizeof(double) * nc * nc, st));
            CUDA_CHECK(cudaMemsetAsync(h->coarse_L, 0, sizeof(double) * nc * nc, st));
            k_dense_lower<<<grid_for(h, nc), TPB, 0, st>>>(nc, Lc.A.ptr, Lc.A.col, Lc.A.val, D);
            KERNEL_CHECK();
            k_cholesky<<<1, 1024, 0, st>>>(nc, D, h->coarse_L, S.cnt + 5);
            KERNEL_CHECK();
            if (read_int(S.cnt + 5, S.host, st))
                AMG_THROW(AMG_ERR_NOT_SPD, "coarsest-level Cholesky hit a non-positive pivot");
            k_lower_inverse<<<(nc + 127) / 128, 128, 0, st>>>(nc, h->coarse_L, Y);
            KERNEL_CHECK();
            k_gram<<<(int)(((long long)nc * nc + 255) / 256), 256, 0, st>>>(nc, Y, h->coarse_inv);
            KERNEL_CHECK();
        }
    }
    CUDA_CHECK(cudaStreamSynchronize(st));
    h->prof.flush();
    h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}


// ---------------------------------------------------------------------------
// Matching without any allocation (amg_match_noalloc).
//
// Some callers cannot call cudaMalloc at the point where they need a
// matching: applications that reserve all device memory at start-up and hand
// it out from their own pool or budget, and latency-bound hosts that forbid
// allocation after start-up (cudaMalloc and cudaFree can synchronise the
// device). For them this entry point computes the same edge weights and
// locally-dominant matching as the first sweep of amg_setup using only a fixed
// scratch area that is part of the library image (a file-scope __device__
// array, resident on every GPU that loads the library until the process
// exits). The caller passes A, w and the output array.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t NA_ALIGN = 256;
constexpr size_t na_round(size_t b) { return (b + NA_ALIGN - 1) / NA_ALIGN * NA_ALIGN; }
constexpr size_t NA_DIAG = 0;
constexpr size_t NA_C = NA_DIAG + na_round(sizeof(double) * AMG_NOALLOC_MAX_N);
constexpr size_t NA_CAND = NA_C + na_round(sizeof(double) * (size_t)AMG_NOALLOC_MAX_NNZ);
constexpr size_t NA_L0 = NA_CAND + na_round(sizeof(int) * AMG_NOALLOC_MAX_N);
constexpr size_t NA_L1 = NA_L0 + na_round(sizeof(int) * AMG_NOALLOC_MAX_N);
constexpr size_t NA_M = NA_L1 + na_round(sizeof(int) * AMG_NOALLOC_MAX_N);
constexpr size_t NA_CNT = NA_M + na_round(sizeof(int) * AMG_NOALLOC_MAX_N);
constexpr size_t NA_BYTES = NA_CNT + na_round(sizeof(int) * 16);

static __device__ __align__(256) unsigned char g_match_scratch[NA_BYTES];

std::mutex g_na_mu;
unsigned char* g_na_ptr[256] = {};   // device address of g_match_scratch, per device ordinal

// Device address of the scratch array for the current device. Looked up once
// per device with that device current (the host-side symbol is only a
// stand-in and must never be handed to a kernel).
unsigned char* noalloc_scratch(int dev) {
    std::lock_guard<std::mutex> g(g_na_mu);
    if (dev < 0 || dev >= 256) AMG_THROW(AMG_ERR_ARG, "device ordinal %d out of range", dev);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        CUDA_CHECK(cudaGetSymbolAddress(&p, g_match_scratch));
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    return g_na_ptr[dev];
}

__global__ void k_mate_normalize(int n, int* mate) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (mate[i] < 0) mate[i] = -1;
}

int noalloc_read_int(const int* dev, cudaStream_t st) {
    int v = 0;
    CUDA_CHECK(cudaMemcpyAsync(&v, dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    return v;
}

}  // namespace

amg_status match_noalloc(const amg_csr* A, const double* w, int32_t* mate, void* stream, int32_t* rounds_out) {
    const int n = A->n, nnz = A->nnz;
    if (n > AMG_NOALLOC_MAX_N || nnz > AMG_NOALLOC_MAX_NNZ)
        AMG_THROW(AMG_ERR_TOO_LARGE, "amg_match_noalloc: n = %d, nnz = %d exceed the fixed scratch limits (%d, %d)", n,
                  nnz, AMG_NOALLOC_MAX_N, AMG_NOALLOC_MAX_NNZ);
    int dev = 0, sms = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    unsigned char* base = noalloc_scratch(dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* diag = reinterpret_cast<double*>(base + NA_DIAG);
    double* c = reinterpret_cast<double*>(base + NA_C);
    int* cand = reinterpret_cast<int*>(base + NA_CAND);
    int* lists[2] = {reinterpret_cast<int*>(base + NA_L0), reinterpret_cast<int*>(base + NA_L1)};
    int* mlist = reinterpret_cast<int*>(base + NA_M);
    int* cnt = reinterpret_cast<int*>(base + NA_CNT);   // [0,1] lists, [2,3] matches, [4] rounds, [5] flags
    const int grid = blocks_for(n, TPB, sms * 16);
    const int* ptr = A->row_ptr;
    const int* col = A->col;
    const double* val = A->val;

    // every counter starts at zero on every call (the array keeps the last call's contents)
    CUDA_CHECK(cudaMemsetAsync(cnt, 0, sizeof(int) * 16, st));
    k_check_ptr<<<blocks_for(n + 1, TPB, sms * 16), TPB, 0, st>>>(n, nnz, ptr, cnt + 5);
    KERNEL_CHECK();
    int f = noalloc_read_int(cnt + 5, st);
    if (f & F_SHAPE) AMG_THROW(AMG_ERR_ARG, "row_ptr is not a valid CSR row pointer");
    k_check_rows<<<grid, TPB, 0, st>>>(n, ptr, col, val, w, diag, cnt + 5);
    KERNEL_CHECK();
    f = noalloc_read_int(cnt + 5, st);
    if (f & F_SHAPE) AMG_THROW(AMG_ERR_ARG, "CSR columns unsorted, out of range, or pattern not symmetric");
    if (f & F_NOT_SPD) AMG_THROW(AMG_ERR_NOT_SPD, "non-finite value or diagonal entry missing or <= 0");
    if (f & F_BAD_W) AMG_THROW(AMG_ERR_BAD_W, "smooth vector w has a zero or non-finite entry");

    k_dww<<<grid, TPB, 0, st>>>(n, diag, w);
    KERNEL_CHECK();
    launch_weights(weights_group(nnz, n), sms * 16, st, n, ptr, col, val, diag, w, c);
    CUDA_CHECK(cudaMemsetAsync(mate, 0xff, sizeof(int) * n, st));
    k_ld_init<<<grid, TPB, 0, st>>>(n, ptr, col, c, cand, mate);
    KERNEL_CHECK();
    const int rgrid = sms * 8;
    const long long max_rounds = (long long)n + 4;
    long long r = 0;
    for (;;) {
        for (int b = 0; b < 16; ++b, ++r) {
            const int cur = (int)(r & 1), nxt = (int)((r + 1) & 1);
            k_ld_match<<<rgrid, TPB, 0, st>>>(n, r == 0 ? nullptr : lists[cur], &cnt[cur], cand, mate, mlist,
                                              &cnt[2 + cur], &cnt[nxt], cnt + 4);
            KERNEL_CHECK();
            k_ld_update<<<rgrid, TPB, 0, st>>>(n, ptr, col, c, cand, mate, mlist, &cnt[2 + cur], lists[nxt], &cnt[nxt],
                                               &cnt[2 + nxt]);
            KERNEL_CHECK();
        }
        if (noalloc_read_int(&cnt[r & 1], st) == 0) break;
        if (r > max_rounds) AMG_THROW(AMG_ERR_TIMEOUT, "matching did not settle after %lld rounds", r);
    }
    k_mate_normalize<<<grid, TPB, 0, st>>>(n, mate);
    KERNEL_CHECK();
    const int rounds = noalloc_read_int(cnt + 4, st);
    if (rounds_out) *rounds_out = rounds;
    return AMG_OK;
}

}  // namespace amg

namespace amg {
namespace {
__global__ void k_cat_ptr(int n, const int* __restrict__ src, int nnz_off, int* __restrict__ dst, int last) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
        if (i < n || last) dst[i] = src[i] + nnz_off;
}
__global__ void k_cat_col(long long nnz, const int* __restrict__ src, int col_off, int* __restrict__ dst) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x)
        dst[k] = src[k] + col_off;
}
}  // namespace

// Block-diagonal union of m systems (device arrays), set up as one hierarchy
// that keeps every system's row offsets.
// ---------------------------------------------- smooth vector (Section 3.2) --
// One l1-Jacobi sweep on A w = 0: w_i - (omega / M_ii) (A w)_i, the row sum in
// column order and every operation rounded on its own (the oracle's order).
__global__ void k_smooth_sweep(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                               const double* __restrict__ val, const double* __restrict__ minv, double omega,
                               const double* __restrict__ w, double* __restrict__ wout) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = ptr[i]; k < ptr[i + 1]; ++k) s = __dadd_rn(s, __dmul_rn(val[k], w[col[k]]));
        wout[i] = __dsub_rn(w[i], __dmul_rn(__dmul_rn(omega, minv[i]), s));
    }
}

void smooth_vector(const amg_csr* A, const double* w0, double* w, int sweeps, double omega, cudaStream_t st) {
    const int n = A->n;
    int dev = 0, sms = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevArena tmp;
    tmp.stream = st;
    double* minv = tmp.alloc<double>(n);
    double* other = tmp.alloc<double>(n);
    int* flags = tmp.alloc<int>(1);
    const int grid = blocks_for(n, TPB, sms * 8);
    // the same checks as amg_setup: CSR shape, SPD diagonal, usable sample vector
    CUDA_CHECK(cudaMemsetAsync(flags, 0, sizeof(int), st));
    k_check_ptr<<<blocks_for(n + 1, TPB, sms * 8), TPB, 0, st>>>(n, A->nnz, A->row_ptr, flags);
    KERNEL_CHECK();
    int f = 0;
    CUDA_CHECK(cudaMemcpyAsync(&f, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    if (f & F_SHAPE) AMG_THROW(AMG_ERR_ARG, "row_ptr is not a valid CSR row pointer");
    k_check_rows<<<grid, TPB, 0, st>>>(n, A->row_ptr, A->col, A->val, w0, minv, flags);
    KERNEL_CHECK();
    CUDA_CHECK(cudaMemcpyAsync(&f, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    if (f & F_SHAPE) AMG_THROW(AMG_ERR_ARG, "CSR columns unsorted, out of range, or pattern not symmetric");
    if (f & F_NOT_SPD) AMG_THROW(AMG_ERR_NOT_SPD, "non-finite value or diagonal entry missing or <= 0");
    if (f & F_BAD_W) AMG_THROW(AMG_ERR_BAD_W, "sample vector w0 has a zero or non-finite entry");
    k_l1_jacobi<<<grid, TPB, 0, st>>>(n, A->row_ptr, A->col, A->val, minv, nullptr);
    KERNEL_CHECK();
    // ping-pong between w and the scratch vector so that the last sweep lands in w
    double* cur = (sweeps % 2 == 0) ? w : other;
    double* nxt = (sweeps % 2 == 0) ? other : w;
    if (cur != w0) CUDA_CHECK(cudaMemcpyAsync(cur, w0, sizeof(double) * n, cudaMemcpyDefault, st));
    for (int k = 0; k < sweeps; ++k) {
        k_smooth_sweep<<<grid, TPB, 0, st>>>(n, A->row_ptr, A->col, A->val, minv, omega, cur, nxt);
        KERNEL_CHECK();
        std::swap(cur, nxt);
    }
    CUDA_CHECK(cudaStreamSynchronize(st));
}

void setup_many(amg_hierarchy* h, int m, const amg_csr* As, const double* const* ws) {
    cudaStream_t st = h->stream;
    long long n = 0, nnz = 0;
    h->seg0.assign(m + 1, 0);
    for (int s = 0; s < m; ++s) {
        n += As[s].n;
        nnz += As[s].nnz;
        h->seg0[s + 1] = (int)n;
        if (n > 0x7ffffffe || nnz > 0x7ffffffe) AMG_THROW(AMG_ERR_TOO_LARGE, "the union exceeds int32 sizes");
    }
    DevArena tmp;
    tmp.stream = st;
    int* ptr = tmp.alloc<int>(n + 1);
    int* col = tmp.alloc<int>(nnz);
    double* val = tmp.alloc<double>(nnz);
    double* w = tmp.alloc<double>(n);
    long long ro = 0, no = 0;
    for (int s = 0; s < m; ++s) {
        const amg_csr& A = As[s];
        k_cat_ptr<<<blocks_for(A.n + 1, TPB, h->num_sms * 8), TPB, 0, st>>>(A.n, A.row_ptr, (int)no, ptr + ro,
                                                                          s == m - 1);
        KERNEL_CHECK();
        k_cat_col<<<blocks_for(A.nnz, TPB, h->num_sms * 8), TPB, 0, st>>>(A.nnz, A.col, (int)ro, col + no);
        KERNEL_CHECK();
        CUDA_CHECK(cudaMemcpyAsync(val + no, A.val, sizeof(double) * (size_t)A.nnz, cudaMemcpyDefault, st));
        CUDA_CHECK(cudaMemcpyAsync(w + ro, ws[s], sizeof(double) * (size_t)A.n, cudaMemcpyDefault, st));
        ro += A.n;
        no += A.nnz;
    }
    amg_csr U{(int32_t)n, (int32_t)nnz, ptr, col, val};
    setup_hierarchy(h, &U, w);
}

}  // namespace amg
