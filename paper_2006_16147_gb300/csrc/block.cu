// block.cu -- several right-hand sides at once (multi-RHS block solve).
//
// Every column runs its own preconditioned CG (its own alpha, beta, rho and
// convergence), while each sparse product and the V-cycle (Eq. 2) serve all k
// columns in one pass over the matrices: the matrix is read once per k
// columns. Vectors are row-major n x k. A group of G lanes (G = the power of
// two >= k, at most 32) handles one row; lane gl owns columns gl, gl + G, ...
// so the group reads each matrix entry once (broadcast) and the k values of a
// gathered row of X as one coalesced segment.
//
// Columns carry a state (ColMode): START columns enter at the V-cycle half of
// a step (r given, z = B r, p = z), ACTIVE columns take a full CG step, a
// column whose recursive residual meets rtol goes to CHECK, where the true
// residual decides DONE or a restart. Columns in other states are carried
// along but never updated, so columns can join and leave between steps.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "amg_internal.cuh"
#include "device_util.cuh"

namespace amg {

BlockWork::~BlockWork() {
    if (mode_host) cudaFreeHost(mode_host);
    if (iters_host) cudaFreeHost(iters_host);
    if (rr_host) cudaFreeHost(rr_host);
    if (bb_host) cudaFreeHost(bb_host);
}

namespace {

constexpr int TPB = 256;
constexpr int WARPS = TPB / 32;
constexpr int MAXK = 256;

struct SellV {
    int n, nslices;
    const int* __restrict__ sptr;
    const int* __restrict__ col;
    const int* __restrict__ perm;
};

__device__ __forceinline__ int rowid(const SellV& S, int ip) { return S.perm ? __ldg(S.perm + ip) : ip; }

struct Grp {
    int G, gl, gw, ngroups;
};

__device__ __forceinline__ Grp make_grp(int G) {
    Grp g;
    g.G = G;
    const int lane = threadIdx.x & 31;
    g.gl = lane & (G - 1);
    const int gpw = 32 / G;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    g.gw = warp * gpw + lane / G;
    g.ngroups = (int)((gridDim.x * blockDim.x) >> 5) * gpw;
    return g;
}

// acc[m] += sum_e val_e * xv(col_e, c) for the row at SELL position ip.
template <typename T, int CPL, typename XV>
__device__ __forceinline__ void sell_row_k(const SellV& S, const T* __restrict__ val, int ip, const Grp& g, int k,
                                           XV&& xv, T (&acc)[CPL]) {
    const int s = ip >> 5, r = ip & 31;
    long long base = (long long)__ldg(S.sptr + s) * 32 + r;
    const int w = __ldg(S.sptr + s + 1) - __ldg(S.sptr + s);
    for (int e = 0; e < w; ++e, base += 32) {
        const int j = __ldg(S.col + base);
        const T a = __ldg(val + base);
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = g.gl + m * g.G;
            if (c < k) acc[m] = fma(a, xv(j, c), acc[m]);
        }
    }
}

// Per-column sums of (v0, v1) over the rows of the whole grid in a fixed
// order (groups of a warp, warps of a block, then blocks); the last block to
// finish calls fin(c, sum0, sum1) for every column. Deterministic for a fixed
// (grid, k).
template <int CPL, typename FIN>
__device__ __forceinline__ void colsum2(double (&v0)[CPL], double (&v1)[CPL], const Grp& g, int k, double* partial,
                                        unsigned* ticket, FIN&& fin) {
    __shared__ double sm[WARPS][2][MAXK];
    __shared__ bool last;
#pragma unroll
    for (int m = 0; m < CPL; ++m)
        for (int o = g.G; o < 32; o <<= 1) {
            v0[m] += __shfl_xor_sync(FULL_MASK, v0[m], o);
            v1[m] += __shfl_xor_sync(FULL_MASK, v1[m], o);
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < g.G) {
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = lane + m * g.G;
            if (c < k) {
                sm[warp][0][c] = v0[m];
                sm[warp][1][c] = v1[m];
            }
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < WARPS; ++w) {
            a += sm[w][0][c];
            b += sm[w][1][c];
        }
        partial[((size_t)blockIdx.x * 2 + 0) * k + c] = a;
        partial[((size_t)blockIdx.x * 2 + 1) * k + c] = b;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int blk = 0; blk < (int)gridDim.x; ++blk) {
            a += __ldcg(partial + ((size_t)blk * 2 + 0) * k + c);
            b += __ldcg(partial + ((size_t)blk * 2 + 1) * k + c);
        }
        fin(c, a, b);
    }
    __syncthreads();
    if (threadIdx.x == 0) *ticket = 0u;
}

// ---------------------------------------------------------- V-cycle --------
template <typename T, typename TB, int CPL>
__global__ void __launch_bounds__(TPB) bk_pre(SellV S, const T* __restrict__ valm, const T* __restrict__ minv, T omega,
                                              const TB* __restrict__ B, T* __restrict__ X, T* __restrict__ R, int k,
                                              int G) {
    const Grp g = make_grp(G);
    for (int ip = g.gw; ip < S.n; ip += g.ngroups) {
        T acc[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) acc[m] = 0;
        sell_row_k<T, CPL>(S, valm, ip, g, k, [&](int j, int c) { return (T)__ldg(B + (size_t)j * k + c); }, acc);
        const int i = rowid(S, ip);
        const T mi = omega * minv[i];
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = g.gl + m * g.G;
            if (c < k) {
                const size_t o = (size_t)i * k + c;
                const T bi = (T)B[o];
                X[o] = mi * bi;
                R[o] = fma(-omega, acc[m], bi);
            }
        }
    }
}

template <typename T, int CPL>
__global__ void __launch_bounds__(TPB) bk_restrict(int nc, const int* __restrict__ pt_ptr,
                                                   const int* __restrict__ pt_idx, const T* __restrict__ p,
                                                   const T* __restrict__ R, T* __restrict__ Bc, int k, int G) {
    const Grp g = make_grp(G);
    for (int q = g.gw; q < nc; q += g.ngroups) {
        T acc[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) acc[m] = 0;
        for (int e = pt_ptr[q]; e < pt_ptr[q + 1]; ++e) {
            const int i = __ldg(pt_idx + e);
            const T pi = __ldg(p + i);
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                const int c = g.gl + m * g.G;
                if (c < k) acc[m] = fma(pi, __ldg(R + (size_t)i * k + c), acc[m]);
            }
        }
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = g.gl + m * g.G;
            if (c < k) Bc[(size_t)q * k + c] = acc[m];
        }
    }
}

// X = A_L^{-1} B on the coarsest level, FP64 arithmetic.
template <typename TI, typename TO, int CPL>
__global__ void __launch_bounds__(TPB) bk_coarse_dense(int n, const double* __restrict__ Ainv, const TI* __restrict__ B,
                                                       TO* __restrict__ X, int k, int G) {
    const Grp g = make_grp(G);
    for (int i = g.gw; i < n; i += g.ngroups) {
        double acc[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) acc[m] = 0.0;
        const double* row = Ainv + (size_t)i * n;
        for (int j = 0; j < n; ++j) {
            const double a = __ldg(row + j);
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                const int c = g.gl + m * g.G;
                if (c < k) acc[m] = fma(a, (double)__ldg(B + (size_t)j * k + c), acc[m]);
            }
        }
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = g.gl + m * g.G;
            if (c < k) X[(size_t)i * k + c] = (TO)acc[m];
        }
    }
}

// Column c of a row-major n x k array to / from a contiguous FP64 vector.
template <typename T>
__global__ void bk_gather_col(int n, const T* __restrict__ A, int k, int c, double* __restrict__ v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = (double)A[(size_t)i * k + c];
}
template <typename T>
__global__ void bk_scatter_col(int n, const double* __restrict__ v, int k, int c, T* __restrict__ A) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) A[(size_t)i * k + c] = (T)v[i];
}

// r . z finisher: START columns take rho and beta = 0 and become ACTIVE;
// ACTIVE columns update beta (PCG, or flexible CG from z . q) and rho.
__device__ __forceinline__ void fin_rz(const BlockScalars& sc, int c, double rz, double zq, int flexible) {
    const int mode = sc.mode[c];
    if (mode == COL_START) {
        sc.rho[c] = rz;
        sc.beta[c] = 0.0;
        sc.mode[c] = isfinite(rz) ? COL_ACTIVE : COL_FAILED;
    } else if (mode == COL_ACTIVE) {
        const double beta = flexible ? -sc.alpha[c] * zq / sc.rho[c] : rz / sc.rho[c];
        sc.beta[c] = beta;
        sc.rho[c] = rz;
        if (!isfinite(beta)) sc.mode[c] = COL_FAILED;
    }
}

// out = x + P e + omega M^-1 (r - (A P) e); on level 0 also r_cg . out and
// (flexible CG) q . out per column.
template <typename T, typename TO, int CPL, bool DOT>
__global__ void __launch_bounds__(TPB) bk_post(SellV SAP, const T* __restrict__ apval, const T* __restrict__ minv,
                                               T omega, const int* __restrict__ agg, const T* __restrict__ p,
                                               const T* __restrict__ E, const T* __restrict__ X,
                                               const T* __restrict__ R, const double* __restrict__ Bdot,
                                               const double* __restrict__ Q2, TO* __restrict__ Out, int k, int G,
                                               double* partial, unsigned* ticket, BlockScalars sc, int flexible) {
    const Grp g = make_grp(G);
    double d0[CPL], d1[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) d0[m] = d1[m] = 0.0;
    for (int ip = g.gw; ip < SAP.n; ip += g.ngroups) {
        T acc[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) acc[m] = 0;
        sell_row_k<T, CPL>(SAP, apval, ip, g, k, [&](int q, int c) { return __ldg(E + (size_t)q * k + c); }, acc);
        const int i = rowid(SAP, ip);
        const int a = agg[i];
        const T pi = p[i];
        const T mi = omega * minv[i];
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = g.gl + m * g.G;
            if (c < k) {
                const size_t o = (size_t)i * k + c;
                const T y = fma(pi, E[(size_t)a * k + c], X[o]);
                const T v = fma(mi, R[o] - acc[m], y);
                Out[o] = (TO)v;
                if (DOT) {
                    d0[m] = fma(Bdot[o], (double)(TO)v, d0[m]);
                    if (Q2) d1[m] = fma(Q2[o], (double)(TO)v, d1[m]);
                }
            }
        }
    }
    if (DOT) colsum2<CPL>(d0, d1, g, k, partial, ticket, [&](int c, double a, double b) { fin_rz(sc, c, a, b, flexible); });
}

// ------------------------------------------------------------- CG ----------
// Q = A P; p . q per column; alpha = rho / p.q for ACTIVE columns, else 0.
template <int CPL>
__global__ void __launch_bounds__(TPB) bk_spmv_dot(SellV S, const double* __restrict__ val,
                                                   const double* __restrict__ P, double* __restrict__ Q, int k, int G,
                                                   double* partial, unsigned* ticket, BlockScalars sc) {
    const Grp g = make_grp(G);
    double d0[CPL], d1[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) d0[m] = d1[m] = 0.0;
    for (int ip = g.gw; ip < S.n; ip += g.ngroups) {
        double acc[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) acc[m] = 0.0;
        sell_row_k<double, CPL>(S, val, ip, g, k, [&](int j, int c) { return __ldg(P + (size_t)j * k + c); }, acc);
        const int i = rowid(S, ip);
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = g.gl + m * g.G;
            if (c < k) {
                const size_t o = (size_t)i * k + c;
                Q[o] = acc[m];
                d0[m] = fma(P[o], acc[m], d0[m]);
            }
        }
    }
    colsum2<CPL>(d0, d1, g, k, partial, ticket, [&](int c, double pq, double) {
        sc.pq[c] = pq;
        if (sc.mode[c] == COL_ACTIVE) {
            const double alpha = sc.rho[c] / pq;
            if (!(pq > 0.0) || !isfinite(alpha)) {
                sc.mode[c] = COL_FAILED;
                sc.alpha[c] = 0.0;
            } else {
                sc.alpha[c] = alpha;
            }
        } else {
            sc.alpha[c] = 0.0;
        }
    });
}

// ACTIVE columns: X += alpha P, R -= alpha Q, ||R||^2; convergence -> CHECK.
template <int CPL>
__global__ void __launch_bounds__(TPB) bk_update_xr(int n, const double* __restrict__ P, const double* __restrict__ Q,
                                                    double* __restrict__ X, double* __restrict__ R, int k, int G,
                                                    double* partial, unsigned* ticket, BlockScalars sc) {
    const Grp g = make_grp(G);
    double al[CPL];
    bool on[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) {
        const int c = g.gl + m * g.G;
        on[m] = c < k && sc.mode[c] == COL_ACTIVE;
        al[m] = on[m] ? sc.alpha[c] : 0.0;
    }
    double d0[CPL], d1[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) d0[m] = d1[m] = 0.0;
    for (int i = g.gw; i < n; i += g.ngroups) {
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            if (!on[m]) continue;
            const size_t o = (size_t)i * k + g.gl + m * g.G;
            X[o] = fma(al[m], P[o], X[o]);
            const double ri = fma(-al[m], Q[o], R[o]);
            R[o] = ri;
            d0[m] = fma(ri, ri, d0[m]);
        }
    }
    colsum2<CPL>(d0, d1, g, k, partial, ticket, [&](int c, double rr, double) {
        if (sc.mode[c] != COL_ACTIVE) return;
        sc.rr[c] = rr;
        sc.iters[c] += 1;
        if (rr <= sc.rtol[c] * sc.rtol[c] * sc.bb[c]) sc.mode[c] = COL_CHECK;
    });
}

// ACTIVE columns: P = Z + beta P (P = Z when beta = 0, whatever P held).
template <int CPL>
__global__ void __launch_bounds__(TPB) bk_update_p(int n, const double* __restrict__ Z, double* __restrict__ P, int k,
                                                   int G, BlockScalars sc) {
    const Grp g = make_grp(G);
    double be[CPL];
    bool on[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) {
        const int c = g.gl + m * g.G;
        on[m] = c < k && sc.mode[c] == COL_ACTIVE;
        be[m] = on[m] ? sc.beta[c] : 0.0;
    }
    for (int i = g.gw; i < n; i += g.ngroups) {
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            if (!on[m]) continue;
            const size_t o = (size_t)i * k + g.gl + m * g.G;
            P[o] = be[m] == 0.0 ? Z[o] : fma(be[m], P[o], Z[o]);
        }
    }
}

// R = B - A X for the selected columns, ||R||^2 and ||B||^2.
//   stage 0 (start): every non-idle column; DONE when ||B|| = 0, else START.
//   stage 1 (check): CHECK columns; true residual below rtol -> DONE, else the
//                    column restarts from R (START).
//   stage 2 (report): every column; only records ||R||^2 in rr.
template <int CPL>
__global__ void __launch_bounds__(TPB) bk_residual(SellV S, const double* __restrict__ val,
                                                   const double* __restrict__ X, const double* __restrict__ B,
                                                   double* __restrict__ R, int k, int G, double* partial,
                                                   unsigned* ticket, BlockScalars sc, int stage) {
    const Grp g = make_grp(G);
    bool on[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) {
        const int c = g.gl + m * g.G;
        const int md = c < k ? sc.mode[c] : COL_IDLE;
        on[m] = c < k && (stage == 0 ? md != COL_IDLE : (stage == 1 ? md == COL_CHECK : true));
    }
    double d0[CPL], d1[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) d0[m] = d1[m] = 0.0;
    for (int ip = g.gw; ip < S.n; ip += g.ngroups) {
        double acc[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) acc[m] = 0.0;
        sell_row_k<double, CPL>(S, val, ip, g, k, [&](int j, int c) { return __ldg(X + (size_t)j * k + c); }, acc);
        const int i = rowid(S, ip);
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            if (!on[m]) continue;
            const size_t o = (size_t)i * k + g.gl + m * g.G;
            const double bi = B[o];
            const double ri = bi - acc[m];
            R[o] = ri;
            d0[m] = fma(ri, ri, d0[m]);
            d1[m] = fma(bi, bi, d1[m]);
        }
    }
    colsum2<CPL>(d0, d1, g, k, partial, ticket, [&](int c, double rr, double bb) {
        const int md = sc.mode[c];
        if (stage == 0) {
            if (md == COL_IDLE) return;
            sc.bb[c] = bb;
            sc.rr[c] = rr;
            sc.iters[c] = 0;
            sc.mode[c] = bb == 0.0 ? COL_DONE : (rr <= sc.rtol[c] * sc.rtol[c] * bb ? COL_DONE : COL_START);
        } else if (stage == 1) {
            if (md != COL_CHECK) return;
            sc.rr[c] = rr;
            sc.mode[c] = rr <= sc.rtol[c] * sc.rtol[c] * sc.bb[c] ? COL_DONE : COL_START;
        } else {
            sc.rr[c] = rr;
        }
    });
}

__global__ void bk_zero_cols(int n, double* __restrict__ X, int k, const int* __restrict__ mode,
                             const double* __restrict__ bb) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * k;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % k);
        if (bb[c] == 0.0 && mode[c] == COL_DONE) X[t] = 0.0;
    }
}

// ------------------------------------------------------------- host --------
SellV sv(const DevSell& S) { return SellV{S.n, S.nslices, S.sptr, S.col, S.perm}; }

void group_shape(int k, int* G, int* cpl) {
    int g = 1;
    while (g < k && g < 32) g <<= 1;
    int c = (k + g - 1) / g;
    int p = 1;
    while (p < c) p <<= 1;
    *G = g;
    *cpl = p;
}

#define DISPATCH_CPL(cpl, ...)                          \
    switch (cpl) {                                      \
        case 1: { constexpr int CPL = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int CPL = 2; __VA_ARGS__; } break; \
        case 4: { constexpr int CPL = 4; __VA_ARGS__; } break; \
        default: { constexpr int CPL = 8; __VA_ARGS__; } break; \
    }

int grid_rows(const amg_hierarchy* h, long long rows, int G) {
    const long long groups_per_block = (long long)WARPS * (32 / G);
    return blocks_for(rows, (int)groups_per_block, h->num_sms * 8);
}

BlockWork& ensure_work(amg_hierarchy* h, int K) {
    if (h->blk && h->blk->K == K) return *h->blk;
    if (h->blk) {
        CUDA_CHECK(cudaStreamSynchronize(h->stream));
        delete h->blk;
        h->blk = nullptr;
    }
    BlockWork* W = new BlockWork;
    h->blk = W;
    W->K = K;
    const bool f32 = h->opt.precision == AMG_FP32_VCYCLE;
    const size_t V = f32 ? 4 : 8;
    for (auto& L : h->lev) {
        const size_t m = (size_t)L.A.n * K;
        W->b.push_back(W->mem.alloc<char>(m * V));
        W->x.push_back(W->mem.alloc<char>(m * V));
        W->r.push_back(W->mem.alloc<char>(m * V));
        W->y.push_back(W->mem.alloc<char>(m * V));
    }
    const size_t m0 = (size_t)h->lev[0].A.n * K;
    W->R = W->mem.alloc<double>(m0);
    W->Z = W->mem.alloc<double>(m0);
    W->P = W->mem.alloc<double>(m0);
    W->Q = W->mem.alloc<double>(m0);
    W->T = W->mem.alloc<double>(m0);
    W->sc.mode = W->mem.alloc<int>(K);
    W->sc.iters = W->mem.alloc<int>(K);
    W->sc.rho = W->mem.alloc<double>(K);
    W->sc.alpha = W->mem.alloc<double>(K);
    W->sc.beta = W->mem.alloc<double>(K);
    W->sc.pq = W->mem.alloc<double>(K);
    W->sc.rr = W->mem.alloc<double>(K);
    W->sc.bb = W->mem.alloc<double>(K);
    W->sc.rtol = W->mem.alloc<double>(K);
    W->grid = h->num_sms * 8;
    W->partial = W->mem.alloc<double>((size_t)W->grid * 2 * K);
    W->ticket = W->mem.alloc<unsigned>(1);
    CUDA_CHECK(cudaMemsetAsync(W->ticket, 0, sizeof(unsigned), h->stream));
    CUDA_CHECK(cudaMemsetAsync(W->sc.mode, 0, sizeof(int) * K, h->stream));
    CUDA_CHECK(cudaMemsetAsync(W->sc.iters, 0, sizeof(int) * K, h->stream));
    CUDA_CHECK(cudaHostAlloc(&W->mode_host, sizeof(int) * K, cudaHostAllocDefault));
    CUDA_CHECK(cudaHostAlloc(&W->iters_host, sizeof(int) * K, cudaHostAllocDefault));
    CUDA_CHECK(cudaHostAlloc(&W->rr_host, sizeof(double) * K, cudaHostAllocDefault));
    CUDA_CHECK(cudaHostAlloc(&W->bb_host, sizeof(double) * K, cudaHostAllocDefault));
    if (h->coarse_cg) {
        W->cb = W->mem.alloc<double>(h->nc);
        W->cx = W->mem.alloc<double>(h->nc);
    }
    return *W;
}

// Z = B R for all K columns (block V-cycle); level 0 finishes r . z per column.
template <typename T>
void block_vcycle(amg_hierarchy* h, BlockWork& W, int flexible) {
    cudaStream_t st = h->stream;
    const int K = W.K;
    const int L = (int)h->lev.size() - 1;
    const bool f32 = sizeof(T) == 4;
    const T omega = (T)h->opt.omega;
    int G, cpl;
    group_shape(K, &G, &cpl);
    auto lv = [&](std::vector<void*>& v, int l) { return static_cast<T*>(v[l]); };
    if (L == 0) {
        // single level: the whole operator is the coarsest solve
        AMG_THROW(AMG_ERR_ARG, "block solves need at least two levels");
    }
    for (int l = 0; l < L; ++l) {
        Level& Lv = h->lev[l];
        const T* valm = f32 ? (const T*)Lv.valm32 : (const T*)Lv.valm;
        const T* minv = f32 ? (const T*)Lv.minv32 : (const T*)Lv.minv;
        const int g = grid_rows(h, Lv.S.n, G);
        Scope sc_(&h->prof, st, l == 0 ? K_PRE_L0 : K_PRE,
                  (double)Lv.A.nnz * (sizeof(T) + 4) + (double)Lv.A.n * K * ((l == 0 ? 8 : sizeof(T)) + 2.0 * sizeof(T)));
        if (l == 0)
            DISPATCH_CPL(cpl, bk_pre<T, double, CPL><<<g, TPB, 0, st>>>(sv(Lv.S), valm, minv, omega, W.R, lv(W.x, 0),
                                                                       lv(W.r, 0), K, G))
        else
            DISPATCH_CPL(cpl, bk_pre<T, T, CPL><<<g, TPB, 0, st>>>(sv(Lv.S), valm, minv, omega, lv(W.b, l), lv(W.x, l),
                                                                  lv(W.r, l), K, G))
        KERNEL_CHECK();
        const int nc = h->lev[l + 1].A.n;
        const T* p = f32 ? (const T*)Lv.p32 : (const T*)Lv.p;
        DISPATCH_CPL(cpl, bk_restrict<T, CPL><<<grid_rows(h, nc, G), TPB, 0, st>>>(nc, Lv.pt_ptr, Lv.pt_idx, p,
                                                                                   lv(W.r, l), lv(W.b, l + 1), K, G))
        KERNEL_CHECK();
    }
    {
        Scope sc_(&h->prof, st, K_COARSE, 8.0 * h->nc * h->nc + 16.0 * h->nc * K);
        if (!h->coarse_cg) {
            DISPATCH_CPL(cpl, bk_coarse_dense<T, T, CPL><<<grid_rows(h, h->nc, G), TPB, 0, st>>>(
                                  h->nc, h->coarse_inv, lv(W.b, L), lv(W.x, L), K, G))
            KERNEL_CHECK();
        } else {
            const int gg = blocks_for(h->nc, TPB, h->num_sms * 4);
            for (int c = 0; c < K; ++c) {
                bk_gather_col<T><<<gg, TPB, 0, st>>>(h->nc, lv(W.b, L), K, c, W.cb);
                KERNEL_CHECK();
                coarse_cg_solve(h, W.cb, W.cx);
                bk_scatter_col<T><<<gg, TPB, 0, st>>>(h->nc, W.cx, K, c, lv(W.x, L));
                KERNEL_CHECK();
            }
        }
    }
    for (int l = L - 1; l >= 0; --l) {
        Level& Lv = h->lev[l];
        const T* apv = f32 ? (const T*)Lv.AP.val32 : (const T*)Lv.AP.val;
        const T* minv = f32 ? (const T*)Lv.minv32 : (const T*)Lv.minv;
        const T* p = f32 ? (const T*)Lv.p32 : (const T*)Lv.p;
        const T* e = l + 1 == L ? lv(W.x, L) : lv(W.y, l + 1);
        const int g = grid_rows(h, Lv.AP.n, G);
        Scope sc_(&h->prof, st, l == 0 ? K_POST_L0 : K_POST,
                  (double)Lv.ap_nnz * (sizeof(T) + 4) + (double)Lv.A.n * K * (4.0 * sizeof(T) + 8));
        if (l > 0)
            DISPATCH_CPL(cpl, bk_post<T, T, CPL, false><<<g, TPB, 0, st>>>(
                                  sv(Lv.AP), apv, minv, omega, Lv.agg, p, e, lv(W.x, l), lv(W.r, l), nullptr, nullptr,
                                  lv(W.y, l), K, G, W.partial, W.ticket, W.sc, flexible))
        else
            DISPATCH_CPL(cpl, bk_post<T, double, CPL, true><<<W.grid, TPB, 0, st>>>(
                                  sv(Lv.AP), apv, minv, omega, Lv.agg, p, e, lv(W.x, 0), lv(W.r, 0), W.R,
                                  flexible ? W.Q : nullptr, W.Z, K, G, W.partial, W.ticket, W.sc, flexible))
        KERNEL_CHECK();
    }
}

void read_state(amg_hierarchy* h, BlockWork& W) {
    cudaStream_t st = h->stream;
    CUDA_CHECK(cudaMemcpyAsync(W.mode_host, W.sc.mode, sizeof(int) * W.K, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(W.iters_host, W.sc.iters, sizeof(int) * W.K, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(W.rr_host, W.sc.rr, sizeof(double) * W.K, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(W.bb_host, W.sc.bb, sizeof(double) * W.K, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
}

}  // namespace

// One step of every column (see the file comment). Returns after the state
// has been read back into W.mode_host / iters_host / rr_host / bb_host.
void block_step(amg_hierarchy* h, const double* B, double* X) {
    BlockWork& W = *h->blk;
    cudaStream_t st = h->stream;
    const int K = W.K;
    const int flexible = h->opt.krylov == 1;
    int G, cpl;
    group_shape(K, &G, &cpl);
    Level& L0 = h->lev[0];
    const int n = L0.A.n;
    const double nnz = (double)L0.A.nnz;
    bool any_active = false, any_check = false;
    for (int c = 0; c < K; ++c) {
        any_active |= W.mode_host[c] == COL_ACTIVE;
        any_check |= W.mode_host[c] == COL_CHECK;
    }
    if (any_active) {
        {
            Scope sc_(&h->prof, st, K_SPMV_DOT, 12.0 * nnz + 16.0 * n * K);
            DISPATCH_CPL(cpl, bk_spmv_dot<CPL><<<W.grid, TPB, 0, st>>>(sv(L0.S), L0.S.val, W.P, W.Q, K, G, W.partial,
                                                                     W.ticket, W.sc))
            KERNEL_CHECK();
        }
        {
            Scope sc_(&h->prof, st, K_UPDATE_XR, 48.0 * n * K);
            DISPATCH_CPL(cpl, bk_update_xr<CPL><<<W.grid, TPB, 0, st>>>(n, W.P, W.Q, X, W.R, K, G, W.partial, W.ticket,
                                                                      W.sc))
            KERNEL_CHECK();
        }
    }
    if (h->opt.precision == AMG_FP32_VCYCLE) block_vcycle<float>(h, W, flexible);
    else block_vcycle<double>(h, W, flexible);
    {
        Scope sc_(&h->prof, st, K_UPDATE_P, 24.0 * n * K);
        DISPATCH_CPL(cpl, bk_update_p<CPL><<<grid_rows(h, n, G), TPB, 0, st>>>(n, W.Z, W.P, K, G, W.sc))
        KERNEL_CHECK();
    }
    read_state(h, W);
    any_check = false;
    for (int c = 0; c < K; ++c) any_check |= W.mode_host[c] == COL_CHECK;
    if (any_check) {
        Scope sc_(&h->prof, st, K_RESIDUAL, 12.0 * nnz + 24.0 * n * K);
        DISPATCH_CPL(cpl, bk_residual<CPL><<<W.grid, TPB, 0, st>>>(sv(L0.S), L0.S.val, X, B, W.R, K, G, W.partial,
                                                                 W.ticket, W.sc, 1))
        KERNEL_CHECK();
        read_state(h, W);
    }
}

// Marks every column START (or DONE for b = 0) from the residual of X.
void block_begin(amg_hierarchy* h, const double* B, double* X, double rtol) {
    BlockWork& W = *h->blk;
    cudaStream_t st = h->stream;
    const int K = W.K;
    int G, cpl;
    group_shape(K, &G, &cpl);
    Level& L0 = h->lev[0];
    std::vector<double> rt(K, rtol);
    std::vector<int> md(K, COL_START);
    CUDA_CHECK(cudaMemcpyAsync(W.sc.rtol, rt.data(), sizeof(double) * K, cudaMemcpyHostToDevice, st));
    CUDA_CHECK(cudaMemcpyAsync(W.sc.mode, md.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
    DISPATCH_CPL(cpl, bk_residual<CPL><<<W.grid, TPB, 0, st>>>(sv(L0.S), L0.S.val, X, B, W.R, K, G, W.partial,
                                                             W.ticket, W.sc, 0))
    KERNEL_CHECK();
    bk_zero_cols<<<blocks_for((long long)L0.A.n * K, TPB, h->num_sms * 8), TPB, 0, st>>>(L0.A.n, X, K, W.sc.mode,
                                                                                      W.sc.bb);
    KERNEL_CHECK();
    read_state(h, W);
}

amg_status solve_batch(amg_hierarchy* h, int k, const double* B, double* X, double rtol, int maxit,
                       amg_solve_info* infos) {
    auto t0 = std::chrono::steady_clock::now();
    if (k < 1 || k > MAXK) AMG_THROW(AMG_ERR_TOO_LARGE, "block solves take 1..%d columns", MAXK);
    if (h->opt.pre != 1 || h->opt.post != 1) AMG_THROW(AMG_ERR_ARG, "block solves use 1+1 smoothing sweeps");
    if (h->lev.size() < 2) AMG_THROW(AMG_ERR_ARG, "block solves need at least two levels");
    BlockWork& W = ensure_work(h, k);
    block_begin(h, B, X, rtol);
    int steps = 0;
    for (;;) {
        bool live = false;
        for (int c = 0; c < k; ++c) live |= W.mode_host[c] == COL_START || W.mode_host[c] == COL_ACTIVE;
        if (!live) break;
        int maxi = 0;
        for (int c = 0; c < k; ++c) maxi = std::max(maxi, W.iters_host[c]);
        if (maxi >= maxit) break;
        block_step(h, B, X);
        if (++steps > 4 * maxit + 16) break;
    }
    // true residual of every column for the report
    {
        int G, cpl;
        group_shape(k, &G, &cpl);
        Level& L0 = h->lev[0];
        DISPATCH_CPL(cpl, bk_residual<CPL><<<W.grid, TPB, 0, h->stream>>>(sv(L0.S), L0.S.val, X, B, W.T, k, G,
                                                                        W.partial, W.ticket, W.sc, 2))
        KERNEL_CHECK();
        read_state(h, W);
    }
    h->prof.flush();
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    amg_status status = AMG_OK;
    for (int c = 0; c < k; ++c) {
        const int md = W.mode_host[c];
        const double nb = std::sqrt(W.bb_host[c]);
        const double tr = nb > 0.0 ? std::sqrt(W.rr_host[c]) / nb : 0.0;
        if (md == COL_FAILED) status = AMG_ERR_BREAKDOWN;
        else if (md != COL_DONE && status == AMG_OK) status = AMG_NOT_CONVERGED;
        if (infos) {
            infos[c].iterations = W.iters_host[c];
            infos[c].restarts = 0;
            infos[c].relres = tr;
            infos[c].true_relres = tr;
            infos[c].solve_ms = ms;
        }
    }
    return status;
}

void block_free(amg_hierarchy* h) {
    delete h->blk;
    h->blk = nullptr;
}

}  // namespace amg
