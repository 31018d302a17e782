// block.cu -- several right-hand sides at once (multi-RHS block solve).
//
// Every column runs its own preconditioned CG (its own alpha, beta, rho and
// convergence), while each sparse product and the V-cycle (Eq. 2) serve all k
// columns in one pass over the matrices: the matrix is read once per k
// columns. Vectors are row-major n x k. A group of G lanes handles one row;
// lane gl owns the CPL consecutive columns gl * CPL .. gl * CPL + CPL - 1, so
// the group reads each matrix entry once (broadcast) and a gathered row of X
// as one coalesced segment, each lane's part as one vector load (float4,
// float2 or double2) when the row stride is a multiple of CPL.
//
// Columns carry a state (ColMode): START columns enter at the V-cycle half of
// a step (r given, z = B r, p = z), ACTIVE columns take a full CG step, a
// column whose recursive residual meets rtol goes to CHECK, where the true
// residual decides DONE or a restart. Columns in other states are carried
// along but never updated, so columns can join and leave between steps.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>

#include "amg_internal.cuh"
#include "device_util.cuh"

namespace amg {

BlockWork::~BlockWork() {
    for (auto& g : gstep)
        if (g) cudaGraphExecDestroy(g);
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

// The CPL consecutive values at p (a lane's columns of one row; lim of them
// are live columns). With VEC the row stride is a multiple of CPL, so the
// address is aligned to CPL values and all CPL lie inside the row: the loads
// are vectors. Without VEC only the live columns are read. CG reads through
// L2 only (values other blocks write during the launch).
template <bool VEC, bool CG, int CPL, typename T>
__device__ __forceinline__ void ld_cols(const T* p, T (&v)[CPL], int lim) {
    if constexpr (VEC && std::is_same<T, float>::value && CPL >= 4) {
#pragma unroll
        for (int q = 0; q < CPL / 4; ++q) {
            const float4 f = CG ? __ldcg(reinterpret_cast<const float4*>(p) + q)
                                : __ldg(reinterpret_cast<const float4*>(p) + q);
            v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
        }
    } else if constexpr (VEC && std::is_same<T, float>::value && CPL == 2) {
        const float2 f = CG ? __ldcg(reinterpret_cast<const float2*>(p)) : __ldg(reinterpret_cast<const float2*>(p));
        v[0] = f.x; v[1] = f.y;
    } else if constexpr (VEC && std::is_same<T, double>::value && CPL >= 2) {
#pragma unroll
        for (int q = 0; q < CPL / 2; ++q) {
            const double2 f = CG ? __ldcg(reinterpret_cast<const double2*>(p) + q)
                                 : __ldg(reinterpret_cast<const double2*>(p) + q);
            v[2 * q] = f.x; v[2 * q + 1] = f.y;
        }
    } else {
#pragma unroll
        for (int m = 0; m < CPL; ++m) v[m] = m < lim ? (CG ? __ldcg(p + m) : __ldg(p + m)) : T(0);
    }
}

// Plain loads of a lane's columns of a row that this kernel also writes.
template <bool VEC, int CPL, typename T>
__device__ __forceinline__ void ld_own(const T* p, T (&v)[CPL], int lim) {
    if constexpr (VEC && std::is_same<T, float>::value && CPL >= 4) {
#pragma unroll
        for (int q = 0; q < CPL / 4; ++q) {
            const float4 f = reinterpret_cast<const float4*>(p)[q];
            v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
        }
    } else if constexpr (VEC && std::is_same<T, float>::value && CPL == 2) {
        const float2 f = *reinterpret_cast<const float2*>(p);
        v[0] = f.x; v[1] = f.y;
    } else if constexpr (VEC && std::is_same<T, double>::value && CPL >= 2) {
#pragma unroll
        for (int q = 0; q < CPL / 2; ++q) {
            const double2 f = reinterpret_cast<const double2*>(p)[q];
            v[2 * q] = f.x; v[2 * q + 1] = f.y;
        }
    } else {
#pragma unroll
        for (int m = 0; m < CPL; ++m) v[m] = m < lim ? p[m] : T(0);
    }
}

// Stores a lane's columns of a row: one vector store when VEC and all of them
// are live columns (c0 + CPL <= k), else one store per live column.
template <bool VEC, int CPL, typename T>
__device__ __forceinline__ void st_cols(T* p, const T (&v)[CPL], int c0, int k) {
    if constexpr (VEC && std::is_same<T, float>::value && CPL >= 4) {
        if (c0 + CPL <= k) {
#pragma unroll
            for (int q = 0; q < CPL / 4; ++q)
                reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            return;
        }
    } else if constexpr (VEC && std::is_same<T, float>::value && CPL == 2) {
        if (c0 + CPL <= k) {
            *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
            return;
        }
    } else if constexpr (VEC && std::is_same<T, double>::value && CPL >= 2) {
        if (c0 + CPL <= k) {
#pragma unroll
            for (int q = 0; q < CPL / 2; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(v[2 * q], v[2 * q + 1]);
            return;
        }
    }
#pragma unroll
    for (int m = 0; m < CPL; ++m)
        if (c0 + m < k) p[m] = v[m];
}

// acc[m] += sum_e val_e * X[col_e * ld + c0 + m] for the row at SELL position
// ip, in entry order (a lane's columns c0 .. c0 + CPL - 1; a lane without a
// live column returns at once). Four entries at a time (the last group
// predicated): their indices and values are loaded first and the four
// gathered rows of X are in flight together, so a row costs about two memory
// latencies per four entries instead of two per entry.
template <bool VEC, bool CG, int CPL, typename T>
__device__ __forceinline__ void sell_row_k(const SellV& S, const T* __restrict__ val, int ip, int c0, int k,
                                           const T* X, int ld, T (&acc)[CPL]) {
    if (c0 >= k) return;
    const int s = ip >> 5, r = ip & 31;
    const int s0 = __ldg(S.sptr + s);
    const int w = __ldg(S.sptr + s + 1) - s0;
    long long base = (long long)s0 * 32 + r;
    int e = 0;
    for (; e + 4 <= w; e += 4, base += 128) {
        int j[4];
        T a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            j[u] = __ldg(S.col + base + 32 * u);
            a[u] = __ldg(val + base + 32 * u);
        }
        T xs[4][CPL];
#pragma unroll
        for (int u = 0; u < 4; ++u) ld_cols<VEC, CG, CPL>(X + (size_t)j[u] * ld + c0, xs[u], k - c0);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int m = 0; m < CPL; ++m) acc[m] = fma(a[u], xs[u][m], acc[m]);
    }
    if (e < w) {                      // the last 1-3 entries as one predicated group of four
        int j[4];
        T a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ok = e + u < w;
            j[u] = ok ? __ldg(S.col + base + 32 * u) : 0;
            a[u] = ok ? __ldg(val + base + 32 * u) : T(0);
        }
        T xs[4][CPL];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (e + u < w) ld_cols<VEC, CG, CPL>(X + (size_t)j[u] * ld + c0, xs[u], k - c0);
            else
#pragma unroll
                for (int m = 0; m < CPL; ++m) xs[u][m] = T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (e + u < w)
#pragma unroll
                for (int m = 0; m < CPL; ++m) acc[m] = fma(a[u], xs[u][m], acc[m]);
    }
}

// Per-column sums of (v0, v1) over the rows of the whole grid in a fixed
// order (groups of a warp, warps of a block, then blocks); the last block to
// finish calls fin(c, sum0, sum1) for every column. Deterministic for a fixed
// (grid, lanes per row, block width ld): a column's sum never depends on the other columns.
template <int CPL, typename FIN>
__device__ __forceinline__ void colsum2(double (&v0)[CPL], double (&v1)[CPL], const Grp& g, int k, int ld, double* partial,
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
            const int c = lane * CPL + m;
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
    // tpc consecutive lanes per column (a power of two <= 32, set by the
    // block width ld so that it does not depend on how many columns are
    // live): lane j sums the blocks j, j + tpc, ... in order, then the lanes
    // combine by a shuffle tree; a fixed order for a fixed (grid, ld).
    int tpc = 1;
    while (tpc < 32 && tpc * 2 * ld <= (int)blockDim.x) tpc *= 2;
    const int cpb = (int)blockDim.x / tpc;               // columns per pass
    const int j = threadIdx.x & (tpc - 1);
    for (int c0 = 0; c0 < k; c0 += cpb) {
        const int c = c0 + (int)threadIdx.x / tpc;
        double a = 0.0, b = 0.0;
        if (c < k) {
#pragma unroll 4
            for (int blk = j; blk < (int)gridDim.x; blk += tpc) {
                a += __ldcg(partial + ((size_t)blk * 2 + 0) * k + c);
                b += __ldcg(partial + ((size_t)blk * 2 + 1) * k + c);
            }
        }
        for (int o = tpc >> 1; o > 0; o >>= 1) {
            a += __shfl_xor_sync(FULL_MASK, a, o);
            b += __shfl_xor_sync(FULL_MASK, b, o);
        }
        if (c < k && j == 0) fin(c, a, b);
    }
    __syncthreads();
    if (threadIdx.x == 0) *ticket = 0u;
}

// ---------------------------------------------------------- V-cycle --------
template <typename T, int CPL, bool VEC>
__global__ void __launch_bounds__(TPB) bk_pre(SellV S, const T* __restrict__ valm, const T* __restrict__ minv, T omega,
                                              const T* __restrict__ B, T* __restrict__ X, T* __restrict__ R, int k, int ld,
                                              int G) {
    const Grp g = make_grp(G);
    const int c0 = g.gl * CPL;
    if (c0 >= k) return;
    for (int ip = g.gw; ip < S.n; ip += g.ngroups) {
        T acc[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) acc[m] = 0;
        sell_row_k<VEC, false, CPL>(S, valm, ip, c0, k, B, ld, acc);
        const int i = rowid(S, ip);
        const T mi = omega * minv[i];
        const size_t o = (size_t)i * ld + c0;
        T bi[CPL], xo[CPL], ro[CPL];
        ld_cols<VEC, false, CPL>(B + o, bi, k - c0);
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            xo[m] = mi * bi[m];
            ro[m] = fma(-omega, acc[m], bi[m]);
        }
        st_cols<VEC, CPL>(X + o, xo, c0, k);
        st_cols<VEC, CPL>(R + o, ro, c0, k);
    }
}

// FP32 copy of columns [0, k) of the level-0 residual (row-major, leading
// dimension ld) for the FP32 V-cycle: one conversion per entry instead of one
// per gathered matrix entry (the FP64 -> FP32 conversion runs at the FP64 rate).
__global__ void __launch_bounds__(TPB) bk_to_f32(long long n, int k, int ld, const double* __restrict__ a,
                                                 float* __restrict__ b) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * ld;
         t += (long long)gridDim.x * blockDim.x)
        if (k == ld || (int)(t % ld) < k) b[t] = (float)a[t];
}

template <typename T, int CPL, bool VEC>
__global__ void __launch_bounds__(TPB) bk_restrict(int nc, const int* __restrict__ pt_ptr,
                                                   const int* __restrict__ pt_idx, const T* __restrict__ p,
                                                   const T* __restrict__ R, T* __restrict__ Bc, int k, int ld, int G) {
    const Grp g = make_grp(G);
    const int c0 = g.gl * CPL;
    if (c0 >= k) return;
    for (int q = g.gw; q < nc; q += g.ngroups) {
        T acc[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) acc[m] = 0;
        for (int e = pt_ptr[q]; e < pt_ptr[q + 1]; ++e) {
            const int i = __ldg(pt_idx + e);
            const T pi = __ldg(p + i);
            T rv[CPL];
            ld_cols<VEC, false, CPL>(R + (size_t)i * ld + c0, rv, k - c0);
#pragma unroll
            for (int m = 0; m < CPL; ++m) acc[m] = fma(pi, rv[m], acc[m]);
        }
        st_cols<VEC, CPL>(Bc + (size_t)q * ld + c0, acc, c0, k);
    }
}

// X = A_L^{-1} B on the coarsest level, FP64 arithmetic.
template <typename TI, typename TO, int CPL, bool VEC>
__global__ void __launch_bounds__(TPB) bk_coarse_dense(int n, const double* __restrict__ Ainv, const TI* __restrict__ B,
                                                       TO* __restrict__ X, int k, int ld, int G) {
    const Grp g = make_grp(G);
    const int c0 = g.gl * CPL;
    if (c0 >= k) return;
    for (int i = g.gw; i < n; i += g.ngroups) {
        double acc[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) acc[m] = 0.0;
        const double* row = Ainv + (size_t)i * n;
        for (int j = 0; j < n; ++j) {
            const double a = __ldg(row + j);
            TI bv[CPL];
            ld_cols<VEC, false, CPL>(B + (size_t)j * ld + c0, bv, k - c0);
#pragma unroll
            for (int m = 0; m < CPL; ++m) acc[m] = fma(a, (double)bv[m], acc[m]);
        }
        TO xo[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) xo[m] = (TO)acc[m];
        st_cols<VEC, CPL>(X + (size_t)i * ld + c0, xo, c0, k);
    }
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

// out = x + P e + omega M^-1 r - (omega M^-1 A P) e (the stored A P values
// carry the row scaling); on level 0 also r_cg . out and
// (flexible CG) q . out per column.
template <typename T, typename TO, int CPL, bool DOT, bool VEC>
__global__ void __launch_bounds__(TPB) bk_post(SellV SAP, const T* __restrict__ apval, const T* __restrict__ minv,
                                               T omega, const int* __restrict__ agg, const T* __restrict__ p,
                                               const T* __restrict__ E, const T* __restrict__ X,
                                               const T* __restrict__ R, const double* __restrict__ Bdot,
                                               const double* __restrict__ Q2, TO* __restrict__ Out, int k, int ld, int G,
                                               double* partial, unsigned* ticket, BlockScalars sc, int flexible) {
    const Grp g = make_grp(G);
    const int c0 = g.gl * CPL;
    double d0[CPL], d1[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) d0[m] = d1[m] = 0.0;
    if (c0 < k) {
        for (int ip = g.gw; ip < SAP.n; ip += g.ngroups) {
            T acc[CPL];
#pragma unroll
            for (int m = 0; m < CPL; ++m) acc[m] = 0;
            sell_row_k<VEC, false, CPL>(SAP, apval, ip, c0, k, E, ld, acc);
            const int i = rowid(SAP, ip);
            const int a = agg[i];
            const T pi = p[i];
            const T mi = omega * minv[i];
            const size_t o = (size_t)i * ld + c0;
            T ev[CPL], xv[CPL], rv[CPL];
            TO ov[CPL];
            ld_cols<VEC, false, CPL>(E + (size_t)a * ld + c0, ev, k - c0);
            ld_cols<VEC, false, CPL>(X + o, xv, k - c0);
            ld_cols<VEC, false, CPL>(R + o, rv, k - c0);
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                const T y = fma(pi, ev[m], xv[m]);
                ov[m] = (TO)(fma(mi, rv[m], y) - acc[m]);         // acc: rows of omega M^-1 A P
            }
            st_cols<VEC, CPL>(Out + o, ov, c0, k);
            if (DOT) {
                double bd[CPL], qd[CPL];
                ld_cols<VEC, false, CPL>(Bdot + o, bd, k - c0);
                if (Q2) ld_cols<VEC, false, CPL>(Q2 + o, qd, k - c0);
#pragma unroll
                for (int m = 0; m < CPL; ++m) {
                    if (c0 + m >= k) continue;
                    d0[m] = fma(bd[m], (double)ov[m], d0[m]);
                    if (Q2) d1[m] = fma(qd[m], (double)ov[m], d1[m]);
                }
            }
        }
    }
    if (DOT) colsum2<CPL>(d0, d1, g, k, ld, partial, ticket, [&](int c, double a, double b) { fin_rz(sc, c, a, b, flexible); });
}


// ------------------------------------- iterative coarsest solve, k columns
// CG with l1-Jacobi per column to ||r_c|| <= rtol ||b_c|| or maxit, FP64, all
// columns in one cooperative launch (the multi-column form of the
// single-column coarsest solve). Short rows come from the hybrid SELL layout
// through lane groups, rows kept out of it are split over the 32 lanes of a
// warp; per-column sums use one fixed reduction order, and every block sums
// the block partials in the same order after each grid barrier, so all blocks
// hold the same per-column scalars.
__device__ __forceinline__ unsigned long long bk_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned bk_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void bk_grid_sync(unsigned* count, unsigned epoch, int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        const unsigned target = epoch * gridDim.x;
        const unsigned long long t0 = bk_ns();
        while (bk_ld_acquire(count) < target) {
            if (bk_ns() - t0 > 2000000000ull) { atomicExch(err, 1); break; }
        }
        __threadfence();
    }
    __syncthreads();
}

// Block partial of one value per column into out[blockIdx.x * k + c].
template <int CPL>
__device__ __forceinline__ void bk_colpart(double (&v)[CPL], const Grp& g, int k, double* out) {
    __shared__ double sm[WARPS][MAXK];
#pragma unroll
    for (int m = 0; m < CPL; ++m)
        for (int o = g.G; o < 32; o <<= 1) v[m] += __shfl_xor_sync(FULL_MASK, v[m], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < g.G) {
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = lane * CPL + m;
            if (c < k) sm[warp][c] = v[m];
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double a = 0.0;
        for (int w = 0; w < WARPS; ++w) a += sm[w][c];
        out[(size_t)blockIdx.x * k + c] = a;
    }
    __syncthreads();
}

// dst[c] = sum over blocks of part[blk * k + c], same order in every block.
__device__ __forceinline__ void bk_colsum(const double* part, int k, double* dst) {
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double a = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) a += __ldcg(part + (size_t)b * k + c);
        dst[c] = a;
    }
    __syncthreads();
}

template <typename TI, typename TO, int CPL>
__global__ void __launch_bounds__(TPB) bk_coarse_cg(SellV S, const double* __restrict__ sval, int n, int nlong,
                                                    const int* __restrict__ long_rows, const int* __restrict__ cptr,
                                                    const int* __restrict__ ccol, const double* __restrict__ cval,
                                                    const double* __restrict__ minv, const TI* __restrict__ B,
                                                    TO* __restrict__ Xo, int k, int ld, int G, double* x, double* r,
                                                    double* z, double* p, double* q, double* part, unsigned* bar,
                                                    int* err, int maxit, double rtol) {
    __shared__ double s_rho[MAXK], s_bb[MAXK], s_t[MAXK];
    __shared__ int s_live[MAXK];
    __shared__ int s_any;
    const Grp g = make_grp(G);
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const size_t PK = (size_t)gridDim.x * k;
    unsigned epoch = 0;
    int red = 0;
    auto slot = [&]() { return part + (size_t)(red & 1) * PK; };
    double d0[CPL];
    // x = 0, r = b, z = M^-1 r, p = z; rho = r.z and bb = b.b per column
#pragma unroll
    for (int m = 0; m < CPL; ++m) d0[m] = 0.0;
    double d1[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) d1[m] = 0.0;
    for (int i = g.gw; i < n; i += g.ngroups) {
        const double mi = minv[i];
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = g.gl * CPL + m;
            if (c >= k) continue;
            const size_t o = (size_t)i * ld + c;
            const double bi = (double)B[o];
            x[o] = 0.0;
            r[o] = bi;
            const double zi = mi * bi;
            z[o] = zi;
            p[o] = zi;
            d0[m] = fma(bi, zi, d0[m]);
            d1[m] = fma(bi, bi, d1[m]);
        }
    }
    bk_colpart<CPL>(d0, g, k, slot());
    bk_colpart<CPL>(d1, g, k, slot() + PK * 2);
    bk_grid_sync(bar, ++epoch, err);
    if (__ldcg(err)) return;
    bk_colsum(slot(), k, s_rho);
    bk_colsum(slot() + PK * 2, k, s_bb);
    for (int c = threadIdx.x; c < k; c += blockDim.x) s_live[c] = s_bb[c] > 0.0;
    __syncthreads();
    ++red;
    for (int it = 0; it < maxit; ++it) {
        if (threadIdx.x == 0) {
            int a = 0;
            for (int c = 0; c < k; ++c) a |= s_live[c];
            s_any = a;
        }
        __syncthreads();
        if (!s_any) break;
        // q = A p, p . q
#pragma unroll
        for (int m = 0; m < CPL; ++m) d0[m] = 0.0;
        for (int ip = g.gw; ip < S.n; ip += g.ngroups) {
            double acc[CPL];
#pragma unroll
            for (int m = 0; m < CPL; ++m) acc[m] = 0.0;
            sell_row_k<false, true, CPL>(S, sval, ip, g.gl * CPL, k, (const double*)p, ld, acc);
            const int i = rowid(S, ip);
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                const int c = g.gl * CPL + m;
                if (c >= k) continue;
                const size_t o = (size_t)i * ld + c;
                q[o] = acc[m];
                d0[m] = fma(__ldcg(p + o), acc[m], d0[m]);
            }
        }
        for (int lr = gwarp; lr < nlong; lr += nwarps) {
            const int i = __ldg(long_rows + lr);
            const int e0 = __ldg(cptr + i), e1 = __ldg(cptr + i + 1);
            for (int c = 0; c < k; ++c) {
                double a = 0.0;
                for (int e = e0 + lane; e < e1; e += 32) a = fma(__ldg(cval + e), __ldcg(p + (size_t)__ldg(ccol + e) * ld + c), a);
                a = warp_sum(a);
                const size_t o = (size_t)i * ld + c;
                if (lane == 0) q[o] = a;
                // the first group of the warp carries the long rows' share of p . q
#pragma unroll
                for (int m = 0; m < CPL; ++m)
                    if (lane < G && lane * CPL + m == c) d0[m] = fma(__ldcg(p + o), a, d0[m]);
            }
        }
        bk_colpart<CPL>(d0, g, k, slot());
        bk_grid_sync(bar, ++epoch, err);
        if (__ldcg(err)) return;
        bk_colsum(slot(), k, s_t);
        ++red;
        // alpha per live column; x += alpha p, r -= alpha q; r.r
        double al[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = g.gl * CPL + m;
            al[m] = (c < k && s_live[c]) ? s_rho[c] / s_t[c] : 0.0;
            d0[m] = 0.0;
        }
        for (int i = g.gw; i < n; i += g.ngroups) {
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                const int c = g.gl * CPL + m;
                if (c >= k || al[m] == 0.0) continue;
                const size_t o = (size_t)i * ld + c;
                x[o] = fma(al[m], __ldcg(p + o), x[o]);
                const double ri = fma(-al[m], __ldcg(q + o), r[o]);
                r[o] = ri;
                d0[m] = fma(ri, ri, d0[m]);
            }
        }
        bk_colpart<CPL>(d0, g, k, slot());
        bk_grid_sync(bar, ++epoch, err);
        if (__ldcg(err)) return;
        bk_colsum(slot(), k, s_t);
        ++red;
        for (int c = threadIdx.x; c < k; c += blockDim.x)
            if (s_live[c] && s_t[c] <= rtol * rtol * s_bb[c]) s_live[c] = 0;
        __syncthreads();
        // z = M^-1 r; r.z; beta; p = z + beta p
#pragma unroll
        for (int m = 0; m < CPL; ++m) d0[m] = 0.0;
        for (int i = g.gw; i < n; i += g.ngroups) {
            const double mi = minv[i];
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                const int c = g.gl * CPL + m;
                if (c >= k || !s_live[c]) continue;
                const size_t o = (size_t)i * ld + c;
                const double zi = mi * r[o];
                z[o] = zi;
                d0[m] = fma(r[o], zi, d0[m]);
            }
        }
        bk_colpart<CPL>(d0, g, k, slot());
        bk_grid_sync(bar, ++epoch, err);
        if (__ldcg(err)) return;
        bk_colsum(slot(), k, s_t);
        ++red;
        double be[CPL];
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = g.gl * CPL + m;
            be[m] = (c < k && s_live[c]) ? s_t[c] / s_rho[c] : 0.0;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < k; c += blockDim.x)
            if (s_live[c]) s_rho[c] = s_t[c];
        for (int i = g.gw; i < n; i += g.ngroups) {
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                const int c = g.gl * CPL + m;
                if (c >= k || !s_live[c]) continue;
                const size_t o = (size_t)i * ld + c;
                p[o] = fma(be[m], p[o], z[o]);
            }
        }
        bk_grid_sync(bar, ++epoch, err);
        if (__ldcg(err)) return;
    }
    for (int i = g.gw; i < n; i += g.ngroups) {
#pragma unroll
        for (int m = 0; m < CPL; ++m) {
            const int c = g.gl * CPL + m;
            if (c < k) Xo[(size_t)i * ld + c] = (TO)x[(size_t)i * ld + c];
        }
    }
}

// ------------------------------------------------------------- CG ----------
// Q = A P; p . q per column; alpha = rho / p.q for ACTIVE columns, else 0.
template <int CPL, bool VEC>
__global__ void __launch_bounds__(TPB) bk_spmv_dot(SellV S, const double* __restrict__ val,
                                                   const double* __restrict__ P, double* __restrict__ Q, int k, int ld, int G,
                                                   double* partial, unsigned* ticket, BlockScalars sc) {
    const Grp g = make_grp(G);
    const int c0 = g.gl * CPL;
    double d0[CPL], d1[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) d0[m] = d1[m] = 0.0;
    if (c0 < k) {
        for (int ip = g.gw; ip < S.n; ip += g.ngroups) {
            double acc[CPL];
#pragma unroll
            for (int m = 0; m < CPL; ++m) acc[m] = 0.0;
            sell_row_k<VEC, false, CPL>(S, val, ip, c0, k, P, ld, acc);
            const int i = rowid(S, ip);
            const size_t o = (size_t)i * ld + c0;
            double pv[CPL];
            ld_cols<VEC, false, CPL>(P + o, pv, k - c0);
            st_cols<VEC, CPL>(Q + o, acc, c0, k);
#pragma unroll
            for (int m = 0; m < CPL; ++m)
                if (c0 + m < k) d0[m] = fma(pv[m], acc[m], d0[m]);
        }
    }
    colsum2<CPL>(d0, d1, g, k, ld, partial, ticket, [&](int c, double pq, double) {
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
// Other columns are written back unchanged when a vector store covers them.
template <int CPL, bool VEC>
__global__ void __launch_bounds__(TPB) bk_update_xr(int n, const double* __restrict__ P, const double* __restrict__ Q,
                                                    double* __restrict__ X, double* __restrict__ R, int k, int ld, int G,
                                                    double* partial, unsigned* ticket, BlockScalars sc) {
    const Grp g = make_grp(G);
    const int c0 = g.gl * CPL;
    double al[CPL];
    bool on[CPL];
    bool any = false;
#pragma unroll
    for (int m = 0; m < CPL; ++m) {
        const int c = c0 + m;
        on[m] = c < k && sc.mode[c] == COL_ACTIVE;
        al[m] = on[m] ? sc.alpha[c] : 0.0;
        any |= on[m];
    }
    double d0[CPL], d1[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) d0[m] = d1[m] = 0.0;
    if (any) {
        for (int i = g.gw; i < n; i += g.ngroups) {
            const size_t o = (size_t)i * ld + c0;
            double pv[CPL], qv[CPL], xv[CPL], rv[CPL];
            ld_cols<VEC, false, CPL>(P + o, pv, k - c0);
            ld_cols<VEC, false, CPL>(Q + o, qv, k - c0);
            ld_own<VEC, CPL>(X + o, xv, k - c0);
            ld_own<VEC, CPL>(R + o, rv, k - c0);
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                if (!on[m]) continue;
                xv[m] = fma(al[m], pv[m], xv[m]);
                rv[m] = fma(-al[m], qv[m], rv[m]);
                d0[m] = fma(rv[m], rv[m], d0[m]);
            }
            st_cols<VEC, CPL>(X + o, xv, c0, k);
            st_cols<VEC, CPL>(R + o, rv, c0, k);
        }
    }
    colsum2<CPL>(d0, d1, g, k, ld, partial, ticket, [&](int c, double rr, double) {
        if (sc.mode[c] != COL_ACTIVE) return;
        sc.rr[c] = rr;
        sc.iters[c] += 1;
        if (rr <= sc.rtol[c] * sc.rtol[c] * sc.bb[c]) sc.mode[c] = COL_CHECK;
    });
}

// ACTIVE columns: P = Z + beta P (P = Z when beta = 0, whatever P held).
template <int CPL, bool VEC>
__global__ void __launch_bounds__(TPB) bk_update_p(int n, const double* __restrict__ Z, double* __restrict__ P, int k,
                                                   int ld, int G, BlockScalars sc) {
    const Grp g = make_grp(G);
    const int c0 = g.gl * CPL;
    double be[CPL];
    bool on[CPL];
    bool any = false;
#pragma unroll
    for (int m = 0; m < CPL; ++m) {
        const int c = c0 + m;
        on[m] = c < k && sc.mode[c] == COL_ACTIVE;
        be[m] = on[m] ? sc.beta[c] : 0.0;
        any |= on[m];
    }
    if (!any) return;
    for (int i = g.gw; i < n; i += g.ngroups) {
        const size_t o = (size_t)i * ld + c0;
        double zv[CPL], pv[CPL];
        ld_cols<VEC, false, CPL>(Z + o, zv, k - c0);
        ld_own<VEC, CPL>(P + o, pv, k - c0);
#pragma unroll
        for (int m = 0; m < CPL; ++m)
            if (on[m]) pv[m] = be[m] == 0.0 ? zv[m] : fma(be[m], pv[m], zv[m]);
        st_cols<VEC, CPL>(P + o, pv, c0, k);
    }
}

// R = B - A X for the selected columns, ||R||^2 and ||B||^2.
//   stage 0 (start): INIT columns; DONE when ||B|| = 0 or x0 already meets
//                    rtol, else START.
//   stage 1 (check): CHECK columns; true residual below rtol -> DONE, else the
//                    column restarts from R (START).
//   stage 2 (report): every column; only records ||R||^2 in rr.
// Columns not selected keep their R when a vector store covers them.
template <int CPL, bool VEC>
__global__ void __launch_bounds__(TPB) bk_residual(SellV S, const double* __restrict__ val,
                                                   const double* __restrict__ X, const double* __restrict__ B,
                                                   double* __restrict__ R, int k, int ld, int G, double* partial,
                                                   unsigned* ticket, BlockScalars sc, int stage) {
    const Grp g = make_grp(G);
    const int c0 = g.gl * CPL;
    bool on[CPL];
    bool any = false;
#pragma unroll
    for (int m = 0; m < CPL; ++m) {
        const int c = c0 + m;
        const int md = c < k ? sc.mode[c] : COL_IDLE;
        on[m] = c < k && (stage == 0 ? md == COL_INIT : (stage == 1 ? md == COL_CHECK : true));
        any |= on[m];
    }
    double d0[CPL], d1[CPL];
#pragma unroll
    for (int m = 0; m < CPL; ++m) d0[m] = d1[m] = 0.0;
    if (any) {
        for (int ip = g.gw; ip < S.n; ip += g.ngroups) {
            double acc[CPL];
#pragma unroll
            for (int m = 0; m < CPL; ++m) acc[m] = 0.0;
            sell_row_k<VEC, false, CPL>(S, val, ip, c0, k, X, ld, acc);
            const int i = rowid(S, ip);
            const size_t o = (size_t)i * ld + c0;
            double bv[CPL], rv[CPL];
            ld_cols<VEC, false, CPL>(B + o, bv, k - c0);
            ld_own<VEC, CPL>(R + o, rv, k - c0);
#pragma unroll
            for (int m = 0; m < CPL; ++m) {
                if (!on[m]) continue;
                rv[m] = bv[m] - acc[m];
                d0[m] = fma(rv[m], rv[m], d0[m]);
                d1[m] = fma(bv[m], bv[m], d1[m]);
            }
            st_cols<VEC, CPL>(R + o, rv, c0, k);
        }
    }
    colsum2<CPL>(d0, d1, g, k, ld, partial, ticket, [&](int c, double rr, double bb) {
        const int md = sc.mode[c];
        if (stage == 0) {
            if (md != COL_INIT) return;
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

// Slot lists of a request (at most MAXK slots) passed by value.
struct SlotList {
    int n;
    int slot[MAXK];
};

// dst[:, slot[j]] = src[:, j] (src row-major n x k contiguous, dst row stride ld);
// with src == nullptr the slot columns are zeroed.
__global__ void bk_scatter_slots(int n, const double* __restrict__ src, int ld, double* __restrict__ dst,
                                 SlotList sl) {
    const int k = sl.n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * k;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = t / k;
        const int j = (int)(t % k);
        dst[i * ld + sl.slot[j]] = src ? src[t] : 0.0;
    }
}

// dst[:, j] = src[:, slot] for one slot column j of a request (dst n x k).
__global__ void bk_gather_slot(int n, const double* __restrict__ src, int ld, int slot, double* __restrict__ dst,
                               int k, int j) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[(size_t)i * k + j] = src[(size_t)i * ld + slot];
}

__global__ void bk_zero_cols(int n, double* __restrict__ X, int k, int ld, const int* __restrict__ mode,
                             const double* __restrict__ bb) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * k;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % k);
        const long long i = t / k;
        if (bb[c] == 0.0 && mode[c] == COL_DONE) X[i * ld + c] = 0.0;
    }
}

// ------------------------------------------------------------- host --------
SellV sv(const DevSell& S) { return SellV{S.n, S.nslices, S.sptr, S.col, S.perm}; }

int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Group width and columns per lane for k active columns. With a fixed width
// (set by the slot count K, not by k) a column's arithmetic and reduction
// order do not depend on how many columns are in flight.
// The default width gives each lane one vector's worth of columns (4 floats
// or 2 doubles) when the columns fill the group.
void group_shape(const BlockWork& W, int k, int* G, int* cpl) {
    int g = std::min(32, std::max(1, pow2_at_least(W.fixed_width ? W.K : k) / W.vec_cols));
    if (W.tuned_G && !W.fixed_width) g = std::min(W.tuned_G, pow2_at_least(k));
    *G = g;
    *cpl = pow2_at_least((k + g - 1) / g);
}

// CPL columns per lane, as vectors (VEC) when the row stride ld is a multiple of CPL.
#define DISPATCH_ONE(cpl_, vec, ...)                                                               \
    if (vec) { constexpr int CPL = cpl_; constexpr bool VEC = true; (void)VEC; __VA_ARGS__; }        \
    else { constexpr int CPL = cpl_; constexpr bool VEC = false; (void)VEC; __VA_ARGS__; }
#define DISPATCH_CPL(cpl, ld, ...)                                                                 \
    do {                                                                                           \
        const bool vec_ = (cpl) > 1 && (ld) % (cpl) == 0;                                          \
        switch (cpl) {                                                                             \
            case 1: { constexpr int CPL = 1; constexpr bool VEC = false; (void)VEC; __VA_ARGS__; } break; \
            case 2: { DISPATCH_ONE(2, vec_, __VA_ARGS__) } break;                                   \
            case 4: { DISPATCH_ONE(4, vec_, __VA_ARGS__) } break;                                   \
            default: { DISPATCH_ONE(8, vec_, __VA_ARGS__) } break;                                  \
        }                                                                                          \
    } while (0)

int grid_rows(const amg_hierarchy* h, long long rows, int G) {
    const long long groups_per_block = (long long)WARPS * (32 / G);
    return blocks_for(rows, (int)groups_per_block, h->num_sms * 8);
}

// Z = B R for columns [0, k) (block V-cycle); level 0 finishes r . z per column.
template <typename T>
void block_vcycle(amg_hierarchy* h, BlockWork& W, int k, int flexible) {
    cudaStream_t st = h->stream;
    const int ld = W.K;
    const int L = (int)h->lev.size() - 1;
    const bool f32 = sizeof(T) == 4;
    const T omega = (T)h->opt.omega;
    int G, cpl;
    group_shape(W, k, &G, &cpl);
    auto lv = [&](std::vector<void*>& v, int l) { return static_cast<T*>(v[l]); };
    for (int l = 0; l < L; ++l) {
        Level& Lv = h->lev[l];
        const T* valm = f32 ? (const T*)Lv.valm32 : (const T*)Lv.valm;
        const T* minv = f32 ? (const T*)Lv.minv32 : (const T*)Lv.minv;
        const int g = grid_rows(h, Lv.S.n, G);
        Scope sc_(&h->prof, st, l == 0 ? K_PRE_L0 : K_PRE,
                  (double)Lv.A.nnz * (sizeof(T) + 4) + (double)Lv.A.n * k * ((l == 0 ? 8 : sizeof(T)) + 2.0 * sizeof(T)));
        if (l == 0 && f32) {
            bk_to_f32<<<blocks_for((long long)Lv.A.n * ld, TPB, h->num_sms * 8), TPB, 0, st>>>(
                Lv.A.n, k, ld, W.R, reinterpret_cast<float*>(W.b[0]));
            KERNEL_CHECK();
        }
        if (l == 0 && !f32)
            DISPATCH_CPL(cpl, ld, bk_pre<T, CPL, VEC><<<g, TPB, 0, st>>>(sv(Lv.S), valm, minv, omega, (const T*)W.R, lv(W.x, 0),
                                                                       lv(W.r, 0), k, ld, G));
        else
            DISPATCH_CPL(cpl, ld, bk_pre<T, CPL, VEC><<<g, TPB, 0, st>>>(sv(Lv.S), valm, minv, omega, lv(W.b, l), lv(W.x, l),
                                                                  lv(W.r, l), k, ld, G));
        KERNEL_CHECK();
        const int nc = h->lev[l + 1].A.n;
        const T* p = f32 ? (const T*)Lv.p32 : (const T*)Lv.p;
        DISPATCH_CPL(cpl, ld, bk_restrict<T, CPL, VEC><<<grid_rows(h, nc, G), TPB, 0, st>>>(nc, Lv.pt_ptr, Lv.pt_idx, p,
                                                                                   lv(W.r, l), lv(W.b, l + 1), k, ld, G));
        KERNEL_CHECK();
    }
    {
        Scope sc_(&h->prof, st, K_COARSE, 8.0 * h->nc * h->nc + 16.0 * h->nc * k);
        if (!h->coarse_cg) {
            DISPATCH_CPL(cpl, ld, bk_coarse_dense<T, T, CPL, VEC><<<grid_rows(h, h->nc, G), TPB, 0, st>>>(
                                  h->nc, h->coarse_inv, lv(W.b, L), lv(W.x, L), k, ld, G));
            KERNEL_CHECK();
        } else {
            Level& Lc = h->lev[L];
            const SellV Sc = sv(Lc.S);
            const double* sval = Lc.S.val;
            int nrows = Lc.A.n, nlong = Lc.S.nlong, kk = k, ldd = ld, GG = G, maxit = 30;
            const int* long_rows = Lc.S.long_rows;
            const int* cptr = Lc.A.ptr;
            const int* ccol = Lc.A.col;
            const double* cval = Lc.A.val;
            const double* cminv = Lc.minv;
            const T* bin = lv(W.b, L);
            T* xout = lv(W.x, L);
            double rtol = 1e-4;
            unsigned* bar = reinterpret_cast<unsigned*>(W.cctl);
            int* err = W.cctl + 1;
            CUDA_CHECK(cudaMemsetAsync(W.cctl, 0, sizeof(int) * 4, st));
            void* args[] = {(void*)&Sc, (void*)&sval, &nrows, &nlong, (void*)&long_rows, (void*)&cptr, (void*)&ccol,
                            (void*)&cval, (void*)&cminv, (void*)&bin, (void*)&xout, &kk, &ldd, &GG, &W.cw[0],
                            &W.cw[1], &W.cw[2], &W.cw[3], &W.cw[4], &W.cpart, &bar, &err, &maxit, &rtol};
            const void* fn = nullptr;
            DISPATCH_CPL(cpl, ld, fn = (const void*)bk_coarse_cg<T, T, CPL>);
            CUDA_CHECK(cudaLaunchCooperativeKernel(fn, dim3(h->num_sms), dim3(TPB), args, 0, st));
            KERNEL_CHECK();
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
                  (double)Lv.ap_nnz * (sizeof(T) + 4) + (double)Lv.A.n * k * (4.0 * sizeof(T) + 8));
        if (l > 0)
            DISPATCH_CPL(cpl, ld, bk_post<T, T, CPL, false, VEC><<<g, TPB, 0, st>>>(
                                  sv(Lv.AP), apv, minv, omega, Lv.agg, p, e, lv(W.x, l), lv(W.r, l), nullptr, nullptr,
                                  lv(W.y, l), k, ld, G, W.partial, W.ticket, W.sc, flexible));
        else
            DISPATCH_CPL(cpl, ld, bk_post<T, double, CPL, true, VEC><<<W.grid, TPB, 0, st>>>(
                                  sv(Lv.AP), apv, minv, omega, Lv.agg, p, e, lv(W.x, 0), lv(W.r, 0), W.R,
                                  flexible ? W.Q : nullptr, W.Z, k, ld, G, W.partial, W.ticket, W.sc, flexible));
        KERNEL_CHECK();
    }
}

// Lanes per row of the block V-cycle (G; each lane carries ceil(K/G)
// columns, at most 8): the candidates are timed on one V-cycle of all K
// columns, on zeroed work vectors, and the fastest is cached by shape.
void block_autotune(amg_hierarchy* h, BlockWork& W) {
    const bool f32 = h->opt.precision == AMG_FP32_VCYCLE;
    const int V = f32 ? 4 : 8;
    const Level& L0 = h->lev[0];
    const std::string key = tune_key("block", V, L0.A.n, L0.A.nnz, (long long)h->lev.size(), W.K, h->num_sms);
    int best = 0;
    if (!tune_get(key, &best)) {
        cudaStream_t st = h->stream;
        for (size_t l = 0; l < h->lev.size(); ++l) {
            const size_t m = (size_t)h->lev[l].A.n * W.K * V;
            for (void* v : {W.b[l], W.x[l], W.r[l], W.y[l]}) CUDA_CHECK(cudaMemsetAsync(v, 0, m, st));
        }
        const size_t m0 = (size_t)L0.A.n * W.K * 8;
        for (double* v : {W.R, W.Z, W.Q}) CUDA_CHECK(cudaMemsetAsync(v, 0, m0, st));
        const bool prof_on = h->prof.on;
        h->prof.on = false;
        double tbest = 1e30;
        try {
            for (int G = std::min(32, pow2_at_least(W.K)); G >= 1; G /= 2) {
                if (pow2_at_least((W.K + G - 1) / G) > 8) break;
                W.tuned_G = G;
                const double t = time_launches(st, [&]() {
                    if (f32) block_vcycle<float>(h, W, W.K, 0);
                    else block_vcycle<double>(h, W, W.K, 0);
                }, 2);
                if (t < tbest) {
                    tbest = t;
                    best = G;
                }
            }
        } catch (...) {
            h->prof.on = prof_on;
            W.tuned_G = 0;
            throw;
        }
        h->prof.on = prof_on;
        CUDA_CHECK(cudaMemsetAsync(W.sc.mode, 0, sizeof(int) * W.K, st));
        CUDA_CHECK(cudaMemsetAsync(W.sc.iters, 0, sizeof(int) * W.K, st));
        CUDA_CHECK(cudaStreamSynchronize(st));
        tune_put(key, best);
    }
    W.tuned_G = best;
}

void copy_state_async(amg_hierarchy* h, BlockWork& W) {
    cudaStream_t st = h->stream;
    CUDA_CHECK(cudaMemcpyAsync(W.mode_host, W.sc.mode, sizeof(int) * W.K, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(W.iters_host, W.sc.iters, sizeof(int) * W.K, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(W.rr_host, W.sc.rr, sizeof(double) * W.K, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(W.bb_host, W.sc.bb, sizeof(double) * W.K, cudaMemcpyDeviceToHost, st));
}

}  // namespace

BlockWork& block_ensure(amg_hierarchy* h, int K, bool fixed_width) {
    if (h->blk && h->blk->K == K && h->blk->fixed_width == fixed_width) return *h->blk;
    if (K < 1 || K > MAXK) AMG_THROW(AMG_ERR_TOO_LARGE, "block solves take 1..%d columns", MAXK);
    if (h->opt.pre != 1 || h->opt.post != 1) AMG_THROW(AMG_ERR_ARG, "block solves use 1+1 smoothing sweeps");
    if (h->lev.size() < 2) AMG_THROW(AMG_ERR_ARG, "block solves need at least two levels");
    if (!h->seg0.empty()) AMG_THROW(AMG_ERR_ARG, "block solves take a hierarchy of one system");
    if (h->opt.cycle > 0 || h->opt.smooth_p) AMG_THROW(AMG_ERR_ARG, "block solves use the unsmoothed V-cycle");
    if (h->blk) {
        CUDA_CHECK(cudaStreamSynchronize(h->stream));
        delete h->blk;
        h->blk = nullptr;
    }
    BlockWork* W = new BlockWork;
    W->mem.stream = h->stream;
    h->blk = W;
    W->K = K;
    W->fixed_width = fixed_width;
    const bool f32 = h->opt.precision == AMG_FP32_VCYCLE;
    W->vec_cols = f32 ? 4 : 2;
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
    for (int c = 0; c < K; ++c) W->mode_host[c] = COL_IDLE;
    if (h->coarse_cg) {
        for (int v = 0; v < 5; ++v) W->cw[v] = W->mem.alloc<double>((size_t)h->nc * K);
        W->cpart = W->mem.alloc<double>((size_t)h->num_sms * K * 4);
        W->cctl = W->mem.alloc<int>(4);
        int per_sm = 0;
        CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bk_coarse_cg<double, double, 8>, TPB, 0));
        if (per_sm < 1) AMG_THROW(AMG_ERR_CUDA, "multi-column coarsest CG kernel cannot be resident");
    }
    if (h->opt.autotune && !fixed_width) block_autotune(h, *W);
    return *W;
}

size_t block_bytes_per_column(const amg_hierarchy* h) {
    const size_t V = h->opt.precision == AMG_FP32_VCYCLE ? 4 : 8;
    size_t rows = 0;
    for (auto& L : h->lev) rows += (size_t)L.A.n;
    return rows * 4 * V + (size_t)h->lev[0].A.n * 5 * 8;
}

// INIT columns among [0, k): residual of X, then START (or DONE for b = 0,
// whose X column is zeroed). Launches only.
void block_init_launch(amg_hierarchy* h, const double* B, double* X, int k) {
    BlockWork& W = *h->blk;
    cudaStream_t st = h->stream;
    int G, cpl;
    group_shape(W, k, &G, &cpl);
    Level& L0 = h->lev[0];
    DISPATCH_CPL(cpl, W.K, bk_residual<CPL, VEC><<<W.grid, TPB, 0, st>>>(sv(L0.S), L0.S.val, X, B, W.R, k, W.K, G, W.partial,
                                                             W.ticket, W.sc, 0));
    KERNEL_CHECK();
    bk_zero_cols<<<blocks_for((long long)L0.A.n * k, TPB, h->num_sms * 8), TPB, 0, st>>>(L0.A.n, X, k, W.K, W.sc.mode,
                                                                                      W.sc.bb);
    KERNEL_CHECK();
}

namespace {

// The kernels of one step of columns [0, k): with `any_active` the CG half
// (q = A p, x and r updates), then the V-cycle and p = z + beta p.
void block_step_kernels(amg_hierarchy* h, double* X, int k, bool any_active) {
    BlockWork& W = *h->blk;
    cudaStream_t st = h->stream;
    const int ld = W.K;
    const int flexible = h->opt.krylov == 1;
    int G, cpl;
    group_shape(W, k, &G, &cpl);
    Level& L0 = h->lev[0];
    const int n = L0.A.n;
    const double nnz = (double)L0.A.nnz;
    if (any_active) {
        {
            Scope sc_(&h->prof, st, K_SPMV_DOT, 12.0 * nnz + 16.0 * n * k);
            DISPATCH_CPL(cpl, ld, bk_spmv_dot<CPL, VEC><<<W.grid, TPB, 0, st>>>(sv(L0.S), L0.S.val, W.P, W.Q, k, ld, G,
                                                                     W.partial, W.ticket, W.sc));
            KERNEL_CHECK();
        }
        {
            Scope sc_(&h->prof, st, K_UPDATE_XR, 48.0 * n * k);
            DISPATCH_CPL(cpl, ld, bk_update_xr<CPL, VEC><<<W.grid, TPB, 0, st>>>(n, W.P, W.Q, X, W.R, k, ld, G, W.partial,
                                                                      W.ticket, W.sc));
            KERNEL_CHECK();
        }
    }
    if (h->opt.precision == AMG_FP32_VCYCLE) block_vcycle<float>(h, W, k, flexible);
    else block_vcycle<double>(h, W, k, flexible);
    {
        Scope sc_(&h->prof, st, K_UPDATE_P, 24.0 * n * k);
        DISPATCH_CPL(cpl, ld, bk_update_p<CPL, VEC><<<grid_rows(h, n, G), TPB, 0, st>>>(n, W.Z, W.P, k, ld, G, W.sc));
        KERNEL_CHECK();
    }
}

bool any_active_column(const BlockWork& W, int k) {
    for (int c = 0; c < k; ++c)
        if (W.mode_host[c] == COL_ACTIVE) return true;
    return false;
}

// The same step as one CUDA graph launch: the step's kernels are captured
// once per (active columns or not) on a private stream (the caller's may be
// the legacy default stream, which cannot capture) and replayed on the
// hierarchy's stream. Used while profiling is off and the coarsest level is
// dense (the coarsest CG is a cooperative launch).
void block_step_graph(amg_hierarchy* h, double* X, int k) {
    BlockWork& W = *h->blk;
    if (W.gk != k || W.gX != X) {
        for (auto& g : W.gstep)
            if (g) {
                CUDA_CHECK(cudaGraphExecDestroy(g));
                g = nullptr;
            }
        W.gk = k;
        W.gX = X;
    }
    const bool act = any_active_column(W, k);
    cudaGraphExec_t& ge = W.gstep[act ? 1 : 0];
    if (!ge) {
        cudaStream_t st = h->stream;
        cudaStream_t cs = nullptr;
        CUDA_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        h->stream = cs;
        cudaGraph_t graph = nullptr;
        try {
            CUDA_CHECK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            const long long before = launch_counter().load();
            try {
                block_step_kernels(h, X, k, act);
                W.gkernels[act ? 1 : 0] = launch_counter().load() - before;
            } catch (...) {
                cudaStreamEndCapture(cs, &graph);
                if (graph) cudaGraphDestroy(graph);
                throw;
            }
            CUDA_CHECK(cudaStreamEndCapture(cs, &graph));
            CUDA_CHECK(cudaGraphInstantiate(&ge, graph, 0));
            CUDA_CHECK(cudaGraphDestroy(graph));
        } catch (...) {
            h->stream = st;
            cudaStreamDestroy(cs);
            throw;
        }
        h->stream = st;
        CUDA_CHECK(cudaStreamDestroy(cs));
    }
    CUDA_CHECK(cudaGraphLaunch(ge, h->stream));
    launch_counter().fetch_add(W.gkernels[act ? 1 : 0], std::memory_order_relaxed);
    copy_state_async(h, W);
}

}  // namespace

// One step of columns [0, k) (see the file comment), then an asynchronous
// copy of the column states to the host mirrors. Launches only.
void block_step_launch(amg_hierarchy* h, const double* B, double* X, int k) {
    (void)B;
    BlockWork& W = *h->blk;
    block_step_kernels(h, X, k, any_active_column(W, k));
    copy_state_async(h, W);
}

// After a synchronised step: true residual of the CHECK columns (DONE or
// restart). Returns whether anything was launched.
bool block_check_launch(amg_hierarchy* h, const double* B, double* X, int k) {
    BlockWork& W = *h->blk;
    bool any_check = false;
    for (int c = 0; c < k; ++c) any_check |= W.mode_host[c] == COL_CHECK;
    if (!any_check) return false;
    int G, cpl;
    group_shape(W, k, &G, &cpl);
    Level& L0 = h->lev[0];
    const double nnz = (double)L0.A.nnz;
    Scope sc_(&h->prof, h->stream, K_RESIDUAL, 12.0 * nnz + 24.0 * L0.A.n * k);
    DISPATCH_CPL(cpl, W.K, bk_residual<CPL, VEC><<<W.grid, TPB, 0, h->stream>>>(sv(L0.S), L0.S.val, X, B, W.R, k, W.K, G,
                                                                    W.partial, W.ticket, W.sc, 1));
    KERNEL_CHECK();
    copy_state_async(h, W);
    return true;
}

void block_report_launch(amg_hierarchy* h, const double* B, const double* X, int k) {
    BlockWork& W = *h->blk;
    int G, cpl;
    group_shape(W, k, &G, &cpl);
    Level& L0 = h->lev[0];
    DISPATCH_CPL(cpl, W.K, bk_residual<CPL, VEC><<<W.grid, TPB, 0, h->stream>>>(sv(L0.S), L0.S.val, X, B, W.T, k, W.K, G,
                                                                    W.partial, W.ticket, W.sc, 2));
    KERNEL_CHECK();
    copy_state_async(h, W);
}

void block_set_columns(amg_hierarchy* h, int c0, int cnt, int mode, double rtol) {
    BlockWork& W = *h->blk;
    std::vector<int> md(cnt, mode);
    std::vector<double> rt(cnt, rtol);
    std::vector<int> zi(cnt, 0);
    CUDA_CHECK(cudaMemcpyAsync(W.sc.mode + c0, md.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, h->stream));
    CUDA_CHECK(cudaMemcpyAsync(W.sc.rtol + c0, rt.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, h->stream));
    CUDA_CHECK(cudaMemcpyAsync(W.sc.iters + c0, zi.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, h->stream));
    // host buffers are pageable: make sure they are consumed before they go out of scope
    CUDA_CHECK(cudaStreamSynchronize(h->stream));
    for (int c = c0; c < c0 + cnt; ++c) W.mode_host[c] = mode;
}

amg_status solve_batch(amg_hierarchy* h, int k, const double* B, double* X, double rtol, int maxit,
                       amg_solve_info* infos) {
    auto t0 = std::chrono::steady_clock::now();
    BlockWork& W = block_ensure(h, k, false);
    block_set_columns(h, 0, k, COL_INIT, rtol);
    block_init_launch(h, B, X, k);
    copy_state_async(h, W);
    CUDA_CHECK(cudaStreamSynchronize(h->stream));
    int steps = 0;
    const bool graphs = !h->prof.on && !h->coarse_cg;
    for (;;) {
        bool live = false;
        int maxi = 0;
        for (int c = 0; c < k; ++c) {
            live |= W.mode_host[c] == COL_START || W.mode_host[c] == COL_ACTIVE;
            maxi = std::max(maxi, W.iters_host[c]);
        }
        if (!live || maxi >= maxit || ++steps > 4 * maxit + 16) break;
        if (graphs) block_step_graph(h, X, k);
        else block_step_launch(h, B, X, k);
        CUDA_CHECK(cudaStreamSynchronize(h->stream));
        if (block_check_launch(h, B, X, k)) CUDA_CHECK(cudaStreamSynchronize(h->stream));
    }
    block_report_launch(h, B, X, k);
    CUDA_CHECK(cudaStreamSynchronize(h->stream));
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

void block_scatter_request(amg_hierarchy* h, const double* src, int k, const int* slots, double* dst) {
    SlotList sl;
    sl.n = k;
    for (int j = 0; j < k; ++j) sl.slot[j] = slots[j];
    const int n = h->lev[0].A.n;
    bk_scatter_slots<<<blocks_for((long long)n * k, TPB, h->num_sms * 8), TPB, 0, h->stream>>>(n, src, h->blk->K, dst,
                                                                                            sl);
    KERNEL_CHECK();
}

void block_gather_column(amg_hierarchy* h, const double* src, int slot, double* dst, int k, int j) {
    const int n = h->lev[0].A.n;
    bk_gather_slot<<<blocks_for(n, TPB, h->num_sms * 4), TPB, 0, h->stream>>>(n, src, h->blk->K, slot, dst, k, j);
    KERNEL_CHECK();
}

}  // namespace amg
