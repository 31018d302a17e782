// solve.cu -- V-cycle (Eq. 2) with l1-Jacobi smoothing and preconditioned CG.
//
// Every level holds its matrix in SELL-32: one warp per 32-row slice, one
// lane per row, entries of a slice stored column-major so that each step of
// the row loop is one fully coalesced 128-byte (float) / 256-byte (double)
// load of values and a 128-byte load of column indices.
//
// V-cycle for level l < L (input b_l, zero initial guess):
//   pre-smooth + residual (fused):  x = omega M^-1 b;  r = b - A x
//   restriction:                    b_{l+1} = P^T r   (member lists, no atomics)
//   coarse correction:              e = B_{l+1} b_{l+1}
//   prolongation + post-smooth (fused): y = x + P e;  y += omega M^-1 (b - A y)
// where the neighbours' x, resp. x + P e, are recomputed inside the row loop
// instead of being stored and re-read. On level 0 the post-smoothing kernel
// also forms the dot product r . z needed by CG.
#include <chrono>
#include <cmath>

#include "amg_internal.cuh"
#include "device_util.cuh"

namespace amg {

namespace {

constexpr int TPB = 256;
constexpr int WARPS = TPB / 32;

enum FinMode : int {
    FIN_NORMS = 0, FIN_PQ = 1, FIN_RR = 2, FIN_RHO_INIT = 3, FIN_RHO_UPDATE = 4, FIN_NONE = 5, FIN_RHO_UPDATE_FCG = 6
};

__device__ void finish(int mode, double a, double b, PcgScalars* sc) {
    switch (mode) {
        case FIN_NORMS: sc->rr = a; sc->bb = b; break;
        case FIN_PQ: {
            sc->pq = a;
            const double alpha = sc->rho / a;
            sc->alpha = alpha;
            if (!(a > 0.0) || !isfinite(alpha)) sc->breakdown = 1;
            break;
        }
        case FIN_RR: sc->rr = a; break;
        case FIN_RHO_INIT: sc->rho = a; if (!isfinite(a)) sc->breakdown = 1; break;
        case FIN_RHO_UPDATE: {
            const double beta = a / sc->rho;
            sc->rho_new = a;
            sc->beta = beta;
            sc->rho = a;
            if (!isfinite(beta)) sc->breakdown = 1;
            break;
        }
        case FIN_RHO_UPDATE_FCG: {
            // flexible CG, one direction kept: beta = z'^T (r' - r) / rho with
            // r' - r = -alpha q, so beta = -alpha (z' . q) / rho  (b = z' . q)
            const double beta = -sc->alpha * b / sc->rho;
            sc->rho_new = a;
            sc->beta = beta;
            sc->rho = a;
            if (!isfinite(beta)) sc->breakdown = 1;
            break;
        }
        default: break;
    }
}

// Block partial sums, then the last block to arrive combines all partials in
// a fixed order (deterministic for a fixed grid) and calls fin(sum_a, sum_b)
// on one thread.
template <typename FIN>
__device__ __forceinline__ void reduce_then(double a, double b, Reducer red, FIN&& fin) {
    __shared__ bool last;
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        red.partial[2 * blockIdx.x] = a;
        red.partial[2 * blockIdx.x + 1] = b;
        __threadfence();
        last = atomicAdd(red.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double sa = 0.0, sb = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        sa += __ldcg(&red.partial[2 * k]);
        sb += __ldcg(&red.partial[2 * k + 1]);
    }
    sa = block_sum(sa);
    sb = block_sum(sb);
    if (threadIdx.x == 0) {
        fin(sa, sb);
        *red.ticket = 0u;
    }
}

__device__ __forceinline__ void reduce_and_finish(double a, double b, Reducer red, PcgScalars* sc, int mode) {
    reduce_then(a, b, red, [&](double sa, double sb) { finish(mode, sa, sb, sc); });
}

struct SellView {
    int n, nslices;
    const int* __restrict__ sptr;
    const int* __restrict__ col;
    const int* __restrict__ perm;   // row held by slice position (null: identity)
};

// Row index held by SELL position ip (rows may be permuted by length).
__device__ __forceinline__ int sell_rowid(const SellView& S, int ip) { return S.perm ? __ldg(S.perm + ip) : ip; }

template <typename T>
__device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

// Row dot product of one SELL slice lane: sum_k val[k] * xv(col[k]). The
// loop is unrolled by four so that the column, value and gather loads of four
// entries are in flight together. Two accumulators shorten the FMA chain
// (latency-bound kernels); one accumulator saves the final add, which pays in
// the fused smoothers, where the FP64 pipe (this GPU's FP64 rate is 1/64 of
// its FP32 rate) is the bound.
template <typename T, int NACC = 2, typename F>
__device__ __forceinline__ T sell_row(const int* __restrict__ col, const T* __restrict__ val, long long base, int w,
                                      F&& xv) {
    T a0 = 0, a1 = 0;
    int k = 0;
    for (; k + 4 <= w; k += 4, base += 128) {
        const int j0 = ld(col + base), j1 = ld(col + base + 32), j2 = ld(col + base + 64), j3 = ld(col + base + 96);
        const T v0 = ld(val + base), v1 = ld(val + base + 32), v2 = ld(val + base + 64), v3 = ld(val + base + 96);
        const T x0 = xv(j0), x1 = xv(j1), x2 = xv(j2), x3 = xv(j3);
        if (NACC == 1) {
            a0 = fma(v0, x0, a0);
            a0 = fma(v1, x1, a0);
            a0 = fma(v2, x2, a0);
            a0 = fma(v3, x3, a0);
        } else {
            a0 = fma(v0, x0, a0);
            a1 = fma(v1, x1, a1);
            a0 = fma(v2, x2, a0);
            a1 = fma(v3, x3, a1);
        }
    }
    for (; k < w; ++k, base += 32) a0 = fma(ld(val + base), xv(ld(col + base)), a0);
    return NACC == 1 ? a0 : a0 + a1;
}

#define SELL_LOOP(S)                                                                 \
    const int lane = threadIdx.x & 31;                                               \
    const int nw_ = gridDim.x * WARPS;                                               \
    for (int s = blockIdx.x * WARPS + (threadIdx.x >> 5); s < (S).nslices; s += nw_)

#define SELL_ROW_ARGS(S) (S).col, (long long)(S).sptr[s] * 32 + lane, (S).sptr[s + 1] - (S).sptr[s]

// --------------------------------------------------------- V-cycle ---------
// First pre-smoothing sweep from a zero guess, fused with the residual:
//   x = omega M^-1 b,  r = b - omega (A M^-1) b,
// with the column-scaled values valm = A M^-1 (one FMA per stored entry) and
// wm = omega M^-1. With U (one pre-smoothing sweep), x is not stored but
// u = x + omega M^-1 r = omega M^-1 (b + r), the part of the post-smoother
// that does not depend on the coarse correction.
template <typename T, typename TB, bool U>
__global__ void __launch_bounds__(TPB) k_pre(SellView S, const T* __restrict__ valm, const T* __restrict__ wm,
                                             T omega, const TB* __restrict__ b, T* __restrict__ x,
                                             T* __restrict__ r) {
    SELL_LOOP(S) {
        const T acc = sell_row<T, 1>(S.col, valm, (long long)S.sptr[s] * 32 + lane, S.sptr[s + 1] - S.sptr[s],
                               [&](int j) { return (T)ld(b + j); });
        const int ip = s * 32 + lane;
        if (ip < S.n) {
            const int i = sell_rowid(S, ip);
            const T bi = (T)b[i];
            const T ri = fma(-omega, acc, bi);
            r[i] = ri;
            x[i] = U ? wm[i] * (bi + ri) : wm[i] * bi;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(TPB) k_restrict(int nc, const int* __restrict__ pt_ptr, const int* __restrict__ pt_idx,
                                                  const T* __restrict__ p, const T* __restrict__ r, T* __restrict__ bc) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
        T s = 0;
        for (int k = pt_ptr[q]; k < pt_ptr[q + 1]; ++k) {
            const int i = pt_idx[k];
            s = fma(ld(p + i), ld(r + i), s);
        }
        bc[q] = s;
    }
}

// Coarse correction and first post-smoothing sweep, fused:
//   y = x + P e,  out = y + omega M^-1 (b - A y),
// evaluated as out = (x + omega M^-1 r) + P e - (omega M^-1 A P) e, since
// b - A y = r - A P e with r = b - A x from the pre-smoother. The stored
// apw = omega M^-1 A P has about half the entries of A and gathers only the
// short coarse vector e. With U the first term u = x + omega M^-1 r comes
// ready from the pre-smoother; otherwise it is formed here from x, r and
// wm = omega M^-1. With DOT, also bdot . out (r . z of CG on level 0),
// finished into the CG scalars. FP64 work per row: one FMA per entry of
// apw, two more, and the dot.
template <typename T, typename TB, typename TO, bool DOT, bool U>
__global__ void __launch_bounds__(TPB) k_post(SellView SAP, const T* __restrict__ apw, const T* __restrict__ wm,
                                              const int* __restrict__ agg, const T* __restrict__ p,
                                              const T* __restrict__ e, const T* __restrict__ x,
                                              const T* __restrict__ r, const TB* __restrict__ bdot,
                                              TO* __restrict__ out, Reducer red, PcgScalars* sc, int mode,
                                              const double* __restrict__ q2) {
    double dot = 0.0, dot2 = 0.0;
    SELL_LOOP(SAP) {
        const T acc = sell_row<T, 1>(SAP.col, apw, (long long)SAP.sptr[s] * 32 + lane, SAP.sptr[s + 1] - SAP.sptr[s],
                               [&](int q) { return ld(e + q); });
        const int ip = s * 32 + lane;
        if (ip < SAP.n) {
            const int i = sell_rowid(SAP, ip);
            const T ui = U ? x[i] : fma(wm[i], r[i], x[i]);
            const T o = fma(p[i], e[agg[i]], ui) - acc;
            out[i] = (TO)o;
            if (DOT) {
                dot = fma((double)bdot[i], (double)(TO)o, dot);
                if (q2) dot2 = fma(q2[i], (double)(TO)o, dot2);
            }
        }
    }
    if (DOT) reduce_and_finish(dot, dot2, red, sc, mode);
}

template <typename T, typename TB>
void launch_pre(bool u, int grid, cudaStream_t st, SellView S, const T* valm, const T* wm, T omega, const TB* b, T* x,
                T* r) {
    if (u) k_pre<T, TB, true><<<grid, TPB, 0, st>>>(S, valm, wm, omega, b, x, r);
    else k_pre<T, TB, false><<<grid, TPB, 0, st>>>(S, valm, wm, omega, b, x, r);
    KERNEL_CHECK();
}

template <typename T, typename TB, typename TO, bool DOT>
void launch_post(bool u, int grid, cudaStream_t st, SellView SAP, const T* apw, const T* wm, const int* agg,
                 const T* p, const T* e, const T* x, const T* r, const TB* bdot, TO* out, Reducer red, PcgScalars* sc,
                 int mode, const double* q2) {
    if (u) k_post<T, TB, TO, DOT, true><<<grid, TPB, 0, st>>>(SAP, apw, wm, agg, p, e, x, r, bdot, out, red, sc, mode, q2);
    else k_post<T, TB, TO, DOT, false><<<grid, TPB, 0, st>>>(SAP, apw, wm, agg, p, e, x, r, bdot, out, red, sc, mode, q2);
    KERNEL_CHECK();
}

// ------------------------------------------------------------ K-cycle ------
// The coarse correction of a K-cycle on level m: two flexible CG iterations
// on A_m e = b from e = 0, preconditioned by the cycle that starts on level m
// (Section 3.2). d1 = B b; q1 = A d1; alpha1 = d1.b / d1.q1; e = alpha1 d1;
// r2 = b - alpha1 q1; z2 = B r2; beta = z2.q1 / d1.q1; d2 = z2 - beta d1;
// q2 = A d2 = A z2 - beta q1; alpha2 = d2.r2 / d2.q2; e += alpha2 d2. The
// scalars stay on the device; dot products are summed in FP64.
enum KcMode : int { KC_ALPHA1 = 0, KC_BETA = 1, KC_ALPHA2 = 2 };

__device__ __forceinline__ void kc_finish(KcScalars* ks, int mode, double a, double b) {
    if (mode == KC_ALPHA1) {
        ks->rho1 = a;
        ks->alpha1 = a != 0.0 ? b / a : 0.0;
    } else if (mode == KC_BETA) {
        ks->beta = ks->rho1 != 0.0 ? a / ks->rho1 : 0.0;
    } else {
        ks->alpha2 = a != 0.0 ? b / a : 0.0;
    }
}

// q1 = A d1; d1.q1 and d1.b -> rho1, alpha1.
template <typename T>
__global__ void __launch_bounds__(TPB) k_kc_spmv_dot(SellView S, const T* __restrict__ val, const T* __restrict__ d1,
                                                     T* __restrict__ q1, const T* __restrict__ b, Reducer red,
                                                     KcScalars* ks) {
    double dq = 0.0, db = 0.0;
    SELL_LOOP(S) {
        const T acc = sell_row(S.col, val, (long long)S.sptr[s] * 32 + lane, S.sptr[s + 1] - S.sptr[s],
                               [&](int j) { return ld(d1 + j); });
        const int ip = s * 32 + lane;
        if (ip < S.n) {
            const int i = sell_rowid(S, ip);
            q1[i] = acc;
            const double di = (double)d1[i];
            dq = fma(di, (double)acc, dq);
            db = fma(di, (double)b[i], db);
        }
    }
    reduce_then(dq, db, red, [&](double a, double c) { kc_finish(ks, KC_ALPHA1, a, c); });
}

// e = alpha1 d1; r2 = b - alpha1 q1.
template <typename T>
__global__ void __launch_bounds__(TPB) k_kc_update1(int n, const T* __restrict__ d1, const T* __restrict__ q1,
                                                    const T* __restrict__ b, T* __restrict__ e, T* __restrict__ r2,
                                                    const KcScalars* ks) {
    const T a = (T)ks->alpha1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        e[i] = a * d1[i];
        r2[i] = fma(-a, q1[i], b[i]);
    }
}

// z2.q1 -> beta.
template <typename T>
__global__ void __launch_bounds__(TPB) k_kc_dot(int n, const T* __restrict__ z2, const T* __restrict__ q1, Reducer red,
                                                KcScalars* ks) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s = fma((double)z2[i], (double)q1[i], s);
    reduce_then(s, 0.0, red, [&](double a, double) { kc_finish(ks, KC_BETA, a, 0.0); });
}

// d2 = z2 - beta d1; q2 = A z2 - beta q1 (= A d2, without a second product);
// d2.q2 and d2.r2 -> alpha2.
template <typename T>
__global__ void __launch_bounds__(TPB) k_kc_spmv2(SellView S, const T* __restrict__ val, const T* __restrict__ z2,
                                                  const T* __restrict__ q1, const T* __restrict__ d1,
                                                  const T* __restrict__ r2, T* __restrict__ d2, Reducer red,
                                                  KcScalars* ks) {
    const T be = (T)ks->beta;
    double dq = 0.0, dr = 0.0;
    SELL_LOOP(S) {
        const T acc = sell_row(S.col, val, (long long)S.sptr[s] * 32 + lane, S.sptr[s + 1] - S.sptr[s],
                               [&](int j) { return ld(z2 + j); });
        const int ip = s * 32 + lane;
        if (ip < S.n) {
            const int i = sell_rowid(S, ip);
            const T q2 = fma(-be, q1[i], acc);
            const T di = fma(-be, d1[i], z2[i]);
            d2[i] = di;
            dq = fma((double)di, (double)q2, dq);
            dr = fma((double)di, (double)r2[i], dr);
        }
    }
    reduce_then(dq, dr, red, [&](double a, double c) { kc_finish(ks, KC_ALPHA2, a, c); });
}

// e += alpha2 d2.
template <typename T>
__global__ void __launch_bounds__(TPB) k_kc_update2(int n, const T* __restrict__ d2, T* __restrict__ e,
                                                    const KcScalars* ks) {
    const T a = (T)ks->alpha2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) e[i] = fma(a, d2[i], e[i]);
}

// ------------------------------------------- smoothed prolongator (SA) ----
// Restriction b_c = Pbar^T r (rows of Pbar^T in SELL).
template <typename T>
__global__ void __launch_bounds__(TPB) k_sell_spmv(SellView S, const T* __restrict__ val, const T* __restrict__ x,
                                                   T* __restrict__ y) {
    SELL_LOOP(S) {
        const T acc = sell_row(S.col, val, (long long)S.sptr[s] * 32 + lane, S.sptr[s + 1] - S.sptr[s],
                               [&](int j) { return ld(x + j); });
        const int ip = s * 32 + lane;
        if (ip < S.n) y[sell_rowid(S, ip)] = acc;
    }
}

// Wide rows (the dense coarse levels of smoothed hierarchies), FP64, CSR,
// one warp per row: lanes take the row's entries k = lane, lane + 32, ...,
// the partial sums meet in a shuffle reduction, lane 0 applies the row's
// step. s_i = sum_j v_ij x_j with v_ij = a_ij, or (a_ij m_j) x_j for W_PRE
// (the same rounded products as the column-scaled values of the SELL path).
//   W_SPMV    y_i = s_i                              (restriction Pbar^T r)
//   W_ADD     y_i = y_i + s_i                        (prolongation x + Pbar e)
//   W_PRE     y_i = b_i - omega s_i, xo_i = wm_i b_i (pre-smoothing from zero)
//   W_SMOOTH  y_i = x_i + omega m_i (b_i - s_i)      (smoothing sweep)
//   W_RES     y_i = b_i - s_i                           (residual)
enum WideOp : int { W_SPMV = 0, W_ADD = 1, W_PRE = 2, W_SMOOTH = 3, W_RES = 4 };
constexpr int WIDE_MIN_A = 64;   // mean entries per row from which a level matrix takes this path
constexpr int WIDE_MIN_P = 64;   // the same for Pbar and its transpose
template <int OP>
__global__ void __launch_bounds__(TPB) k_wide(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                                              const double* __restrict__ val, const double* __restrict__ x,
                                              const double* __restrict__ minv, const double* __restrict__ wm,
                                              double omega, const double* __restrict__ b, double* __restrict__ y,
                                              double* __restrict__ xo) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const int kb = ptr[i], ke = ptr[i + 1];
        double acc0 = 0.0, acc1 = 0.0;
        int k = kb + lane;
        auto xv = [&](int j) { return ld(x + j); };
        for (; k + 32 < ke; k += 64) {
            const int j0 = col[k], j1 = col[k + 32];
            const double v0 = OP == W_PRE ? val[k] * minv[j0] : val[k];
            const double v1 = OP == W_PRE ? val[k + 32] * minv[j1] : val[k + 32];
            acc0 = fma(v0, xv(j0), acc0);
            acc1 = fma(v1, xv(j1), acc1);
        }
        if (k < ke) {
            const int j0 = col[k];
            const double v0 = OP == W_PRE ? val[k] * minv[j0] : val[k];
            acc0 = fma(v0, xv(j0), acc0);
        }
        double acc = acc0 + acc1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);
        if (lane == 0) {
            if (OP == W_SPMV) y[i] = acc;
            if (OP == W_ADD) y[i] = y[i] + acc;
            if (OP == W_PRE) {
                const double bi = b[i];
                y[i] = fma(-omega, acc, bi);
                xo[i] = wm[i] * bi;
            }
            if (OP == W_SMOOTH) y[i] = fma(omega * minv[i], b[i] - acc, x[i]);
            if (OP == W_RES) y[i] = b[i] - acc;
        }
    }
}

bool wide(const DevCsr& M, int min_mean) { return M.n > 0 && (long long)M.nnz >= (long long)min_mean * M.n; }

// Prolongation x <- x + Pbar e (rows of Pbar in SELL).
template <typename T>
__global__ void __launch_bounds__(TPB) k_prolong(SellView S, const T* __restrict__ val, const T* __restrict__ e,
                                                 T* __restrict__ x) {
    SELL_LOOP(S) {
        const T acc = sell_row(S.col, val, (long long)S.sptr[s] * 32 + lane, S.sptr[s + 1] - S.sptr[s],
                               [&](int q) { return ld(e + q); });
        const int ip = s * 32 + lane;
        if (ip < S.n) {
            const int i = sell_rowid(S, ip);
            x[i] = x[i] + acc;
        }
    }
}

// FP32 copy of the level-0 residual for the FP32 V-cycle: one conversion per
// row here instead of one per gathered matrix entry in the sweep (on this GPU
// the FP64 -> FP32 conversion runs at the FP64 rate).
__global__ void __launch_bounds__(TPB) k_to_f32(int n, const double* __restrict__ a, float* __restrict__ b) {
    const int stride = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + stride < n; i += 2 * stride) {
        const double a0 = a[i], a1 = a[i + stride];
        b[i] = (float)a0;
        b[i + stride] = (float)a1;
    }
    if (i < n) b[i] = (float)a[i];
}

// Residual after the last of several pre-smoothing sweeps: r = b - A x.
// (Sweeps between the first and the last are k_smooth, the first is k_pre
// storing x + omega M^-1 r; each reads one gathered vector, one FMA per
// stored entry.)
template <typename T, typename TB>
__global__ void __launch_bounds__(TPB) k_resid(SellView S, const T* __restrict__ val, const TB* __restrict__ b,
                                               const T* __restrict__ x, T* __restrict__ r) {
    SELL_LOOP(S) {
        const T acc = sell_row(S.col, val, (long long)S.sptr[s] * 32 + lane, S.sptr[s + 1] - S.sptr[s],
                               [&](int j) { return ld(x + j); });
        const int ip = s * 32 + lane;
        if (ip < S.n) {
            const int i = sell_rowid(S, ip);
            r[i] = (T)b[i] - acc;
        }
    }
}

// Extra post-smoothing sweep: y' = y + omega M^-1 (b - A y).
template <typename T, typename TB, typename TO>
__global__ void __launch_bounds__(TPB) k_smooth(SellView S, const T* __restrict__ val, const T* __restrict__ minv,
                                                T omega, const TB* __restrict__ b, const T* __restrict__ yin,
                                                TO* __restrict__ yout) {
    SELL_LOOP(S) {
        const T acc = sell_row(S.col, val, (long long)S.sptr[s] * 32 + lane, S.sptr[s + 1] - S.sptr[s],
                               [&](int j) { return ld(yin + j); });
        const int ip = s * 32 + lane;
        if (ip < S.n) {
            const int i = sell_rowid(S, ip);
            yout[i] = (TO)fma(omega * minv[i], (T)b[i] - acc, yin[i]);
        }
    }
}

// a . b and, if c is given, b . c.
__global__ void __launch_bounds__(TPB) k_dot(int n, const double* __restrict__ a, const double* __restrict__ b,
                                             const double* __restrict__ c, Reducer red, PcgScalars* sc, int mode) {
    double d = 0.0, d2 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        d = fma(a[i], b[i], d);
        if (c) d2 = fma(b[i], c[i], d2);
    }
    reduce_and_finish(d, d2, red, sc, mode);
}

// x = A_L^{-1} b on the coarsest level, in FP64 whatever T is.
template <typename T, typename TO>
__global__ void k_coarse_solve(int n, const double* __restrict__ Ainv, const T* __restrict__ b, TO* __restrict__ x) {
    extern __shared__ double bs[];
    for (int j = threadIdx.x; j < n; j += blockDim.x) bs[j] = (double)b[j];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (int i = blockIdx.x * warps + (threadIdx.x >> 5); i < n; i += gridDim.x * warps) {
        double s = 0.0;
        const double* row = Ainv + (size_t)i * n;
        for (int j = lane; j < n; j += 32) s = fma(row[j], bs[j], s);
        s = warp_sum(s);
        if (lane == 0) x[i] = (TO)s;
    }
}


// ------------------------------------- iterative coarsest solve (large n_L)
// When the coarsest level is too large for the dense factor, it is solved
// with CG preconditioned by l1-Jacobi from x = 0 to ||r|| <= rtol ||b|| or
// maxit iterations, all in FP64 and in one cooperative launch. Scalars are
// block partials written to a double buffer; after each grid barrier every
// block sums the partials in the same order, so all blocks hold identical
// scalars without a broadcast step. Waits are bounded (2 s).
__device__ __forceinline__ unsigned long long cg_global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned cg_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void cg_grid_sync(unsigned* count, unsigned epoch, int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        const unsigned target = epoch * gridDim.x;
        const unsigned long long t0 = cg_global_ns();
        while (cg_ld_acquire(count) < target) {
            if (cg_global_ns() - t0 > 2000000000ull) { atomicExch(err, 1); break; }
        }
        __threadfence();
    }
    __syncthreads();
}

// Sum of the G block partials of slot k in buffer `buf`, same order in every block.
__device__ __forceinline__ double cg_sum(const double* part, int G) {
    double s = 0.0;
    for (int k = threadIdx.x; k < G; k += blockDim.x) s += __ldcg(part + k);
    return block_sum(s);
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(512) k_coarse_cg(SellView S, const double* __restrict__ val, int n,
                                                   int nlong, const int* __restrict__ long_rows,
                                                   const int* __restrict__ cptr, const int* __restrict__ ccol,
                                                   const double* __restrict__ cval,
                                                   const double* __restrict__ minv, const TI* __restrict__ b,
                                                   TO* __restrict__ xout, double* x, double* r, double* z, double* p,
                                                   double* q, double* part, unsigned* bar, int* err, int maxit,
                                                   double rtol) {
    const int G = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = G * blockDim.x;
    unsigned epoch = 0;
    int red = 0;   // reduction counter: buffer = red & 1, two slots per buffer
    auto slot = [&](int k) { return part + (size_t)((red & 1) * 2 + k) * G; };
    double a = 0.0, c = 0.0;
    for (int i = tid; i < n; i += stride) {
        const double bi = (double)b[i];
        x[i] = 0.0;
        r[i] = bi;
        const double zi = minv[i] * bi;
        z[i] = zi;
        p[i] = zi;
        a = fma(bi, zi, a);
        c = fma(bi, bi, c);
    }
    a = block_sum(a);
    c = block_sum(c);
    if (threadIdx.x == 0) { slot(0)[blockIdx.x] = a; slot(1)[blockIdx.x] = c; }
    cg_grid_sync(bar, ++epoch, err);
    if (__ldcg(err)) return;
    double rho = cg_sum(slot(0), G);
    const double bb = cg_sum(slot(1), G);
    ++red;
    if (bb > 0.0) {
        const double stop2 = rtol * rtol * bb;
        for (int it = 0; it < maxit; ++it) {
            // q = A p, p . q
            double pq = 0.0;
            const int lane = threadIdx.x & 31, nw = G * (blockDim.x >> 5);
            for (int sl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sl < S.nslices; sl += nw) {
                const double acc = sell_row(S.col, val, (long long)S.sptr[sl] * 32 + lane, S.sptr[sl + 1] - S.sptr[sl],
                                            [&](int j) { return __ldcg(p + j); });
                const int ip = sl * 32 + lane;
                if (ip < S.n) {
                    const int i = sell_rowid(S, ip);
                    q[i] = acc;
                    pq = fma(__ldcg(p + i), acc, pq);
                }
            }
            // long rows: one warp per row, straight from the CSR
            for (int lr = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); lr < nlong; lr += nw) {
                const int i = __ldg(long_rows + lr);
                double acc = 0.0;
                for (int k = __ldg(cptr + i) + lane; k < __ldg(cptr + i + 1); k += 32)
                    acc = fma(__ldg(cval + k), __ldcg(p + __ldg(ccol + k)), acc);
                acc = warp_sum(acc);
                if (lane == 0) {
                    q[i] = acc;
                    pq = fma(__ldcg(p + i), acc, pq);
                }
            }
            pq = block_sum(pq);
            if (threadIdx.x == 0) slot(0)[blockIdx.x] = pq;
            cg_grid_sync(bar, ++epoch, err);
            if (__ldcg(err)) return;
            const double alpha = rho / cg_sum(slot(0), G);
            ++red;
            // x += alpha p, r -= alpha q, z = M^-1 r: r . r and r . z in one
            // reduction (z is formed even on the last step, where it is unused)
            double rr = 0.0, rz = 0.0;
            for (int i = tid; i < n; i += stride) {
                x[i] = fma(alpha, __ldcg(p + i), x[i]);
                const double ri = fma(-alpha, __ldcg(q + i), r[i]);
                r[i] = ri;
                rr = fma(ri, ri, rr);
                const double zi = minv[i] * ri;
                z[i] = zi;
                rz = fma(ri, zi, rz);
            }
            rr = block_sum(rr);
            rz = block_sum(rz);
            if (threadIdx.x == 0) { slot(0)[blockIdx.x] = rr; slot(1)[blockIdx.x] = rz; }
            cg_grid_sync(bar, ++epoch, err);
            if (__ldcg(err)) return;
            const double rr_all = cg_sum(slot(0), G);
            const double rho_new = cg_sum(slot(1), G);
            ++red;
            if (rr_all <= stop2) break;
            const double beta = rho_new / rho;
            rho = rho_new;
            for (int i = tid; i < n; i += stride) p[i] = fma(beta, p[i], z[i]);
            cg_grid_sync(bar, ++epoch, err);
            if (__ldcg(err)) return;
        }
    }
    for (int i = tid; i < n; i += stride) xout[i] = (TO)x[i];
}

// Block-diagonal coarsest level of a batch of systems: x_i = sum_j of the
// system's dense inverse block times b, one warp per row.
template <typename T, typename TO>
__global__ void k_coarse_solve_seg(int n, int m, const int* __restrict__ segp, const long long* __restrict__ blk,
                                   const double* __restrict__ Ainv, const T* __restrict__ b, TO* __restrict__ x) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        int lo = 0, hi = m;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (segp[mid] <= i) lo = mid; else hi = mid;
        }
        const int r0 = segp[lo], ns = segp[lo + 1] - r0;
        const double* row = Ainv + blk[lo] + (long long)(i - r0) * ns;
        double acc = 0.0;
        for (int j = lane; j < ns; j += 32) acc = fma(row[j], (double)b[r0 + j], acc);
        acc = warp_sum(acc);
        if (lane == 0) x[i] = (TO)acc;
    }
}

// ------------------------------------------------------------- PCG ---------
// r = b - A x; ||r||^2 and ||b||^2.
__global__ void __launch_bounds__(TPB) k_residual(SellView S, const double* __restrict__ val,
                                                  const double* __restrict__ x, const double* __restrict__ b,
                                                  double* __restrict__ r, Reducer red, PcgScalars* sc) {
    double rr = 0.0, bb = 0.0;
    SELL_LOOP(S) {
        const double acc = sell_row(S.col, val, (long long)S.sptr[s] * 32 + lane, S.sptr[s + 1] - S.sptr[s],
                                    [&](int j) { return ld(x + j); });
        const int ip = s * 32 + lane;
        if (ip < S.n) {
            const int i = sell_rowid(S, ip);
            const double bi = b[i];
            const double ri = bi - acc;
            r[i] = ri;
            rr = fma(ri, ri, rr);
            bb = fma(bi, bi, bb);
        }
    }
    reduce_and_finish(rr, bb, red, sc, FIN_NORMS);
}

// q = A p; p . q; alpha = rho / p.q.
__global__ void __launch_bounds__(TPB) k_spmv_dot(SellView S, const double* __restrict__ val,
                                                  const double* __restrict__ p, double* __restrict__ q, Reducer red,
                                                  PcgScalars* sc) {
    double pq = 0.0;
    SELL_LOOP(S) {
        const int ip = s * 32 + lane;
        const bool live = ip < S.n;
        const int i = live ? sell_rowid(S, ip) : 0;
        const double pi = live ? ld(p + i) : 0.0;
        const double acc = sell_row(S.col, val, (long long)S.sptr[s] * 32 + lane, S.sptr[s + 1] - S.sptr[s],
                                    [&](int j) { return ld(p + j); });
        if (live) {
            q[i] = acc;
            pq = fma(pi, acc, pq);
        }
    }
    reduce_and_finish(pq, 0.0, red, sc, FIN_PQ);
}

// x += alpha p; r -= alpha q; ||r||^2.
// With r32 set (FP32 V-cycle), also the float copy of the new r that the
// V-cycle's level 0 reads (the conversion of k_to_f32, without its pass).
__global__ void __launch_bounds__(TPB) k_update_xr(int n, const double* __restrict__ p, const double* __restrict__ q,
                                                   double* __restrict__ x, double* __restrict__ r,
                                                   float* __restrict__ r32, Reducer red, PcgScalars* sc) {
    const double alpha = sc->alpha;
    double rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        if (r32) r32[i] = (float)ri;
        rr = fma(ri, ri, rr);
    }
    reduce_and_finish(rr, 0.0, red, sc, FIN_RR);
}

// p = z + beta p.
__global__ void __launch_bounds__(TPB) k_update_p(int n, const double* __restrict__ z, double* __restrict__ p,
                                                  const PcgScalars* sc) {
    const double beta = sc->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = fma(beta, p[i], z[i]);
}

// ------------------------------------------------------------ host ---------
// Algorithmic bytes of one launch: every array the kernel must touch, read
// or written once (index 4 B, value V B, the level-0 input/output in FP64);
// matrix entries counted without SELL padding.
double by_pre(const Level& L, int V, int Vb) { return (double)L.A.nnz * (V + 4) + (double)L.A.n * (Vb + 3.0 * V); }
// post: omega M^-1 A P entries + u, p (V) [x, r, omega M^-1 instead of u without
// the fused u: 3V] + agg (4) + out (Vo) [+ CG r for the dot] + e (n_c)
double by_post2(const Level& L, int nc, int V, int Vo, bool dot, bool u) {
    return (double)L.ap_nnz * (V + 4) + (double)L.A.n * ((u ? 2.0 : 4.0) * V + 4 + Vo + (dot ? 8 : 0)) +
           (double)nc * V;
}
double by_resid(const Level& L, int V, int Vb) { return (double)L.A.nnz * (V + 4) + (double)L.A.n * (Vb + 2.0 * V); }
double by_restrict(int n, int nc, int V) { return (double)n * (4 + 2.0 * V) + (double)nc * (4 + V); }
double by_smooth(const Level& L, int V, int Vb, int Vo) { return (double)L.A.nnz * (V + 4) + (double)L.A.n * (2.0 * V + Vb + Vo); }
double by_coarse(int nc, int Vi, int Vo) { return 8.0 * nc * nc + (double)nc * (Vi + Vo); }

SellView view(const Level& L) { return SellView{L.S.n, L.S.nslices, L.S.sptr, L.S.col, L.S.perm}; }

int sell_grid(const amg_hierarchy* h, int nslices) {
    int g = (nslices + WARPS - 1) / WARPS;
    int cap = h->num_sms * 8;
    return g < 1 ? 1 : (g > cap ? cap : g);
}

int vec_grid(const amg_hierarchy* h, long long n) { return blocks_for(n, TPB, h->num_sms * 8); }

// Fixed grid of every reducing kernel (deterministic partial order).
int red_grid(const amg_hierarchy* h) { return h->red.blocks; }
int wide_grid(const amg_hierarchy* h, long long rows) { return blocks_for(rows * 32, TPB, h->num_sms * 16); }

void coarse_solve_launch(amg_hierarchy* h, const void* b, void* x, bool fp32_in, bool fp64_out) {
    const int n = h->nc;
    if (h->segL_ptr) {
        const int m = (int)h->seg0.size() - 1;
        const int grid = blocks_for((long long)n * 32, 256, h->num_sms * 8);
        Scope sc_(&h->prof, h->stream, K_COARSE, 16.0 * n);
        if (!fp32_in)
            k_coarse_solve_seg<double, double><<<grid, 256, 0, h->stream>>>(n, m, h->segL_ptr, h->segL_blk,
                                                                            h->coarse_inv, (const double*)b, (double*)x);
        else if (fp64_out)
            k_coarse_solve_seg<float, double><<<grid, 256, 0, h->stream>>>(n, m, h->segL_ptr, h->segL_blk,
                                                                           h->coarse_inv, (const float*)b, (double*)x);
        else
            k_coarse_solve_seg<float, float><<<grid, 256, 0, h->stream>>>(n, m, h->segL_ptr, h->segL_blk,
                                                                          h->coarse_inv, (const float*)b, (float*)x);
        KERNEL_CHECK();
        return;
    }
    if (h->coarse_cg) {
        Level& Lc = h->lev.back();
        CoarseCg& C = h->ccg;
        Scope sc_(&h->prof, h->stream, K_COARSE, 8.0 * 30 * (3.0 * Lc.A.nnz + 10.0 * n));
        CUDA_CHECK(cudaMemsetAsync(C.ctl, 0, sizeof(int) * 4, h->stream));
        SellView S{Lc.S.n, Lc.S.nslices, Lc.S.sptr, Lc.S.col, Lc.S.perm};
        const double* val = Lc.S.val;
        int nrows = Lc.A.n;
        int nlong = Lc.S.nlong;
        const int* long_rows = Lc.S.long_rows;
        const int* cptr = Lc.A.ptr;
        const int* ccol = Lc.A.col;
        const double* cval = Lc.A.val;
        const double* minv = Lc.minv;
        unsigned* bar = reinterpret_cast<unsigned*>(C.ctl);
        int* err = C.ctl + 1;
        int maxit = 30;
        double rtol = 1e-4;
        void* args[] = {&S, &val, &nrows, &nlong, &long_rows, &cptr, &ccol, &cval, &minv, const_cast<void**>(&b), &x,
                        &C.x, &C.r, &C.z, &C.p, &C.q, &C.part, &bar, &err, &maxit, &rtol};
        const void* fn = !fp32_in ? (const void*)k_coarse_cg<double, double>
                                  : (fp64_out ? (const void*)k_coarse_cg<float, double> : (const void*)k_coarse_cg<float, float>);
        CUDA_CHECK(cudaLaunchCooperativeKernel(fn, dim3(C.blocks), dim3(512), args, 0, h->stream));
        KERNEL_CHECK();
        return;
    }
    const int threads = 256;
    int grid = (n + (threads / 32) - 1) / (threads / 32);
    if (grid > h->num_sms * 2) grid = h->num_sms * 2;
    const size_t sh = sizeof(double) * (size_t)n;
    Scope sc_(&h->prof, h->stream, K_COARSE, by_coarse(n, fp32_in ? 4 : 8, fp64_out ? 8 : 4));
    if (!fp32_in)
        k_coarse_solve<double, double><<<grid, threads, sh, h->stream>>>(n, h->coarse_inv, (const double*)b, (double*)x);
    else if (fp64_out)
        k_coarse_solve<float, double><<<grid, threads, sh, h->stream>>>(n, h->coarse_inv, (const float*)b, (double*)x);
    else
        k_coarse_solve<float, float><<<grid, threads, sh, h->stream>>>(n, h->coarse_inv, (const float*)b, (float*)x);
    KERNEL_CHECK();
}

// z = B r on level 0. With rz_mode != FIN_NONE, also finishes r . z.
template <typename T>
void vcycle_typed(amg_hierarchy* h, const double* r, double* z, int rz_mode) {
    cudaStream_t st = h->stream;
    const double* q2 = rz_mode == FIN_RHO_UPDATE_FCG ? h->q : nullptr;
    const int L = (int)h->lev.size() - 1;
    const bool f32 = sizeof(T) == 4;
    const T omega = (T)h->opt.omega;
    const int n0 = h->lev[0].A.n;
    if (L == 0) {
        coarse_solve_launch(h, r, z, false, true);
        if (rz_mode != FIN_NONE) {
            Scope sc_(&h->prof, st, K_DOT, 16.0 * n0);
            k_dot<<<red_grid(h), TPB, 0, st>>>(n0, r, z, q2, h->red, h->sc, rz_mode);
            KERNEL_CHECK();
        }
        return;
    }
    auto val = [&](Level& Lv) -> const T* { return f32 ? (const T*)Lv.S.val32 : (const T*)Lv.S.val; };
    auto valm = [&](Level& Lv) -> const T* { return f32 ? (const T*)Lv.valm32 : (const T*)Lv.valm; };
    auto apv = [&](Level& Lv) -> const T* { return f32 ? (const T*)Lv.AP.val32 : (const T*)Lv.AP.val; };
    auto minv = [&](Level& Lv) -> const T* { return f32 ? (const T*)Lv.minv32 : (const T*)Lv.minv; };
    auto wm = [&](Level& Lv) -> const T* { return f32 ? (const T*)Lv.wminv32 : (const T*)Lv.wminv; };
    auto pv = [&](Level& Lv) -> const T* { return f32 ? (const T*)Lv.p32 : (const T*)Lv.p; };
    auto vec = [&](Level& Lv, int which) -> T* {
        if (f32) {
            float* v[6] = {Lv.b32, Lv.x32, Lv.r32, Lv.y32, Lv.t32, Lv.u32};
            return (T*)v[which];
        }
        double* v[6] = {Lv.b, Lv.x, Lv.r, Lv.y, Lv.t, Lv.u};
        return (T*)v[which];
    };
    enum { VB = 0, VX = 1, VR = 2, VY = 3, VT = 4, VU = 5 };
    const int V = sizeof(T);
    const int pre = h->opt.pre < 1 ? 1 : h->opt.pre;
    const int post = h->opt.post < 1 ? 1 : h->opt.post;
    const bool SA = h->opt.smooth_p != 0;   // smoothed prolongator: explicit Pbar^T, Pbar, then A-smoothing
    const bool U = pre == 1 && !SA;         // the pre-smoother hands u = x + omega M^-1 r to the post-smoother
    std::vector<T*> xcur(L + 1), rcur(L + 1), out(L + 1), spare(L + 1);

    // downward: level 0 reads the FP64 r directly
    for (int l = 0; l < L; ++l) {
        Level& Lv = h->lev[l];
        const SellView S = view(Lv);
        const int g = Lv.grid_pre[f32] ? Lv.grid_pre[f32] : sell_grid(h, S.nslices);
        T *xa = vec(Lv, VX), *ra = vec(Lv, VR), *xb = vec(Lv, VT);
        const int Vb = l == 0 ? 8 : V;
        if (l == 0 && f32 && !h->r32_ready) {           // else the CG update already wrote it
            Scope sc_(&h->prof, st, K_CONVERT, 12.0 * Lv.A.n);
            k_to_f32<<<vec_grid(h, Lv.A.n), TPB, 0, st>>>(Lv.A.n, r, (float*)vec(Lv, VB));
            KERNEL_CHECK();
        }
        const bool wideA = SA && !f32 && wide(Lv.A, WIDE_MIN_A);       // dense coarse level of a smoothed hierarchy
        // pre sweeps: x_1 = omega M^-1 b with r_1 = b - A x_1 (k_pre, which with
        // more sweeps to come stores x_2 = x_1 + omega M^-1 r_1 instead of x_1),
        // x_{k+1} = x_k + omega M^-1 (b - A x_k) for k = 2 .. pre - 1, then the
        // residual r = b - A x_pre
        const bool more = pre > 1;
        if (wideA) {
            Scope sc_(&h->prof, st, l == 0 ? K_PRE_L0 : K_PRE, by_pre(Lv, V, l == 0 ? 8 : V));
            const double* bl = l == 0 ? r : (const double*)vec(Lv, VB);
            k_wide<W_PRE><<<wide_grid(h, Lv.A.n), TPB, 0, st>>>(Lv.A.n, Lv.A.ptr, Lv.A.col, Lv.A.val, bl, Lv.minv,
                                                                Lv.wminv, (double)omega, bl, (double*)ra,
                                                                (double*)xa);
            KERNEL_CHECK();
        } else {
            Scope sc_(&h->prof, st, l == 0 ? K_PRE_L0 : K_PRE, by_pre(Lv, V, l == 0 && !f32 ? 8 : V));
            if (l == 0 && !f32) launch_pre<T, double>(U || more, g, st, S, valm(Lv), wm(Lv), omega, r, xa, ra);
            else launch_pre<T, T>(U || more, g, st, S, valm(Lv), wm(Lv), omega, vec(Lv, VB), xa, ra);
        }
        // the dense-level path stored x_1: it takes one sweep more here
        for (int k = wideA ? 1 : 2; k < pre; ++k) {
            Scope sc_(&h->prof, st, K_PRE_STEP, by_smooth(Lv, V, Vb, V));
            if (wideA)
                k_wide<W_SMOOTH><<<wide_grid(h, Lv.A.n), TPB, 0, st>>>(
                    Lv.A.n, Lv.A.ptr, Lv.A.col, Lv.A.val, (const double*)xa, Lv.minv, nullptr, (double)omega,
                    l == 0 ? r : (const double*)vec(Lv, VB), (double*)xb, nullptr);
            else if (l == 0) k_smooth<T, double, T><<<g, TPB, 0, st>>>(S, val(Lv), minv(Lv), omega, r, xa, xb);
            else k_smooth<T, T, T><<<g, TPB, 0, st>>>(S, val(Lv), minv(Lv), omega, vec(Lv, VB), xa, xb);
            KERNEL_CHECK();
            std::swap(xa, xb);
        }
        if (more) {
            Scope sc_(&h->prof, st, K_PRE_STEP, by_resid(Lv, V, Vb));
            if (wideA)
                k_wide<W_RES><<<wide_grid(h, Lv.A.n), TPB, 0, st>>>(
                    Lv.A.n, Lv.A.ptr, Lv.A.col, Lv.A.val, (const double*)xa, nullptr, nullptr, 0.0,
                    l == 0 ? r : (const double*)vec(Lv, VB), (double*)ra, nullptr);
            else if (l == 0) k_resid<T, double><<<g, TPB, 0, st>>>(S, val(Lv), r, xa, ra);
            else k_resid<T, T><<<g, TPB, 0, st>>>(S, val(Lv), vec(Lv, VB), xa, ra);
            KERNEL_CHECK();
        }
        xcur[l] = xa;
        rcur[l] = ra;
        spare[l] = (xa == vec(Lv, VX)) ? vec(Lv, VT) : vec(Lv, VX);
        const int nc = h->lev[l + 1].A.n;
        if (SA) {
            const SellView SPT{Lv.PBT.n, Lv.PBT.nslices, Lv.PBT.sptr, Lv.PBT.col, Lv.PBT.perm};
            Scope sc_(&h->prof, st, K_RESTRICT, (double)Lv.pbar_t.nnz * (V + 4) + (double)(Lv.A.n + nc) * V);
            if (!f32 && wide(Lv.pbar_t, WIDE_MIN_P))
                k_wide<W_SPMV><<<wide_grid(h, nc), TPB, 0, st>>>(nc, Lv.pbar_t.ptr, Lv.pbar_t.col, Lv.pbar_t.val,
                                                                 (const double*)ra, nullptr, nullptr, 0.0, nullptr,
                                                                 (double*)vec(h->lev[l + 1], VB), nullptr);
            else
                k_sell_spmv<T><<<sell_grid(h, SPT.nslices), TPB, 0, st>>>(
                    SPT, f32 ? (const T*)Lv.PBT.val32 : (const T*)Lv.PBT.val, ra, vec(h->lev[l + 1], VB));
            KERNEL_CHECK();
            continue;
        }
        Scope sc_(&h->prof, st, K_RESTRICT, by_restrict(Lv.A.n, nc, V));
        k_restrict<T><<<Lv.grid_restrict[f32] ? Lv.grid_restrict[f32] : vec_grid(h, nc), TPB, 0, st>>>(
            nc, Lv.pt_ptr, Lv.pt_idx, pv(Lv), ra, vec(h->lev[l + 1], VB));
        KERNEL_CHECK();
    }
    // coarsest: FP64 dense solve
    out[L] = vec(h->lev[L], VX);
    coarse_solve_launch(h, vec(h->lev[L], VB), out[L], f32, !f32);
    // upward
    for (int l = L - 1; l >= 0; --l) {
        Level& Lv = h->lev[l];
        const SellView S = view(Lv);
        const SellView SAP{Lv.AP.n, Lv.AP.nslices, Lv.AP.sptr, Lv.AP.col, Lv.AP.perm};
        const int g = Lv.grid_post[f32] ? Lv.grid_post[f32] : sell_grid(h, S.nslices);
        const T* e = out[l + 1];
        const int nc = h->lev[l + 1].A.n;
        if (SA) {
            // x <- x + Pbar e, then one l1-Jacobi sweep on A (the unfused post-smoother)
            const SellView SPB{Lv.PB.n, Lv.PB.nslices, Lv.PB.sptr, Lv.PB.col, Lv.PB.perm};
            {
                Scope sc_(&h->prof, st, l == 0 ? K_POST_L0 : K_POST,
                          (double)Lv.pbar.nnz * (V + 4) + 2.0 * Lv.A.n * V + (double)nc * V);
                if (!f32 && wide(Lv.pbar, WIDE_MIN_P))
                    k_wide<W_ADD><<<wide_grid(h, Lv.A.n), TPB, 0, st>>>(Lv.A.n, Lv.pbar.ptr, Lv.pbar.col,
                                                                       Lv.pbar.val, (const double*)e, nullptr,
                                                                       nullptr, 0.0, nullptr, (double*)xcur[l],
                                                                       nullptr);
                else
                    k_prolong<T><<<sell_grid(h, SPB.nslices), TPB, 0, st>>>(
                        SPB, f32 ? (const T*)Lv.PB.val32 : (const T*)Lv.PB.val, e, xcur[l]);
                KERNEL_CHECK();
            }
            // post sweeps alternate between y and the x buffer the pre-smoother left free
            T* cur = xcur[l];
            T* bufs[2] = {vec(Lv, VY), spare[l]};
            if (l > 0) {
                for (int k = 0; k < post; ++k) {
                    T* dst = bufs[k & 1];
                    Scope sc_(&h->prof, st, K_SMOOTH, by_smooth(Lv, V, V, V));
                    if (!f32 && wide(Lv.A, WIDE_MIN_A))
                        k_wide<W_SMOOTH><<<wide_grid(h, Lv.A.n), TPB, 0, st>>>(
                            Lv.A.n, Lv.A.ptr, Lv.A.col, Lv.A.val, (const double*)cur, Lv.minv, nullptr,
                            (double)omega, (const double*)vec(Lv, VB), (double*)dst, nullptr);
                    else
                        k_smooth<T, T, T><<<g, TPB, 0, st>>>(S, val(Lv), minv(Lv), omega, vec(Lv, VB), cur, dst);
                    KERNEL_CHECK();
                    cur = dst;
                }
                out[l] = cur;
                continue;
            }
            for (int k = 0; k + 1 < post; ++k) {
                T* dst = bufs[k & 1];
                Scope sc_(&h->prof, st, K_SMOOTH, by_smooth(Lv, V, 8, V));
                k_smooth<T, double, T><<<g, TPB, 0, st>>>(S, val(Lv), minv(Lv), omega, r, cur, dst);
                KERNEL_CHECK();
                cur = dst;
            }
            {
                Scope sc_(&h->prof, st, K_SMOOTH, by_smooth(Lv, V, 8, 8));
                k_smooth<T, double, double><<<g, TPB, 0, st>>>(S, val(Lv), minv(Lv), omega, r, cur, z);
                KERNEL_CHECK();
            }
            if (rz_mode != FIN_NONE) {
                Scope sc_(&h->prof, st, K_DOT, 16.0 * n0);
                k_dot<<<red_grid(h), TPB, 0, st>>>(n0, r, z, q2, h->red, h->sc, rz_mode);
                KERNEL_CHECK();
            }
            continue;
        }
        if (l > 0) {
            T *ya = vec(Lv, VY), *yb = spare[l];
            {
                Scope sc_(&h->prof, st, K_POST, by_post2(Lv, nc, V, V, false, U));
                launch_post<T, T, T, false>(U, g, st, SAP, apv(Lv), wm(Lv), Lv.agg, pv(Lv), e, xcur[l], rcur[l],
                                            (const T*)nullptr, ya, h->red, h->sc, FIN_NONE, nullptr);
            }
            for (int k = 1; k < post; ++k) {
                Scope sc_(&h->prof, st, K_SMOOTH, by_smooth(Lv, V, V, V));
                k_smooth<T, T, T><<<g, TPB, 0, st>>>(S, val(Lv), minv(Lv), omega, vec(Lv, VB), ya, yb);
                KERNEL_CHECK();
                std::swap(ya, yb);
            }
            out[l] = ya;
            continue;
        }
        if (post == 1) {
            Scope sc_(&h->prof, st, K_POST_L0, by_post2(Lv, nc, V, 8, rz_mode != FIN_NONE, U));
            if (rz_mode != FIN_NONE)
                launch_post<T, double, double, true>(U, red_grid(h), st, SAP, apv(Lv), wm(Lv), Lv.agg, pv(Lv), e,
                                                     xcur[0], rcur[0], r, z, h->red, h->sc, rz_mode, q2);
            else
                launch_post<T, double, double, false>(U, g, st, SAP, apv(Lv), wm(Lv), Lv.agg, pv(Lv), e, xcur[0],
                                                      rcur[0], r, z, h->red, h->sc, FIN_NONE, nullptr);
        } else {
            T *ya = vec(Lv, VY), *yb = spare[0];
            {
                Scope sc_(&h->prof, st, K_POST_L0, by_post2(Lv, nc, V, V, false, U));
                launch_post<T, double, T, false>(U, g, st, SAP, apv(Lv), wm(Lv), Lv.agg, pv(Lv), e, xcur[0], rcur[0],
                                                 r, ya, h->red, h->sc, FIN_NONE, nullptr);
            }
            for (int k = 1; k < post - 1; ++k) {
                Scope sc_(&h->prof, st, K_SMOOTH, by_smooth(Lv, V, 8, V));
                k_smooth<T, double, T><<<g, TPB, 0, st>>>(S, val(Lv), minv(Lv), omega, r, ya, yb);
                KERNEL_CHECK();
                std::swap(ya, yb);
            }
            {
                Scope sc_(&h->prof, st, K_SMOOTH, by_smooth(Lv, V, 8, 8));
                k_smooth<T, double, double><<<g, TPB, 0, st>>>(S, val(Lv), minv(Lv), omega, r, ya, z);
                KERNEL_CHECK();
            }
            if (rz_mode != FIN_NONE) {
                Scope sc_(&h->prof, st, K_DOT, 16.0 * n0);
                k_dot<<<red_grid(h), TPB, 0, st>>>(n0, r, z, q2, h->red, h->sc, rz_mode);
                KERNEL_CHECK();
            }
        }
    }
}

// ---- K-cycle (host side) ---------------------------------------------------
template <typename T>
T* lvec(Level& Lv, int which) {
    if (sizeof(T) == 4) {
        float* v[4] = {Lv.b32, Lv.x32, Lv.r32, Lv.y32};
        return (T*)v[which];
    }
    double* v[4] = {Lv.b, Lv.x, Lv.r, Lv.y};
    return (T*)v[which];
}

template <typename T>
struct LevelOps {
    Level& Lv;
    bool f32 = sizeof(T) == 4;
    explicit LevelOps(Level& L) : Lv(L) {}
    const T* val() const { return f32 ? (const T*)Lv.S.val32 : (const T*)Lv.S.val; }
    const T* valm() const { return f32 ? (const T*)Lv.valm32 : (const T*)Lv.valm; }
    const T* apw() const { return f32 ? (const T*)Lv.AP.val32 : (const T*)Lv.AP.val; }
    const T* wm() const { return f32 ? (const T*)Lv.wminv32 : (const T*)Lv.wminv; }
    const T* p() const { return f32 ? (const T*)Lv.p32 : (const T*)Lv.p; }
    T* kv(int i) const { return (T*)Lv.kv[i]; }
};

template <typename T>
void kc_fcg2(amg_hierarchy* h, int m, const T* b, T* e);

// out = B_l in on a level l >= 1 of a K-cycle: pre-smoothing from zero,
// restriction, coarse correction (two FCG iterations on the first `cycle`
// coarse levels, the V-cycle below them, the coarsest solve at the bottom),
// prolongation and post-smoothing; vectors in the cycle's type.
template <typename T>
void kc_apply(amg_hierarchy* h, int l, const T* in, T* out) {
    cudaStream_t st = h->stream;
    const int L = (int)h->lev.size() - 1;
    const bool f32 = sizeof(T) == 4;
    if (l == L) {
        coarse_solve_launch(h, in, out, f32, !f32);
        return;
    }
    Level& Lv = h->lev[l];
    Level& Ln = h->lev[l + 1];
    const LevelOps<T> O(Lv);
    const SellView S = view(Lv);
    const SellView SAP{Lv.AP.n, Lv.AP.nslices, Lv.AP.sptr, Lv.AP.col, Lv.AP.perm};
    const int V = sizeof(T), nc = Ln.A.n;
    const T omega = (T)h->opt.omega;
    T* xa = lvec<T>(Lv, 1);
    T* ra = lvec<T>(Lv, 2);
    {
        Scope sc_(&h->prof, st, K_PRE, by_pre(Lv, V, V));
        launch_pre<T, T>(true, Lv.grid_pre[f32] ? Lv.grid_pre[f32] : sell_grid(h, S.nslices), st, S, O.valm(), O.wm(),
                         omega, in, xa, ra);
    }
    {
        Scope sc_(&h->prof, st, K_RESTRICT, by_restrict(Lv.A.n, nc, V));
        k_restrict<T><<<Lv.grid_restrict[f32] ? Lv.grid_restrict[f32] : vec_grid(h, nc), TPB, 0, st>>>(
            nc, Lv.pt_ptr, Lv.pt_idx, O.p(), ra, lvec<T>(Ln, 0));
        KERNEL_CHECK();
    }
    // coarse correction on level l+1: the coarsest solve, two FCG iterations
    // (the first `cycle` coarse levels) or the V-cycle from level l+1
    T* e;
    if (l + 1 == L) {
        e = lvec<T>(Ln, 1);
        coarse_solve_launch(h, lvec<T>(Ln, 0), e, f32, !f32);
    } else if (l + 1 <= h->opt.cycle) {
        e = LevelOps<T>(Ln).kv(5);
        kc_fcg2<T>(h, l + 1, lvec<T>(Ln, 0), e);
    } else {
        e = lvec<T>(Ln, 3);
        kc_apply<T>(h, l + 1, lvec<T>(Ln, 0), e);
    }
    Scope sc_(&h->prof, st, K_POST, by_post2(Lv, nc, V, V, false, true));
    launch_post<T, T, T, false>(true, Lv.grid_post[f32] ? Lv.grid_post[f32] : sell_grid(h, S.nslices), st, SAP, O.apw(),
                                O.wm(), Lv.agg, O.p(), e, xa, ra, (const T*)nullptr, out, h->red, h->sc, FIN_NONE,
                                nullptr);
}

template <typename T>
void kc_fcg2(amg_hierarchy* h, int m, const T* b, T* e) {
    cudaStream_t st = h->stream;
    Level& Lm = h->lev[m];
    const LevelOps<T> O(Lm);
    const SellView S = view(Lm);
    const int n = Lm.A.n, V = sizeof(T);
    KcScalars* ks = h->ks + m;
    T *d1 = O.kv(0), *q1 = O.kv(1), *r2 = O.kv(2), *z2 = O.kv(3), *d2 = O.kv(4);
    const double by_spmv = (double)Lm.A.nnz * (V + 4) + (double)n * 3 * V;
    kc_apply<T>(h, m, b, d1);
    {
        Scope sc_(&h->prof, st, K_KFCG, by_spmv);
        k_kc_spmv_dot<T><<<red_grid(h), TPB, 0, st>>>(S, O.val(), d1, q1, b, h->red, ks);
        KERNEL_CHECK();
    }
    {
        Scope sc_(&h->prof, st, K_KFCG, 5.0 * n * V);
        k_kc_update1<T><<<vec_grid(h, n), TPB, 0, st>>>(n, d1, q1, b, e, r2, ks);
        KERNEL_CHECK();
    }
    kc_apply<T>(h, m, r2, z2);
    {
        Scope sc_(&h->prof, st, K_KFCG, 2.0 * n * V);
        k_kc_dot<T><<<red_grid(h), TPB, 0, st>>>(n, z2, q1, h->red, ks);
        KERNEL_CHECK();
    }
    {
        Scope sc_(&h->prof, st, K_KFCG, (double)Lm.A.nnz * (V + 4) + (double)n * 5 * V);
        k_kc_spmv2<T><<<red_grid(h), TPB, 0, st>>>(S, O.val(), z2, q1, d1, r2, d2, h->red, ks);
        KERNEL_CHECK();
    }
    {
        Scope sc_(&h->prof, st, K_KFCG, 3.0 * n * V);
        k_kc_update2<T><<<vec_grid(h, n), TPB, 0, st>>>(n, d2, e, ks);
        KERNEL_CHECK();
    }
}

// z = B r with the K-cycle on level 0 (FP64 r and z; with rz_mode the r.z
// (and q.z) sums of the outer CG are finished as in the V-cycle).
template <typename T>
void kcycle_typed(amg_hierarchy* h, const double* r, double* z, int rz_mode) {
    const int L = (int)h->lev.size() - 1;
    if (L <= 1) {                          // no intermediate level: the K-cycle is the V-cycle
        vcycle_typed<T>(h, r, z, rz_mode);
        return;
    }
    cudaStream_t st = h->stream;
    const bool f32 = sizeof(T) == 4;
    const double* q2 = rz_mode == FIN_RHO_UPDATE_FCG ? h->q : nullptr;
    Level& L0 = h->lev[0];
    Level& L1 = h->lev[1];
    const LevelOps<T> O(L0);
    const SellView S = view(L0);
    const SellView SAP{L0.AP.n, L0.AP.nslices, L0.AP.sptr, L0.AP.col, L0.AP.perm};
    const int V = sizeof(T), n0 = L0.A.n, nc = L1.A.n;
    const T omega = (T)h->opt.omega;
    T* xa = lvec<T>(L0, 1);
    T* ra = lvec<T>(L0, 2);
    const int g = L0.grid_pre[f32] ? L0.grid_pre[f32] : sell_grid(h, S.nslices);
    if (f32 && !h->r32_ready) {                         // else the CG update already wrote it
        Scope sc_(&h->prof, st, K_CONVERT, 12.0 * n0);
        k_to_f32<<<vec_grid(h, n0), TPB, 0, st>>>(n0, r, (float*)lvec<T>(L0, 0));
        KERNEL_CHECK();
    }
    {
        Scope sc_(&h->prof, st, K_PRE_L0, by_pre(L0, V, f32 ? V : 8));
        if (f32) launch_pre<T, T>(true, g, st, S, O.valm(), O.wm(), omega, lvec<T>(L0, 0), xa, ra);
        else launch_pre<T, double>(true, g, st, S, O.valm(), O.wm(), omega, r, xa, ra);
    }
    {
        Scope sc_(&h->prof, st, K_RESTRICT, by_restrict(n0, nc, V));
        k_restrict<T><<<L0.grid_restrict[f32] ? L0.grid_restrict[f32] : vec_grid(h, nc), TPB, 0, st>>>(
            nc, L0.pt_ptr, L0.pt_idx, O.p(), ra, lvec<T>(L1, 0));
        KERNEL_CHECK();
    }
    T* e = LevelOps<T>(L1).kv(5);
    kc_fcg2<T>(h, 1, lvec<T>(L1, 0), e);
    Scope sc_(&h->prof, st, K_POST_L0, by_post2(L0, nc, V, 8, rz_mode != FIN_NONE, true));
    const int gp = L0.grid_post[f32] ? L0.grid_post[f32] : sell_grid(h, S.nslices);
    if (rz_mode != FIN_NONE)
        launch_post<T, double, double, true>(true, red_grid(h), st, SAP, O.apw(), O.wm(), L0.agg, O.p(), e, xa, ra, r, z,
                                             h->red, h->sc, rz_mode, q2);
    else
        launch_post<T, double, double, false>(true, gp, st, SAP, O.apw(), O.wm(), L0.agg, O.p(), e, xa, ra, r, z,
                                              h->red, h->sc, FIN_NONE, nullptr);
}

void vcycle_dispatch(amg_hierarchy* h, const double* r, double* z, int rz_mode) {
    const bool f32 = h->opt.precision == AMG_FP32_VCYCLE;
    if (h->opt.cycle > 0) {
        if (f32) kcycle_typed<float>(h, r, z, rz_mode);
        else kcycle_typed<double>(h, r, z, rz_mode);
    } else {
        if (f32) vcycle_typed<float>(h, r, z, rz_mode);
        else vcycle_typed<double>(h, r, z, rz_mode);
    }
}

// Launch-shape candidates of a grid-stride kernel that needs at most `need`
// blocks: 1, 2, 4, ..., 32 blocks per SM, capped at `need`.
std::vector<int> grid_candidates(const amg_hierarchy* h, long long need) {
    std::vector<int> c;
    for (int m = 1; m <= 32; m *= 2) {
        long long g = (long long)h->num_sms * m;
        if (g > need) g = need;
        if (g < 1) g = 1;
        if (c.empty() || c.back() != (int)g) c.push_back((int)g);
        if (g == need) break;
    }
    return c;
}

// Fastest candidate grid for `launch(g)`, from the cache or timed now.
template <typename F>
int tune_grid(amg_hierarchy* h, const std::string& key, const std::vector<int>& cand, F&& launch) {
    int best = 0;
    if (tune_get(key, &best)) return best;
    double tbest = 1e30;
    for (int g : cand) {
        const double t = time_launches(h->stream, [&]() { launch(g); }, 3);
        if (t < tbest) {
            tbest = t;
            best = g;
        }
    }
    tune_put(key, best);
    return best;
}

// Times the SELL sweeps and the restriction of every level for value type T
// on the hierarchy's own work vectors (zeroed first) and records the fastest
// grids in the levels.
template <typename T>
void autotune_levels(amg_hierarchy* h) {
    cudaStream_t st = h->stream;
    const bool f32 = sizeof(T) == 4;
    const int V = sizeof(T);
    const T omega = (T)h->opt.omega;
    const int L = (int)h->lev.size() - 1;
    auto zero = [&](void* p, size_t bytes) {
        if (p) CUDA_CHECK(cudaMemsetAsync(p, 0, bytes, st));
    };
    for (auto& Lv : h->lev) {
        const size_t n = (size_t)Lv.A.n;
        if (f32) {
            for (float* v : {Lv.b32, Lv.x32, Lv.r32, Lv.y32}) zero(v, n * 4);
        } else {
            for (double* v : {Lv.b, Lv.x, Lv.r, Lv.y}) zero(v, n * 8);
        }
    }
    const size_t n0 = (size_t)h->lev[0].A.n;
    zero(h->r, n0 * 8);
    zero(h->z, n0 * 8);
    auto vb = [&](Level& Lv) -> T* { return f32 ? (T*)Lv.b32 : (T*)Lv.b; };
    auto vx = [&](Level& Lv) -> T* { return f32 ? (T*)Lv.x32 : (T*)Lv.x; };
    auto vr = [&](Level& Lv) -> T* { return f32 ? (T*)Lv.r32 : (T*)Lv.r; };
    auto vy = [&](Level& Lv) -> T* { return f32 ? (T*)Lv.y32 : (T*)Lv.y; };
    for (int l = 0; l < L; ++l) {
        Level& Lv = h->lev[l];
        Level& Ln = h->lev[l + 1];
        const SellView S = view(Lv);
        const SellView SAP{Lv.AP.n, Lv.AP.nslices, Lv.AP.sptr, Lv.AP.col, Lv.AP.perm};
        const T* valm = f32 ? (const T*)Lv.valm32 : (const T*)Lv.valm;
        const T* apv = f32 ? (const T*)Lv.AP.val32 : (const T*)Lv.AP.val;
        const T* wm = f32 ? (const T*)Lv.wminv32 : (const T*)Lv.wminv;
        const T* p = f32 ? (const T*)Lv.p32 : (const T*)Lv.p;
        const bool U = h->opt.pre <= 1;
        const long long need = (S.nslices + WARPS - 1) / WARPS;
        const auto cand = grid_candidates(h, need);
        const int z0 = l == 0;
        Lv.grid_pre[f32] = tune_grid(h, tune_key(z0 ? "pre0" : "pre", V, S.n, Lv.A.nnz, S.nslices, 1, h->num_sms),
                                     cand, [&](int g) {
                                         if (z0 && !f32)
                                             launch_pre<T, double>(U, g, st, S, valm, wm, omega, h->r, vx(Lv), vr(Lv));
                                         else
                                             launch_pre<T, T>(U, g, st, S, valm, wm, omega, vb(Lv), vx(Lv), vr(Lv));
                                     });
        if (h->opt.smooth_p) continue;     // the smoothed path has no fused post-smoother or member lists
        Lv.grid_post[f32] = tune_grid(
            h, tune_key(z0 ? "post0" : "post", V, SAP.n, Lv.ap_nnz, SAP.nslices, 1, h->num_sms), cand, [&](int g) {
                if (z0)
                    launch_post<T, double, double, false>(U, g, st, SAP, apv, wm, Lv.agg, p, vx(Ln), vx(Lv), vr(Lv),
                                                          h->r, h->z, h->red, h->sc, FIN_NONE, nullptr);
                else
                    launch_post<T, T, T, false>(U, g, st, SAP, apv, wm, Lv.agg, p, vx(Ln), vx(Lv), vr(Lv),
                                                (const T*)nullptr, vy(Lv), h->red, h->sc, FIN_NONE, nullptr);
            });
        const int nc = Ln.A.n;
        Lv.grid_restrict[f32] = tune_grid(h, tune_key("restrict", V, nc, Lv.A.n, 0, 1, h->num_sms),
                                          grid_candidates(h, (nc + TPB - 1) / TPB), [&](int g) {
                                              k_restrict<T><<<g, TPB, 0, st>>>(nc, Lv.pt_ptr, Lv.pt_idx, p, vr(Lv),
                                                                               vb(Ln));
                                              KERNEL_CHECK();
                                          });
    }
    CUDA_CHECK(cudaStreamSynchronize(st));
}

void read_scalars(amg_hierarchy* h) {
    CUDA_CHECK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, h->stream));
    CUDA_CHECK(cudaStreamSynchronize(h->stream));
}

}  // namespace

void prepare_solve(amg_hierarchy* h) {
    const bool f32 = h->opt.precision == AMG_FP32_VCYCLE;
    const bool extra = h->opt.pre > 1 || h->opt.post > 1;
    for (auto& L : h->lev) {
        const int n = L.A.n;
        if (f32) {
            L.b32 = h->mem.alloc<float>(n);
            L.x32 = h->mem.alloc<float>(n);
            L.r32 = h->mem.alloc<float>(n);
            L.y32 = h->mem.alloc<float>(n);
            if (extra) { L.t32 = h->mem.alloc<float>(n); L.u32 = h->mem.alloc<float>(n); }
        } else {
            L.b = h->mem.alloc<double>(n);
            L.x = h->mem.alloc<double>(n);
            L.r = h->mem.alloc<double>(n);
            L.y = h->mem.alloc<double>(n);
            if (extra) { L.t = h->mem.alloc<double>(n); L.u = h->mem.alloc<double>(n); }
        }
    }
    if (h->coarse_cg) {
        const int nc = h->lev.back().A.n;
        CoarseCg& C = h->ccg;
        int per_sm = 0;
        CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_cg<double, double>, 512, 0));
        if (per_sm < 1) AMG_THROW(AMG_ERR_CUDA, "coarsest CG kernel cannot be resident");
        C.blocks = h->num_sms;
        C.x = h->mem.alloc<double>(nc);
        C.r = h->mem.alloc<double>(nc);
        C.z = h->mem.alloc<double>(nc);
        C.p = h->mem.alloc<double>(nc);
        C.q = h->mem.alloc<double>(nc);
        C.part = h->mem.alloc<double>(4 * (size_t)C.blocks);
        C.ctl = h->mem.alloc<int>(4);
    }
    if (h->opt.cycle > 0) {
        // K-cycle: FCG(2) vectors on the levels that take it, scalars per level
        const size_t V = f32 ? 4 : 8;
        for (size_t l = 1; l + 1 < h->lev.size() && (int)l <= h->opt.cycle; ++l)
            for (int i = 0; i < 6; ++i) h->lev[l].kv[i] = h->mem.alloc<char>((size_t)h->lev[l].A.n * V);
        h->ks = h->mem.alloc<KcScalars>(h->lev.size());
        CUDA_CHECK(cudaMemsetAsync(h->ks, 0, sizeof(KcScalars) * h->lev.size(), h->stream));
    }
    const int n0 = h->lev[0].A.n;
    h->r = h->mem.alloc<double>(n0);
    h->z = h->mem.alloc<double>(n0);
    h->p = h->mem.alloc<double>(n0);
    h->q = h->mem.alloc<double>(n0);
    h->t = h->mem.alloc<double>(n0);
    h->sc = h->mem.alloc<PcgScalars>(1);
    CUDA_CHECK(cudaMemsetAsync(h->sc, 0, sizeof(PcgScalars), h->stream));
    if (!h->sc_host) CUDA_CHECK(cudaHostAlloc(&h->sc_host, sizeof(PcgScalars), cudaHostAllocDefault));
    h->red.blocks = h->num_sms * 8;
    h->red.partial = h->mem.alloc<double>(2 * (size_t)h->red.blocks);
    h->red.ticket = h->mem.alloc<unsigned>(1);
    CUDA_CHECK(cudaMemsetAsync(h->red.ticket, 0, sizeof(unsigned), h->stream));
    CUDA_CHECK(cudaStreamSynchronize(h->stream));
}

void autotune_vcycle(amg_hierarchy* h) {
    if (h->lev.size() < 2) return;
    const bool prof_on = h->prof.on;
    h->prof.on = false;
    try {
        if (h->opt.precision == AMG_FP32_VCYCLE) autotune_levels<float>(h);
        else autotune_levels<double>(h);
    } catch (...) {
        h->prof.on = prof_on;
        throw;
    }
    h->prof.on = prof_on;
}

void coarse_cg_solve(amg_hierarchy* h, const double* b, double* x) { coarse_solve_launch(h, b, x, false, true); }

void vcycle_plain(amg_hierarchy* h, const double* r, double* z) { vcycle_dispatch(h, r, z, FIN_NONE); }

void vcycle_apply(amg_hierarchy* h, const double* r, double* z) {
    vcycle_dispatch(h, r, z, FIN_NONE);
    CUDA_CHECK(cudaStreamSynchronize(h->stream));
    h->prof.flush();
}

amg_status solve(amg_hierarchy* h, const double* b, double* x, double rtol, int maxit, amg_solve_info* info) {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = h->stream;
    Level& L0 = h->lev[0];
    const int n = L0.A.n;
    const SellView S = view(L0);
    const double* A = L0.S.val;
    PcgScalars* hs = h->sc_host;

    const double nnz = (double)L0.A.nnz;
    const double by_res = 12.0 * nnz + 24.0 * n, by_spmv = 12.0 * nnz + 16.0 * n;
    CUDA_CHECK(cudaMemsetAsync(h->sc, 0, sizeof(PcgScalars), st));
    {
        Scope sc_(&h->prof, st, K_RESIDUAL, by_res);
        k_residual<<<red_grid(h), TPB, 0, st>>>(S, A, x, b, h->r, h->red, h->sc);
        KERNEL_CHECK();
    }
    read_scalars(h);
    const double nb = std::sqrt(hs->bb);
    amg_solve_info inf{};
    amg_status status = AMG_NOT_CONVERGED;
    if (nb == 0.0) {
        CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
        CUDA_CHECK(cudaStreamSynchronize(st));
        inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (info) *info = inf;
        return AMG_OK;
    }
    double rel = std::sqrt(hs->rr) / nb;
    double true_rel = rel;
    bool have_true = true;          // r currently equals b - A x exactly
    int it = 0;
    bool restart = true;
    // FP32 V-cycle: the CG update also writes level 0's float copy of r
    float* r32 = h->opt.precision == AMG_FP32_VCYCLE ? h->lev[0].b32 : nullptr;
    h->r32_ready = false;
    struct Ev {
        cudaEvent_t e = nullptr;
        ~Ev() { if (e) cudaEventDestroy(e); }
    } ev;
    CUDA_CHECK(cudaEventCreateWithFlags(&ev.e, cudaEventDisableTiming));
    // z = B r for the next iteration, then p = z + beta p
    auto precondition = [&]() {
        h->r32_ready = r32 != nullptr;                  // level 0's float r is the one k_update_xr wrote
        vcycle_dispatch(h, h->r, h->z,
                        h->opt.krylov == 1 || h->opt.cycle > 0 ? FIN_RHO_UPDATE_FCG : FIN_RHO_UPDATE);
        h->r32_ready = false;
        Scope sc_(&h->prof, st, K_UPDATE_P, 24.0 * n);
        k_update_p<<<vec_grid(h, n), TPB, 0, st>>>(n, h->z, h->p, h->sc);
        KERNEL_CHECK();
    };
    if (rel <= rtol) status = AMG_OK;
    while (status != AMG_OK && it < maxit) {
        if (restart) {
            vcycle_dispatch(h, h->r, h->z, FIN_RHO_INIT);
            CUDA_CHECK(cudaMemcpyAsync(h->p, h->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            restart = false;
        }
        {
            Scope sc_(&h->prof, st, K_SPMV_DOT, by_spmv);
            k_spmv_dot<<<red_grid(h), TPB, 0, st>>>(S, A, h->p, h->q, h->red, h->sc);
            KERNEL_CHECK();
        }
        {
            Scope sc_(&h->prof, st, K_UPDATE_XR, 48.0 * n + (r32 ? 4.0 * n : 0.0));
            k_update_xr<<<red_grid(h), TPB, 0, st>>>(n, h->p, h->q, x, h->r, r32, h->red, h->sc);
            KERNEL_CHECK();
        }
        ++it;
        // The scalars go to the host. While the residual is well above the
        // tolerance, the next iteration's preconditioner and direction update
        // (which write only z, p and the device scalars) are queued behind the
        // copy before the host waits for it, so the round trip overlaps the
        // V-cycle; if the check below ends the loop after all, x and r are
        // final and that work goes unused, and a restart recomputes rho and p
        // from the true residual. Near the tolerance the host checks first.
        const bool ahead = rel > 4.0 * rtol;
        CUDA_CHECK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
        CUDA_CHECK(cudaEventRecord(ev.e, st));
        if (ahead) precondition();
        CUDA_CHECK(cudaEventSynchronize(ev.e));
        if (hs->breakdown) { status = AMG_ERR_BREAKDOWN; break; }
        rel = std::sqrt(hs->rr) / nb;
        have_true = false;
        if (rel <= rtol) {
            {
                Scope sc_(&h->prof, st, K_RESIDUAL, by_res);
                k_residual<<<red_grid(h), TPB, 0, st>>>(S, A, x, b, h->t, h->red, h->sc);
                KERNEL_CHECK();
            }
            read_scalars(h);
            true_rel = std::sqrt(hs->rr) / nb;
            have_true = true;
            if (true_rel <= rtol) { status = AMG_OK; break; }
            CUDA_CHECK(cudaMemcpyAsync(h->r, h->t, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            rel = true_rel;
            restart = true;
            ++inf.restarts;
            continue;
        }
        if (!ahead) precondition();
    }
    if (!have_true) {
        {
            Scope sc_(&h->prof, st, K_RESIDUAL, by_res);
            k_residual<<<red_grid(h), TPB, 0, st>>>(S, A, x, b, h->t, h->red, h->sc);
            KERNEL_CHECK();
        }
        read_scalars(h);
        true_rel = std::sqrt(hs->rr) / nb;
    }
    CUDA_CHECK(cudaStreamSynchronize(st));
    h->prof.flush();
    inf.iterations = it;
    inf.relres = rel;
    inf.true_relres = true_rel;
    inf.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return status;
}

}  // namespace amg
