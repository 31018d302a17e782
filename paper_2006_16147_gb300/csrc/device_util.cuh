// device_util.cuh -- warp/block reductions and scans used by the kernels.
#pragma once

#include <cuda_runtime.h>

namespace amg {

constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

__device__ __forceinline__ int warp_max_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL_MASK, v, o));
    return v;
}

// Block-wide sum (any blockDim multiple of 32, <= 1024). All threads get it.
__device__ __forceinline__ int block_sum_int(int v) {
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_int(v);
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    int t = (lane < nw) ? ws[lane] : 0;
    t = warp_sum_int(t);
    __syncthreads();
    return t;
}

// Block-wide maximum (any blockDim multiple of 32, <= 1024). All threads get it.
__device__ __forceinline__ int block_max_int(int v) {
    __shared__ int wm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max_int(v);
    if (lane == 0) wm[wid] = v;
    __syncthreads();
    int t = (lane < nw) ? wm[lane] : 0;
    t = warp_max_int(t);
    __syncthreads();
    return t;
}

// Block-wide sum in a fixed combination order (deterministic for a fixed
// blockDim). All threads get the result.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    double t = (lane < nw) ? ws[lane] : 0.0;
    t = warp_sum(t);
    __syncthreads();
    return t;
}

// Block-wide exclusive scan of ints.
__device__ __forceinline__ int block_exclusive_scan_int(int v) {
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = (lane < nw) ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL_MASK, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    int r = x - v + (wid > 0 ? ws[wid - 1] : 0);
    __syncthreads();
    return r;
}

// Warp-aggregated append of one item per participating lane to list[*cnt];
// items past `cap` are dropped (the caller sizes lists so this cannot happen).
__device__ __forceinline__ void warp_append(bool take, int item, int* list, int* cnt, int cap) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, take);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(act, base, leader);
    const int pos = base + __popc(m & ((1u << lane) - 1));
    if (take && pos < cap) list[pos] = item;
}

}  // namespace amg
