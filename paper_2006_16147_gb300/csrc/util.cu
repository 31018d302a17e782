// util.cu -- device prefix sum and error-message plumbing.
#include "amg_internal.cuh"
#include "device_util.cuh"

namespace amg {

namespace {
thread_local std::string g_last_error;

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Sum of one tile of SCAN_TILE inputs.
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_sum(const int* __restrict__ in, int n, int* __restrict__ bsum) {
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    int s = 0;
    for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_THREADS) {
        long long i = base + k;
        if (i < n) s += in[i];
    }
    s = block_sum_int(s);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s;
}

// Exclusive scan of one tile, offset by the scanned tile sums. Each thread
// owns SCAN_ITEMS consecutive items, so in-place use is safe.
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const int* in, int* out, int n,
                                                            const int* __restrict__ boff, int* total) {
    const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int run = block_exclusive_scan_int(s) + (boff ? boff[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) *total = run;
}
}  // namespace

void set_last_error(const std::string& m) { g_last_error = m; }

std::atomic<long long>& launch_counter() {
    static std::atomic<long long> c{0};
    return c;
}
const char* last_error_cstr() { return g_last_error.c_str(); }

size_t scan_scratch_ints(int n) {
    size_t s = 0;
    long long m = n;
    while (m > SCAN_TILE) {
        m = (m + SCAN_TILE - 1) / SCAN_TILE;
        s += (size_t)m + 1;
    }
    return s + 1;
}

void scan_exclusive(const int* in, int* out, int n, int* total_dev, cudaStream_t st, int* scratch) {
    if (n <= 0) {
        if (total_dev) CUDA_CHECK(cudaMemsetAsync(total_dev, 0, sizeof(int), st));
        return;
    }
    const int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        k_tile_scan<<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr, total_dev);
        KERNEL_CHECK();
        return;
    }
    int* bsum = scratch;
    k_tile_sum<<<nb, SCAN_THREADS, 0, st>>>(in, n, bsum);
    KERNEL_CHECK();
    scan_exclusive(bsum, bsum, nb, nullptr, st, scratch + nb + 1);
    k_tile_scan<<<nb, SCAN_THREADS, 0, st>>>(in, out, n, bsum, total_dev);
    KERNEL_CHECK();
}

void keep_pool_reserved() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> g(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done[dev] = true;
}

}  // namespace amg
