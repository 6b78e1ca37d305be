// Device-wide exclusive prefix sum of int32 or int64 (reduce-then-scan, 4096-item tiles).
#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;

// Exclusive scan of one value per thread across the block; returns the block total.
template <typename T>
__device__ T block_exclusive_scan(T v, T &total) {
    __shared__ T warp_tot[kThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T t = lane < kThreads / 32 ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kThreads / 32) warp_tot[lane] = t;   // inclusive
    }
    __syncthreads();
    T before = warp > 0 ? warp_tot[warp - 1] : T(0);
    total = warp_tot[kThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

template <typename T>
__global__ void k_tile_reduce(const T *__restrict__ in, int64_t n, T *__restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * kTile;
    T s = 0;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        if (g < n) s += in[g];
    }
    T tot;
    block_exclusive_scan<T>(s, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// out[base + i] = offset + exclusive scan within the tile; the last tile writes out[n].
template <typename T>
__global__ void k_tile_scan(const T *__restrict__ in, T *__restrict__ out, int64_t n, const T *__restrict__ tile_off) {
    __shared__ T buf[kTile];
    int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        buf[i] = g < n ? in[g] : 0;
    }
    __syncthreads();
    T loc[kItems];
    T s = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        loc[j] = s;
        s += buf[threadIdx.x * kItems + j];
    }
    T tot;
    T pre = block_exclusive_scan<T>(s, tot);
    T off = tile_off ? tile_off[blockIdx.x] : T(0);
#pragma unroll
    for (int j = 0; j < kItems; ++j) buf[threadIdx.x * kItems + j] = loc[j] + pre + off;
    __syncthreads();
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        if (g < n) out[g] = buf[i];
    }
    if (threadIdx.x == 0 && base + kTile >= n) out[n] = off + tot;
}

template <typename T>
void scan_exclusive(const T *in, T *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        RBF_CUDA(cudaMemsetAsync(out, 0, sizeof(T), s));
        return;
    }
    int64_t ntiles = ceil_div(n, kTile);
    if (ntiles == 1) {
        k_tile_scan<T><<<1, kThreads, 0, s>>>(in, out, n, nullptr);
        RBF_LAUNCHED();
        return;
    }
    DevBuf<T> sums, offs;
    sums.alloc(ntiles, s);
    offs.alloc(ntiles + 1, s);
    k_tile_reduce<T><<<(unsigned)ntiles, kThreads, 0, s>>>(in, n, sums.p);
    RBF_LAUNCHED();
    scan_exclusive<T>(sums.p, offs.p, ntiles, s);
    k_tile_scan<T><<<(unsigned)ntiles, kThreads, 0, s>>>(in, out, n, offs.p);
    RBF_LAUNCHED();
}

}  // namespace

void scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) { scan_exclusive<int32_t>(in, out, n, s); }
void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) { scan_exclusive<int64_t>(in, out, n, s); }
