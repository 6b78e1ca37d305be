// Device-wide exclusive prefix sum of int32 (reduce-then-scan, 4096-item tiles).
#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;

// Exclusive scan of one value per thread across the block; returns the block total.
__device__ int block_exclusive_scan(int v, int &total) {
    __shared__ int warp_tot[kThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < kThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kThreads / 32) warp_tot[lane] = t;   // inclusive
    }
    __syncthreads();
    int before = warp > 0 ? warp_tot[warp - 1] : 0;
    total = warp_tot[kThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void k_tile_reduce(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * kTile;
    int s = 0;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        if (g < n) s += in[g];
    }
    int tot;
    block_exclusive_scan(s, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// out[base + i] = offset + exclusive scan within the tile; the last tile writes out[n].
__global__ void k_tile_scan(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t n,
                            const int32_t *__restrict__ tile_off) {
    __shared__ int buf[kTile];
    int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        buf[i] = g < n ? in[g] : 0;
    }
    __syncthreads();
    int loc[kItems];
    int s = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        loc[j] = s;
        s += buf[threadIdx.x * kItems + j];
    }
    int tot;
    int pre = block_exclusive_scan(s, tot);
    int off = tile_off ? tile_off[blockIdx.x] : 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) buf[threadIdx.x * kItems + j] = loc[j] + pre + off;
    __syncthreads();
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t g = base + i;
        if (g < n) out[g] = buf[i];
    }
    if (threadIdx.x == 0 && base + kTile >= n) out[n] = off + tot;
}

}  // namespace

void scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        RBF_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
        return;
    }
    int64_t ntiles = ceil_div(n, kTile);
    if (ntiles == 1) {
        k_tile_scan<<<1, kThreads, 0, s>>>(in, out, n, nullptr);
        RBF_LAUNCHED();
        return;
    }
    DevBuf<int32_t> sums, offs;
    sums.alloc(ntiles, s);
    offs.alloc(ntiles + 1, s);
    k_tile_reduce<<<(unsigned)ntiles, kThreads, 0, s>>>(in, n, sums.p);
    RBF_LAUNCHED();
    scan_exclusive_i32(sums.p, offs.p, ntiles, s);
    k_tile_scan<<<(unsigned)ntiles, kThreads, 0, s>>>(in, out, n, offs.p);
    RBF_LAUNCHED();
}
