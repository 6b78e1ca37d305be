// Stable LSD radix sort of (uint32 key, int32 value) pairs, 8-bit digits.
//
// Per pass: (1) every 4096-key tile counts its digits, (2) an exclusive scan over
// the digit-major [256][tiles] count matrix gives each (digit, tile) its output
// base, (3) every tile scatters its keys in input order: inside a 256-key round
// the rank of a key among equal digits comes from __match_any_sync (within a
// warp) plus the counts of the lower warps, so the scatter is stable.
#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRounds = 16;
constexpr int kTile = kThreads * kRounds;
constexpr int kRadix = 256;

__global__ void k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift, uint32_t mask,
                             int ntiles, int32_t *__restrict__ hist) {
    __shared__ int h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += kThreads) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kRounds; ++r) {
        int64_t g = base + r * kThreads + threadIdx.x;
        if (g < n) atomicAdd(&h[(keys[g] >> shift) & mask], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kThreads) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

__global__ void k_radix_scatter(const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin,
                                uint32_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t n,
                                int shift, uint32_t mask, int ntiles, const int32_t *__restrict__ offs) {
    __shared__ int base_d[kRadix];
    __shared__ int wcnt[kWarps][kRadix];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kRadix; d += kThreads) {
        base_d[d] = offs[(int64_t)d * ntiles + blockIdx.x];
        for (int w = 0; w < kWarps; ++w) wcnt[w][d] = 0;
    }
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t tbase = (int64_t)blockIdx.x * kTile;
    for (int r = 0; r < kRounds; ++r) {
        int64_t g = tbase + r * kThreads + threadIdx.x;
        bool valid = g < n;
        uint32_t key = valid ? kin[g] : 0u;
        int val = valid ? vin[g] : 0;
        int d = valid ? (int)((key >> shift) & mask) : kRadix;   // kRadix = "no key"
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt_mask);
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int off = base_d[d] + rank;
            for (int w = 0; w < warp; ++w) off += wcnt[w][d];
            kout[off] = key;
            vout[off] = val;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < kRadix; dd += kThreads) {
            int t = 0;
            for (int w = 0; w < kWarps; ++w) {
                t += wcnt[w][dd];
                wcnt[w][dd] = 0;
            }
            base_d[dd] += t;
        }
        __syncthreads();
    }
}

}  // namespace

void radix_sort_pairs(uint32_t *keys, int32_t *vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return;
    int ntiles = (int)ceil_div(n, kTile);
    DevBuf<uint32_t> k2;
    DevBuf<int32_t> v2, hist, offs;
    k2.alloc(n, s);
    v2.alloc(n, s);
    hist.alloc((size_t)kRadix * ntiles, s);
    offs.alloc((size_t)kRadix * ntiles + 1, s);
    uint32_t *ka = keys, *kb = k2.p;
    int32_t *va = vals, *vb = v2.p;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        int w = bits - shift < 8 ? bits - shift : 8;
        uint32_t mask = (1u << w) - 1u;
        k_radix_hist<<<ntiles, kThreads, 0, s>>>(ka, n, shift, mask, ntiles, hist.p);
        RBF_LAUNCHED();
        scan_exclusive_i32(hist.p, offs.p, (int64_t)kRadix * ntiles, s);
        k_radix_scatter<<<ntiles, kThreads, 0, s>>>(ka, va, kb, vb, n, shift, mask, ntiles, offs.p);
        RBF_LAUNCHED();
        std::swap(ka, kb);
        std::swap(va, vb);
        ++passes;
    }
    if (passes & 1) {
        RBF_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        RBF_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
}
