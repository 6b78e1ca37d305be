// Dense contractions of the learned preconditioner's network on the tensor cores
// (tcgen05.mma, kind::tf32, accumulator in tensor memory).
//
//   C[m][n] = epilogue( sum_k A(m, k) B(n, k) )        0 <= m < M, 0 <= n < N
//
// A(m, k) = A[m * a_sr + k * a_sk] (float32), B(n, k) = B[n * b_sr + k * b_sk]
// (float32 or bfloat16), so one kernel serves the forward layers (activations
// times W^T) and both backward contractions (dC W and dC^T A) by strides alone.
// A CTA computes a 128 x 64 tile of C; it stages 128 rows of A and 64 rows of B per
// K chunk of 32 into shared memory as no-swizzle K-major core matrices (8 rows x 16 bytes),
// splitting float32 values into a tf32 head and a tf32 tail (x = h + l to about
// 22 significant bits).  Per 8-wide K step one thread issues
//   h_A h_B                      (kProducts = 1),
//   h_A h_B + l_A h_B            (kProducts = 2: B exact in tf32, e.g. bf16 weights),
//   h_A h_B + l_A h_B + h_A l_B  (kProducts = 3: both operands float32),
// so kProducts = 2 with bf16 weights and 3 with float32 weights give float32-class
// results.  Two stages alternate: the CTA loads chunk c + 1 while the MMAs of
// chunk c run (every thread issues its loads of a chunk before it waits for the
// stage); tcgen05.commit on a per-stage mbarrier says when a stage may be
// overwritten.  The epilogue reads the 128 x 64 float32 accumulator with
// tcgen05.ld (warp w: rows 32w .. 32w + 31), passes each 32 x 32 piece through
// shared memory so that stores run along rows, and applies bias, ReLU and a skip
// term.  Short, wide-K contractions (the weight gradients: 64 or 256 rows, a
// batch of K) are split along K over more CTAs; the partial tiles are then added
// in a fixed order, so results do not depend on scheduling.  Every wait is bounded (1 s): on expiry the context's error word is
// raised and the CTA returns after the issued MMAs finish (bounded again).
#include <cuda_bf16.h>

#include "gemm_tc.cuh"
#include "tcgen05.cuh"

namespace {

constexpr int kGT = 128;                     // threads: 4 warps, one per 32 accumulator lanes
constexpr int kBM = 128;                     // rows of A (and of C) per CTA
constexpr int kBK = 16;                      // K per stage (small stages: 4-5 CTAs per SM hide latency)
constexpr uint32_t kLbo = 128;               // next 16-byte K chunk of the same 8 rows
constexpr uint32_t kSbo = (kBK / 4) * 128;   // next group of 8 rows: kBK / 4 chunks of 128 bytes
constexpr uint64_t kWaitNs = 1000000000ull;

__host__ __device__ constexpr int tile_bytes(int rows) { return rows / 8 * (int)kSbo; }

__device__ __forceinline__ uint32_t core_off(int row, int chunk) {
    return (uint32_t)((row >> 3) * kSbo + chunk * kLbo + (row & 7) * 16);
}

__device__ __forceinline__ float ld_val(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_val(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// Four consecutive-k values of row r starting at k (zero outside the matrix); one
// vector load when k is contiguous, all four are inside and the address is aligned.
__device__ __forceinline__ bool vec_ok(const float *q) { return ((uintptr_t)q & 15u) == 0; }
__device__ __forceinline__ bool vec_ok(const __nv_bfloat16 *q) { return ((uintptr_t)q & 7u) == 0; }
__device__ __forceinline__ float4 vec_ld(const float *q) { return __ldg(reinterpret_cast<const float4 *>(q)); }
__device__ __forceinline__ float4 vec_ld(const __nv_bfloat16 *q) {
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(q));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                       __uint_as_float(u.y & 0xffff0000u));
}
template <typename T, bool kCont>
__device__ __forceinline__ float4 load4(const T *src, int64_t sr, int64_t sk, int r, int R, int k, int K) {
    if (r >= R) return make_float4(0.f, 0.f, 0.f, 0.f);
    const T *q = src + (int64_t)r * sr + (int64_t)k * sk;
    if (kCont && k + 3 < K && vec_ok(q)) return vec_ld(q);
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = k + i < K ? ld_val(q + (int64_t)i * sk) : 0.f;
    return make_float4(v[0], v[1], v[2], v[3]);
}

__device__ __forceinline__ float4 head4(float4 v) {
    return make_float4(tc5::to_tf32(v.x), tc5::to_tf32(v.y), tc5::to_tf32(v.z), tc5::to_tf32(v.w));
}
__device__ __forceinline__ float4 tail4(float4 v, float4 h) {
    return make_float4(tc5::to_tf32(v.x - h.x), tc5::to_tf32(v.y - h.y), tc5::to_tf32(v.z - h.z),
                       tc5::to_tf32(v.w - h.w));
}

// One operand's share of a K chunk of 32, per thread: kItems float4 (4 consecutive k
// of one row).  kCont: k is the contiguous index (a warp walks chunks of a few rows);
// otherwise rows are (a warp walks 32 rows), so every warp-wide load reads consecutive
// addresses.  The loads of a chunk are all issued before any is used.
template <typename T, bool kCont, int kRows>
struct Stager {
    static constexpr int kItems = kRows * (kBK / 4) / kGT;
    float4 v[kItems];
    __device__ __forceinline__ static void coords(int it, int &row, int &ch) {
        row = kCont ? it / (kBK / 4) : it % kRows;
        ch = kCont ? it % (kBK / 4) : it / kRows;
    }
    __device__ __forceinline__ void load(const T *src, int64_t sr, int64_t sk, int r0, int R, int k0, int K) {
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            int row, ch;
            coords((int)threadIdx.x + i * kGT, row, ch);
            v[i] = load4<T, kCont>(src, sr, sk, r0 + row, R, k0 + 4 * ch, K);
        }
    }
    __device__ __forceinline__ void store(uint8_t *hi, uint8_t *lo) const {
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            int row, ch;
            coords((int)threadIdx.x + i * kGT, row, ch);
            const float4 h = head4(v[i]);
            *reinterpret_cast<float4 *>(hi + core_off(row, ch)) = h;
            if (lo) *reinterpret_cast<float4 *>(lo + core_off(row, ch)) = tail4(v[i], h);
        }
    }
};

template <int kBN, int kProducts>
struct GemmSmem {
    static constexpr int kA = tile_bytes(kBM), kB = tile_bytes(kBN);
    static constexpr bool kSplitB = kProducts == 3;
    static constexpr int kStage = 2 * kA + (kSplitB ? 2 : 1) * kB;
    static constexpr int kEpi = kGT / 32 * 32 * 33 * 4;        // per-warp 32 x 33 float tiles
    static constexpr int kBody = 2 * kStage > kEpi ? 2 * kStage : kEpi;
    static constexpr int kBytes = kBody + 64;                   // then barriers and flags
};

// Wait (every thread, bounded) for the phase of a stage barrier; false for all threads
// when any of them gave up (the decision is made uniform through shared memory).
__device__ __forceinline__ bool wait_all(uint64_t *bar, uint32_t parity, volatile int *abort_flag, uint64_t lim,
                                         unsigned *err) {
    if (!tc5::mbar_wait(bar, parity, (const volatile int *)abort_flag, lim)) {
        *abort_flag = 1;
        if (err) atomicOr(err, 1u);
    }
    __syncthreads();
    return *abort_flag == 0;
}

// Grid: (row tiles of 128, column tiles of kBN, K slices of g.kslice chunks).  With more
// than one K slice, slice z writes its partial C to g.C + z g.c_zstride (no epilogue).
template <int kBN, int kProducts, typename TB, bool kACont, bool kBCont>
__global__ void __launch_bounds__(kGT) k_gemm_tc(GemmArgs g, const float *__restrict__ A,
                                                 const TB *__restrict__ B, unsigned *err) {
    using L = GemmSmem<kBN, kProducts>;
    constexpr uint32_t kCols = kBN <= 32 ? 32 : kBN <= 64 ? 64 : kBN <= 128 ? 128 : 256;
    constexpr uint32_t kIdesc = tc5::idesc_tf32(kBM, kBN);
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *done = reinterpret_cast<uint64_t *>(smem + L::kBody);
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(done + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_base + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;

    if (warp == 0) {
        tc5::tmem_alloc(tmem_base, kCols);
        tc5::tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        tc5::mbar_init(&done[0], 1);
        tc5::mbar_init(&done[1], 1);
        *abort_flag = 0;
        tc5::mbar_init_fence();
    }
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tmem = *tmem_base;

    const int nch = (g.K + kBK - 1) / kBK;
    const int c0 = blockIdx.z * g.kslice, c1 = min(nch, c0 + g.kslice);
    const TB *Bn = B + (int64_t)n0 * g.b_sr;
    // two register sets: chunk c + 1's loads are in flight while chunk c is converted
    Stager<float, kACont, kBM> sa0, sa1;
    Stager<TB, kBCont, kBN> sb0, sb1;
    int last = -1;   // last chunk whose MMAs were committed
    auto step = [&](Stager<float, kACont, kBM> &ca, Stager<TB, kBCont, kBN> &cb, Stager<float, kACont, kBM> &na,
                    Stager<TB, kBCont, kBN> &nb, int c) -> bool {
        const int j = c - c0, s = j & 1;
        uint8_t *ahi = smem + s * L::kStage, *alo = ahi + L::kA, *bhi = ahi + 2 * L::kA;
        uint8_t *blo = L::kSplitB ? bhi + L::kB : nullptr;
        if (c + 1 < c1) {
            na.load(A, g.a_sr, g.a_sk, m0, g.M, (c + 1) * kBK, g.K);
            nb.load(Bn, g.b_sr, g.b_sk, 0, g.N - n0, (c + 1) * kBK, g.K);
        }
        // the MMAs of chunk c - 2 read this stage: wait until they are done
        if (j >= 2 && !wait_all(&done[s], (uint32_t)((j - 2) >> 1) & 1u, abort_flag, kWaitNs, err)) return false;
        ca.store(ahi, alo);
        cb.store(bhi, blo);
        tc5::fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc5::fence_after_sync();
            const uint64_t da = tc5::smem_desc(tc5::smem_u32(ahi), kLbo, kSbo);
            const uint64_t dal = tc5::smem_desc(tc5::smem_u32(alo), kLbo, kSbo);
            const uint64_t db = tc5::smem_desc(tc5::smem_u32(bhi), kLbo, kSbo);
            const uint64_t dbl = L::kSplitB ? tc5::smem_desc(tc5::smem_u32(blo), kLbo, kSbo) : 0ull;
#pragma unroll
            for (int i = 0; i < kBK / 8; ++i) {
                const uint64_t st = (uint64_t)((i * 2 * kLbo) >> 4);   // two 16-byte chunks per K step of 8
                tc5::mma_tf32(tmem, da + st, db + st, kIdesc, (j > 0 || i > 0) ? 1u : 0u);
                if (kProducts >= 2) tc5::mma_tf32(tmem, dal + st, db + st, kIdesc, 1u);
                if (kProducts >= 3) tc5::mma_tf32(tmem, da + st, dbl + st, kIdesc, 1u);
            }
            tc5::mma_commit(&done[s]);
        }
        last = j;
        return true;
    };
    if (c0 < c1) {
        sa0.load(A, g.a_sr, g.a_sk, m0, g.M, c0 * kBK, g.K);
        sb0.load(Bn, g.b_sr, g.b_sk, 0, g.N - n0, c0 * kBK, g.K);
    }
    for (int c = c0; c < c1; c += 2) {
        if (!step(sa0, sb0, sa1, sb1, c)) break;
        if (c + 1 < c1 && !step(sa1, sb1, sa0, sb0, c + 1)) break;
    }
    // the accumulator is complete when the last committed chunk's MMAs are (after an
    // abort, wait a shorter bounded time so that no MMA is in flight at the release)
    bool ok = *abort_flag == 0;   // uniform: read after the CTA's last barrier
    if (last >= 0) {
        const uint32_t par = (uint32_t)(last >> 1) & 1u;
        if (ok) ok = wait_all(&done[last & 1], par, abort_flag, kWaitNs, err);
        if (!ok) {
            const uint64_t t0 = tc5::global_ns();
            while (!tc5::mbar_try_wait(&done[last & 1], par) && tc5::global_ns() - t0 < kWaitNs / 10) {
            }
            __syncthreads();
        }
    }
    tc5::fence_after_sync();
    if (ok) {
        // warp w holds rows 32w .. 32w + 31; each 32 x 32 piece goes through this warp's
        // shared tile so that the stores run along rows (one 128-byte row per instruction)
        float *tile = reinterpret_cast<float *>(smem) + warp * 32 * 33;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        float *C = g.C + (int64_t)blockIdx.z * g.c_zstride;
        const bool epi = gridDim.z == 1;
#pragma unroll 1
        for (int q = 0; q < kBN; q += 32) {
            float v[32];
            if (last >= 0) {
                tc5::tmem_ld_32x32(trow + (uint32_t)q, v);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.f;    // an empty K slice contributes zero
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) tile[lane * 33 + i] = v[i];   // row `lane`, column i
            __syncwarp();
            const int n = n0 + q + lane;
            const float bn = (epi && g.bias && n < g.N) ? g.bias[n] : 0.f;
#pragma unroll 4
            for (int r = 0; r < 32; ++r) {
                const int m = m0 + warp * 32 + r;
                if (m < g.M && n < g.N) {
                    float x = tile[r * 33 + lane];
                    if (epi) {
                        x += bn;
                        if (g.relu) x = fmaxf(x, 0.f);
                        if (g.skip) x += g.skip[(int64_t)m * g.ldskip + n];
                    }
                    C[(int64_t)m * g.ldc + n] = x;
                }
            }
            __syncwarp();
        }
    }
    tc5::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc5::fence_after_sync();
        tc5::tmem_dealloc(tmem, kCols);
    }
}

// out[i] = sum_z part[z * stride + i], slices added in order
__global__ void k_sum_slices(const float *__restrict__ part, int nz, int64_t stride, int M, int N, int64_t ldc,
                             float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * N) return;
    const int64_t m = i / N, n = i % N;
    float acc = 0.f;
    for (int z = 0; z < nz; ++z) acc += part[z * stride + m * N + n];
    out[m * ldc + n] = acc;
}

template <int kBN, int kProducts, typename TB, bool kACont, bool kBCont>
void launch(const GemmArgs &g0, const float *A, const TB *B, unsigned *err, cudaStream_t s) {
    constexpr int smem = GemmSmem<kBN, kProducts>::kBytes;
    static_assert(smem <= 227 * 1024, "shared memory");
    auto k = k_gemm_tc<kBN, kProducts, TB, kACont, kBCont>;
    static bool attr_set[64] = {};      // once per device and kernel instance
    int dev = 0;
    RBF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        RBF_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    if (g0.M <= 0) return;
    GemmArgs g = g0;
    const int mt = (g.M + kBM - 1) / kBM, nt = (g.N + kBN - 1) / kBN, nch = (g.K + kBK - 1) / kBK;
    // split K when the tiles alone cannot fill the GPU (the weight gradients: few rows,
    // a long batch); slices of at least 2 chunks, partial sums added in a fixed order
    int nz = 1;
    if (g.bias == nullptr && g.skip == nullptr && !g.relu && mt * nt < 64 && nch >= 4)
        nz = std::min((nch + 1) / 2, std::max(1, 128 / (mt * nt)));
    g.kslice = (nch + nz - 1) / nz;
    nz = (nch + g.kslice - 1) / g.kslice;
    if (nz == 1) {
        g.c_zstride = 0;
        k<<<dim3((unsigned)mt, (unsigned)nt, 1), kGT, smem, s>>>(g, A, B, err);
        RBF_LAUNCHED();
        return;
    }
    DevBuf<float> part;
    part.alloc((size_t)nz * g.M * g.N, s);
    GemmArgs gp = g;
    gp.C = part.p;
    gp.ldc = g.N;
    gp.c_zstride = (int64_t)g.M * g.N;
    k<<<dim3((unsigned)mt, (unsigned)nt, (unsigned)nz), kGT, smem, s>>>(gp, A, B, err);
    RBF_LAUNCHED();
    const int64_t tot = (int64_t)g.M * g.N;
    k_sum_slices<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part.p, nz, gp.c_zstride, g.M, g.N, g.ldc, g.C);
    RBF_LAUNCHED();
}

template <typename TB>
void dispatch_layout(const GemmArgs &g, const float *A, const TB *B, int products, unsigned *err, cudaStream_t s) {
    const bool ac = g.a_sk == 1, bc = g.b_sk == 1;
    RBF_CHECK(ac || g.a_sr == 1, RBF_ERR_INVALID, "tensor-core GEMM: A needs a unit stride");
    RBF_CHECK(bc || g.b_sr == 1, RBF_ERR_INVALID, "tensor-core GEMM: B needs a unit stride");
    if (products == 2) {
        RBF_CHECK(ac && bc, RBF_ERR_INVALID, "tensor-core GEMM: two products only for K-contiguous operands");
        launch<64, 2, TB, true, true>(g, A, B, err, s);
    } else if (ac && bc) {
        launch<64, 3, TB, true, true>(g, A, B, err, s);
    } else if (ac && !bc) {
        launch<64, 3, TB, true, false>(g, A, B, err, s);
    } else if (!ac && !bc) {
        launch<64, 3, TB, false, false>(g, A, B, err, s);
    } else {
        launch<64, 3, TB, false, true>(g, A, B, err, s);
    }
}

}  // namespace

void gemm_tc(const GemmArgs &g, const float *A, const float *B, int products, unsigned *err, cudaStream_t s) {
    RBF_CHECK(g.N > 0 && g.K > 0 && g.M >= 0, RBF_ERR_INVALID, "tensor-core GEMM: empty operand");
    RBF_CHECK(products == 2 || products == 3, RBF_ERR_INVALID, "tensor-core GEMM: 2 or 3 products");
    dispatch_layout<float>(g, A, B, products, err, s);
}

void gemm_tc(const GemmArgs &g, const float *A, const __nv_bfloat16 *B, int products, unsigned *err,
             cudaStream_t s) {
    RBF_CHECK(g.N > 0 && g.K > 0 && g.M >= 0, RBF_ERR_INVALID, "tensor-core GEMM: empty operand");
    RBF_CHECK(products == 2, RBF_ERR_INVALID, "tensor-core GEMM: bf16 operands are exact in tf32 (2 products)");
    dispatch_layout<__nv_bfloat16>(g, A, B, 2, err, s);
}
