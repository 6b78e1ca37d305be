// Throughput probes for the rooflines: MUFU.EX2 and FP32 FMA (scalar and packed
// f32x2) per SM per clock for the product kernels, FP64 FMA per SM per clock for
// the float64 Arnoldi vector work, with the SM clock read from the cycle counter
// against the global nanosecond timer during the run.
#include "common.cuh"
#include "tcgen05.cuh"
#include "../../include/rbf_probe.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// mode 0: ex2.approx chains; 1: scalar FFMA chains; 2: packed f32x2 FMA chains;
// 3: float64 FMA chains
template <int kMode>
__global__ void __launch_bounds__(kThreads) k_probe(int iters, float seed, float *out, unsigned long long *clk) {
    unsigned long long c0 = clock64(), t0 = gtimer();
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed * (float)(threadIdx.x + c + 1) * 1e-9f;
    if (kMode == 0) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = ex2_approx(v[c]) - 1.0f;   // stays near 0
        }
    } else if (kMode == 1) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], 0.999999f, 1e-7f);
        }
    } else if (kMode == 3) {
        double d[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) d[c] = (double)v[c];
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) d[c] = fma(d[c], 0.999999, 1e-7);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = (float)d[c];
    } else {
        unsigned long long p[kChains / 2], a, b;
        asm("mov.b64 %0, {%1,%2};" : "=l"(a) : "f"(0.999999f), "f"(0.999999f));
        asm("mov.b64 %0, {%1,%2};" : "=l"(b) : "f"(1e-7f), "f"(1e-7f));
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) asm("mov.b64 %0, {%1,%2};" : "=l"(p[c]) : "f"(v[2 * c]), "f"(v[2 * c + 1]));
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains / 2; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[c]) : "l"(a), "l"(b));
        }
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) asm("mov.b64 {%0,%1}, %2;" : "=f"(v[2 * c]), "=f"(v[2 * c + 1]) : "l"(p[c]));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 12345.678f) out[0] = s;   // keeps the chains alive
    unsigned long long c1 = clock64(), t1 = gtimer();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        clk[0] = c1 - c0;
        clk[1] = t1 - t0;
    }
}

// Latency of the product's tensor-core step: thread 0 of each CTA issues `stages` pairs of
// dependent tf32 MMAs (M 128, N 32, K 8; operands zero) into distinct TMEM columns, each
// pair followed by a commit to its own mbarrier, then waits for every phase; averaged
// over `rounds`.  Every wait gives up after 100 ms and reports it in out[2].
__global__ void __launch_bounds__(128) k_probe_mma(int rounds, int stages, unsigned long long *out) {
    __shared__ __align__(1024) uint8_t A[128 * 64];
    __shared__ __align__(1024) uint8_t B[32 * 64];
    __shared__ uint64_t bar[4];
    __shared__ uint32_t tm;
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (int)(sizeof(A) / 4); i += blockDim.x) reinterpret_cast<float *>(A)[i] = 0.f;
    for (int i = threadIdx.x; i < (int)(sizeof(B) / 4); i += blockDim.x) reinterpret_cast<float *>(B)[i] = 0.f;
    if (warp == 0) {
        tc5::tmem_alloc(&tm, 128);
        tc5::tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < 4; ++s) tc5::mbar_init(&bar[s], 1);
        tc5::mbar_init_fence();
    }
    tc5::fence_async_smem();
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tmem = tm;
    if (threadIdx.x == 0) {
        const uint32_t idesc = tc5::idesc_tf32(128, 32), a = tc5::smem_u32(A), b = tc5::smem_u32(B);
        unsigned long long tot = 0;
        bool late = false;
        for (int it = 0; it < rounds && !late; ++it) {
            const long long t0 = clock64();
            for (int s = 0; s < stages; ++s) {
                const uint32_t d = tmem + 32u * (uint32_t)s;
                tc5::mma_tf32(d, tc5::smem_desc(a, 128, 512), tc5::smem_desc(b, 128, 512), idesc, 0u);
                tc5::mma_tf32(d, tc5::smem_desc(a + 256, 128, 512), tc5::smem_desc(b + 256, 128, 512), idesc, 1u);
                tc5::mma_commit(&bar[s]);
            }
            for (int s = 0; s < stages; ++s) {
                const uint64_t g0 = tc5::global_ns();
                while (!tc5::mbar_try_wait(&bar[s], (uint32_t)it & 1u)) {
                    if (tc5::global_ns() - g0 > 100000000ull) {
                        late = true;
                        break;
                    }
                }
            }
            tot += (unsigned long long)(clock64() - t0);
        }
        if (late) atomicAdd(&out[2], 1ull);
        atomicAdd(&out[0], tot / (unsigned long long)rounds);
        atomicAdd(&out[1], 1ull);
    }
    tc5::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc5::fence_after_sync();
        tc5::tmem_dealloc(tmem, 128);
    }
}

double run_probe_mma(int num_sms, int stages, cudaStream_t s) {
    DevBuf<unsigned long long> out;
    out.alloc(3, s);
    out.zero(s);
    k_probe_mma<<<num_sms, 128, 0, s>>>(200, stages, out.p);
    RBF_LAUNCHED();
    unsigned long long h[3];
    RBF_CUDA(cudaMemcpyAsync(h, out.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    RBF_CHECK(h[2] == 0, RBF_ERR_TIMEOUT, "tensor-core latency probe: an mbarrier wait expired");
    return h[1] ? (double)h[0] / (double)h[1] : 0.0;
}

template <int kMode>
double run_probe(int num_sms, double ops_per_iter_per_thread, double *mhz, cudaStream_t s) {
    const int blocks = num_sms * 8, iters = kMode == 3 ? 1000 : 20000;   // float64 runs far slower
    DevBuf<float> out;
    DevBuf<unsigned long long> clk;
    out.alloc(1, s);
    clk.alloc(2, s);
    cudaEvent_t a, b;
    RBF_CUDA(cudaEventCreate(&a));
    RBF_CUDA(cudaEventCreate(&b));
    k_probe<kMode><<<blocks, kThreads, 0, s>>>(iters / 10, 0.5f, out.p, clk.p);   // warm-up
    RBF_LAUNCHED();
    RBF_CUDA(cudaEventRecord(a, s));
    k_probe<kMode><<<blocks, kThreads, 0, s>>>(iters, 0.5f, out.p, clk.p);
    RBF_LAUNCHED();
    RBF_CUDA(cudaEventRecord(b, s));
    RBF_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    RBF_CUDA(cudaEventElapsedTime(&ms, a, b));
    unsigned long long hc[2];
    RBF_CUDA(cudaMemcpy(hc, clk.p, sizeof(hc), cudaMemcpyDeviceToHost));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    double f = hc[1] > 0 ? (double)hc[0] / (double)hc[1] * 1e3 : 0.0;   // MHz
    *mhz = f;
    double ops = (double)blocks * kThreads * iters * ops_per_iter_per_thread;
    double per_s = ops / (ms * 1e-3);
    return per_s / ((double)num_sms * f * 1e6);   // per SM per clock
}

// A wait that nothing completes (see rbf_probe_wait_expiry).
__global__ void k_expiring_wait(unsigned *err, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        tc5::mbar_init(&bar, 1);
        tc5::mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc5::mbar_wait(&bar, 0u, &abort_flag, limit_ns)) atomicOr(err, kErrTimeout);
}

}  // namespace

extern "C" rbf_status rbf_probe_peaks(int device, rbf_probe_result *r) {
    if (!r) return RBF_ERR_INVALID;
    try {
        RBF_CUDA(cudaSetDevice(device));
        int sms = 0;
        RBF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        r->num_sms = sms;
        double m0, m1, m2;
        r->ex2_per_clk_sm = run_probe<0>(sms, kChains, &m0, 0);
        r->ffma_per_clk_sm = run_probe<1>(sms, kChains, &m1, 0);
        r->ffma2_lanes_per_clk_sm = run_probe<2>(sms, kChains, &m2, 0);
        r->sm_mhz = (m0 + m1 + m2) / 3.0;
        double m3;
        r->dfma_per_clk_sm = run_probe<3>(sms, kChains, &m3, 0);
        r->mma_commit_cycles = run_probe_mma(sms, 1, 0);
        r->mma_commit4_cycles = run_probe_mma(sms, 4, 0);
        return RBF_OK;
    } catch (const RbfError &e) {
        return e.status;
    }
}

void launch_expiring_wait(unsigned *err, uint64_t limit_ns, cudaStream_t s) {
    const uint64_t lim = limit_ns < 1000ull ? 1000ull : (limit_ns > 1000000000ull ? 1000000000ull : limit_ns);
    k_expiring_wait<<<1, 32, 0, s>>>(err, (unsigned long long)lim);
    RBF_LAUNCHED();
}
