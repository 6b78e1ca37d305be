// Throughput probes for the roofline of the product kernels: MUFU.EX2 and
// FP32 FMA (scalar and packed f32x2) per SM per clock, with the SM clock read
// from the cycle counter against the global nanosecond timer during the run.
#include "common.cuh"
#include "../../include/rbf_probe.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// mode 0: ex2.approx chains; 1: scalar FFMA chains; 2: packed f32x2 FMA chains
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

template <int kMode>
double run_probe(int num_sms, double ops_per_iter_per_thread, double *mhz, cudaStream_t s) {
    const int blocks = num_sms * 8, iters = 20000;
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
        return RBF_OK;
    } catch (const RbfError &e) {
        return e.status;
    }
}
