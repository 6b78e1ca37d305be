// Allocation-free untruncated product y = A z (rbf_matvec_dense_noalloc).
//
// Some callers cannot allocate device memory when they call in: a host that
// reserves all of its device memory up front and forbids later allocation (a
// fixed-budget service or an embedded controller), or code running where an
// allocation would synchronise or fail, such as inside another framework's
// memory pool or in a real-time loop.  This entry point serves them: it uses no
// plan, allocates nothing, and keeps its only scratch - the per-segment
// partial sums of the split over sources - in the file-scope device array
// below, which every GPU that loads the library holds until the process exits.
//
// Modules load lazily, and loading this file's module is what allocates the
// array, so the context does it when it is created (noalloc_prepare): it loads
// the module and both kernels and keeps the array's device address.  A call
// then only launches.
#include <cmath>

#include "common.cuh"

namespace {

constexpr int kNoAllocMaxN = 32768;                 // largest n accepted
constexpr int kSegLen = 1024;                       // sources per segment
constexpr int kMaxSegs = kNoAllocMaxN / kSegLen;    // 32
constexpr int kThreads = 128;                       // targets per CTA

// 32 x 32768 floats = 4 MiB: partial sums [segment][target].
static __device__ __align__(256) float g_noalloc_partial[kMaxSegs * kNoAllocMaxN];

__global__ void __launch_bounds__(kThreads) k_dense_noalloc(const float4 *__restrict__ C, const float *__restrict__ z,
                                                            int n, float c, float *__restrict__ part) {
    __shared__ float4 sp[kThreads];
    __shared__ float sw[kThreads];
    const int i = blockIdx.x * kThreads + threadIdx.x;
    const int seg = blockIdx.y;
    const float4 p = i < n ? C[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int j0 = seg * kSegLen, j1 = min(n, j0 + kSegLen);
    float acc = 0.f;
    for (int jb = j0; jb < j1; jb += kThreads) {
        const int j = jb + threadIdx.x;
        __syncthreads();
        sp[threadIdx.x] = j < j1 ? C[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        sw[threadIdx.x] = j < j1 ? z[j] : 0.f;
        __syncthreads();
        const int cnt = min(kThreads, j1 - jb);
        for (int k = 0; k < cnt; ++k) {
            const float4 q = sp[k];
            const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            acc = fmaf(sw[k], ex2_approx(-r2 * c), acc);
        }
    }
    // every (segment, target) entry read by the reduction is written here first
    if (i < n) part[(int64_t)seg * n + i] = acc;
}

__global__ void k_dense_noalloc_reduce(const float *__restrict__ part, int n, int nseg, float *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = 0.f;
    for (int s = 0; s < nseg; ++s) v += part[(int64_t)s * n + i];
    y[i] = v;
}

}  // namespace

cudaError_t noalloc_prepare(rbf_ctx *ctx) {
    // the name g_noalloc_partial is only a host-side stand-in: a kernel needs the
    // device address, which depends on the device current here
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partial);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_dense_noalloc);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_dense_noalloc_reduce);
    if (e != cudaSuccess || !ptr) {
        (void)cudaGetLastError();
        return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    }
    ctx->noalloc_scratch = (float *)ptr;
    return cudaSuccess;
}

extern "C" rbf_status rbf_matvec_dense_noalloc(rbf_ctx *ctx, const float *centers, int64_t n, float sigma,
                                               const float *z, float *y, void *stream) {
    if (!ctx) return RBF_ERR_INVALID;
    ctx->last_error.clear();
    if (!centers || !z || !y || z == y || ((uintptr_t)centers & 15u) != 0) {
        ctx->last_error = "centers (16-byte aligned), z and y must be distinct device pointers";
        return RBF_ERR_INVALID;
    }
    if (!(std::isfinite(sigma) && sigma > 0.f)) {
        ctx->last_error = "sigma must be finite and > 0";
        return RBF_ERR_INVALID;
    }
    if (n <= 0 || n > kNoAllocMaxN) {
        char buf[160];
        snprintf(buf, sizeof(buf), "n = %lld is outside 1..%d, the size the allocation-free scratch holds",
                 (long long)n, kNoAllocMaxN);
        ctx->last_error = buf;
        return n <= 0 ? RBF_ERR_INVALID : RBF_ERR_UNSUPPORTED;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        ctx->last_error = std::string("device selection: ") + cudaGetErrorString(e);
        return RBF_ERR_CUDA;
    }
    float *part = ctx->noalloc_scratch;          // resolved when the context was created
    if (!part) {
        ctx->last_error = "the allocation-free scratch was not resolved for this context";
        return RBF_ERR_CUDA;
    }
    const int nn = (int)n;
    const int nseg = (nn + kSegLen - 1) / kSegLen;
    const double c = 1.4426950408889634 / (2.0 * (double)sigma * (double)sigma);
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid((nn + kThreads - 1) / kThreads, nseg);
    k_dense_noalloc<<<grid, kThreads, 0, s>>>((const float4 *)centers, z, nn, (float)c, part);
    rbf_count_launch();
    k_dense_noalloc_reduce<<<(nn + 255) / 256, 256, 0, s>>>(part, nn, nseg, y);
    rbf_count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->last_error = std::string("kernel launch: ") + cudaGetErrorString(e);
        return RBF_ERR_CUDA;
    }
    return RBF_OK;
}
