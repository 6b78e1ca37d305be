// Step 1 of Algorithm 1 (Sec. II.A.1-2): the extended data set and its targets,
// plus the bounding-box reduction used for the default offset and the binning.
#include <cmath>

#include "centers.cuh"

namespace {

constexpr int kThreads = 256;

// Per-CTA min/max of points given with a stride (3 floats or float4) and a
// non-finite flag; partial results [cta] = (min xyz, max xyz).
__global__ void k_bbox_partial(const float *__restrict__ p, int64_t n, int stride, float *__restrict__ part,
                               int *__restrict__ bad) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int nonfinite = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float v = p[i * stride + d];
            if (!isfinite(v)) nonfinite = 1;
            mn[d] = fminf(mn[d], v);
            mx[d] = fmaxf(mx[d], v);
        }
    }
    __shared__ float s[6][kThreads / 32];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    }
    nonfinite = __any_sync(0xffffffffu, nonfinite);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        for (int d = 0; d < 3; ++d) {
            s[d][warp] = mn[d];
            s[3 + d][warp] = mx[d];
        }
        if (nonfinite) atomicOr(bad, 1);
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = s[threadIdx.x][0];
        for (int w = 1; w < kThreads / 32; ++w)
            v = threadIdx.x < 3 ? fminf(v, s[threadIdx.x][w]) : fmaxf(v, s[threadIdx.x][w]);
        part[blockIdx.x * 6 + threadIdx.x] = v;
    }
}

__global__ void k_bbox_final(const float *__restrict__ part, int nparts, float *__restrict__ out) {
    if (threadIdx.x < 6) {
        float v = part[threadIdx.x];
        for (int b = 1; b < nparts; ++b)
            v = threadIdx.x < 3 ? fminf(v, part[b * 6 + threadIdx.x]) : fmaxf(v, part[b * 6 + threadIdx.x]);
        out[threadIdx.x] = v;
    }
}

__global__ void k_build_centers(const float *__restrict__ pts, const float *__restrict__ nrm, int64_t N,
                                float delta, float tval, float4 *__restrict__ C, float *__restrict__ b,
                                int *__restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    float nx = nrm[3 * i], ny = nrm[3 * i + 1], nz = nrm[3 * i + 2];
    if (!(isfinite(nx) && isfinite(ny) && isfinite(nz))) atomicOr(bad, 2);
    C[i] = make_float4(x, y, z, 0.f);
    C[N + i] = make_float4(fmaf(delta, nx, x), fmaf(delta, ny, y), fmaf(delta, nz, z), 0.f);
    C[2 * N + i] = make_float4(fmaf(-delta, nx, x), fmaf(-delta, ny, y), fmaf(-delta, nz, z), 0.f);
    b[i] = 0.f;
    b[N + i] = tval;
    b[2 * N + i] = -tval;
}

}  // namespace

// Bounding box of n points (stride floats apart) -> host lo[3], hi[3];
// returns true if every coordinate is finite.  Synchronises the stream.
bool bbox_host(const float *p, int64_t n, int stride, float lo[3], float hi[3], cudaStream_t s) {
    int nparts = (int)std::min<int64_t>(ceil_div(n, kThreads), 4 * 148);
    if (nparts < 1) nparts = 1;
    DevBuf<float> part, out;
    DevBuf<int> bad;
    part.alloc((size_t)nparts * 6, s);
    out.alloc(6, s);
    bad.alloc(1, s);
    bad.zero(s);
    k_bbox_partial<<<nparts, kThreads, 0, s>>>(p, n, stride, part.p, bad.p);
    RBF_LAUNCHED();
    k_bbox_final<<<1, 32, 0, s>>>(part.p, nparts, out.p);
    RBF_LAUNCHED();
    float h[6];
    int hb = 0;
    RBF_CUDA(cudaMemcpyAsync(h, out.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    for (int d = 0; d < 3; ++d) {
        lo[d] = h[d];
        hi[d] = h[3 + d];
    }
    return hb == 0;
}

float build_centers(const float *pts, const float *nrm, int64_t N, float delta, float target, float *centers,
                    float *targets, cudaStream_t s) {
    float lo[3], hi[3];
    bool finite = bbox_host(pts, N, 3, lo, hi, s);
    RBF_CHECK(finite, RBF_ERR_INVALID, "non-finite point coordinate");
    if (!(delta > 0.f)) {
        double d2 = 0;
        for (int d = 0; d < 3; ++d) d2 += (double)(hi[d] - lo[d]) * (double)(hi[d] - lo[d]);
        delta = (float)(0.01 * std::sqrt(d2));
        RBF_CHECK(delta > 0.f, RBF_ERR_INVALID, "degenerate bounding box: default delta is zero");
    }
    float tval = target > 0.f ? target : delta;
    DevBuf<int> bad;
    bad.alloc(1, s);
    bad.zero(s);
    k_build_centers<<<(unsigned)ceil_div(N, kThreads), kThreads, 0, s>>>(pts, nrm, N, delta, tval,
                                                                        (float4 *)centers, targets, bad.p);
    RBF_LAUNCHED();
    int hb = 0;
    RBF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    RBF_CHECK(hb == 0, RBF_ERR_INVALID, "non-finite normal component");
    return delta;
}
