// Density measures of the point cloud (Sec. IV): the nearest-neighbour distance
// of every point, the separation distance q = 1/2 min_{i!=j} |x_i - x_j|
// (Eq. sepDist), h_max = max_j min_{i!=j} |x_i - x_j|, their mean, and, over
// caller-given probe points of the domain, the fill distance
// max_p min_j |p - x_j| (Eq. fillDist); the sigma rules 2 q (Eq. h1),
// fill sqrt(2) (Eq. h2) and h_max sqrt(2) (Eq. hmax) are derived on the host.
//
// The points are binned with the plan's binning (coarse cells of edge e).  A
// thread searches the cells around its point ring by ring (Chebyshev distance
// rho = 0, 1, ...); once ring rho is done, every unvisited point lies at least
// rho e away (it is separated by rho whole cells along some axis), so the search
// stops when the best distance found is <= rho e.  Distances are float32 from
// the float32 coordinates; min, max and sum are reduced in the device.
#include <cmath>
#include <cstring>

#include "centers.cuh"
#include "plan.cuh"

namespace {

constexpr int kThr = 256;

struct DensityAcc {
    unsigned int min_bits;     // float bits of the smallest nearest-neighbour distance (>= 0)
    unsigned int max_bits;     // largest
    unsigned int fill_bits;    // largest probe distance
    unsigned int pad;
    double sum;
};

struct Grid {
    float lo[3];
    float inv;          // fine cells per unit length
    int levels;
    int cdim;           // coarse cells per axis
    float e;            // coarse cell edge
};

__device__ __forceinline__ int coarse(float x, float lo, const Grid &g) {
    float f = floorf((x - lo) * g.inv);
    f = fminf(fmaxf(f, 0.f), (float)((g.cdim << g.levels) - 1));
    return ((int)f) >> g.levels;
}

// Nearest distance from p to the points (binned order), skipping index `self`.
__device__ float nearest(const Grid &g, const float4 *__restrict__ pos, const int32_t *__restrict__ cstart,
                         const int32_t *__restrict__ cend, float px, float py, float pz, int64_t self) {
    const int cx = coarse(px, g.lo[0], g), cy = coarse(py, g.lo[1], g), cz = coarse(pz, g.lo[2], g);
    float best2 = INFINITY;
    for (int rho = 0; rho <= g.cdim; ++rho) {
        for (int dz = -rho; dz <= rho; ++dz) {
            const int z = cz + dz;
            if (z < 0 || z >= g.cdim) continue;
            for (int dy = -rho; dy <= rho; ++dy) {
                const int y = cy + dy;
                if (y < 0 || y >= g.cdim) continue;
                const bool face = (dz == -rho || dz == rho || dy == -rho || dy == rho);
                const int step = face ? 1 : (rho > 0 ? 2 * rho : 1);
                for (int dx = -rho; dx <= rho; dx += step) {
                    const int x = cx + dx;
                    if (x < 0 || x >= g.cdim) continue;
                    const uint32_t code = part1by2_u32(x) | (part1by2_u32(y) << 1) | (part1by2_u32(z) << 2);
                    const int j0 = cstart[code], j1 = cend[code];
                    for (int j = j0; j < j1; ++j) {
                        if ((int64_t)j == self) continue;
                        const float4 q = pos[j];
                        const float ax = px - q.x, ay = py - q.y, az = pz - q.z;
                        best2 = fminf(best2, fmaf(ax, ax, fmaf(ay, ay, az * az)));
                    }
                }
            }
        }
        const float reach = (float)rho * g.e;
        if (best2 <= reach * reach) break;
    }
    return sqrtf(best2);
}

__device__ __forceinline__ void block_reduce(float mn, float mx, double sm, DensityAcc *acc) {
    __shared__ float s_mn[kThr / 32], s_mx[kThr / 32];
    __shared__ double s_sm[kThr / 32];
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_mn[w] = mn;
        s_mx[w] = mx;
        s_sm[w] = sm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kThr / 32; ++i) {
            mn = fminf(mn, s_mn[i]);
            mx = fmaxf(mx, s_mx[i]);
        }
        double t = s_sm[0];
        for (int i = 1; i < kThr / 32; ++i) t += s_sm[i];
        if (mn < INFINITY) atomicMin(&acc->min_bits, __float_as_uint(mn));
        if (mx >= 0.f) atomicMax(&acc->max_bits, __float_as_uint(mx));
        atomicAdd(&acc->sum, t);
    }
}

__global__ void __launch_bounds__(kThr) k_nn_points(Grid g, const float4 *__restrict__ pos,
                                                    const int32_t *__restrict__ cstart,
                                                    const int32_t *__restrict__ cend,
                                                    const int32_t *__restrict__ perm, int64_t n, float *nn,
                                                    DensityAcc *acc) {
    const int64_t i = (int64_t)blockIdx.x * kThr + threadIdx.x;
    float d = -1.f;
    if (i < n) {
        const float4 p = pos[i];
        d = nearest(g, pos, cstart, cend, p.x, p.y, p.z, i);
        if (nn) nn[perm[i]] = d;
    }
    block_reduce(i < n ? d : INFINITY, d, i < n ? (double)d : 0.0, acc);
}

__global__ void __launch_bounds__(kThr) k_nn_probes(Grid g, const float4 *__restrict__ pos,
                                                    const int32_t *__restrict__ cstart,
                                                    const int32_t *__restrict__ cend, const float4 *__restrict__ pr,
                                                    int64_t m, DensityAcc *acc) {
    const int64_t i = (int64_t)blockIdx.x * kThr + threadIdx.x;
    float d = -1.f;
    if (i < m) {
        const float4 p = pr[i];
        d = nearest(g, pos, cstart, cend, p.x, p.y, p.z, -1);
    }
    __shared__ float s_mx[kThr / 32];
    for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
    if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThr / 32; ++k) d = fmaxf(d, s_mx[k]);
        if (d >= 0.f) atomicMax(&acc->fill_bits, __float_as_uint(d));
    }
}

__global__ void k_check_finite(const float4 *__restrict__ p, int64_t m, int *bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        const float4 q = p[i];
        if (!isfinite(q.x) || !isfinite(q.y) || !isfinite(q.z)) atomicOr(bad, 1);
    }
}

float bits_to_float(unsigned int b) {
    float f;
    std::memcpy(&f, &b, sizeof(f));
    return f;
}

}  // namespace

void density_measures(rbf_ctx *ctx, const float4 *pts, int64_t n, const float4 *probes, int64_t m, float cell,
                      float *nn, rbf_density *out, cudaStream_t s) {
    RBF_CHECK(n >= 2, RBF_ERR_INVALID, "density measures need at least 2 points (n = %lld)", (long long)n);
    RBF_CHECK(m >= 0 && (m == 0 || probes), RBF_ERR_INVALID, "probes: m = %lld", (long long)m);
    if (m > 0) {
        DevBuf<int> bad;
        bad.alloc(1, s);
        bad.zero(s);
        k_check_finite<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(probes, m, bad.p);
        RBF_LAUNCHED();
        int hb = 0;
        RBF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(cudaStreamSynchronize(s));
        RBF_CHECK(hb == 0, RBF_ERR_INVALID, "non-finite probe coordinate");
    }
    // binning: coarse cells of edge e (the plan with sigma = e, k = 1); e at least
    // 8 x extent / 1023 (the binning's limit of 1024 fine cells per axis at 3 levels)
    rbf_plan P;
    P.ctx = ctx;
    P.n = n;
    P.cells_per_cutoff = 1;
    P.levels = 3;
    P.k = 1.f;
    {
        float lo[3], hi[3];
        RBF_CHECK(bbox_host((const float *)pts, n, 4, lo, hi, s), RBF_ERR_INVALID, "non-finite point coordinate");
        double ext = 0.0;
        for (int d = 0; d < 3; ++d) ext = std::max(ext, (double)hi[d] - (double)lo[d]);
        double e = cell > 0.f ? (double)cell : 2.0 * ext / std::sqrt((double)n);
        e = std::max(e, 8.0 * ext / 1020.0);
        if (!(e > 0.0)) e = 1.0;   // all points equal
        P.sigma = (float)e;
    }
    plan_build(&P, pts, s, true);
    Grid g;
    for (int d = 0; d < 3; ++d) g.lo[d] = P.lo[d];
    g.inv = P.inv;
    g.levels = P.levels;
    g.cdim = P.cdim;
    g.e = P.rc;
    DevBuf<DensityAcc> acc;
    acc.alloc(1, s);
    DensityAcc h0{0x7f800000u, 0u, 0u, 0u, 0.0};
    RBF_CUDA(cudaMemcpyAsync(acc.p, &h0, sizeof(h0), cudaMemcpyHostToDevice, s));
    k_nn_points<<<(unsigned)ceil_div(n, kThr), kThr, 0, s>>>(g, P.pos.p, P.cell_start.p, P.cell_end.p, P.perm.p, n,
                                                            nn, acc.p);
    RBF_LAUNCHED();
    if (m > 0) {   // probes in cell order, so that neighbouring threads search neighbouring cells
        DevBuf<float4> sp;
        sp.alloc(m, s);
        plan_sorted_copy(&P, probes, m, sp.p, s);
        k_nn_probes<<<(unsigned)ceil_div(m, kThr), kThr, 0, s>>>(g, P.pos.p, P.cell_start.p, P.cell_end.p, sp.p, m,
                                                                acc.p);
        RBF_LAUNCHED();
    }
    DensityAcc h;
    RBF_CUDA(cudaMemcpyAsync(&h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    out->q = 0.5 * (double)bits_to_float(h.min_bits);
    out->h_max = (double)bits_to_float(h.max_bits);
    out->mean_nn = h.sum / (double)n;
    out->fill = m > 0 ? (double)bits_to_float(h.fill_bits) : NAN;
    out->sigma_q = 2.0 * out->q;
    out->sigma_fill = out->fill * std::sqrt(2.0);
    out->sigma_hmax = out->h_max * std::sqrt(2.0);
    out->cell = P.rc;
}
