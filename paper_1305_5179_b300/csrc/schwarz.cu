// Restricted additive Schwarz preconditioner (Sec. III.A, RASM).
//
// Subdomain i of the binned order is the run [d0_i, d0_i + B) around the core
// [s_i, s_i + core) (B = min(block, n), d0_i = clamp(s_i - (block - core)/2, 0,
// n - B)).  Set-up: one CTA per subdomain assembles the untruncated Gaussian
// block A_i + shift I in shared memory (float32, exp2 on the SFU) and factorises
// it in place by a blocked right-looking Cholesky on 32 x 32 tiles; a failed
// pivot retries with a 10x larger shift when escalation is on.  Apply: one warp
// per subdomain gathers v, solves L y = v and L^T x = y tile by tile (ras::solve_block),
// and writes the core entries (restricted) or adds the whole local solution (additive).
#include <cmath>

#include "plan.cuh"
#include "schwarz.cuh"

namespace {

constexpr int kMaxB = 128;
constexpr int kSetupThreads = 128;

__device__ __forceinline__ void dom_of(int64_t blkid, int core, int B, int64_t n, int64_t &d0, int64_t &c0,
                                       int &cl) {
    int64_t s = blkid * core;
    int64_t e = s + core < n ? s + core : n;
    int o = B - core;
    int64_t st = s - o / 2;
    if (st > n - B) st = n - B;
    if (st < 0) st = 0;
    d0 = st;
    c0 = s;
    cl = (int)(e - s);
}

// Blocked Cholesky of the padded matrix (Bp = B rounded up to 32, identity beyond B) in
// shared memory, tiles of 32 x 32, right-looking: the diagonal tile by one warp in
// registers (per column: pivot, column scaled by its reciprocal, the tile's trailing
// triangle), the panel below it by one
// thread per row (substitution against the diagonal tile), the trailing tiles by the
// four warps (each lane one column of a tile, the panel rows broadcast from shared
// memory).  A pivot that is not positive and finite fails the attempt.
__global__ void __launch_bounds__(kSetupThreads) k_schwarz_setup(const float4 *__restrict__ pos, int64_t n, int core,
                                                                 int B, float scl, float imq_beta, float shift,
                                                                 int escalate,
                                                                 float *__restrict__ Lout, float *__restrict__ shift_used,
                                                                 int32_t *__restrict__ failed) {
    extern __shared__ float sm[];
    const int Bp = (B + 31) & ~31, T = Bp >> 5, ld = Bp + 1;
    float *A = sm;                                  // Bp x (Bp + 1), padded rows
    float4 *P = reinterpret_cast<float4 *>(sm + Bp * ld);   // the block's positions
    __shared__ int s_fail;
    __shared__ float s_rcp[32];     // reciprocal pivots of the current diagonal tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t d0, c0;
    int cl;
    dom_of(blockIdx.x, core, B, n, d0, c0, cl);
    for (int i = threadIdx.x; i < B; i += blockDim.x) P[i] = pos[d0 + i];
    __syncthreads();
    float lam = shift;
    int attempts = escalate ? 5 : 1;
    int ok = 0;
    for (int att = 0; att < attempts && !ok; ++att, lam *= 10.f) {
        for (int idx = threadIdx.x; idx < Bp * Bp; idx += blockDim.x) {
            const int i = idx / Bp, j = idx % Bp;
            if (j > i) continue;
            float v;
            if (i >= B) {
                v = i == j ? 1.f : 0.f;                 // padding: identity
            } else if (i == j) {
                v = 1.f + lam;
            } else {
                const float4 pi = P[i], pj = P[j];   // difference before scaling keeps it exact-ish
                float dx = (pi.x - pj.x) * scl, dy = (pi.y - pj.y) * scl, dz = (pi.z - pj.z) * scl;
                const float t = dx * dx + dy * dy + dz * dz;   // |d|^2 log2(e) / (2 sigma^2)
                // Gaussian 2^-t; inverse multiquadric (1 + |d|^2 / sigma^2)^-beta, |d|^2 / sigma^2 = 2 ln(2) t
                v = imq_beta > 0.f ? ex2_approx(-imq_beta * __log2f(fmaf(t, 1.3862943611198906f, 1.f)))
                                   : ex2_approx(-t);
            }
            A[i * ld + j] = v;
        }
        if (threadIdx.x == 0) s_fail = 0;
        __syncthreads();
        for (int k = 0; k < T; ++k) {
            const int k0 = 32 * k;
            // 1. diagonal tile by warp 0, in registers: lane r holds row k0 + r; per column jj
            //    the pivot, the column scaled by it (shuffled to the other rows), then the
            //    tile's remaining lower triangle updated, with no CTA barrier in between
            if (warp == 0) {
                float x[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) x[c] = A[(k0 + lane) * ld + k0 + c];
                bool bad = false;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const float d = __shfl_sync(0xffffffffu, x[jj], jj);
                    bad |= !(d > 0.f) || !isfinite(d);
                    const float ljj = sqrtf(fmaxf(d, 1e-30f)), rl = __frcp_rn(ljj);
                    if (lane == jj) {
                        x[jj] = ljj;
                        s_rcp[jj] = rl;     // for the panel below
                    } else if (lane > jj) {
                        x[jj] *= rl;
                    }
#pragma unroll
                    for (int cc = 0; cc < 32; ++cc) {
                        if (cc <= jj) continue;
                        const float lc = __shfl_sync(0xffffffffu, x[jj], cc);   // L[k0 + cc][k0 + jj]
                        if (lane >= cc) x[cc] = fmaf(-x[jj], lc, x[cc]);
                    }
                }
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c <= lane) A[(k0 + lane) * ld + k0 + c] = x[c];
                if (lane == 0 && bad) s_fail = 1;
            }
            __syncthreads();
            if (s_fail) break;
            // 2. panel: rows below the diagonal tile, X = A_ik L_kk^-T
            const int r = k0 + 32 + threadIdx.x;
            if (r < Bp) {
                float x[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) x[c] = A[r * ld + k0 + c];
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    float acc = x[c];
#pragma unroll
                    for (int m = 0; m < c; ++m) acc = fmaf(-x[m], A[(k0 + c) * ld + k0 + m], acc);
                    x[c] = acc * s_rcp[c];
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) A[r * ld + k0 + c] = x[c];
            }
            __syncthreads();
            // 3. trailing tiles (i, l), k < l <= i: A_il -= X_i X_l^T
            const int Tr = T - 1 - k;
            const int ntiles = Tr * (Tr + 1) / 2;
            for (int q = warp; q < ntiles; q += kSetupThreads / 32) {
                int i = 0, l = q;                        // q -> (i, l) with l <= i over the trailing tiles
                while (l > i) {
                    l -= i + 1;
                    ++i;
                }
                const int ri = k0 + 32 + 32 * i, cl0 = k0 + 32 + 32 * l;
                float xl[32];
#pragma unroll
                for (int m = 0; m < 32; ++m) xl[m] = A[(cl0 + lane) * ld + k0 + m];
                for (int rr = 0; rr < 32; ++rr) {
                    const float *xi = A + (ri + rr) * ld + k0;
                    float acc = 0.f;
#pragma unroll
                    for (int m = 0; m < 32; ++m) acc = fmaf(xi[m], xl[m], acc);
                    A[(ri + rr) * ld + cl0 + lane] -= acc;
                }
            }
            __syncthreads();
        }
        ok = !s_fail;
        __syncthreads();
    }
    float *L = Lout + (int64_t)blockIdx.x * B * B;
    for (int idx = threadIdx.x; idx < B * B; idx += blockDim.x) {
        int i = idx / B, j = idx % B;
        float v;
        if (ok)
            v = j <= i ? A[i * ld + j] : 0.f;
        else
            v = (i == j) ? 1.f : 0.f;
        L[idx] = v;
    }
    if (threadIdx.x == 0) {
        failed[blockIdx.x] = ok ? 0 : 1;
        shift_used[blockIdx.x] = ok ? lam / 10.f : -1.f;
    }
}

template <typename Tin, bool kOne>   // kOne: B <= 32 (one factor tile)
__global__ void k_schwarz_apply(const Tin *__restrict__ v, int64_t n, int core, int B, int64_t nblocks,
                                const float *__restrict__ Lall, int restricted, float *__restrict__ z) {
    int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (blk >= nblocks) return;
    int64_t d0, c0;
    int cl;
    dom_of(blk, core, B, n, d0, c0, cl);
    const float *L = Lall + blk * (int64_t)B * B;
    constexpr int Q = kMaxB / 32;
    float y[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        int k = lane + 32 * q;
        y[q] = k < B ? (float)v[d0 + k] : 0.f;
    }
    if (kOne) ras::solve_block32(L, B, y[0], lane);
    else ras::solve_block(L, B, y, lane);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        int k = lane + 32 * q;
        if (k >= B) continue;
        int64_t gi = d0 + k;
        if (restricted) {
            if (gi >= c0 && gi < c0 + cl) z[gi] = y[q];
        } else {
            atomicAdd(&z[gi], y[q]);
        }
    }
}

}  // namespace

void schwarz_setup(rbf_plan *P, const rbf_schwarz_params &p, int64_t *failed_host, cudaStream_t s) {
    RBF_CHECK(p.block >= 1 && p.block <= kMaxB, RBF_ERR_UNSUPPORTED, "schwarz block %d outside 1..%d", p.block, kMaxB);
    RBF_CHECK(p.core >= 1 && p.core <= p.block, RBF_ERR_INVALID, "schwarz core %d outside 1..block", p.core);
    RBF_CHECK(p.shift >= 0.f && std::isfinite(p.shift), RBF_ERR_INVALID, "schwarz shift must be finite and >= 0");
    SchwarzData &S = P->sz;
    S.ready = false;
    S.core = p.core;
    S.block = (int)std::min<int64_t>(p.block, P->n);
    S.restricted = p.restricted ? 1 : 0;
    S.shift = p.shift;
    S.nblocks = ceil_div(P->n, p.core);
    const int B = S.block;
    S.L.alloc((size_t)S.nblocks * B * B, s);
    S.shift_used.alloc(S.nblocks, s);
    S.failed.alloc(S.nblocks, s);
    const int Bp = (B + 31) & ~31;
    size_t smem = (size_t)Bp * (Bp + 1) * sizeof(float) + (size_t)Bp * sizeof(float4);
    RBF_CUDA(cudaFuncSetAttribute(k_schwarz_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const float imq_beta = P->kernel == RBF_KERNEL_IMQ ? P->beta : 0.f;
    k_schwarz_setup<<<(unsigned)S.nblocks, kSetupThreads, smem, s>>>(P->pos.p, P->n, S.core, B, P->scl, imq_beta,
                                                                     p.shift, p.escalate, S.L.p, S.shift_used.p,
                                                                     S.failed.p);
    RBF_LAUNCHED();
    if (failed_host) {
        std::vector<int32_t> f(S.nblocks);
        RBF_CUDA(cudaMemcpyAsync(f.data(), S.failed.p, S.nblocks * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(cudaStreamSynchronize(s));
        int64_t c = 0;
        for (auto x : f) c += x;
        *failed_host = c;
    }
    S.ready = true;
}

void schwarz_apply_binned(rbf_plan *P, const double *vd, const float *vf, float *z, cudaStream_t s) {
    SchwarzData &S = P->sz;
    RBF_CHECK(S.ready, RBF_ERR_INVALID, "schwarz preconditioner not set up");
    if (!S.restricted) RBF_CUDA(cudaMemsetAsync(z, 0, P->n * sizeof(float), s));
    unsigned grid = (unsigned)ceil_div(S.nblocks * 32, 256);
    if (S.block <= 32) {
        if (vd)
            k_schwarz_apply<double, true><<<grid, 256, 0, s>>>(vd, P->n, S.core, S.block, S.nblocks, S.L.p,
                                                                S.restricted, z);
        else
            k_schwarz_apply<float, true><<<grid, 256, 0, s>>>(vf, P->n, S.core, S.block, S.nblocks, S.L.p,
                                                               S.restricted, z);
    } else if (vd) {
        k_schwarz_apply<double, false><<<grid, 256, 0, s>>>(vd, P->n, S.core, S.block, S.nblocks, S.L.p,
                                                             S.restricted, z);
    } else {
        k_schwarz_apply<float, false><<<grid, 256, 0, s>>>(vf, P->n, S.core, S.block, S.nblocks, S.L.p,
                                                            S.restricted, z);
    }
    RBF_LAUNCHED();
}
