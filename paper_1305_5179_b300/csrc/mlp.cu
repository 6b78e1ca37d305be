// Learned block preconditioner: a small MLP approximating the action of the
// shifted subdomain inverse (A_i + lambda I)^-1 on a residual (not in the paper;
// it replaces the exact block solve of the restricted additive Schwarz method of
// Sec. III.A by a trained approximation).
//
// Blocks are the Schwarz subdomains of 64 centres.  Features of block i and
// vector r: the 64 offsets (c_k - c_mean)/sigma (192 values, x y z per centre)
// and rho = 8 r_i / |r_i|_2 (64 values of unit mean square).  Network:
// 256 -> 256 -> 256 -> 64 with ReLU and a skip connection adding rho to the
// output, weights W[out][in] (FP32 master copy for training, BF16 copy for
// inference), FP32 accumulation.  Output v approximates
// 8 lambda (A_i + lambda I)^-1 r_i / |r_i|, so the block correction is
// v |r_i| / (8 lambda).  Training data are exact float64 solves of the shifted
// blocks for caller-supplied random right-hand sides; the loss is the mean
// squared error; Adam updates the master weights.
#include <cmath>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "gemm_tc.cuh"
#include "plan.cuh"

namespace {

constexpr int kIn = 256, kH = 256, kOut = 64, kBlkN = 64;
constexpr float kRhoScale = 8.f;   // sqrt(64): the normalised residual with unit mean square
constexpr int64_t kNW1 = (int64_t)kH * kIn, kNW2 = (int64_t)kH * kH, kNW3 = (int64_t)kOut * kH;
constexpr int64_t kOffW1 = 0, kOffB1 = kNW1, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kNW2, kOffW3 = kOffB2 + kH,
                  kOffB3 = kOffW3 + kNW3, kNParams = kOffB3 + kOut;

// ------------------------------------------------------------------ features
// One warp per block: X[row] = [offsets/sigma (3 x 64, centre-major), r/|r|]; nrm[row] = |r|.
// The residual comes from the vector v (binned order, v[d0 + k]) or, for training
// samples, from rows of R (R[row * 64 + k]).
template <typename Tv>
__global__ void k_features(const float4 *__restrict__ pos, const Tv *__restrict__ v, const float *__restrict__ Rrows,
                           int64_t n, int core, int B, const int32_t *__restrict__ block_ids, int64_t nrows,
                           float inv_sigma, float *__restrict__ X, float *__restrict__ nrm) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= nrows) return;
    const int64_t blk = block_ids ? block_ids[row] : row;
    int64_t s = blk * core;
    int64_t d0 = s - (B - core) / 2;
    if (d0 > n - B) d0 = n - B;
    if (d0 < 0) d0 = 0;
    float4 p0 = pos[d0 + lane], p1 = pos[d0 + lane + 32];
    float cx = p0.x + p1.x, cy = p0.y + p1.y, cz = p0.z + p1.z;
    for (int o = 16; o > 0; o >>= 1) {
        cx += __shfl_xor_sync(0xffffffffu, cx, o);
        cy += __shfl_xor_sync(0xffffffffu, cy, o);
        cz += __shfl_xor_sync(0xffffffffu, cz, o);
    }
    cx *= 1.f / 64.f;
    cy *= 1.f / 64.f;
    cz *= 1.f / 64.f;
    float *xr = X + row * kIn;
    xr[3 * lane] = (p0.x - cx) * inv_sigma;
    xr[3 * lane + 1] = (p0.y - cy) * inv_sigma;
    xr[3 * lane + 2] = (p0.z - cz) * inv_sigma;
    xr[3 * (lane + 32)] = (p1.x - cx) * inv_sigma;
    xr[3 * (lane + 32) + 1] = (p1.y - cy) * inv_sigma;
    xr[3 * (lane + 32) + 2] = (p1.z - cz) * inv_sigma;
    float r0, r1;
    if (Rrows) {
        r0 = Rrows[row * 64 + lane];
        r1 = Rrows[row * 64 + lane + 32];
    } else {
        r0 = (float)v[d0 + lane];
        r1 = (float)v[d0 + lane + 32];
    }
    float ss = r0 * r0 + r1 * r1;
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float nr = sqrtf(ss);
    const float inv = nr > 0.f ? kRhoScale / nr : 0.f;
    xr[192 + lane] = r0 * inv;
    xr[192 + lane + 32] = r1 * inv;
    if (lane == 0 && nrm) nrm[row] = nr;
}

// ------------------------------------------------------------------ exact shifted block solves (training data)
// One CTA (64 threads) per sample: Y = lambda (A_i + lambda I)^-1 r / |r| in float64,
// A_i untruncated over the subdomain's 64 centres, r the sample's right-hand side.
__global__ void __launch_bounds__(64) k_block_solve64(const float4 *__restrict__ pos, int64_t n, int core,
                                                      const int32_t *__restrict__ block_ids,
                                                      const float *__restrict__ R, double inv2s2, double lambda,
                                                      float *__restrict__ Y, int *__restrict__ failed) {
    __shared__ double A[kBlkN][kBlkN + 1];
    __shared__ double u[kBlkN];
    __shared__ double px[kBlkN], py[kBlkN], pz[kBlkN];
    __shared__ double nr2;
    __shared__ int bad;
    const int t = threadIdx.x;
    const int64_t row = blockIdx.x;
    const int64_t blk = block_ids[row];
    int64_t s = blk * core;
    int64_t d0 = s - (kBlkN - core) / 2;
    if (d0 > n - kBlkN) d0 = n - kBlkN;
    if (d0 < 0) d0 = 0;
    float4 p = pos[d0 + t];
    px[t] = p.x;
    py[t] = p.y;
    pz[t] = p.z;
    const double r = (double)R[row * kBlkN + t];
    if (t == 0) {
        bad = 0;
        nr2 = 0.0;
    }
    __syncthreads();
    for (int j = 0; j <= t; ++j) {
        double dx = px[t] - px[j], dy = py[t] - py[j], dz = pz[t] - pz[j];
        double a = exp(-(dx * dx + dy * dy + dz * dz) * inv2s2);
        A[t][j] = (j == t) ? a + lambda : a;
    }
    atomicAdd(&nr2, r * r);
    __syncthreads();
    // right-looking Cholesky, column j by thread rows
    for (int j = 0; j < kBlkN; ++j) {
        if (t == j) {
            double d = A[j][j];
            if (!(d > 0.0)) bad = 1;
            A[j][j] = sqrt(d > 0.0 ? d : 1e-300);
        }
        __syncthreads();
        if (t > j) A[t][j] /= A[j][j];
        __syncthreads();
        if (t > j)
            for (int c = j + 1; c <= t; ++c) A[t][c] -= A[t][j] * A[c][j];
        __syncthreads();
    }
    const double nr = sqrt(nr2);
    u[t] = nr > 0.0 ? r / nr : 0.0;
    __syncthreads();
    if (t == 0) {
        for (int i = 0; i < kBlkN; ++i) {
            double acc = u[i];
            for (int c = 0; c < i; ++c) acc -= A[i][c] * u[c];
            u[i] = acc / A[i][i];
        }
        for (int i = kBlkN - 1; i >= 0; --i) {
            double acc = u[i];
            for (int c = i + 1; c < kBlkN; ++c) acc -= A[c][i] * u[c];
            u[i] = acc / A[i][i];
        }
        if (bad) atomicAdd(failed, 1);
    }
    __syncthreads();
    Y[row * kOut + t] = (float)((double)kRhoScale * lambda * u[t]);
}

// ------------------------------------------------------------------ dense layers
// The three contractions (forward, dA = dC W, dW = dC^T A) run on the tensor cores
// (gemm_tc.cu); the bias gradient is a column sum.

// db[n] = sum_m dC[m][n] (fixed order per column)
__global__ void k_colsum(const float *__restrict__ dC, int M, int N, float *__restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float acc = 0.f;
    for (int m = 0; m < M; ++m) acc += dC[(int64_t)m * N + n];
    db[n] = acc;
}

// g = g * (act > 0)
__global__ void k_relu_mask(float *__restrict__ g, const float *__restrict__ act, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(act[i] > 0.f)) g[i] = 0.f;
}

// dY = 2 (Y - T) / (M * N); per-block partial sums of the squared error
__global__ void k_mse(const float *__restrict__ Y, const float *__restrict__ T, int64_t n, float scale,
                      float *__restrict__ dY, double *__restrict__ part) {
    __shared__ double sh[8];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float d = Y[i] - T[i];
        if (dY) dY[i] = 2.f * d * scale;
        s += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// Adam (Kingma and Ba, 2015) on the master weights; refreshes the bf16 copy
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, __nv_bfloat16 *__restrict__ wb, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float a = b1 * m1[i] + (1.f - b1) * gi;
    float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    float v = w[i] - lr * (a * c1) / (sqrtf(b * c2) + eps);
    w[i] = v;
    wb[i] = __float2bfloat16_rn(v);
}

__global__ void k_to_bf16(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

// z[core of block] = out * nrm / lambda (restricted); blocks with a non-finite output are flagged
__global__ void k_mlp_scatter(const float *__restrict__ out, const float *__restrict__ nrm, int64_t n, int core,
                              int B, int64_t nblocks, float inv_lambda, float *__restrict__ z,
                              int *__restrict__ bad_blocks, int *__restrict__ nbad) {
    const int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 6;
    const int k = threadIdx.x & 63;
    if (blk >= nblocks) return;
    int64_t s = blk * core, e = s + core < n ? s + core : n;
    int64_t d0 = s - (B - core) / 2;
    if (d0 > n - B) d0 = n - B;
    if (d0 < 0) d0 = 0;
    const float v = out[blk * kOut + k] * nrm[blk] * inv_lambda;
    const int64_t gi = d0 + k;
    const bool fin = isfinite(v);
    if (!fin && k == 0) {
        int slot = atomicAdd(nbad, 1);
        bad_blocks[slot] = (int)blk;
    }
    if (gi >= s && gi < e) z[gi] = fin ? v : 0.f;
}

inline unsigned g1(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

}  // namespace

// ------------------------------------------------------------------ host
struct rbf_mlp {
    rbf_ctx *ctx = nullptr;
    PBuf<float> w, g, m1, m2;
    PBuf<__nv_bfloat16> wb;
    int64_t step = 0;
    // activations of the last training batch
    PBuf<float> a1, a2, y, d3, d2, d1, dx;
    PBuf<double> part;
    int cap = 0;
};

static void mlp_ensure(rbf_mlp *M, int rows, cudaStream_t s) {
    if (rows <= M->cap) return;
    M->a1.alloc((size_t)rows * kH, s);
    M->a2.alloc((size_t)rows * kH, s);
    M->y.alloc((size_t)rows * kOut, s);
    M->d3.alloc((size_t)rows * kOut, s);
    M->d2.alloc((size_t)rows * kH, s);
    M->d1.alloc((size_t)rows * kH, s);
    M->dx.alloc((size_t)rows * kIn, s);
    M->part.alloc(1024, s);
    M->cap = rows;
}

int64_t mlp_nparams() { return kNParams; }

rbf_mlp *mlp_create(rbf_ctx *ctx, const float *host_params, cudaStream_t s) {
    rbf_mlp *M = new rbf_mlp();
    try {
        M->ctx = ctx;
        M->w.alloc(kNParams, s);
        M->g.alloc(kNParams, s);
        M->m1.alloc(kNParams, s);
        M->m2.alloc(kNParams, s);
        M->wb.alloc(kNParams, s);
        M->m1.zero(s);
        M->m2.zero(s);
        RBF_CUDA(cudaMemcpyAsync(M->w.p, host_params, kNParams * sizeof(float), cudaMemcpyHostToDevice, s));
        k_to_bf16<<<g1(kNParams), 256, 0, s>>>(M->w.p, M->wb.p, kNParams);
        RBF_LAUNCHED();
        RBF_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        delete M;
        throw;
    }
    return M;
}

void mlp_destroy(rbf_mlp *M) { delete M; }
rbf_ctx *mlp_ctx(rbf_mlp *M) { return M->ctx; }

void mlp_get_params(rbf_mlp *M, float *host, cudaStream_t s) {
    RBF_CUDA(cudaMemcpyAsync(host, M->w.p, kNParams * sizeof(float), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
}

// C[rows x N] = act(A[rows x K] W^T + bias) (+ skip), W [N x K] row-major
template <typename Tw>
static void dense_fwd(rbf_mlp *M, const float *A, const Tw *W, const float *bias, float *C, int rows, int N, int K,
                      bool relu, const float *skip, int ldskip, cudaStream_t s) {
    GemmArgs g;
    g.M = rows;
    g.N = N;
    g.K = K;
    g.a_sr = K;
    g.a_sk = 1;
    g.b_sr = K;
    g.b_sk = 1;
    g.C = C;
    g.ldc = N;
    g.bias = bias;
    g.relu = relu ? 1 : 0;
    g.skip = skip;
    g.ldskip = ldskip;
    gemm_tc(g, A, W, std::is_same<Tw, __nv_bfloat16>::value ? 2 : 3, ctx_error_word(M->ctx), s);
}

// forward of `rows` inputs; bf16 = inference weights (exact in tf32: head and tail of the
// activations times the weights), else the FP32 master weights (three tf32 products)
static void mlp_forward_dev(rbf_mlp *M, const float *X, int rows, float *Y, bool bf16, cudaStream_t s) {
    mlp_ensure(M, rows, s);
    const float *w = M->w.p;
    if (bf16) {
        const __nv_bfloat16 *wb = M->wb.p;
        dense_fwd(M, X, wb + kOffW1, w + kOffB1, M->a1.p, rows, kH, kIn, true, nullptr, 0, s);
        dense_fwd(M, M->a1.p, wb + kOffW2, w + kOffB2, M->a2.p, rows, kH, kH, true, nullptr, 0, s);
        dense_fwd(M, M->a2.p, wb + kOffW3, w + kOffB3, Y, rows, kOut, kH, false, X + 192, kIn, s);
    } else {
        dense_fwd(M, X, w + kOffW1, w + kOffB1, M->a1.p, rows, kH, kIn, true, nullptr, 0, s);
        dense_fwd(M, M->a1.p, w + kOffW2, w + kOffB2, M->a2.p, rows, kH, kH, true, nullptr, 0, s);
        dense_fwd(M, M->a2.p, w + kOffW3, w + kOffB3, Y, rows, kOut, kH, false, X + 192, kIn, s);
    }
}

// dW[N x K] = dC^T A over the batch (dC [rows x N], A [rows x K]), db = column sums of dC
static void dense_bwd_weight(rbf_mlp *M, const float *dC, const float *A, float *dW, float *db, int rows, int N, int K,
                             cudaStream_t s) {
    GemmArgs g;
    g.M = N;
    g.N = K;
    g.K = rows;
    g.a_sr = 1;
    g.a_sk = N;
    g.b_sr = 1;
    g.b_sk = K;
    g.C = dW;
    g.ldc = K;
    gemm_tc(g, dC, A, 3, ctx_error_word(M->ctx), s);
    k_colsum<<<g1(N, 128), 128, 0, s>>>(dC, rows, N, db);
    RBF_LAUNCHED();
}

// dA[rows x K] = dC [rows x N] W [N x K]
static void dense_bwd_data(rbf_mlp *M, const float *dC, const float *W, float *dA, int rows, int N, int K,
                           cudaStream_t s) {
    GemmArgs g;
    g.M = rows;
    g.N = K;
    g.K = N;
    g.a_sr = N;
    g.a_sk = 1;
    g.b_sr = 1;
    g.b_sk = K;
    g.C = dA;
    g.ldc = K;
    gemm_tc(g, dC, W, 3, ctx_error_word(M->ctx), s);
}

void mlp_forward(rbf_mlp *M, const float *X, int64_t rows, float *Y, int bf16, cudaStream_t s) {
    for (int64_t r0 = 0; r0 < rows; r0 += 65536) {
        int r = (int)std::min<int64_t>(65536, rows - r0);
        mlp_forward_dev(M, X + r0 * kIn, r, Y + r0 * kOut, bf16 != 0, s);
    }
}

// loss = mean (Y - T)^2 over rows x 64; gradient of the FP32 master weights into M->g
double mlp_loss_grad(rbf_mlp *M, const float *X, const float *T, int rows, bool want_grad, cudaStream_t s) {
    mlp_ensure(M, rows, s);   // before taking M->y.p: the forward writes into it
    mlp_forward_dev(M, X, rows, M->y.p, false, s);
    const int64_t ny = (int64_t)rows * kOut;
    const int nblk = (int)std::min<int64_t>(1024, ceil_div(ny, 256));
    k_mse<<<nblk, 256, 0, s>>>(M->y.p, T, ny, 1.f / (float)ny, want_grad ? M->d3.p : nullptr, M->part.p);
    RBF_LAUNCHED();
    if (want_grad) {
        float *g = M->g.p;
        const float *w = M->w.p;
        // layer 3
        dense_bwd_weight(M, M->d3.p, M->a2.p, g + kOffW3, g + kOffB3, rows, kOut, kH, s);
        dense_bwd_data(M, M->d3.p, w + kOffW3, M->d2.p, rows, kOut, kH, s);
        k_relu_mask<<<g1((int64_t)rows * kH), 256, 0, s>>>(M->d2.p, M->a2.p, (int64_t)rows * kH);
        RBF_LAUNCHED();
        // layer 2
        dense_bwd_weight(M, M->d2.p, M->a1.p, g + kOffW2, g + kOffB2, rows, kH, kH, s);
        dense_bwd_data(M, M->d2.p, w + kOffW2, M->d1.p, rows, kH, kH, s);
        k_relu_mask<<<g1((int64_t)rows * kH), 256, 0, s>>>(M->d1.p, M->a1.p, (int64_t)rows * kH);
        RBF_LAUNCHED();
        // layer 1
        dense_bwd_weight(M, M->d1.p, X, g + kOffW1, g + kOffB1, rows, kH, kIn, s);
    }
    std::vector<double> part(nblk);
    RBF_CUDA(cudaMemcpyAsync(part.data(), M->part.p, nblk * sizeof(double), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    double tot = 0.0;
    for (double v : part) tot += v;
    return tot / (double)ny;
}

void mlp_get_grad(rbf_mlp *M, float *host, cudaStream_t s) {
    RBF_CUDA(cudaMemcpyAsync(host, M->g.p, kNParams * sizeof(float), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
}

void mlp_adam_step(rbf_mlp *M, float lr, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    M->step += 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)M->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)M->step)));
    k_adam<<<g1(kNParams), 256, 0, s>>>(M->w.p, M->g.p, M->m1.p, M->m2.p, M->wb.p, kNParams, lr, b1, b2, eps, c1, c2);
    RBF_LAUNCHED();
}

// Training data: for every sample, the features of its block (offsets/sigma and r/|r|) and
// Y = lambda (A_i + lambda I)^-1 r/|r| from an exact float64 solve.
int64_t mlp_make_data(rbf_plan *P, float lambda, const int32_t *block_ids, const float *R, int64_t ns, float *X,
                      float *Y, cudaStream_t s) {
    RBF_CHECK(P->n >= kBlkN, RBF_ERR_INVALID, "plan has fewer than %d centres", kBlkN);
    RBF_CHECK(lambda > 0.f && std::isfinite(lambda), RBF_ERR_INVALID, "lambda must be finite and > 0");
    DevBuf<int> failed;
    failed.alloc(1, s);
    failed.zero(s);
    if (ns > 0) {
        k_block_solve64<<<(unsigned)ns, 64, 0, s>>>(P->pos.p, P->n, kBlkN, block_ids, R, P->inv2s2_64, (double)lambda,
                                                    Y, failed.p);
        RBF_LAUNCHED();
        k_features<float><<<g1(ns * 32), 256, 0, s>>>(P->pos.p, nullptr, R, P->n, kBlkN, kBlkN, block_ids, ns,
                                                      1.f / P->sigma, X, nullptr);
        RBF_LAUNCHED();
    }
    int hf = 0;
    RBF_CUDA(cudaMemcpyAsync(&hf, failed.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    return hf;
}

// Preconditioner z = M^-1 v (binned order) with the network on the plan's 64-centre
// subdomains (core `core`); blocks whose output is not finite fall back to the
// plan's restricted additive Schwarz factor when it has one of the same geometry,
// else to the identity.  Returns the number of fallback blocks.
int64_t mlp_apply(rbf_mlp *M, rbf_plan *P, float lambda, int core, const double *vd, float *z, cudaStream_t s) {
    const int B = kBlkN;
    RBF_CHECK(P->n >= B, RBF_ERR_INVALID, "plan has fewer than %d centres", B);
    const int64_t nblocks = ceil_div(P->n, core);
    P->mlp_x.ensure((size_t)nblocks * kIn, s);
    P->mlp_y.ensure((size_t)nblocks * kOut, s);
    P->mlp_n.ensure(nblocks, s);
    P->mlp_bad.ensure(nblocks + 1, s);
    k_features<double><<<g1(nblocks * 32), 256, 0, s>>>(P->pos.p, vd, nullptr, P->n, core, B, nullptr, nblocks,
                                                        1.f / P->sigma, P->mlp_x.p, P->mlp_n.p);
    RBF_LAUNCHED();
    mlp_forward(M, P->mlp_x.p, nblocks, P->mlp_y.p, 1, s);
    RBF_CUDA(cudaMemsetAsync(P->mlp_bad.p + nblocks, 0, sizeof(int32_t), s));
    k_mlp_scatter<<<g1(nblocks * 64), 256, 0, s>>>(P->mlp_y.p, P->mlp_n.p, P->n, core, B, nblocks,
                                                   1.f / (kRhoScale * lambda), z,
                                                   P->mlp_bad.p, P->mlp_bad.p + nblocks);
    RBF_LAUNCHED();
    int nbad = 0;
    RBF_CUDA(cudaMemcpyAsync(&nbad, P->mlp_bad.p + nblocks, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    if (nbad > 0 && P->sz.ready && P->sz.block == B && P->sz.core == core) schwarz_apply_binned(P, vd, nullptr, z, s);
    return nbad;
}
