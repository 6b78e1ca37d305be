// Flexible GMRES(m) with right preconditioning (Saad 1993), the Krylov method
// of Sec. III.A, in binned order.
//
// Precision split: the product A~ z and the preconditioner run in float32; the
// Arnoldi basis V (float64), classical Gram-Schmidt applied twice, the
// Hessenberg matrix, its Givens rotations and least-squares solve, and the
// iterate x are float64.  Every restart recomputes the true residual
// r = b - A~ x with a float64-accurate product (double-float on the float32
// pipes by default, or native float64), so the outer loop is iterative
// refinement x <- x + FGMRES(r).
//
// Per inner step j: Z_j = M^-1 V_j; w = A~ Z_j; two passes of h = V^T w,
// w -= V h (fused multi-dot and multi-axpy kernels with fixed-order reductions);
// V_{j+1} = w / |w|.  Each step's column of H goes to its own device slot; the host
// applies the rotations after reading it back, once per step when a tolerance is
// checked, once per cycle for a fixed iteration count (nothing on the device waits
// for the host in between).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "plan.cuh"

namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ double ld(const T *p, int64_t i) { return (double)p[i]; }

__device__ double block_sum_d(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
    return t;   // valid in thread 0
}

// partial[k * G + g] = sum over CTA g's range of V[k][i] * w[i], k < nv.  Eight vectors
// per sweep of the range (eight independent loads in flight per element); each thread
// sums its elements in index order, the warp reduces by a butterfly reduce-scatter and
// the block sums its warps in order.
constexpr int kDotGroup = 8;   // the reduce-scatter below is written for 8
template <typename Tw>
__global__ void __launch_bounds__(kThreads) k_mdot(const double *__restrict__ V, int64_t ldv, int nv,
                                                   const Tw *__restrict__ w, int64_t n, double *__restrict__ partial) {
    __shared__ double sh[kDotGroup][kThreads / 32];
    const int G = gridDim.x;
    const int64_t per = (n + G - 1) / G;
    const int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k0 = 0; k0 < nv; k0 += kDotGroup) {
        const int kn = min(kDotGroup, nv - k0);
        const double *v0 = V + (int64_t)k0 * ldv;
        double s[kDotGroup];
#pragma unroll
        for (int q = 0; q < kDotGroup; ++q) s[q] = 0.0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += kThreads) {
            const double wi = ld(w, i);
#pragma unroll
            for (int q = 0; q < kDotGroup; ++q)
                if (q < kn) s[q] += v0[q * ldv + i] * wi;
        }
        // butterfly reduce-scatter over the warp (9 float64 adds per lane instead of 40):
        // each level keeps half of the values and adds the partner's copy of them, so that
        // lane l ends with the warp's sum for vector q = (l >> 2) & 7
        const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
        double t4[4], t2[2];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            t4[i] = (b4 ? s[4 + i] : s[i]) + __shfl_xor_sync(0xffffffffu, b4 ? s[i] : s[4 + i], 16);
#pragma unroll
        for (int i = 0; i < 2; ++i)
            t2[i] = (b3 ? t4[2 + i] : t4[i]) + __shfl_xor_sync(0xffffffffu, b3 ? t4[i] : t4[2 + i], 8);
        double v = (b2 ? t2[1] : t2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? t2[0] : t2[1], 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if ((lane & 3) == 0) sh[(lane >> 2) & 7][warp] = v;
        __syncthreads();
        if ((int)threadIdx.x < kn) {
            double t = 0.0;
            for (int u = 0; u < kThreads / 32; ++u) t += sh[threadIdx.x][u];
            partial[(int64_t)(k0 + threadIdx.x) * G + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

// out[k] (+)= sum_g partial[k * G + g] in a fixed tree order; one CTA per k.
__global__ void k_mdot_final(const double *__restrict__ partial, int G, double *__restrict__ out, int accumulate) {
    __shared__ double sh[kThreads / 32];
    int k = blockIdx.x;
    double s = 0.0;
    for (int g = threadIdx.x; g < G; g += kThreads) s += partial[(int64_t)k * G + g];
    double t = block_sum_d(s, sh);
    if (threadIdx.x == 0) out[k] = accumulate ? out[k] + t : t;
}

// wout[i] = win[i] - sum_k h[k] V[k][i]; optional partial sums of wout^2.
template <typename Tw>
__global__ void __launch_bounds__(kThreads) k_maxpy(const double *__restrict__ V, int64_t ldv, int nv,
                                                    const double *__restrict__ h, const Tw *__restrict__ win,
                                                    double *__restrict__ wout, int64_t n, double *__restrict__ nrm_part) {
    __shared__ double sh[kThreads / 32];
    __shared__ double hs[520];
    for (int k = threadIdx.x; k < nv; k += kThreads) hs[k] = h[k];
    __syncthreads();
    int G = gridDim.x;
    int64_t per = (n + G - 1) / G;
    int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    double sq = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kThreads) {
        double v = ld(win, i);
#pragma unroll 8
        for (int k = 0; k < nv; ++k) v -= hs[k] * V[k * ldv + i];
        wout[i] = v;
        sq += v * v;
    }
    if (nrm_part) {
        double t = block_sum_d(sq, sh);
        if (threadIdx.x == 0) nrm_part[blockIdx.x] = t;
    }
}

// dst = src * (1 / s) (s on the device), float64.  One thread per CTA forms the
// reciprocal: a float64 division costs many float64 FMA slots on this GPU.
__global__ void k_scale(const double *__restrict__ src, const double *__restrict__ sptr, double *__restrict__ dst,
                        int64_t n) {
    __shared__ double s_inv;
    if (threadIdx.x == 0) s_inv = 1.0 / *sptr;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] * s_inv;
}

__global__ void k_sqrt(double *p) { *p = sqrt(*p); }

__global__ void k_b_to_r(const float *__restrict__ b, double *__restrict__ r, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = (double)b[i];
}

__global__ void k_b_minus(const float *__restrict__ b, const float *__restrict__ y, double *__restrict__ r, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = (double)b[i] - (double)y[i];
}

__global__ void k_f32_to_f64(const float *__restrict__ a, double *__restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

__global__ void k_f32_scaled_to_f64(const float *__restrict__ a, double alpha, double *__restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = alpha * (double)a[i];
}

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// x[i] += sum_j y[j] Z[j][i]
__global__ void k_update_x(double *__restrict__ x, const float *__restrict__ Z, int64_t ldz, int k,
                           const double *__restrict__ y, int64_t n) {
    __shared__ double ys[512];
    for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[j];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = x[i];
    for (int j = 0; j < k; ++j) v += ys[j] * (double)Z[j * ldz + i];
    x[i] = v;
}

inline unsigned g1(int64_t n) { return (unsigned)std::max<int64_t>(1, ceil_div(n, kThreads)); }

// Accumulates CUDA-event intervals on a stream (read once, at the end).
struct Intervals {
    std::vector<cudaEvent_t> ev;
    int count = 0;
    void begin(cudaStream_t s) {
        cudaEvent_t a, b;
        RBF_CUDA(cudaEventCreate(&a));
        RBF_CUDA(cudaEventCreate(&b));
        ev.push_back(a);
        ev.push_back(b);
        RBF_CUDA(cudaEventRecord(a, s));
    }
    void end(cudaStream_t s) {
        RBF_CUDA(cudaEventRecord(ev.back(), s));
        ++count;
    }
    double total_ms() {
        double t = 0;
        for (size_t i = 0; i + 1 < ev.size(); i += 2) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) t += ms;
        }
        return t;
    }
    ~Intervals() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

}  // namespace

// Fixed-order norm^2 of a float64 vector: device scalar out.
static void norm2_dev(const double *v, int64_t n, int G, double *part, double *out, cudaStream_t s) {
    k_mdot<double><<<G, kThreads, 0, s>>>(v, 0, 1, v, n, part);
    RBF_LAUNCHED();
    k_mdot_final<<<1, kThreads, 0, s>>>(part, G, out, 0);
    RBF_LAUNCHED();
}

rbf_status fgmres_solve(rbf_plan *P, const float *b_caller, const rbf_solve_params &p, double *x_caller,
                        rbf_report *rep, cudaStream_t s) {
    const int64_t n = P->n;
    const int m = p.m > 0 ? p.m : 50;
    const int max_it = p.max_it > 0 ? p.max_it : 500;
    const double tol = p.tol > 0 ? p.tol : 1e-6;
    RBF_CHECK(m <= 512, RBF_ERR_INVALID, "restart length %d > 512", m);
    const bool each_restart = p.true_residual_each_restart != 0;
    const int G = std::max(1, std::min<int>(4 * P->ctx->num_sms, (int)ceil_div(n, kThreads)));
    RBF_CHECK(!p.assembled || P->csr.ready, RBF_ERR_INVALID,
              "assembled operator requested but the plan has no assembled matrix");
    // the float32 operator: matrix-free product, or the assembled matrix (Algorithm 2)
    auto op = [&](const float *in, float *out) {
        if (p.assembled) spmv_binned(P, in, out, s);
        else matvec_binned(P, in, out, s);
    };

    rbf_report R{};
    Timer tm_setup, tm_solve;
    cudaEventRecord(tm_setup.a, s);
    if (p.precond == RBF_PRECOND_SCHWARZ) {
        int64_t failed = 0;
        schwarz_setup(P, p.schwarz, &failed, s);
        R.precond_failed_blocks = (int)failed;
    } else if (p.precond == RBF_PRECOND_MLP) {
        RBF_CHECK(P->kernel == RBF_KERNEL_GAUSSIAN, RBF_ERR_UNSUPPORTED,
                  "the learned preconditioner is trained on Gaussian blocks");
        RBF_CHECK(p.mlp && p.mlp_lambda > 0.f, RBF_ERR_INVALID, "MLP preconditioner needs a network and lambda > 0");
        rbf_schwarz_params fb{};
        fb.core = 64;
        fb.block = 64;
        fb.shift = p.mlp_lambda;
        fb.restricted = 1;
        fb.escalate = 1;
        int64_t failed = 0;
        schwarz_setup(P, fb, &failed, s);   // the fallback of blocks with a non-finite output
    }
    cudaEventRecord(tm_setup.b, s);
    cudaEventRecord(tm_solve.a, s);

    DevBuf<float> bs, Z, w32;
    DevBuf<double> V, w64, part, hdev, x, r, y, scal;
    bs.alloc(n, s);
    permute_to_binned_f32(P, b_caller, bs.p, s);
    V.alloc((size_t)(m + 1) * n, s);
    Z.alloc((size_t)m * n, s);
    w32.alloc(n, s);
    w64.alloc(n, s);
    part.alloc((size_t)(m + 1) * G, s);
    hdev.alloc((size_t)m * 3 * (m + 1), s);   // per Arnoldi step of a cycle: h, h2, |w|
    x.alloc(n, s);
    x.zero(s);
    r.alloc(n, s);
    y.alloc(m, s);
    scal.alloc(2, s);

    // x0 = 0, so r0 = b exactly
    k_b_to_r<<<g1(n), kThreads, 0, s>>>(bs.p, r.p, n);
    RBF_LAUNCHED();
    norm2_dev(r.p, n, G, part.p, scal.p, s);
    double bnorm2 = 0;
    RBF_CUDA(cudaMemcpyAsync(&bnorm2, scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    const double bnorm = std::sqrt(bnorm2);
    int64_t mlp_fallbacks = 0;
    bool x_nonzero = false;
    Intervals t_mv, t_res, t_pc;
    if (p.precond == RBF_PRECOND_MLP && p.mlp_initial_guess && bnorm > 0) {
        // g = network applied to b, u = A~ g (float32 product); x0 = a g with the a that
        // minimises |b - a u|, a = <b, u> / <u, u>, so that |r0| <= |b| whatever the network
        // returns (a = 0 drops the guess)
        mlp_fallbacks += mlp_apply(p.mlp, P, p.mlp_lambda, 64, r.p, w32.p, s);
        t_mv.begin(s);
        op(w32.p, Z.p);                                   // Z's first column as scratch
        t_mv.end(s);
        k_f32_to_f64<<<g1(n), kThreads, 0, s>>>(Z.p, w64.p, n);
        RBF_LAUNCHED();
        k_mdot<double><<<G, kThreads, 0, s>>>(r.p, n, 1, w64.p, n, part.p);   // r holds b here
        RBF_LAUNCHED();
        k_mdot_final<<<1, kThreads, 0, s>>>(part.p, G, scal.p, 0);
        RBF_LAUNCHED();
        norm2_dev(w64.p, n, G, part.p, scal.p + 1, s);
        double bu_uu[2] = {0, 0};
        RBF_CUDA(cudaMemcpyAsync(bu_uu, scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(cudaStreamSynchronize(s));
        ctx_check_device_error(P->ctx);
        const double bu = bu_uu[0], uu = bu_uu[1];
        const double alpha = (uu > 0 && std::isfinite(uu) && std::isfinite(bu)) ? bu / uu : 0.0;
        R.guess_scale = alpha;
        R.guess_residual = alpha != 0.0 ? std::sqrt(std::max(0.0, bnorm2 - bu * alpha)) / bnorm : 1.0;
        if (alpha != 0.0) {
            k_f32_scaled_to_f64<<<g1(n), kThreads, 0, s>>>(w32.p, alpha, x.p, n);
            RBF_LAUNCHED();
            x_nonzero = true;
        }
    }

    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hcol(m + 2), yh(m),
        hbuf((size_t)m * 3 * (m + 1));
    int it = 0, cycles = 0;
    double beta = bnorm, est = 1.0, true_rel = bnorm > 0 ? 1.0 : 0.0;
    bool converged = bnorm == 0.0, breakdown = false;
    bool have_true = !x_nonzero;   // r holds b - A~ x for the current x

    while (!converged && it < max_it && !breakdown) {
        if (!have_true) {
            if (each_restart) {
                t_res.begin(s);
                residual_binned(P, p.residual_mode, bs.p, x.p, r.p, s);
                t_res.end(s);
                have_true = true;   // a solve that stops here needs no second residual for this x
            } else {
                // float32 product for the restart vector; the float64 residual runs once at the end
                k_to_f32<<<g1(n), kThreads, 0, s>>>(x.p, w32.p, n);
                RBF_LAUNCHED();
                op(w32.p, Z.p);
                k_b_minus<<<g1(n), kThreads, 0, s>>>(bs.p, Z.p, r.p, n);
                RBF_LAUNCHED();
            }
        }
        norm2_dev(r.p, n, G, part.p, scal.p, s);
        k_sqrt<<<1, 1, 0, s>>>(scal.p);
        RBF_LAUNCHED();
        RBF_CUDA(cudaMemcpyAsync(&beta, scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(cudaStreamSynchronize(s));
        ctx_check_device_error(P->ctx);   // a true residual out of range, or an expired wait
        true_rel = beta / bnorm;
        if (!std::isfinite(beta)) {
            breakdown = true;
            break;
        }
        if (!p.fixed_iterations && beta <= tol * bnorm) {
            converged = true;
            break;
        }
        k_scale<<<g1(n), kThreads, 0, s>>>(r.p, scal.p, V.p, n);
        RBF_LAUNCHED();
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0, k = 0;
        // Host side of Arnoldi step jj: Hessenberg column from its slot (h + h2, |w|), Givens
        // rotations, residual estimate.  False ends the cycle (breakdown, an exact solution
        // in the Krylov space, or the tolerance met).
        auto take_column = [&](int jj, const double *hb) -> bool {
            const int nv = jj + 1;
            for (int i = 0; i < nv; ++i) hcol[i] = hb[i] + hb[m + 1 + i];
            hcol[nv] = hb[2 * (m + 1)];
            bool finite = true;
            for (int i = 0; i <= nv; ++i) finite = finite && std::isfinite(hcol[i]);
            if (!finite) {
                breakdown = true;
                return false;
            }
            for (int i = 0; i <= nv; ++i) H[(size_t)i * m + jj] = hcol[i];
            for (int i = 0; i < jj; ++i) {
                double t = cs[i] * H[(size_t)i * m + jj] + sn[i] * H[(size_t)(i + 1) * m + jj];
                H[(size_t)(i + 1) * m + jj] = -sn[i] * H[(size_t)i * m + jj] + cs[i] * H[(size_t)(i + 1) * m + jj];
                H[(size_t)i * m + jj] = t;
            }
            double a = H[(size_t)jj * m + jj], bb = H[(size_t)(jj + 1) * m + jj];
            double rho = std::hypot(a, bb);
            cs[jj] = rho > 0 ? a / rho : 1.0;
            sn[jj] = rho > 0 ? bb / rho : 0.0;
            H[(size_t)jj * m + jj] = rho;
            H[(size_t)(jj + 1) * m + jj] = 0.0;
            g[jj + 1] = -sn[jj] * g[jj];
            g[jj] = cs[jj] * g[jj];
            est = std::fabs(g[jj + 1]) / bnorm;
            k = jj + 1;
            if (hcol[nv] == 0.0) return false;                            // exact solution in the Krylov space
            if (!p.fixed_iterations && est <= tol) return false;
            return true;
        };
        for (j = 0; j < m && it < max_it; ++j) {
            double *Vj = V.p + (size_t)j * n;
            float *Zj = Z.p + (size_t)j * n;
            if (p.precond == RBF_PRECOND_SCHWARZ) {
                t_pc.begin(s);
                schwarz_apply_binned(P, Vj, nullptr, Zj, s);
                t_pc.end(s);
            } else if (p.precond == RBF_PRECOND_MLP) {
                t_pc.begin(s);
                mlp_fallbacks += mlp_apply(p.mlp, P, p.mlp_lambda, 64, Vj, Zj, s);
                t_pc.end(s);
            } else {
                k_to_f32<<<g1(n), kThreads, 0, s>>>(Vj, Zj, n);
                RBF_LAUNCHED();
            }
            t_mv.begin(s);
            op(Zj, w32.p);
            t_mv.end(s);
            const int nv = j + 1;
            double *h1 = hdev.p + (size_t)j * 3 * (m + 1);   // this step's slot
            double *h2 = h1 + (m + 1);
            double *hn = h1 + 2 * (m + 1);
            // pass 1
            k_mdot<float><<<G, kThreads, 0, s>>>(V.p, n, nv, w32.p, n, part.p);
            RBF_LAUNCHED();
            k_mdot_final<<<nv, kThreads, 0, s>>>(part.p, G, h1, 0);
            RBF_LAUNCHED();
            k_maxpy<float><<<G, kThreads, 0, s>>>(V.p, n, nv, h1, w32.p, w64.p, n, nullptr);
            RBF_LAUNCHED();
            // pass 2 (re-orthogonalisation), accumulating into h, with |w|^2 partials
            k_mdot<double><<<G, kThreads, 0, s>>>(V.p, n, nv, w64.p, n, part.p);
            RBF_LAUNCHED();
            k_mdot_final<<<nv, kThreads, 0, s>>>(part.p, G, h2, 0);
            RBF_LAUNCHED();
            k_maxpy<double><<<G, kThreads, 0, s>>>(V.p, n, nv, h2, w64.p, w64.p, n, part.p);
            RBF_LAUNCHED();
            k_mdot_final<<<1, kThreads, 0, s>>>(part.p, G, hn, 0);
            RBF_LAUNCHED();
            k_sqrt<<<1, 1, 0, s>>>(hn);
            RBF_LAUNCHED();
            k_scale<<<g1(n), kThreads, 0, s>>>(w64.p, hn, V.p + (size_t)(j + 1) * n, n);
            RBF_LAUNCHED();
            ++it;
            // with a fixed iteration count nothing on the device waits for the host: the
            // columns are read back once at the end of the cycle
            if (p.fixed_iterations) continue;
            RBF_CUDA(cudaMemcpyAsync(hbuf.data(), h1, 3 * (m + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
            RBF_CUDA(cudaStreamSynchronize(s));
            if (!take_column(j, hbuf.data())) break;
        }
        if (p.fixed_iterations && j > 0) {
            // steps after a breakdown ran on non-finite or zero-scaled vectors; their columns
            // are never used
            RBF_CUDA(cudaMemcpyAsync(hbuf.data(), hdev.p, (size_t)j * 3 * (m + 1) * sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
            RBF_CUDA(cudaStreamSynchronize(s));
            int used = j;
            for (int jj = 0; jj < j; ++jj)
                if (!take_column(jj, hbuf.data() + (size_t)jj * 3 * (m + 1))) {
                    used = jj + 1;
                    break;
                }
            it -= j - used;   // count the steps the cycle used, as the step-by-step form does
        }
        if (k == 0) break;
        // back substitution for y (k x k upper triangular)
        for (int i = k - 1; i >= 0; --i) {
            double t = g[i];
            for (int c = i + 1; c < k; ++c) t -= H[(size_t)i * m + c] * yh[c];
            yh[i] = H[(size_t)i * m + i] != 0.0 ? t / H[(size_t)i * m + i] : 0.0;
        }
        RBF_CUDA(cudaMemcpyAsync(y.p, yh.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
        k_update_x<<<g1(n), kThreads, 0, s>>>(x.p, Z.p, n, k, y.p, n);
        RBF_LAUNCHED();
        ++cycles;
        have_true = false;
    }
    // final true residual (float64)
    if (!have_true || !each_restart) {
        t_res.begin(s);
        residual_binned(P, p.residual_mode, bs.p, x.p, r.p, s);
        t_res.end(s);
        norm2_dev(r.p, n, G, part.p, scal.p, s);
        double r2 = 0;
        RBF_CUDA(cudaMemcpyAsync(&r2, scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(cudaStreamSynchronize(s));
        true_rel = bnorm > 0 ? std::sqrt(r2) / bnorm : 0.0;
        converged = true_rel <= tol;
    }
    permute_from_binned_f64(P, x.p, x_caller, s);
    cudaEventRecord(tm_solve.b, s);
    RBF_CUDA(cudaStreamSynchronize(s));
    ctx_check_device_error(P->ctx);   // a product launch of this solve gave up on a bounded wait
    float ms_a = 0, ms_b = 0;
    cudaEventElapsedTime(&ms_a, tm_setup.a, tm_setup.b);
    cudaEventElapsedTime(&ms_b, tm_solve.a, tm_solve.b);
    if (p.precond == RBF_PRECOND_MLP) R.precond_failed_blocks = (int)mlp_fallbacks;
    R.iterations = it;
    R.restarts = cycles;
    R.converged = converged ? 1 : 0;
    R.residual_estimate = est;
    R.residual_true = true_rel;
    R.ms_setup = ms_a;
    R.ms_solve = ms_b;
    R.matvec_pairs = P->pairs >= 0 ? P->pairs * (int64_t)t_mv.count : 0;
    R.matvec_launches = t_mv.count;
    R.residual_launches = t_res.count;
    R.ms_matvec = t_mv.total_ms();
    R.ms_residual = t_res.total_ms();
    R.ms_precond = t_pc.total_ms();
    if (rep) *rep = R;
    if (breakdown) return RBF_ERR_BREAKDOWN;
    if (!converged && !p.fixed_iterations) return RBF_ERR_NOT_CONVERGED;
    return RBF_OK;
}
