// extern "C" entry points (include/rbf.h): argument checks, device selection,
// error translation.  No arithmetic of the method lives here.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "../../include/rbf_probe.h"
#include "centers.cuh"
#include "plan.cuh"

static std::atomic<long long> g_launches{0};
void rbf_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void rbf_count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

template <typename F>
rbf_status guarded(rbf_ctx *ctx, F &&f) {
    if (!ctx) return RBF_ERR_INVALID;
    try {
        ctx->last_error.clear();
        (void)cudaGetLastError();   // a stale (non-sticky) error of earlier, unrelated work is not this call's
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            ctx->last_error = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
            return RBF_ERR_CUDA;
        }
        return f();
    } catch (const RbfError &err) {
        ctx->last_error = err.msg;
        return err.status;
    } catch (const std::bad_alloc &) {
        ctx->last_error = "host allocation failed";
        return RBF_ERR_OOM;
    } catch (...) {
        ctx->last_error = "unknown exception";
        return RBF_ERR_CUDA;
    }
}

inline cudaStream_t S(void *s) { return (cudaStream_t)s; }

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

void check_plan_params(const rbf_plan_params *p) {
    RBF_CHECK(p, RBF_ERR_INVALID, "null plan parameters");
    RBF_CHECK(std::isfinite(p->sigma) && p->sigma > 0.f, RBF_ERR_INVALID, "sigma must be finite and > 0");
    RBF_CHECK(std::isfinite(p->k) && p->k >= 0.f && p->k <= 12.f, RBF_ERR_INVALID, "k must be in [0, 12]");
    RBF_CHECK(p->cells_per_cutoff >= 0 && p->cells_per_cutoff <= 4, RBF_ERR_INVALID, "cells_per_cutoff in 0..4");
    RBF_CHECK(p->levels >= -1 && p->levels <= 7, RBF_ERR_INVALID, "levels in -1..7");
    RBF_CHECK(p->product == RBF_PRODUCT_TC || p->product == RBF_PRODUCT_SIMT, RBF_ERR_INVALID,
              "product must be RBF_PRODUCT_TC or RBF_PRODUCT_SIMT");
    RBF_CHECK(p->kernel == RBF_KERNEL_GAUSSIAN || p->kernel == RBF_KERNEL_IMQ, RBF_ERR_INVALID,
              "kernel must be RBF_KERNEL_GAUSSIAN or RBF_KERNEL_IMQ");
    RBF_CHECK(p->kernel != RBF_KERNEL_IMQ || (std::isfinite(p->beta) && p->beta > 0.f && p->beta <= 16.f),
              RBF_ERR_INVALID, "inverse multiquadric beta must be in (0, 16]");
    RBF_CHECK(std::isfinite(p->cell_edge) && p->cell_edge >= 0.f, RBF_ERR_INVALID,
              "cell_edge must be finite and >= 0 (0 selects the default)");
}

}  // namespace

unsigned *ctx_error_word(rbf_ctx *ctx) { return ctx->err_dev; }

void ctx_check_device_error(rbf_ctx *ctx) {
    const unsigned w = ctx->err_host ? *(volatile unsigned *)ctx->err_host : 0u;
    if (w) {
        *(volatile unsigned *)ctx->err_host = 0u;
        if (w & kErrTimeout)
            rbf_fail(RBF_ERR_TIMEOUT, "a bounded wait inside a product kernel expired (results of that launch invalid)");
        rbf_fail(RBF_ERR_RANGE, "double-float true residual: a row's share exceeded the fixed-point accumulator's "
                                "range (weights too large; residual_mode = RBF_RESIDUAL_F64 has no such limit)");
    }
}

namespace {

rbf_plan *make_plan(rbf_ctx *ctx, const float *centers, int64_t n, const rbf_plan_params *p, cudaStream_t s) {
    check_plan_params(p);
    RBF_CHECK(centers && aligned16(centers), RBF_ERR_INVALID, "centers must be a 16-byte aligned device pointer");
    RBF_CHECK(n > 0 && n < (1LL << 31) - 1, RBF_ERR_INVALID, "n = %lld out of range", (long long)n);
    rbf_plan *P = new rbf_plan();
    try {
        P->ctx = ctx;
        P->device = ctx->device;
        P->n = n;
        P->sigma = p->sigma;
        P->k = p->k;
        P->cells_per_cutoff = p->cells_per_cutoff > 0 ? p->cells_per_cutoff : 1;
        P->levels = p->levels >= 0 ? p->levels : 3;
        P->product = p->product;
        P->kernel = p->kernel;
        P->beta = p->kernel == RBF_KERNEL_IMQ ? p->beta : 0.f;
        P->cell_edge = p->cell_edge;
        plan_build(P, (const float4 *)centers, s);
    } catch (...) {
        delete P;
        throw;
    }
    return P;
}

}  // namespace

extern "C" {

int rbf_version(void) { return RBF_VERSION; }

int64_t rbf_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

const char *rbf_status_string(rbf_status s) {
    switch (s) {
        case RBF_OK: return "RBF_OK";
        case RBF_ERR_INVALID: return "RBF_ERR_INVALID";
        case RBF_ERR_OOM: return "RBF_ERR_OOM";
        case RBF_ERR_CUDA: return "RBF_ERR_CUDA";
        case RBF_ERR_NOT_CONVERGED: return "RBF_ERR_NOT_CONVERGED";
        case RBF_ERR_BREAKDOWN: return "RBF_ERR_BREAKDOWN";
        case RBF_ERR_TIMEOUT: return "RBF_ERR_TIMEOUT";
        case RBF_ERR_NOT_SPD: return "RBF_ERR_NOT_SPD";
        case RBF_ERR_UNSUPPORTED: return "RBF_ERR_UNSUPPORTED";
        case RBF_ERR_RANGE: return "RBF_ERR_RANGE";
    }
    return "RBF_UNKNOWN_STATUS";
}

rbf_status rbf_ctx_create(rbf_ctx **ctx, int device) {
    if (!ctx) return RBF_ERR_INVALID;
    *ctx = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        (void)cudaGetLastError();
        return RBF_ERR_CUDA;
    }
    rbf_ctx *c = new (std::nothrow) rbf_ctx();
    if (!c) return RBF_ERR_OOM;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaHostAlloc((void **)&c->err_host, sizeof(unsigned), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c->err_dev, c->err_host, 0) != cudaSuccess ||
        noalloc_prepare(c) != cudaSuccess) {
        if (c->err_host) cudaFreeHost(c->err_host);
        (void)cudaGetLastError();
        delete c;
        return RBF_ERR_CUDA;
    }
    *c->err_host = 0u;
    *ctx = c;
    return RBF_OK;
}

rbf_status rbf_ctx_destroy(rbf_ctx *ctx) {
    if (ctx && ctx->err_host) cudaFreeHost(ctx->err_host);
    delete ctx;
    return RBF_OK;
}

const char *rbf_last_error(const rbf_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

rbf_status rbf_build_centers(rbf_ctx *ctx, const float *pts, const float *nrm, int64_t N, float delta, float target,
                             float *centers, float *targets, float *delta_out, void *stream) {
    return guarded(ctx, [&]() {
        RBF_CHECK(pts && nrm && centers && targets, RBF_ERR_INVALID, "null pointer argument");
        RBF_CHECK(aligned16(centers), RBF_ERR_INVALID, "centers must be 16-byte aligned");
        RBF_CHECK(N > 0 && 3 * N < (1LL << 31) - 1, RBF_ERR_INVALID, "N = %lld out of range", (long long)N);
        RBF_CHECK(std::isfinite(delta) && std::isfinite(target), RBF_ERR_INVALID, "non-finite delta or target");
        float d = build_centers(pts, nrm, N, delta, target, centers, targets, S(stream));
        if (delta_out) *delta_out = d;
        return RBF_OK;
    });
}

rbf_status rbf_plan_create(rbf_ctx *ctx, const float *centers, int64_t n, const rbf_plan_params *p, rbf_plan **plan,
                           void *stream) {
    if (plan) *plan = nullptr;
    return guarded(ctx, [&]() {
        RBF_CHECK(plan, RBF_ERR_INVALID, "null plan output");
        *plan = make_plan(ctx, centers, n, p, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_plan_destroy(rbf_plan *plan) {
    if (!plan) return RBF_OK;
    int cur = 0;
    const bool have = cudaGetDevice(&cur) == cudaSuccess;
    cudaSetDevice(plan->device);     // its buffers belong to this device
    delete plan;
    if (have) cudaSetDevice(cur);
    (void)cudaGetLastError();        // leave no error behind for the caller's next check
    return RBF_OK;
}

rbf_status rbf_plan_get_info(const rbf_plan *P, rbf_plan_info *info) {
    if (!P || !info) return RBF_ERR_INVALID;
    std::memset(info, 0, sizeof(*info));
    info->n = P->n;
    info->ncells = P->ncells;
    info->nblocks = P->nblk;
    info->nchunks = P->nchk;
    info->pairlist_len = P->pl.len;
    info->nsegments = P->pl.nseg;
    info->nbits = P->nbits;
    info->levels = P->levels;
    for (int d = 0; d < 3; ++d) info->lo[d] = P->lo[d];
    info->inv = P->inv;
    info->cell_edge = P->hc;
    info->symmetric = P->sym_ready ? 1 : 0;
    info->sigma = P->sigma;
    info->k = P->k;
    return RBF_OK;
}

rbf_status rbf_plan_export_binning(rbf_plan *P, int32_t *perm, uint32_t *keys, int32_t *cell_start, int32_t *cell_end,
                                   void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        cudaStream_t s = S(stream);
        if (perm) RBF_CUDA(cudaMemcpyAsync(perm, P->perm.p, P->n * 4, cudaMemcpyDeviceToDevice, s));
        if (keys) RBF_CUDA(cudaMemcpyAsync(keys, P->keys.p, P->n * 4, cudaMemcpyDeviceToDevice, s));
        if (cell_start) RBF_CUDA(cudaMemcpyAsync(cell_start, P->cell_start.p, P->ncells * 4, cudaMemcpyDeviceToDevice, s));
        if (cell_end) RBF_CUDA(cudaMemcpyAsync(cell_end, P->cell_end.p, P->ncells * 4, cudaMemcpyDeviceToDevice, s));
        return RBF_OK;
    });
}

rbf_status rbf_matvec(rbf_plan *P, const float *z, float *y, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(z && y && z != y, RBF_ERR_INVALID, "z and y must be distinct device pointers");
        cudaStream_t s = S(stream);
        P->zs.ensure(P->n, s);
        P->ys.ensure(P->n, s);
        permute_to_binned_f32(P, z, P->zs.p, s);
        matvec_binned(P, P->zs.p, P->ys.p, s);
        permute_from_binned_f32(P, P->ys.p, y, s);
        return RBF_OK;
    });
}

rbf_status rbf_count_pairs(rbf_plan *P, int64_t *count, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(count, RBF_ERR_INVALID, "null count");
        *count = count_pairs(P, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_probe_wait_expiry(rbf_ctx *ctx, uint64_t limit_ns, void *stream) {
    return guarded(ctx, [&]() {
        cudaStream_t s = S(stream);
        launch_expiring_wait(ctx_error_word(ctx), limit_ns, s);
        RBF_CUDA(cudaStreamSynchronize(s));
        ctx_check_device_error(ctx);
        return RBF_OK;
    });
}

rbf_status rbf_count_candidate_pairs(rbf_plan *P, int64_t *count, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(count, RBF_ERR_INVALID, "null count");
        *count = count_candidates(P, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_residual(rbf_plan *P, const float *b, const double *x, double *r, double *norms, int mode,
                        void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(b && x && r, RBF_ERR_INVALID, "null pointer argument");
        cudaStream_t s = S(stream);
        DevBuf<float> bs;
        DevBuf<double> xs, rs;
        bs.alloc(P->n, s);
        xs.alloc(P->n, s);
        rs.alloc(P->n, s);
        permute_to_binned_f32(P, b, bs.p, s);
        permute_to_binned_f64(P, x, xs.p, s);
        RBF_CHECK(mode == RBF_RESIDUAL_DF || mode == RBF_RESIDUAL_F64, RBF_ERR_INVALID, "unknown residual mode %d",
                  mode);
        residual_binned(P, mode, bs.p, xs.p, rs.p, s);
        permute_from_binned_f64(P, rs.p, r, s);
        if (norms) {
            std::vector<double> hr(P->n);
            std::vector<float> hb(P->n);
            RBF_CUDA(cudaMemcpyAsync(hr.data(), rs.p, P->n * 8, cudaMemcpyDeviceToHost, s));
            RBF_CUDA(cudaMemcpyAsync(hb.data(), bs.p, P->n * 4, cudaMemcpyDeviceToHost, s));
            RBF_CUDA(cudaStreamSynchronize(s));
            double a = 0, c = 0;
            for (int64_t i = 0; i < P->n; ++i) {
                a += hr[i] * hr[i];
                c += (double)hb[i] * (double)hb[i];
            }
            norms[0] = std::sqrt(a);
            norms[1] = std::sqrt(c);
            ctx_check_device_error(P->ctx);
        }
        return RBF_OK;
    });
}

rbf_status rbf_plan_assemble(rbf_plan *P, int64_t max_bytes, int64_t *nnz, int64_t *stored, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(nnz && stored, RBF_ERR_INVALID, "nnz and stored are required");
        *nnz = 0;
        *stored = 0;
        assemble_csr(P, max_bytes, nnz, stored, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_plan_release_csr(rbf_plan *P) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        P->csr.release();
        return RBF_OK;
    });
}

rbf_status rbf_plan_export_csr(rbf_plan *P, int64_t *row_ptr, int32_t *col, float *val, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        const CsrData &M = P->csr;
        RBF_CHECK(M.ready, RBF_ERR_INVALID, "the plan has no assembled matrix");
        cudaStream_t s = S(stream);
        if (row_ptr)
            RBF_CUDA(cudaMemcpyAsync(row_ptr, M.row_ptr.p, (P->n + 1) * 8, cudaMemcpyDeviceToDevice, s));
        if (col) RBF_CUDA(cudaMemcpyAsync(col, M.col.p, M.stored * 4, cudaMemcpyDeviceToDevice, s));
        if (val) RBF_CUDA(cudaMemcpyAsync(val, M.val.p, M.stored * 4, cudaMemcpyDeviceToDevice, s));
        return RBF_OK;
    });
}

rbf_status rbf_spmv(rbf_plan *P, const float *z, float *y, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(z && y && z != y, RBF_ERR_INVALID, "z and y must be distinct device pointers");
        RBF_CHECK(P->csr.ready, RBF_ERR_INVALID, "the plan has no assembled matrix (call rbf_plan_assemble first)");
        cudaStream_t s = S(stream);
        P->zs.ensure(P->n, s);
        P->ys.ensure(P->n, s);
        permute_to_binned_f32(P, z, P->zs.p, s);
        spmv_binned(P, P->zs.p, P->ys.p, s);
        permute_from_binned_f32(P, P->ys.p, y, s);
        return RBF_OK;
    });
}

rbf_status rbf_schwarz_setup(rbf_plan *P, const rbf_schwarz_params *p, int64_t *failed, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(p, RBF_ERR_INVALID, "null schwarz parameters");
        int64_t f = 0;
        schwarz_setup(P, *p, &f, S(stream));
        if (failed) *failed = f;
        return f > 0 ? RBF_ERR_NOT_SPD : RBF_OK;
    });
}

rbf_status rbf_schwarz_apply(rbf_plan *P, const float *v, float *z, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(v && z && v != z, RBF_ERR_INVALID, "v and z must be distinct device pointers");
        cudaStream_t s = S(stream);
        P->zs.ensure(P->n, s);
        P->ys.ensure(P->n, s);
        permute_to_binned_f32(P, v, P->zs.p, s);
        schwarz_apply_binned(P, nullptr, P->zs.p, P->ys.p, s);
        permute_from_binned_f32(P, P->ys.p, z, s);
        return RBF_OK;
    });
}

rbf_status rbf_plan_solve(rbf_plan *P, const float *b, const rbf_solve_params *p, double *x, rbf_report *report,
                          void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(b && p && x, RBF_ERR_INVALID, "null pointer argument");
        RBF_CHECK(p->precond == RBF_PRECOND_NONE || p->precond == RBF_PRECOND_SCHWARZ ||
                      p->precond == RBF_PRECOND_MLP,
                  RBF_ERR_INVALID, "unknown preconditioner %d", p->precond);
        RBF_CHECK(std::isfinite(p->tol) && p->tol >= 0, RBF_ERR_INVALID, "tol must be finite and >= 0");
        RBF_CHECK(p->residual_mode == RBF_RESIDUAL_DF || p->residual_mode == RBF_RESIDUAL_F64, RBF_ERR_INVALID,
                  "unknown residual mode %d", p->residual_mode);
        return fgmres_solve(P, b, *p, x, report, S(stream));
    });
}

rbf_status rbf_solve(rbf_ctx *ctx, const float *centers, const float *targets, int64_t n, const rbf_plan_params *pp,
                     const rbf_solve_params *sp, double *weights, rbf_report *report, void *stream) {
    return guarded(ctx, [&]() {
        RBF_CHECK(targets && sp && weights, RBF_ERR_INVALID, "null pointer argument");
        rbf_plan *P = make_plan(ctx, centers, n, pp, S(stream));
        rbf_status st;
        try {
            st = fgmres_solve(P, targets, *sp, weights, report, S(stream));
        } catch (...) {
            delete P;
            throw;
        }
        cudaStreamSynchronize(S(stream));
        delete P;
        return st;
    });
}

rbf_status rbf_plan_eval_grid(rbf_plan *P, const double *weights, const rbf_grid *g, float *f, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(weights && g && f, RBF_ERR_INVALID, "null pointer argument");
        eval_grid(P, weights, *g, f, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_count_grid_pairs(rbf_plan *P, const rbf_grid *g, int64_t *count, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(g && count, RBF_ERR_INVALID, "null pointer argument");
        *count = count_grid_pairs(P, *g, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_count_grid_candidate_pairs(rbf_plan *P, const rbf_grid *g, int64_t *count, void *stream) {
    if (!P) return RBF_ERR_INVALID;
    return guarded(P->ctx, [&]() {
        RBF_CHECK(g && count, RBF_ERR_INVALID, "null pointer argument");
        *count = count_grid_candidates(P, *g, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_isosurface(rbf_ctx *ctx, const float *f, const rbf_grid *g, float iso, const float *points,
                          int64_t npoints, float band, float *triangles, int64_t capacity, int64_t *ntri,
                          void *stream) {
    return guarded(ctx, [&]() {
        RBF_CHECK(f && g && ntri, RBF_ERR_INVALID, "null pointer argument");
        RBF_CHECK(!points || aligned16(points), RBF_ERR_INVALID, "points must be 16-byte aligned");
        RBF_CHECK(npoints >= 0 && npoints < (1LL << 31) - 1, RBF_ERR_INVALID, "npoints out of range");
        *ntri = isosurface(ctx, f, *g, iso, (const float4 *)points, npoints, band, triangles, capacity, S(stream));
        RBF_CHECK(!triangles || *ntri <= capacity, RBF_ERR_INVALID, "triangle buffer holds %lld, the level set has %lld",
                  (long long)capacity, (long long)*ntri);
        return RBF_OK;
    });
}

rbf_status rbf_density_measures(rbf_ctx *ctx, const float *points, int64_t n, const float *probes, int64_t m,
                                float cell, float *nn, rbf_density *out, void *stream) {
    return guarded(ctx, [&]() {
        RBF_CHECK(points && out && aligned16(points), RBF_ERR_INVALID,
                  "points must be a 16-byte aligned device pointer, out non-null");
        RBF_CHECK(m == 0 || (probes && aligned16(probes)), RBF_ERR_INVALID, "probes must be 16-byte aligned");
        RBF_CHECK(n < (1LL << 31) - 1 && m < (1LL << 31) - 1, RBF_ERR_INVALID, "n or m out of range");
        RBF_CHECK(std::isfinite(cell), RBF_ERR_INVALID, "cell must be finite");
        density_measures(ctx, (const float4 *)points, n, (const float4 *)probes, m, cell, nn, out, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_eval_grid(rbf_ctx *ctx, const float *centers, const double *weights, int64_t n,
                         const rbf_plan_params *pp, const rbf_grid *g, float *f, void *stream) {
    return guarded(ctx, [&]() {
        RBF_CHECK(weights && g && f, RBF_ERR_INVALID, "null pointer argument");
        rbf_plan *P = make_plan(ctx, centers, n, pp, S(stream));
        try {
            eval_grid(P, weights, *g, f, S(stream));
        } catch (...) {
            delete P;
            throw;
        }
        cudaStreamSynchronize(S(stream));
        delete P;
        return RBF_OK;
    });
}

rbf_status rbf_mlp_create(rbf_ctx *ctx, const float *host_params, rbf_mlp **mlp) {
    if (mlp) *mlp = nullptr;
    return guarded(ctx, [&]() {
        RBF_CHECK(host_params && mlp, RBF_ERR_INVALID, "null pointer argument");
        *mlp = mlp_create(ctx, host_params, 0);
        return RBF_OK;
    });
}

rbf_status rbf_mlp_destroy(rbf_mlp *mlp) {
    if (mlp) mlp_destroy(mlp);
    return RBF_OK;
}

rbf_status rbf_mlp_get_params(rbf_mlp *mlp, float *host_params) {
    if (!mlp) return RBF_ERR_INVALID;
    return guarded(mlp_ctx(mlp), [&]() {
        RBF_CHECK(host_params, RBF_ERR_INVALID, "null pointer argument");
        mlp_get_params(mlp, host_params, 0);
        return RBF_OK;
    });
}

rbf_status rbf_mlp_make_data(rbf_plan *plan, float lambda, const int32_t *block_ids, const float *R, int64_t ns,
                             float *X, float *Y, int64_t *failed, void *stream) {
    if (!plan) return RBF_ERR_INVALID;
    return guarded(plan->ctx, [&]() {
        RBF_CHECK(block_ids && R && X && Y && ns >= 0, RBF_ERR_INVALID, "null pointer argument");
        RBF_CHECK(plan->kernel == RBF_KERNEL_GAUSSIAN, RBF_ERR_UNSUPPORTED,
                  "the learned preconditioner is trained on Gaussian blocks");
        int64_t f = mlp_make_data(plan, lambda, block_ids, R, ns, X, Y, S(stream));
        if (failed) *failed = f;
        return RBF_OK;
    });
}

rbf_status rbf_mlp_forward(rbf_mlp *mlp, const float *X, int64_t rows, float *Y, int use_bf16, void *stream) {
    if (!mlp) return RBF_ERR_INVALID;
    return guarded(mlp_ctx(mlp), [&]() {
        RBF_CHECK(X && Y && rows >= 0, RBF_ERR_INVALID, "null pointer argument");
        mlp_forward(mlp, X, rows, Y, use_bf16, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_mlp_loss_grad(rbf_mlp *mlp, const float *X, const float *T, int64_t rows, double *loss,
                             float *host_grad, void *stream) {
    if (!mlp) return RBF_ERR_INVALID;
    return guarded(mlp_ctx(mlp), [&]() {
        RBF_CHECK(X && T && loss && rows > 0 && rows <= 65536, RBF_ERR_INVALID, "bad arguments");
        *loss = mlp_loss_grad(mlp, X, T, (int)rows, host_grad != nullptr, S(stream));
        if (host_grad) mlp_get_grad(mlp, host_grad, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_mlp_train(rbf_mlp *mlp, const float *X, const float *T, int64_t ns, const rbf_train_params *p,
                         double *loss_history, void *stream) {
    if (!mlp) return RBF_ERR_INVALID;
    return guarded(mlp_ctx(mlp), [&]() {
        RBF_CHECK(X && T && p && ns > 0 && p->epochs > 0 && p->batch > 0 && p->batch <= 65536 && p->lr > 0.f,
                  RBF_ERR_INVALID, "bad training arguments");
        cudaStream_t s = S(stream);
        for (int e = 0; e < p->epochs; ++e) {
            double sum = 0.0;
            int64_t nb = 0;
            for (int64_t r0 = 0; r0 < ns; r0 += p->batch) {
                const int rows = (int)std::min<int64_t>(p->batch, ns - r0);
                sum += mlp_loss_grad(mlp, X + r0 * RBF_MLP_IN, T + r0 * RBF_MLP_OUT, rows, true, s);
                mlp_adam_step(mlp, p->lr, s);
                ++nb;
            }
            if (loss_history) loss_history[e] = sum / (double)nb;
        }
        RBF_CUDA(cudaStreamSynchronize(s));
        return RBF_OK;
    });
}

rbf_status rbf_batch_create(rbf_ctx *ctx, rbf_plan *const *plans, int nplans, rbf_batch **batch, void *stream) {
    if (batch) *batch = nullptr;
    return guarded(ctx, [&]() {
        RBF_CHECK(batch, RBF_ERR_INVALID, "null batch output");
        *batch = batch_create(ctx, plans, nplans, S(stream));
        return RBF_OK;
    });
}

rbf_status rbf_batch_destroy(rbf_batch *batch) {
    if (!batch) return RBF_OK;
    batch_destroy(batch);
    return RBF_OK;
}

int64_t rbf_batch_size(const rbf_batch *batch) { return batch ? batch_size(batch) : 0; }

rbf_status rbf_batch_matvec(rbf_batch *batch, const float *z, float *y, void *stream) {
    if (!batch) return RBF_ERR_INVALID;
    rbf_ctx *ctx = batch_ctx(batch);
    return guarded(ctx, [&]() {
        RBF_CHECK(z && y && z != y, RBF_ERR_INVALID, "z and y must be distinct device pointers");
        cudaStream_t s = S(stream);
        const int64_t N = batch_size(batch);
        ctx_check_device_error(ctx);
        DevBuf<float> zs, ys;
        zs.alloc(N, s);
        ys.alloc(N, s);
        batch_gather_f32(batch, z, zs.p, s);
        batch_matvec_binned(batch, zs.p, ys.p, s);
        batch_scatter_f32(batch, ys.p, y, s);
        return RBF_OK;
    });
}

rbf_status rbf_batch_solve(rbf_batch *batch, const float *b, const rbf_solve_params *p, double *x,
                           rbf_report *reports, rbf_batch_stats *stats, void *stream) {
    if (!batch) return RBF_ERR_INVALID;
    return guarded(batch_ctx(batch), [&]() {
        RBF_CHECK(b && p && x, RBF_ERR_INVALID, "null pointer argument");
        return batch_solve(batch, b, *p, x, reports, stats, S(stream));
    });
}

rbf_status rbf_batch_autotune(rbf_batch *batch, const float *b, const rbf_solve_params *p, const int *candidates,
                              int ncand, int *best, double *scores, void *stream) {
    if (!batch) return RBF_ERR_INVALID;
    return guarded(batch_ctx(batch), [&]() {
        RBF_CHECK(b && p && candidates && ncand > 0 && best, RBF_ERR_INVALID, "null pointer argument");
        for (int c = 0; c < ncand; ++c)
            RBF_CHECK(candidates[c] >= 1 && candidates[c] <= 128, RBF_ERR_UNSUPPORTED, "block %d outside 1..128",
                      candidates[c]);
        *best = batch_autotune(batch, b, *p, candidates, ncand, scores, S(stream));
        return RBF_OK;
    });
}

}  // extern "C"
