/* The whole path through the C interface alone (no Python): a golden-spiral sphere of
 * 400 points -> extended centres (Sec. II.A) -> plan -> RAS-preconditioned FGMRES
 * (Sec. III.A) -> P_f on a 24^3 grid (Eq. matxvet).  Checks what the method fixes
 * for a sphere: P_f < 0 at 0.85 u and > 0 at 1.15 u on the six axis directions u
 * (single-node grids, 1.5 sigma from the surface), the grid values finite, the
 * reported float64 residual below the tolerance, and an invalid call reported as such.
 * Exit status 0 and the line "c abi ok" on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "rbf.h"

#define CHECK(call)                                                                           \
    do {                                                                                      \
        rbf_status st_ = (call);                                                              \
        if (st_ != RBF_OK) {                                                                  \
            fprintf(stderr, "%s failed: %s (%s)\n", #call, rbf_status_string(st_),            \
                    ctx ? rbf_last_error(ctx) : "");                                          \
            return 1;                                                                         \
        }                                                                                     \
    } while (0)

#define CUDA(call)                                                                            \
    do {                                                                                      \
        if ((call) != cudaSuccess) {                                                          \
            fprintf(stderr, "%s failed\n", #call);                                            \
            return 1;                                                                         \
        }                                                                                     \
    } while (0)

int main(void) {
    const int64_t N = 400, n = 3 * N;
    const int G = 24;
    rbf_ctx *ctx = NULL;
    float *hp = malloc(N * 3 * sizeof(float));
    for (int64_t i = 0; i < N; ++i) {   /* golden-angle spiral on the unit sphere */
        double z = 1.0 - (2.0 * i + 1.0) / N, r = sqrt(1.0 - z * z), a = 3.14159265358979323846 * (3.0 - sqrt(5.0)) * i;
        hp[3 * i] = (float)(r * cos(a));
        hp[3 * i + 1] = (float)(r * sin(a));
        hp[3 * i + 2] = (float)z;
    }
    float *pts, *centers, *targets, *f;
    double *x;
    CUDA(cudaMalloc((void **)&pts, N * 3 * sizeof(float)));
    CUDA(cudaMalloc((void **)&centers, n * 4 * sizeof(float)));
    CUDA(cudaMalloc((void **)&targets, n * sizeof(float)));
    CUDA(cudaMalloc((void **)&x, n * sizeof(double)));
    CUDA(cudaMalloc((void **)&f, (size_t)G * G * G * sizeof(float)));
    CUDA(cudaMemcpy(pts, hp, N * 3 * sizeof(float), cudaMemcpyHostToDevice));

    CHECK(rbf_ctx_create(&ctx, 0));
    /* the unit sphere's outward normal is the position itself */
    CHECK(rbf_build_centers(ctx, pts, pts, N, 0.05f, 0.f, centers, targets, NULL, NULL));

    rbf_plan_params pp = {0};
    pp.sigma = 0.1f;            /* about half the point spacing: a well-conditioned system */
    pp.k = 0.f;                 /* untruncated */
    pp.levels = -1;
    pp.product = RBF_PRODUCT_TC;
    pp.kernel = RBF_KERNEL_GAUSSIAN;
    rbf_plan *plan = NULL;
    CHECK(rbf_plan_create(ctx, centers, n, &pp, &plan, NULL));

    rbf_solve_params sp = {0};
    sp.m = 50;
    sp.max_it = 400;
    sp.tol = 1e-6;
    sp.precond = RBF_PRECOND_SCHWARZ;
    sp.schwarz.core = 96;
    sp.schwarz.block = 128;
    sp.schwarz.shift = 1e-4f;
    sp.schwarz.restricted = 1;
    sp.schwarz.escalate = 1;
    sp.true_residual_each_restart = 1;
    rbf_report rep;
    CHECK(rbf_plan_solve(plan, targets, &sp, x, &rep, NULL));

    rbf_grid g = {{-1.2f, -1.2f, -1.2f}, {1.2f, 1.2f, 1.2f}, {G, G, G}};
    CHECK(rbf_plan_eval_grid(plan, x, &g, f, NULL));
    float *hf = malloc((size_t)G * G * G * sizeof(float));
    CUDA(cudaMemcpy(hf, f, (size_t)G * G * G * sizeof(float), cudaMemcpyDeviceToHost));

    int fails = 0;
    for (int64_t i = 0; i < (int64_t)G * G * G; ++i)
        if (!isfinite(hf[i])) { fprintf(stderr, "grid value %lld not finite\n", (long long)i); ++fails; break; }
    /* inside and outside the surface along the axes: single-node grids (lo = hi) */
    for (int a = 0; a < 6; ++a) {
        for (int side = 0; side < 2; ++side) {
            const float r = side ? 1.15f : 0.85f, sgn = (a & 1) ? -1.f : 1.f;
            float p[3] = {0.f, 0.f, 0.f};
            p[a >> 1] = sgn * r;
            rbf_grid one = {{p[0], p[1], p[2]}, {p[0], p[1], p[2]}, {1, 1, 1}};
            float v = 0.f;
            CHECK(rbf_plan_eval_grid(plan, x, &one, f, NULL));
            CUDA(cudaMemcpy(&v, f, sizeof(float), cudaMemcpyDeviceToHost));
            if (side ? !(v > 0.f) : !(v < 0.f)) {
                fprintf(stderr, "P_f(%g, %g, %g) = %g has the wrong sign\n", p[0], p[1], p[2], v);
                ++fails;
            }
        }
    }
    if (!(rep.converged == 1 && rep.residual_true <= 1e-6)) {
        fprintf(stderr, "solve: converged %d, residual %g after %d iterations\n", rep.converged, rep.residual_true,
                rep.iterations);
        ++fails;
    }
    rbf_plan_params bad = pp;
    bad.sigma = -1.f;
    rbf_plan *none = NULL;
    if (rbf_plan_create(ctx, centers, n, &bad, &none, NULL) != RBF_ERR_INVALID || none != NULL) {
        fprintf(stderr, "sigma < 0 was not rejected\n");
        ++fails;
    }

    rbf_plan_destroy(plan);
    rbf_ctx_destroy(ctx);
    cudaFree(pts);
    cudaFree(centers);
    cudaFree(targets);
    cudaFree(x);
    cudaFree(f);
    free(hp);
    free(hf);
    if (fails) return 1;
    printf("c abi ok: %d iterations, residual %.3e\n", rep.iterations, rep.residual_true);
    return 0;
}
