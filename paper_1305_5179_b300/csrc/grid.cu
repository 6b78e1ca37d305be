// Step 3 of Algorithm 1 (Eq. matxvet): P_f on the nodes of a structured grid.
//
// The grid is cut into bricks of 8 x 4 x 4 nodes (128 targets, one tile of the
// product kernel; its four quarters of 32 nodes are blocks of 4 x 2 x 4); each brick
// gets a box and a pair list against the source
// blocks exactly like the tiles of centres, so bricks far from every centre
// cost nothing.  The pair list is cached on the plan for repeated grids.
#include <cmath>

#include "plan.cuh"

void matvec_grid_launch(rbf_plan *P, const PairList &pl, const float *ws, const rbf_grid &g, const int64_t bricks[3],
                        float *f, cudaStream_t s);
int64_t count_grid_pairs_launch(rbf_plan *P, const PairList &pl, const rbf_grid &g, const int64_t bricks[3],
                                cudaStream_t s);

namespace {

// Brick boxes, and the boxes of its four quarters of 32 nodes (blocks of 4 x 2 x 4
// nodes, quarter u at x offset 4 (u & 1) and y offset 2 (u >> 1); a quarter entirely
// outside the grid gets lo > hi).
__global__ void k_brick_boxes(int64_t nb, int bx, int by, int gx, int gy, int gz, float lox, float loy, float loz,
                              float sx, float sy, float sz, float4 *__restrict__ lo, float4 *__restrict__ hi,
                              float4 *__restrict__ qlo, float4 *__restrict__ qhi) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    int ix = (int)(t % bx), iy = (int)((t / bx) % by), iz = (int)(t / ((int64_t)bx * by));
    int x0 = ix * 8, y0 = iy * 4, z0 = iz * 4;
    int x1 = min(x0 + 7, gx - 1), y1 = min(y0 + 3, gy - 1), z1 = min(z0 + 3, gz - 1);
    const float X0 = fmaf((float)x0, sx, lox), Y0 = fmaf((float)y0, sy, loy);
    const float X1 = fmaf((float)x1, sx, lox), Y1 = fmaf((float)y1, sy, loy);
    const float Z0 = fmaf((float)z0, sz, loz), Z1 = fmaf((float)z1, sz, loz);
    lo[t] = make_float4(X0, Y0, Z0, 0.f);
    hi[t] = make_float4(X1, Y1, Z1, 0.f);
    for (int u = 0; u < 4; ++u) {
        const int xa = x0 + 4 * (u & 1), ya = y0 + 2 * (u >> 1);
        if (xa < gx && ya < gy) {
            const int xb = min(xa + 3, gx - 1), yb = min(ya + 1, gy - 1);
            qlo[4 * t + u] = make_float4(fmaf((float)xa, sx, lox), fmaf((float)ya, sy, loy), Z0, 0.f);
            qhi[4 * t + u] = make_float4(fmaf((float)xb, sx, lox), fmaf((float)yb, sy, loy), Z1, 0.f);
        } else {
            qlo[4 * t + u] = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
            qhi[4 * t + u] = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
        }
    }
}

bool same_grid(const rbf_grid &a, const rbf_grid &b) {
    for (int d = 0; d < 3; ++d)
        if (a.lo[d] != b.lo[d] || a.hi[d] != b.hi[d] || a.dims[d] != b.dims[d]) return false;
    return true;
}

}  // namespace

static int64_t grid_prepare(rbf_plan *P, const rbf_grid &g, cudaStream_t s);

void eval_grid(rbf_plan *P, const double *weights, const rbf_grid &g, float *f, cudaStream_t s) {
    int64_t total = grid_prepare(P, g, s);
    P->zs.ensure(P->n, s);
    permute_to_binned_f64_to_f32(P, weights, P->zs.p, s);
    GridCache &gc = P->grid;
    // bricks with no source block within the cut-off are never visited: clear the field first
    RBF_CUDA(cudaMemsetAsync(f, 0, (size_t)total * sizeof(float), s));
    matvec_grid_launch(P, gc.pl, P->zs.p, g, gc.bricks, f, s);
}

int64_t count_grid_pairs(rbf_plan *P, const rbf_grid &g, cudaStream_t s) {
    grid_prepare(P, g, s);
    return count_grid_pairs_launch(P, P->grid.pl, g, P->grid.bricks, s);
}

// Validates the grid and (re)builds the brick pair list when the grid changed.
static int64_t grid_prepare(rbf_plan *P, const rbf_grid &g, cudaStream_t s) {
    int64_t total = 1;
    for (int d = 0; d < 3; ++d) {
        RBF_CHECK(g.dims[d] >= 1 && g.dims[d] < (1LL << 24), RBF_ERR_INVALID, "grid dims[%d] = %lld out of range", d,
                  (long long)g.dims[d]);
        RBF_CHECK(std::isfinite(g.lo[d]) && std::isfinite(g.hi[d]), RBF_ERR_INVALID, "non-finite grid bounds");
        total *= g.dims[d];
    }
    RBF_CHECK(total < (1LL << 31), RBF_ERR_INVALID, "grid has %lld nodes (limit 2^31)", (long long)total);
    GridCache &gc = P->grid;
    if (!gc.valid || !same_grid(gc.g, g)) {
        gc.valid = false;
        gc.g = g;
        gc.bricks[0] = ceil_div(g.dims[0], 8);
        gc.bricks[1] = ceil_div(g.dims[1], 4);
        gc.bricks[2] = ceil_div(g.dims[2], 4);
        int64_t nb = gc.bricks[0] * gc.bricks[1] * gc.bricks[2];
        float st[3];
        for (int d = 0; d < 3; ++d)
            st[d] = g.dims[d] > 1 ? (float)(((double)g.hi[d] - (double)g.lo[d]) / (double)(g.dims[d] - 1)) : 0.f;
        DevBuf<float4> blo, bhi, qlo, qhi;
        blo.alloc(nb, s);
        bhi.alloc(nb, s);
        qlo.alloc(4 * nb, s);
        qhi.alloc(4 * nb, s);
        k_brick_boxes<<<(unsigned)ceil_div(nb, 256), 256, 0, s>>>(nb, (int)gc.bricks[0], (int)gc.bricks[1],
                                                                  (int)g.dims[0], (int)g.dims[1], (int)g.dims[2],
                                                                  g.lo[0], g.lo[1], g.lo[2], st[0], st[1], st[2],
                                                                  blo.p, bhi.p, qlo.p, qhi.p);
        RBF_LAUNCHED();
        build_pairlist(P, blo.p, bhi.p, qlo.p, qhi.p, nb, gc.pl, s);
        gc.valid = true;
    }
    return total;
}
