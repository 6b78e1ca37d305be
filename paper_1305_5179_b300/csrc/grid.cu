// Step 3 of Algorithm 1 (Eq. matxvet): P_f on the nodes of a structured grid.
//
// The grid is cut into bricks of 128 nodes (one tile of the product kernel), each
// cut into four quarters of 32 nodes; brick and quarter are powers of two along each
// axis, chosen per grid from its node spacings so that their boxes are compact in
// space (8 x 4 x 4 and 4 x 2 x 4 on an evenly spaced grid).  Each brick gets a box
// and a pair list against the source blocks exactly like the tiles of centres, so
// bricks far from every centre cost nothing.  The pair list is cached on the plan for
// repeated grids.
#include <cmath>

#include "plan.cuh"

void matvec_grid_launch(rbf_plan *P, const PairList &pl, const float *ws, const rbf_grid &g, const GridCache &gc,
                        float *f, cudaStream_t s);
int64_t count_grid_pairs_launch(rbf_plan *P, const PairList &pl, const rbf_grid &g, const GridCache &gc,
                                cudaStream_t s);
namespace {

// Brick boxes, and the boxes of its four quarters (quarter u at offsets (ux, uy, uz) of
// the brick's quarters, x fastest; a quarter entirely outside the grid gets lo > hi).
__global__ void k_brick_boxes(int64_t nb, int bx, int by, int3 blog, int3 qlog, int gx, int gy, int gz, float lox,
                              float loy, float loz, float sx, float sy, float sz, float4 *__restrict__ lo,
                              float4 *__restrict__ hi, float4 *__restrict__ qlo, float4 *__restrict__ qhi) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    int ix = (int)(t % bx), iy = (int)((t / bx) % by), iz = (int)(t / ((int64_t)bx * by));
    int x0 = ix << blog.x, y0 = iy << blog.y, z0 = iz << blog.z;
    int x1 = min(x0 + (1 << blog.x) - 1, gx - 1), y1 = min(y0 + (1 << blog.y) - 1, gy - 1),
        z1 = min(z0 + (1 << blog.z) - 1, gz - 1);
    lo[t] = make_float4(fmaf((float)x0, sx, lox), fmaf((float)y0, sy, loy), fmaf((float)z0, sz, loz), 0.f);
    hi[t] = make_float4(fmaf((float)x1, sx, lox), fmaf((float)y1, sy, loy), fmaf((float)z1, sz, loz), 0.f);
    const int nx = blog.x - qlog.x, ny = blog.y - qlog.y;
    for (int u = 0; u < 4; ++u) {
        const int ux = u & ((1 << nx) - 1), uy = (u >> nx) & ((1 << ny) - 1), uz = u >> (nx + ny);
        const int xa = x0 + (ux << qlog.x), ya = y0 + (uy << qlog.y), za = z0 + (uz << qlog.z);
        if (xa < gx && ya < gy && za < gz) {
            const int xb = min(xa + (1 << qlog.x) - 1, gx - 1), yb = min(ya + (1 << qlog.y) - 1, gy - 1),
                      zb = min(za + (1 << qlog.z) - 1, gz - 1);
            qlo[4 * t + u] = make_float4(fmaf((float)xa, sx, lox), fmaf((float)ya, sy, loy), fmaf((float)za, sz, loz), 0.f);
            qhi[4 * t + u] = make_float4(fmaf((float)xb, sx, lox), fmaf((float)yb, sy, loy), fmaf((float)zb, sz, loz), 0.f);
        } else {
            qlo[4 * t + u] = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
            qhi[4 * t + u] = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
        }
    }
}

// Brick (2^blog, 128 nodes) and quarter (2^qlog, 32 nodes) shapes for a grid with node
// spacings st.  A brick's pair list holds the source blocks within `reach` of its box, so
// the brick minimises (number of bricks) x prod_d (box extent_d + 2 reach), to first order
// the sum of the box's extents; the quarters, which decide how many of those pairs are
// evaluated, minimise prod_d (extent_d + 2 reach) of their own boxes.  Ties keep the first
// shape in the order below, which gives 8 x 4 x 4 bricks of 4 x 2 x 4 quarters on an
// evenly spaced grid.
void choose_shape(const rbf_grid &g, const float st[3], double reach, int blog[3], int qlog[3]) {
    auto ext = [&](int d, int l) { return (double)(std::min<int64_t>(int64_t(1) << l, g.dims[d]) - 1) * st[d]; };
    double best = INFINITY;
    for (int a = 7; a >= 0; --a)
        for (int c = 7 - a; c >= 0; --c) {
            const int b = 7 - a - c;
            const int l[3] = {a, b, c};
            double cost = 1.0;
            for (int d = 0; d < 3; ++d) cost *= (double)ceil_div(g.dims[d], int64_t(1) << l[d]) * (ext(d, l[d]) + 2 * reach);
            if (cost < best * (1.0 - 1e-12)) {
                best = cost;
                for (int d = 0; d < 3; ++d) blog[d] = l[d];
            }
        }
    best = INFINITY;
    for (int a = std::min(5, blog[0]); a >= 0; --a)
        for (int c = std::min(5 - a, blog[2]); c >= 0; --c) {
            const int b = 5 - a - c;
            if (b > blog[1]) continue;
            const int l[3] = {a, b, c};
            double cost = 1.0;
            for (int d = 0; d < 3; ++d) cost *= ext(d, l[d]) + 2 * reach;
            if (cost < best * (1.0 - 1e-12)) {
                best = cost;
                for (int d = 0; d < 3; ++d) qlog[d] = l[d];
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
    matvec_grid_launch(P, gc.pl, P->zs.p, g, gc, f, s);
}

int64_t count_grid_pairs(rbf_plan *P, const rbf_grid &g, cudaStream_t s) {
    grid_prepare(P, g, s);
    return count_grid_pairs_launch(P, P->grid.pl, g, P->grid, s);
}

int64_t count_grid_candidates(rbf_plan *P, const rbf_grid &g, cudaStream_t s) {
    grid_prepare(P, g, s);
    return count_candidates_list(P->grid.pl, nullptr, s);
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
        float st[3];
        for (int d = 0; d < 3; ++d)
            st[d] = g.dims[d] > 1 ? (float)(((double)g.hi[d] - (double)g.lo[d]) / (double)(g.dims[d] - 1)) : 0.f;
        // how far a brick's pair list reaches: the plan's culling radius (the cut-off, or the
        // radius beyond which untruncated Gaussian blocks are skipped); when every block is kept,
        // a large constant leaves each shape's cost proportional to its number of bricks
        const double reach = std::isfinite(P->rc) ? (double)P->rc : 1e30;
        choose_shape(g, st, reach, gc.blog, gc.qlog);
        for (int d = 0; d < 3; ++d) gc.bricks[d] = ceil_div(g.dims[d], int64_t(1) << gc.blog[d]);
        int64_t nb = gc.bricks[0] * gc.bricks[1] * gc.bricks[2];
        DevBuf<float4> blo, bhi, qlo, qhi;
        blo.alloc(nb, s);
        bhi.alloc(nb, s);
        qlo.alloc(4 * nb, s);
        qhi.alloc(4 * nb, s);
        k_brick_boxes<<<(unsigned)ceil_div(nb, 256), 256, 0, s>>>(nb, (int)gc.bricks[0], (int)gc.bricks[1],
                                                                  make_int3(gc.blog[0], gc.blog[1], gc.blog[2]),
                                                                  make_int3(gc.qlog[0], gc.qlog[1], gc.qlog[2]),
                                                                  (int)g.dims[0], (int)g.dims[1], (int)g.dims[2],
                                                                  g.lo[0], g.lo[1], g.lo[2], st[0], st[1], st[2],
                                                                  blo.p, bhi.p, qlo.p, qhi.p);
        RBF_LAUNCHED();
        build_pairlist(P, blo.p, bhi.p, qlo.p, qhi.p, nb, gc.pl, s);
        gc.valid = true;
    }
    return total;
}
