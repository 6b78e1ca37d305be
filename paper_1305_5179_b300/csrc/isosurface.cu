// Step 4 of Algorithm 1 without the rendering: the level set {P_f = iso} of the
// grid field of step 3 as a headless triangle buffer (the paper hands the grid to
// MATLAB's isosurface).  Marching tetrahedra: every grid cell is cut into the six
// tetrahedra around its diagonal from corner 0 = (0,0,0) to corner 7 = (1,1,1)
// (corner c has offsets (c & 1, c >> 1 & 1, c >> 2 & 1)); the same cut in every
// cell makes the faces of neighbouring cells match.  A corner is inside when
// f < iso.  A tetrahedron with one corner on its own side gives one triangle on
// the three edges of that corner, one with two inside corners gives the two
// triangles of the quadrilateral on its four mixed edges; triangles are ordered so
// that (v1 - v0) x (v2 - v0) points from inside to outside.  An edge point is
// interpolated from the edge's corner of smaller node index, so an edge shared by
// several tetrahedra or cells yields the same point.  Cells with a NaN corner
// (nodes the evaluation left out) produce nothing.  With data points and a band
// eps > 0, a cell contributes only when its centre lies within eps of a data point
// (the surrounding volume M_ext^eps of Sec. II.A.3, d(x, M) read as the distance
// to the nearest data point); the test searches the 27 cells (edge >= eps) of a
// binning of the points around the centre and stops at the first hit.
//
// Passes: per-cell triangle counts, an exclusive scan, then the triangles at their
// offsets, in cell order (x fastest), tetrahedron order, triangle order.
#include <algorithm>
#include <cmath>

#include "centers.cuh"
#include "plan.cuh"

namespace {

constexpr int kThr = 256;

// The 6 tetrahedra 0 -> e_a -> e_a + e_b -> 7 (a, b, c a permutation of the axes),
// each listed with positive orientation det(v1 - v0, v2 - v0, v3 - v0) > 0.
__constant__ int c_tet[6][4] = {{0, 1, 3, 7}, {0, 1, 7, 5}, {0, 2, 7, 3}, {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 7, 6}};
// Even permutations of (0 1 2 3) that put corner i first ...
__constant__ int c_first[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 3, 0, 1}, {3, 2, 1, 0}};
// ... and that put a pair of corners first, indexed by the pair's 4-bit mask
// (for a positive tetrahedron (a, b, c, d) with a, b inside, the triangles
// (ac, ad, bd) and (ac, bd, bc) face c and d).
__constant__ int c_pair[16][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 1, 2, 3},   // 0b0011: {0,1}
                                  {0, 0, 0, 0}, {0, 2, 3, 1}, {1, 2, 0, 3}, {0, 0, 0, 0},   // {0,2}, {1,2}
                                  {0, 0, 0, 0}, {0, 3, 1, 2}, {1, 3, 2, 0}, {0, 0, 0, 0},   // {0,3}, {1,3}
                                  {2, 3, 0, 1}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};  // {2,3}

struct IsoArgs {
    const float *f;
    int gx, gy, gz;          // nodes per axis
    float lo[3], step[3];
    float iso;
    // band test (band2 > 0): binned data points and their cell table
    float band2;
    const float4 *pos;
    const int32_t *cstart, *cend;
    float blo[3];
    float inv;
    int levels, cdim;
};

__device__ __forceinline__ int band_cell(float x, float lo, const IsoArgs &a) {
    float f = floorf((x - lo) * a.inv);
    f = fminf(fmaxf(f, 0.f), (float)((a.cdim << a.levels) - 1));
    return ((int)f) >> a.levels;
}

// Some data point within the band of (x, y, z)?  Cells have edge >= band, so the
// points within it lie in the 27 cells around the point's (clamped) cell.
__device__ bool in_band(const IsoArgs &a, float x, float y, float z) {
    const int cx = band_cell(x, a.blo[0], a), cy = band_cell(y, a.blo[1], a), cz = band_cell(z, a.blo[2], a);
    for (int dz = -1; dz <= 1; ++dz) {
        const int zz = cz + dz;
        if (zz < 0 || zz >= a.cdim) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = cy + dy;
            if (yy < 0 || yy >= a.cdim) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int xx = cx + dx;
                if (xx < 0 || xx >= a.cdim) continue;
                const uint32_t code = part1by2_u32(xx) | (part1by2_u32(yy) << 1) | (part1by2_u32(zz) << 2);
                for (int j = a.cstart[code]; j < a.cend[code]; ++j) {
                    const float4 q = a.pos[j];
                    const float ex = x - q.x, ey = y - q.y, ez = z - q.z;
                    if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= a.band2) return true;
                }
            }
        }
    }
    return false;
}

__device__ __forceinline__ void cell_of(const IsoArgs &a, int64_t c, int &kx, int &ky, int &kz) {
    const int64_t cx = a.gx - 1, cy = a.gy - 1;
    kx = (int)(c % cx);
    ky = (int)((c / cx) % cy);
    kz = (int)(c / (cx * cy));
}

// Corner values of a cell; false when a corner is NaN.
__device__ __forceinline__ bool corners(const IsoArgs &a, int kx, int ky, int kz, float (&v)[8]) {
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int64_t i = ((int64_t)(kz + (c >> 2)) * a.gy + (ky + ((c >> 1) & 1))) * a.gx + (kx + (c & 1));
        v[c] = a.f[i];
        ok &= !isnan(v[c]);
    }
    return ok;
}

__device__ __forceinline__ int cell_count(const IsoArgs &a, const float (&v)[8]) {
    unsigned in = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) in |= (v[c] < a.iso ? 1u : 0u) << c;
    if (in == 0u || in == 0xffu) return 0;
    int n = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        int k = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) k += (in >> c_tet[t][i]) & 1u;
        n += (k == 1 || k == 3) ? 1 : (k == 2 ? 2 : 0);
    }
    return n;
}

__global__ void __launch_bounds__(kThr) k_iso_count(IsoArgs a, int64_t ncell, int32_t *__restrict__ cnt) {
    const int64_t c = (int64_t)blockIdx.x * kThr + threadIdx.x;
    if (c >= ncell) return;
    int kx, ky, kz;
    cell_of(a, c, kx, ky, kz);
    float v[8];
    int n = corners(a, kx, ky, kz, v) ? cell_count(a, v) : 0;
    if (n > 0 && a.band2 > 0.f &&
        !in_band(a, fmaf((float)kx + 0.5f, a.step[0], a.lo[0]), fmaf((float)ky + 0.5f, a.step[1], a.lo[1]),
                 fmaf((float)kz + 0.5f, a.step[2], a.lo[2])))
        n = 0;
    cnt[c] = n;
}

__global__ void __launch_bounds__(kThr) k_iso_emit(IsoArgs a, int64_t ncell, const int32_t *__restrict__ off,
                                                   float *__restrict__ tri) {
    const int64_t c = (int64_t)blockIdx.x * kThr + threadIdx.x;
    if (c >= ncell) return;
    int64_t o = off[c];
    if (off[c + 1] == o) return;
    int kx, ky, kz;
    cell_of(a, c, kx, ky, kz);
    float v[8];
    corners(a, kx, ky, kz, v);
    auto node = [&](int corner, int d) {
        const int k = d == 0 ? kx + (corner & 1) : (d == 1 ? ky + ((corner >> 1) & 1) : kz + (corner >> 2));
        return fmaf((float)k, a.step[d], a.lo[d]);
    };
    auto cut = [&](int p, int q, float *out) {
        const int lo = min(p, q), hi = max(p, q);
        const float s = (a.iso - v[lo]) / (v[hi] - v[lo]);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float pl = node(lo, d), ph = node(hi, d);
            out[d] = fmaf(s, ph - pl, pl);
        }
    };
    for (int t = 0; t < 6; ++t) {
        const int *T = c_tet[t];
        unsigned m = 0;
        for (int i = 0; i < 4; ++i) m |= (v[T[i]] < a.iso ? 1u : 0u) << i;
        const int k = __popc(m);
        if (k == 0 || k == 4) continue;
        float *w = tri + o * 9;
        if (k == 1 || k == 3) {
            const unsigned lone_mask = k == 1 ? m : (~m & 15u);
            const int *P = c_first[__ffs(lone_mask) - 1];
            cut(T[P[0]], T[P[1]], w);
            if (k == 1) {
                cut(T[P[0]], T[P[2]], w + 3);
                cut(T[P[0]], T[P[3]], w + 6);
            } else {   // the lone corner is outside: reverse the order
                cut(T[P[0]], T[P[3]], w + 3);
                cut(T[P[0]], T[P[2]], w + 6);
            }
            o += 1;
        } else {
            const int *P = c_pair[m];
            const int A = T[P[0]], B = T[P[1]], Cc = T[P[2]], D = T[P[3]];
            cut(A, Cc, w);          // triangle (ac, ad, bd)
            cut(A, D, w + 3);
            cut(B, D, w + 6);
            cut(A, Cc, w + 9);      // triangle (ac, bd, bc)
            cut(B, D, w + 12);
            cut(B, Cc, w + 15);
            o += 2;
        }
    }
}

}  // namespace

int64_t isosurface(rbf_ctx *ctx, const float *f, const rbf_grid &g, float iso, const float4 *pts, int64_t npts,
                   float band, float *tri, int64_t capacity, cudaStream_t s) {
    int64_t nodes = 1;
    for (int d = 0; d < 3; ++d) {
        RBF_CHECK(g.dims[d] >= 2 && g.dims[d] < (1LL << 24), RBF_ERR_INVALID, "isosurface needs dims[%d] >= 2", d);
        RBF_CHECK(std::isfinite(g.lo[d]) && std::isfinite(g.hi[d]), RBF_ERR_INVALID, "non-finite grid bounds");
        nodes *= g.dims[d];
    }
    RBF_CHECK(nodes < (1LL << 31), RBF_ERR_INVALID, "grid has %lld nodes (limit 2^31)", (long long)nodes);
    RBF_CHECK(std::isfinite(iso), RBF_ERR_INVALID, "iso level must be finite");
    IsoArgs a;
    a.f = f;
    a.gx = (int)g.dims[0];
    a.gy = (int)g.dims[1];
    a.gz = (int)g.dims[2];
    for (int d = 0; d < 3; ++d) {
        a.lo[d] = g.lo[d];
        a.step[d] = (float)(((double)g.hi[d] - (double)g.lo[d]) / (double)(g.dims[d] - 1));
    }
    a.iso = iso;
    a.band2 = 0.f;
    RBF_CHECK(std::isfinite(band) && band >= 0.f, RBF_ERR_INVALID, "band must be finite and >= 0");
    RBF_CHECK(band == 0.f || (pts && npts > 0), RBF_ERR_INVALID, "a band needs data points");
    rbf_plan P;   // binning of the data points when a band is given
    if (band > 0.f) {
        float blo[3], bhi[3];
        RBF_CHECK(bbox_host((const float *)pts, npts, 4, blo, bhi, s), RBF_ERR_INVALID, "non-finite data point");
        double ext = 0.0;
        for (int d = 0; d < 3; ++d) ext = std::max(ext, (double)bhi[d] - (double)blo[d]);
        P.ctx = ctx;
        P.n = npts;
        P.cells_per_cutoff = 1;
        P.levels = 3;
        P.k = 1.f;
        P.sigma = (float)std::max({(double)band, 8.0 * ext / 1020.0, 1e-30});
        plan_build(&P, pts, s, true);
        a.band2 = band * band;
        a.pos = P.pos.p;
        a.cstart = P.cell_start.p;
        a.cend = P.cell_end.p;
        for (int d = 0; d < 3; ++d) a.blo[d] = P.lo[d];
        a.inv = P.inv;
        a.levels = P.levels;
        a.cdim = P.cdim;
    }
    const int64_t ncell = (int64_t)(a.gx - 1) * (a.gy - 1) * (a.gz - 1);
    DevBuf<int32_t> cnt, off;
    cnt.alloc(ncell, s);
    off.alloc(ncell + 1, s);
    k_iso_count<<<(unsigned)ceil_div(ncell, kThr), kThr, 0, s>>>(a, ncell, cnt.p);
    RBF_LAUNCHED();
    scan_exclusive_i32(cnt.p, off.p, ncell, s);
    int32_t total = 0;
    RBF_CUDA(cudaMemcpyAsync(&total, off.p + ncell, sizeof(total), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    RBF_CHECK(total >= 0, RBF_ERR_UNSUPPORTED, "more than 2^31 triangles");
    if (tri && total > 0 && capacity >= total) {
        k_iso_emit<<<(unsigned)ceil_div(ncell, kThr), kThr, 0, s>>>(a, ncell, off.p, tri);
        RBF_LAUNCHED();
        RBF_CUDA(cudaStreamSynchronize(s));
    }
    return total;
}
