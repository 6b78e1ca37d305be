// Cell binning and the block / tile structure of the truncated operator.
//
// The paper restricts each row of A to the "truncation area" of the point
// (Algorithm 2; Sec. III.A, the Gaussian makes A of finite bandwidth).  Here:
//   1. centres are sorted by the Morton code of a fine cell grid (hc / 2^levels,
//      hc = k sigma / s), so that every coarse cell (edge hc) is a contiguous
//      run of the sorted order and consecutive centres are close in space;
//   2. every coarse cell is cut into source blocks of <= 32 consecutive centres
//      (one warp stages one block), with an axis-aligned box each;
//   3. targets are grouped into tiles of 256 consecutive centres, with a box;
//   4. the pair list keeps, per tile, the blocks whose box lies within the
//      cut-off of the tile's box, and flags the blocks that are entirely inside
//      the cut-off for every target (no per-pair test needed).
#include <algorithm>
#include <climits>
#include <cmath>

#include "centers.cuh"
#include "plan.cuh"

namespace {

constexpr int kThreads = 256;

__global__ void k_keys(const float4 *__restrict__ C, int64_t n, float lox, float loy, float loz, float inv,
                       uint32_t qmaxv, uint32_t *__restrict__ keys, int32_t *__restrict__ vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 c = C[i];
    // q = floor((c - lo) * inv) in float32, sub then mul (no contraction possible)
    float fx = floorf(__fmul_rn(__fsub_rn(c.x, lox), inv));
    float fy = floorf(__fmul_rn(__fsub_rn(c.y, loy), inv));
    float fz = floorf(__fmul_rn(__fsub_rn(c.z, loz), inv));
    uint32_t qx = (uint32_t)fminf(fmaxf(fx, 0.f), (float)qmaxv);
    uint32_t qy = (uint32_t)fminf(fmaxf(fy, 0.f), (float)qmaxv);
    uint32_t qz = (uint32_t)fminf(fmaxf(fz, 0.f), (float)qmaxv);
    keys[i] = part1by2_u32(qx) | (part1by2_u32(qy) << 1) | (part1by2_u32(qz) << 2);
    vals[i] = (int32_t)i;
}

__global__ void k_cell_ranges(const uint32_t *__restrict__ keys, int64_t n, int shift, int32_t *__restrict__ start,
                              int32_t *__restrict__ end) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c = keys[i] >> shift;
    if (i == 0 || (keys[i - 1] >> shift) != c) start[c] = (int32_t)i;
    if (i == n - 1 || (keys[i + 1] >> shift) != c) end[c] = (int32_t)(i + 1);
}

__global__ void k_gather_pos(const float4 *__restrict__ C, const int32_t *__restrict__ perm, int64_t n,
                             float4 *__restrict__ pos) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 c = C[perm[i]];
    pos[i] = make_float4(c.x, c.y, c.z, 0.f);
}

__global__ void k_cell_nblocks(const int32_t *__restrict__ start, const int32_t *__restrict__ end, int64_t ncells,
                               int32_t *__restrict__ nb) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int m = end[c] - start[c];
    nb[c] = (m + kBlk - 1) / kBlk;
}

__global__ void k_fill_blocks(const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                              const int32_t *__restrict__ cell_blk, int64_t ncells, int2 *__restrict__ blk) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int s = start[c], m = end[c] - s, b0 = cell_blk[c];
    for (int k = 0; k * kBlk < m; ++k) blk[b0 + k] = make_int2(s + k * kBlk, min(kBlk, m - k * kBlk));
}

// One warp per block: box, centre, overflow guard, and the scaled source offsets.
__global__ void k_block_geom(const float4 *__restrict__ pos, const int2 *__restrict__ blk, int64_t nblk, float scl,
                             float4 *__restrict__ bc, float4 *__restrict__ blo, float4 *__restrict__ bhi,
                             float4 *__restrict__ src) {
    int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (b >= nblk) return;
    int2 bi = blk[b];
    bool v = lane < bi.y;
    float4 p = v ? pos[bi.x + lane] : pos[bi.x];
    float mn[3] = {p.x, p.y, p.z}, mx[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    float cx = 0.5f * (mn[0] + mx[0]), cy = 0.5f * (mn[1] + mx[1]), cz = 0.5f * (mn[2] + mx[2]);
    if (lane == 0) {
        float hx = mx[0] - mn[0], hy = mx[1] - mn[1], hz = mx[2] - mn[2];
        // w: overflow guard U = (32 / r)^2, r the block radius in scaled units (see the product kernel)
        float r = 0.5f * sqrtf(hx * hx + hy * hy + hz * hz) * scl;
        bc[b] = make_float4(cx, cy, cz, r > 0.f ? (32.f / r) * (32.f / r) : INFINITY);
        blo[b] = make_float4(mn[0], mn[1], mn[2], 0.f);
        bhi[b] = make_float4(mx[0], mx[1], mx[2], 0.f);
    }
    if (v) {
        float sx = (p.x - cx) * scl, sy = (p.y - cy) * scl, sz = (p.z - cz) * scl;
        src[bi.x + lane] = make_float4(2.f * sx, 2.f * sy, 2.f * sz, -(sx * sx + sy * sy + sz * sz));
    }
}

// One warp per tile of kChunk consecutive binned centres: its box.
__global__ void k_chunk_boxes(const float4 *__restrict__ pos, int64_t n, int64_t nchk, float4 *__restrict__ lo,
                              float4 *__restrict__ hi) {
    int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (t >= nchk) return;
    int64_t base = t * kChunk;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int r = 0; r < kChunk / 32; ++r) {
        int64_t i = base + lane + 32 * r;
        if (i < n) {
            float4 p = pos[i];
            mn[0] = fminf(mn[0], p.x); mn[1] = fminf(mn[1], p.y); mn[2] = fminf(mn[2], p.z);
            mx[0] = fmaxf(mx[0], p.x); mx[1] = fmaxf(mx[1], p.y); mx[2] = fmaxf(mx[2], p.z);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    if (lane == 0) {
        lo[t] = make_float4(mn[0], mn[1], mn[2], 0.f);
        hi[t] = make_float4(mx[0], mx[1], mx[2], 0.f);
    }
}

struct CellGridArgs {
    float lo[3];
    float inv;
    int levels;
    int cdim;
    float rc;        // culling radius
    float keep2;     // keep block iff min box distance^2 < keep2
    float full2;     // no per-pair test iff max box distance^2 < full2 (0: never)
    int dense;       // every listed block is "full"
};

__device__ __forceinline__ int cell_coord(float x, float lo, float inv, int levels, int cdim) {
    float f = floorf((x - lo) * inv);
    f = fminf(fmaxf(f, 0.f), (float)((cdim << levels) - 1));
    return ((int)f) >> levels;
}

// Visits, in a fixed order, every block of every cell overlapping the tile box
// grown by rc, and applies op(lane_has_block, block, keep, full) warp-wide.
template <typename Op>
__device__ __forceinline__ void visit_blocks(const CellGridArgs &g, float4 tlo, float4 thi,
                                             const int32_t *__restrict__ cell_blk, const float4 *__restrict__ blo,
                                             const float4 *__restrict__ bhi, Op op) {
    int lane = threadIdx.x & 31;
    int c0[3], c1[3];
    float tl[3] = {tlo.x, tlo.y, tlo.z}, th[3] = {thi.x, thi.y, thi.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        c0[d] = cell_coord(tl[d] - g.rc, g.lo[d], g.inv, g.levels, g.cdim);
        c1[d] = cell_coord(th[d] + g.rc, g.lo[d], g.inv, g.levels, g.cdim);
    }
    for (int cz = c0[2]; cz <= c1[2]; ++cz)
        for (int cy = c0[1]; cy <= c1[1]; ++cy)
            for (int cx = c0[0]; cx <= c1[0]; ++cx) {
                uint32_t code = part1by2_u32(cx) | (part1by2_u32(cy) << 1) | (part1by2_u32(cz) << 2);
                int b0 = cell_blk[code], b1 = cell_blk[code + 1];
                for (int bb = b0; bb < b1; bb += 32) {
                    int b = bb + lane;
                    bool keep = false, full = false;
                    if (b < b1) {
                        float4 l = blo[b], h = bhi[b];
                        float gx = fmaxf(0.f, fmaxf(l.x - thi.x, tlo.x - h.x));
                        float gy = fmaxf(0.f, fmaxf(l.y - thi.y, tlo.y - h.y));
                        float gz = fmaxf(0.f, fmaxf(l.z - thi.z, tlo.z - h.z));
                        float dmin2 = gx * gx + gy * gy + gz * gz;
                        keep = dmin2 < g.keep2;
                        if (g.dense) {
                            full = true;
                        } else {
                            float mx = fmaxf(h.x - tlo.x, thi.x - l.x);
                            float my = fmaxf(h.y - tlo.y, thi.y - l.y);
                            float mz = fmaxf(h.z - tlo.z, thi.z - l.z);
                            full = (mx * mx + my * my + mz * mz) < g.full2;
                        }
                    }
                    op(keep, b, full);
                }
            }
}

__global__ void k_pl_count(CellGridArgs g, const float4 *__restrict__ tlo, const float4 *__restrict__ thi,
                           int64_t ntiles, const int32_t *__restrict__ cell_blk, const float4 *__restrict__ blo,
                           const float4 *__restrict__ bhi, int32_t *__restrict__ cnt) {
    int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= ntiles) return;
    int total = 0;
    visit_blocks(g, tlo[t], thi[t], cell_blk, blo, bhi, [&](bool keep, int, bool) {
        total += __popc(__ballot_sync(0xffffffffu, keep));
    });
    if ((threadIdx.x & 31) == 0) cnt[t] = total;
}

__global__ void k_pl_fill(CellGridArgs g, const float4 *__restrict__ tlo, const float4 *__restrict__ thi,
                          int64_t ntiles, const int32_t *__restrict__ cell_blk, const float4 *__restrict__ blo,
                          const float4 *__restrict__ bhi, const int32_t *__restrict__ off,
                          int32_t *__restrict__ ent) {
    int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= ntiles) return;
    int lane = threadIdx.x & 31;
    int w = off[t];
    visit_blocks(g, tlo[t], thi[t], cell_blk, blo, bhi, [&](bool keep, int b, bool full) {
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) ent[w + __popc(m & ((1u << lane) - 1u))] = full ? b : (int)((uint32_t)b | 0x80000000u);
        w += __popc(m);
    });
}

__global__ void k_seg_count(const int32_t *__restrict__ off, int64_t ntiles, int seglen, int32_t *__restrict__ ns) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int64_t c = off[t + 1] - off[t];
    ns[t] = c > 0 ? (int32_t)((c - 1) / seglen + 1) : 0;
}

__global__ void k_seg_fill(const int32_t *__restrict__ off, const int32_t *__restrict__ tseg, int64_t ntiles,
                           int seglen, int4 *__restrict__ seg) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int64_t e0 = off[t], e1 = off[t + 1];
    int s0 = tseg[t];
    for (int64_t k = 0; e0 + k * seglen < e1; ++k) {
        int64_t a = e0 + k * seglen, b = a + seglen < e1 ? a + seglen : e1;
        seg[s0 + k] = make_int4((int)t, (int)a, (int)b, 0);
    }
}

template <typename Tin, typename Tout>
__global__ void k_gather(const Tin *__restrict__ in, const int32_t *__restrict__ perm, int64_t n,
                         Tout *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (Tout)in[perm[i]];
}

template <typename T>
__global__ void k_scatter(const T *__restrict__ in, const int32_t *__restrict__ perm, int64_t n, T *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[perm[i]] = in[i];
}

inline unsigned grid_for(int64_t n, int threads = kThreads) { return (unsigned)std::max<int64_t>(1, ceil_div(n, threads)); }

}  // namespace

void permute_to_binned_f32(const rbf_plan *P, const float *in, float *out, cudaStream_t s) {
    k_gather<float, float><<<grid_for(P->n), kThreads, 0, s>>>(in, P->perm.p, P->n, out);
    RBF_LAUNCHED();
}
void permute_to_binned_f64_to_f32(const rbf_plan *P, const double *in, float *out, cudaStream_t s) {
    k_gather<double, float><<<grid_for(P->n), kThreads, 0, s>>>(in, P->perm.p, P->n, out);
    RBF_LAUNCHED();
}
void permute_to_binned_f64(const rbf_plan *P, const double *in, double *out, cudaStream_t s) {
    k_gather<double, double><<<grid_for(P->n), kThreads, 0, s>>>(in, P->perm.p, P->n, out);
    RBF_LAUNCHED();
}
void permute_from_binned_f32(const rbf_plan *P, const float *in, float *out, cudaStream_t s) {
    k_scatter<float><<<grid_for(P->n), kThreads, 0, s>>>(in, P->perm.p, P->n, out);
    RBF_LAUNCHED();
}
void permute_from_binned_f64(const rbf_plan *P, const double *in, double *out, cudaStream_t s) {
    k_scatter<double><<<grid_for(P->n), kThreads, 0, s>>>(in, P->perm.p, P->n, out);
    RBF_LAUNCHED();
}

void build_pairlist(rbf_plan *P, const float4 *tlo, const float4 *thi, int64_t ntiles, PairList &pl,
                    cudaStream_t s) {
    CellGridArgs g;
    for (int d = 0; d < 3; ++d) g.lo[d] = P->lo[d];
    g.inv = P->inv;
    g.levels = P->levels;
    g.cdim = P->cdim;
    g.rc = P->rc * 1.0001f;   // enumerate cells a little wider than the box test
    g.dense = P->k > 0.f ? 0 : 1;
    // conservative box tests: keep when possibly inside, "full" only when surely inside
    g.keep2 = (P->rc * 1.00001f) * (P->rc * 1.00001f);
    g.full2 = g.dense ? 0.f : (P->rc * 0.99999f) * (P->rc * 0.99999f);

    pl.ntiles = ntiles;
    pl.off.alloc(ntiles + 1, s);
    DevBuf<int32_t> cnt;
    cnt.alloc(ntiles, s);
    unsigned wgrid = grid_for(ntiles * 32);
    k_pl_count<<<wgrid, kThreads, 0, s>>>(g, tlo, thi, ntiles, P->cell_blk.p, P->blk_lo.p, P->blk_hi.p, cnt.p);
    RBF_LAUNCHED();
    scan_exclusive_i32(cnt.p, pl.off.p, ntiles, s);
    int32_t len = 0;
    RBF_CUDA(cudaMemcpyAsync(&len, pl.off.p + ntiles, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    RBF_CHECK(len >= 0, RBF_ERR_UNSUPPORTED, "pair list longer than 2^31 entries");
    pl.len = len;
    pl.ent.alloc(std::max<int64_t>(len, 1), s);
    k_pl_fill<<<wgrid, kThreads, 0, s>>>(g, tlo, thi, ntiles, P->cell_blk.p, P->blk_lo.p, P->blk_hi.p, pl.off.p,
                                         pl.ent.p);
    RBF_LAUNCHED();

    // segments: enough independent work items to fill every SM several times
    int64_t want = 8LL * P->ctx->num_sms;
    int seglen = INT_MAX;
    if (ntiles < want && len > 0) seglen = (int)std::max<int64_t>(8, ceil_div(len, want));
    pl.tile_seg.alloc(ntiles + 1, s);
    k_seg_count<<<grid_for(ntiles), kThreads, 0, s>>>(pl.off.p, ntiles, seglen, cnt.p);
    RBF_LAUNCHED();
    scan_exclusive_i32(cnt.p, pl.tile_seg.p, ntiles, s);
    int32_t nseg = 0;
    RBF_CUDA(cudaMemcpyAsync(&nseg, pl.tile_seg.p + ntiles, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    pl.nseg = nseg;
    pl.seg.alloc(std::max<int64_t>(nseg, 1), s);
    k_seg_fill<<<grid_for(ntiles), kThreads, 0, s>>>(pl.off.p, pl.tile_seg.p, ntiles, seglen, pl.seg.p);
    RBF_LAUNCHED();
    pl.direct = seglen == INT_MAX;
}

void plan_build(rbf_plan *P, const float4 *centers, cudaStream_t s) {
    const int64_t n = P->n;
    bool finite = bbox_host((const float *)centers, n, 4, P->lo, P->hi, s);
    RBF_CHECK(finite, RBF_ERR_INVALID, "non-finite centre coordinate");
    float ext[3];
    for (int d = 0; d < 3; ++d) ext[d] = P->hi[d] - P->lo[d];
    double hc;
    if (P->k > 0.f) {
        hc = (double)P->k * (double)P->sigma / (double)P->cells_per_cutoff;
    } else {
        // untruncated: cells of at most 3 sigma keep blocks compact in scaled units, at least
        // max(ext)/128 keeps the fine grid within 1024 cells per axis
        double m = std::max({(double)ext[0], (double)ext[1], (double)ext[2]});
        hc = m > 0 ? std::max(std::min(m / 8.0, 3.0 * (double)P->sigma), m / 128.0) : 1.0;
    }
    P->inv = (float)(std::ldexp(1.0, P->levels) / hc);
    float qmaxf = 0.f;
    for (int d = 0; d < 3; ++d) qmaxf = std::max(qmaxf, std::floor(ext[d] * P->inv));
    RBF_CHECK(qmaxf < 1024.f, RBF_ERR_UNSUPPORTED,
              "domain spans %.0f fine cells per axis (limit 1024): raise sigma, k or lower levels", qmaxf + 1);
    int qmax = (int)qmaxf, bl = 0;
    while ((1 << bl) <= qmax) ++bl;
    P->nbits = std::max(P->levels, bl);
    P->cdim = 1 << (P->nbits - P->levels);
    P->ncells = (int64_t)P->cdim * P->cdim * P->cdim;

    // Gaussian scaling: phi = exp(-r^2/(2 s^2)) = 2^(-(r*scl)^2)
    double scl = std::sqrt(1.4426950408889634 / (2.0 * (double)P->sigma * (double)P->sigma));
    P->scl = (float)scl;
    P->inv2s2_64 = 1.0 / (2.0 * (double)P->sigma * (double)P->sigma);
    if (P->k > 0.f) {
        P->rc = P->k * P->sigma;
        P->rc2_64 = ((double)P->k * (double)P->sigma) * ((double)P->k * (double)P->sigma);
        P->R = (float)((double)P->k * (double)P->k * 1.4426950408889634 / 2.0);
    } else {
        // untruncated: blocks further than 14 sigma contribute < 3e-43 per unit weight, below
        // float32's normal range, and are skipped
        P->rc = 14.f * P->sigma;
        P->rc2_64 = 0.0;
        P->R = INFINITY;
    }

    // 1-2: keys, stable sort, cell table, binned positions
    P->keys.alloc(n, s);
    P->perm.alloc(n, s);
    k_keys<<<grid_for(n), kThreads, 0, s>>>(centers, n, P->lo[0], P->lo[1], P->lo[2], P->inv,
                                            (uint32_t)((1 << P->nbits) - 1), P->keys.p, P->perm.p);
    RBF_LAUNCHED();
    radix_sort_pairs(P->keys.p, P->perm.p, n, 3 * P->nbits, s);
    P->cell_start.alloc(P->ncells, s);
    P->cell_end.alloc(P->ncells, s);
    P->cell_start.zero(s);
    P->cell_end.zero(s);
    k_cell_ranges<<<grid_for(n), kThreads, 0, s>>>(P->keys.p, n, 3 * P->levels, P->cell_start.p, P->cell_end.p);
    RBF_LAUNCHED();
    P->pos.alloc(n, s);
    k_gather_pos<<<grid_for(n), kThreads, 0, s>>>(centers, P->perm.p, n, P->pos.p);
    RBF_LAUNCHED();

    // 3: source blocks per cell
    DevBuf<int32_t> nb;
    nb.alloc(P->ncells, s);
    k_cell_nblocks<<<grid_for(P->ncells), kThreads, 0, s>>>(P->cell_start.p, P->cell_end.p, P->ncells, nb.p);
    RBF_LAUNCHED();
    P->cell_blk.alloc(P->ncells + 1, s);
    scan_exclusive_i32(nb.p, P->cell_blk.p, P->ncells, s);
    int32_t nblk = 0;
    RBF_CUDA(cudaMemcpyAsync(&nblk, P->cell_blk.p + P->ncells, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    P->nblk = nblk;
    P->blk.alloc(nblk, s);
    k_fill_blocks<<<grid_for(P->ncells), kThreads, 0, s>>>(P->cell_start.p, P->cell_end.p, P->cell_blk.p, P->ncells,
                                                          P->blk.p);
    RBF_LAUNCHED();
    P->blk_c.alloc(nblk, s);
    P->blk_lo.alloc(nblk, s);
    P->blk_hi.alloc(nblk, s);
    P->src.alloc(n, s);
    k_block_geom<<<grid_for((int64_t)nblk * 32), kThreads, 0, s>>>(P->pos.p, P->blk.p, nblk, P->scl, P->blk_c.p,
                                                                   P->blk_lo.p, P->blk_hi.p, P->src.p);
    RBF_LAUNCHED();

    // 4: target tiles and the pair list
    P->nchk = ceil_div(n, kChunk);
    P->chk_lo.alloc(P->nchk, s);
    P->chk_hi.alloc(P->nchk, s);
    k_chunk_boxes<<<grid_for(P->nchk * 32), kThreads, 0, s>>>(P->pos.p, n, P->nchk, P->chk_lo.p, P->chk_hi.p);
    RBF_LAUNCHED();
    build_pairlist(P, P->chk_lo.p, P->chk_hi.p, P->nchk, P->pl, s);
}
