// The truncated Gaussian product y_i = sum_{|c_i - c_j| < k sigma} z_j exp(-|c_i - c_j|^2 / (2 sigma^2))
// (Sec. III.A, Eq. matrixEntries): the operation GMRES repeats (the paper's MatShell).
//
// float32 kernel.  One CTA = one segment of a tile's pair list, 4 warps.  Every
// warp holds all 128 targets of the tile (4 per lane) and walks every 4th block
// of the segment; a block's 32 sources are staged in shared memory as
// structure-of-arrays so that one LDS.128 brings four sources' x (two f32x2
// operands).  For a block with centre c_B and scaled source offsets
// s_j = (x_j - c_B) * scl (precomputed as (2 s_j, -|s_j|^2)), and a target with
// d = (x_i - c_B) * scl:
//      |x_i - x_j|^2 scl^2 = |d|^2 - 2 d.s_j + |s_j|^2,
//      phi_ij = 2^(-|d|^2) * 2^(d.(2 s_j) - |s_j|^2)
// so two sources cost 3 FFMA2 + 2 MUFU.EX2 + 1 FFMA2 per target, and the
// per (target, block) factor 2^(-|d|^2) is applied once per block.  Blocks that
// are not entirely inside the cut-off multiply each term by set.gt(arg, thr),
// thr = |d|^2 - R (R = scaled squared cut-off), before adding.
// When 2 |d| r_B (r_B the scaled block radius) could exceed 64 for some target,
// the block takes a shifted form 2^(-|d|^2 + c) * 2^(d.(2 s_j) - |s_j|^2 - c),
// c = 2 |d| r_B, whose inner exponent is never positive (no overflow).
// Sources of the next block are prefetched into registers while the current
// block is computed.  The 4 warps' partial sums are added in a fixed order.
//
// float64 kernel (true residual): one thread per target, all arithmetic in
// double precision, cut-off decided as |x_i - x_j|^2 < (k sigma)^2 in double.
//
// Inverse multiquadric plans (Table I, phi = (1 + r^2 / sigma^2)^(-beta)) have no
// such factorisation: their float32 product is direct, one thread per target,
// phi = 2^(-beta log2(1 + r^2 / sigma^2)) (two MUFU operations per pair), blocks
// staged in shared memory; entries flagged for the cut-off test keep
// r^2 < (k sigma)^2 (float32).
#include <cmath>

#include "plan.cuh"

#include "product.cuh"

namespace {

using namespace rbfk;

template <bool kGrid>
__global__ void __launch_bounds__(kWarps * 32, RBF_MV_MINBLOCKS) k_matvec_f32(MvArgs a) {
    __shared__ Stage s_st[kWarps];
    __shared__ float s_red[kWarps][kChunk];
    product_segment<kGrid>(a, a.seg[blockIdx.x], blockIdx.x, s_st, s_red);
}

// Sum the segments of each split tile in order (single-segment tiles wrote directly).
template <bool kGrid>
__global__ void k_reduce_segments(MvArgs a, const int32_t *__restrict__ tile_seg, const float *__restrict__ part) {
    int64_t t = blockIdx.x;
    int s0 = tile_seg[t], s1 = tile_seg[t + 1];
    if (s1 - s0 < 2) return;
    for (int q = threadIdx.x; q < kChunk; q += blockDim.x) {
        float x, y, z;
        int64_t oi;
        if (!target_xyz<kGrid>(a, t, q, x, y, z, oi)) continue;
        float v = 0.f;
        for (int sidx = s0; sidx < s1; ++sidx) v += part[(int64_t)sidx * kChunk + q];
        a.out[oi] = v;
    }
}

// Inverse multiquadric product (direct).  One CTA of kChunk threads per segment.
template <bool kGrid>
__global__ void __launch_bounds__(kChunk) k_matvec_imq(MvArgs a) {
    __shared__ float4 s_p[kBlk];
    const int4 sg = a.seg[blockIdx.x];
    float px, py, pz;
    int64_t oi;
    const bool valid = target_xyz<kGrid>(a, sg.x, threadIdx.x, px, py, pz, oi);
    float acc = 0.f;
    for (int e = sg.y; e < sg.z; ++e) {
        const int v = a.ent[e];
        const int2 bi = a.blk[v & 0x7fffffff];
        __syncthreads();
        if ((int)threadIdx.x < bi.y) {
            const float4 q = a.pos[bi.x + threadIdx.x];
            s_p[threadIdx.x] = make_float4(q.x, q.y, q.z, a.w[bi.x + threadIdx.x]);
        }
        __syncthreads();
        const float lim = v < 0 ? a.rc2f : INFINITY;
        for (int j = 0; j < bi.y; ++j) {
            const float4 q = s_p[j];
            const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float phi = ex2_approx(-a.imq_beta * __log2f(fmaf(r2, a.imq_ic, 1.f)));
            acc = fmaf(r2 < lim ? q.w : 0.f, phi, acc);
        }
    }
    if (sg.w) {
        if (valid) a.out[oi] = acc;
    } else {
        a.partial[(int64_t)blockIdx.x * kChunk + threadIdx.x] = acc;
    }
}

// ---------------------------------------------------------------- float64
constexpr int kT64 = kChunk;   // one thread per target

__global__ void __launch_bounds__(kT64) k_resid_f64(const float4 *__restrict__ pos, const int2 *__restrict__ tiles,
                                                   const double *__restrict__ x,
                                                   const int2 *__restrict__ blk, const int32_t *__restrict__ ent,
                                                   const int4 *__restrict__ seg, int64_t n, double rc2, double inv2s2,
                                                   int imq, double imq_ic, double imq_beta,
                                                   const float *__restrict__ b, double *__restrict__ out,
                                                   double *__restrict__ part, unsigned long long *__restrict__ cnt) {
    __shared__ double s_x[kBlk], s_y[kBlk], s_z[kBlk], s_w[kBlk];
    __shared__ unsigned long long s_cnt[kT64 / 32];
    const int4 sg = seg[blockIdx.x];
    const int2 tl = tiles[sg.x];
    const int64_t i = (int64_t)tl.x + threadIdx.x;
    const bool valid = (int)threadIdx.x < tl.y;
    double px = 0, py = 0, pz = 0;
    if (valid) {
        float4 p = pos[i];
        px = p.x; py = p.y; pz = p.z;
    }
    double acc = 0.0;
    unsigned long long c = 0;
    for (int e = sg.y; e < sg.z; ++e) {
        int bidx = ent[e] & 0x7fffffff;
        int2 bi = blk[bidx];
        __syncthreads();
        if (threadIdx.x < kBlk) {
            if ((int)threadIdx.x < bi.y) {
                float4 q = pos[bi.x + threadIdx.x];
                s_x[threadIdx.x] = q.x; s_y[threadIdx.x] = q.y; s_z[threadIdx.x] = q.z;
                s_w[threadIdx.x] = x[bi.x + threadIdx.x];
            }
        }
        __syncthreads();
        for (int j = 0; j < bi.y; ++j) {
            double dx = px - s_x[j], dy = py - s_y[j], dz = pz - s_z[j];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (rc2 <= 0.0 || r2 < rc2) {
                acc += s_w[j] * (imq ? pow(1.0 + r2 * imq_ic, -imq_beta) : exp(-r2 * inv2s2));
                ++c;
            }
        }
    }
    if (sg.w) {
        if (valid) out[i] = (double)b[i] - acc;
    } else {
        part[(int64_t)blockIdx.x * kChunk + threadIdx.x] = acc;
    }
    if (cnt) {
        if (!valid) c = 0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int w = 0; w < kT64 / 32; ++w) t += s_cnt[w];
            atomicAdd(cnt, t);
        }
    }
}

__global__ void k_reduce_resid(const int32_t *__restrict__ tile_seg, const int2 *__restrict__ tiles,
                               const double *__restrict__ part, const float *__restrict__ b, double *__restrict__ out) {
    int64_t t = blockIdx.x;
    int s0 = tile_seg[t], s1 = tile_seg[t + 1];
    if (s1 - s0 < 2) return;
    const int2 tl = tiles[t];
    for (int q = threadIdx.x; q < kChunk; q += blockDim.x) {
        int64_t i = (int64_t)tl.x + q;
        if (q >= tl.y) continue;
        double v = 0.0;
        for (int sidx = s0; sidx < s1; ++sidx) v += part[(int64_t)sidx * kChunk + q];
        out[i] = (double)b[i] - v;
    }
}

MvArgs base_args(const rbf_plan *P, const PairList &pl, const float *w, float *out, float *partial) {
    MvArgs a{};
    a.pos = P->pos.p;
    a.tiles = P->tiles.p;
    a.src = P->src.p;
    a.w = w;
    a.blk = P->blk.p;
    a.blk_c = P->blk_c.p;
    a.ent = pl.ent.p;
    a.ebi = pl.ebi.p;
    a.seg = pl.seg.p;
    a.n = P->n;
    a.scl = P->scl;
    a.R = P->R;
    a.imq_ic = (float)(1.0 / ((double)P->sigma * (double)P->sigma));
    a.imq_beta = P->beta;
    a.rc2f = P->rc2_64 > 0.0 ? (float)P->rc2_64 : INFINITY;
    a.out = out;
    a.partial = partial;
    return a;
}

}  // namespace

void matvec_binned(rbf_plan *P, const float *zs, float *ys, cudaStream_t s) {
    if (P->kernel == RBF_KERNEL_GAUSSIAN && P->product == RBF_PRODUCT_TC && P->sym_ready) {
        // symmetric form: every in-range pair evaluated once (see rbf_plan::sym)
        const PairList &sl = P->sym;
        if (sl.any_split) P->partial.ensure((size_t)sl.nseg * kChunk, s);
        MvArgs a = base_args(P, sl, zs, ys, P->partial.p);
        a.colpart = P->colpart.p;
        ctx_check_device_error(P->ctx);
        product_tc_sym_launch(P, a, s);
        if (sl.any_split) {
            k_reduce_segments<false><<<(unsigned)sl.ntiles, kChunk, 0, s>>>(a, sl.tile_seg.p, P->partial.p);
            RBF_LAUNCHED();
        }
        product_tc_sym_gather(P, ys, s);
        return;
    }
    const PairList &pl = P->pl;
    if (pl.any_split) P->partial.ensure((size_t)pl.nseg * kChunk, s);
    MvArgs a = base_args(P, pl, zs, ys, P->partial.p);
    ctx_check_device_error(P->ctx);
    if (P->kernel == RBF_KERNEL_IMQ) {
        if (pl.nseg > 0) {
            k_matvec_imq<false><<<(unsigned)pl.nseg, kChunk, 0, s>>>(a);
            RBF_LAUNCHED();
        }
    } else if (P->product == RBF_PRODUCT_TC) {
        product_tc_launch(P, pl, a, false, s);
    } else if (pl.nseg > 0) {
        k_matvec_f32<false><<<(unsigned)pl.nseg, kWarps * 32, 0, s>>>(a);
        RBF_LAUNCHED();
    }
    if (pl.any_split) {
        k_reduce_segments<false><<<(unsigned)pl.ntiles, kChunk, 0, s>>>(a, pl.tile_seg.p, P->partial.p);
        RBF_LAUNCHED();
    }
}

void residual_binned_f64(rbf_plan *P, const float *bs, const double *xs, double *rs, unsigned long long *cnt,
                         cudaStream_t s) {
    const PairList &pl = P->pl;
    DevBuf<double> part;
    if (pl.any_split) part.alloc((size_t)pl.nseg * kChunk, s);
    if (pl.nseg > 0) {
        const int imq = P->kernel == RBF_KERNEL_IMQ;
        k_resid_f64<<<(unsigned)pl.nseg, kT64, 0, s>>>(P->pos.p, P->tiles.p, xs, P->blk.p, pl.ent.p, pl.seg.p, P->n,
                                                       P->rc2_64, P->inv2s2_64, imq, 2.0 * P->inv2s2_64,
                                                       (double)P->beta, bs, rs, part.p, cnt);
        RBF_LAUNCHED();
    }
    if (pl.any_split) {
        k_reduce_resid<<<(unsigned)pl.ntiles, kChunk, 0, s>>>(pl.tile_seg.p, P->tiles.p, part.p, bs, rs);
        RBF_LAUNCHED();
    }
}

// Grid evaluation shares the float32 product kernel with grid-generated targets.
// Grid fields of the kernel arguments: node placement, bricks and their shape.
static void set_grid_args(MvArgs &a, const rbf_grid &g, const GridCache &gc) {
    for (int d = 0; d < 3; ++d) {
        a.glo[d] = g.lo[d];
        a.gstep[d] = g.dims[d] > 1 ? (float)(((double)g.hi[d] - (double)g.lo[d]) / (double)(g.dims[d] - 1)) : 0.f;
        a.gdim[d] = (int)g.dims[d];
        a.bdim[d] = (int)gc.bricks[d];
        a.blog[d] = gc.blog[d];
        a.qlog[d] = gc.qlog[d];
    }
}

void matvec_grid_launch(rbf_plan *P, const PairList &pl, const float *ws, const rbf_grid &g, const GridCache &gc,
                        float *f, cudaStream_t s) {
    if (pl.any_split) P->partial.ensure((size_t)pl.nseg * kChunk, s);
    MvArgs a = base_args(P, pl, ws, f, P->partial.p);
    set_grid_args(a, g, gc);
    ctx_check_device_error(P->ctx);
    if (P->kernel == RBF_KERNEL_IMQ) {
        if (pl.nseg > 0) {
            k_matvec_imq<true><<<(unsigned)pl.nseg, kChunk, 0, s>>>(a);
            RBF_LAUNCHED();
        }
    } else if (P->product == RBF_PRODUCT_TC) {
        product_tc_launch(P, pl, a, true, s);
    } else if (pl.nseg > 0) {
        k_matvec_f32<true><<<(unsigned)pl.nseg, kWarps * 32, 0, s>>>(a);
        RBF_LAUNCHED();
    }
    if (pl.any_split) {
        k_reduce_segments<true><<<(unsigned)pl.ntiles, kChunk, 0, s>>>(a, pl.tile_seg.p, P->partial.p);
        RBF_LAUNCHED();
    }
}

// ---------------------------------------------------------------- pair count
namespace {

// Pairs with |x_i - x_j| < k sigma.  The test runs in float32 and is repeated in
// float64 only within 1e-5 (relative) of the cut-off, where float32 rounding of
// the squared distance (< 3e-7 relative) could flip it; so the count equals the
// float64 decision.
__global__ void __launch_bounds__(kT64) k_count_pairs(const float4 *__restrict__ pos, const int2 *__restrict__ tiles,
                                                     const int2 *__restrict__ blk,
                                                     const int32_t *__restrict__ ent, const int4 *__restrict__ seg,
                                                     int64_t n, double rc2, unsigned long long *__restrict__ cnt) {
    __shared__ float4 s_p[kBlk];
    __shared__ unsigned long long s_cnt[kT64 / 32];
    const int4 sg = seg[blockIdx.x];
    const int2 tl = tiles[sg.x];
    const int64_t i = (int64_t)tl.x + threadIdx.x;
    const bool valid = (int)threadIdx.x < tl.y;
    float4 p = valid ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float rc2f = (float)rc2, lo = rc2f * (1.f - 1e-5f), hi = rc2f * (1.f + 1e-5f);
    unsigned long long c = 0;
    for (int e = sg.y; e < sg.z; ++e) {
        int2 bi = blk[ent[e] & 0x7fffffff];
        __syncthreads();
        if ((int)threadIdx.x < bi.y) s_p[threadIdx.x] = pos[bi.x + threadIdx.x];
        __syncthreads();
        for (int j = 0; j < bi.y; ++j) {
            float4 q = s_p[j];
            float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            bool in;
            if (r2 < lo) in = true;
            else if (r2 >= hi) in = false;
            else {
                double ex = (double)p.x - (double)q.x, ey = (double)p.y - (double)q.y, ez = (double)p.z - (double)q.z;
                in = ex * ex + ey * ey + ez * ez < rc2;
            }
            c += in ? 1 : 0;
        }
    }
    if (!valid) c = 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kT64 / 32; ++w) t += s_cnt[w];
        atomicAdd(cnt, t);
    }
}

// Grid version: node coordinates as the float32 product kernel forms them.
__global__ void __launch_bounds__(kT64) k_count_grid_pairs(MvArgs a, double rc2, unsigned long long *__restrict__ cnt) {
    __shared__ float4 s_p[kBlk];
    __shared__ unsigned long long s_cnt[kT64 / 32];
    const int4 sg = a.seg[blockIdx.x];
    float px, py, pz;
    int64_t oi;
    const bool valid = target_xyz<true>(a, sg.x, threadIdx.x, px, py, pz, oi);
    const float rc2f = (float)rc2, lo = rc2f * (1.f - 1e-5f), hi = rc2f * (1.f + 1e-5f);
    unsigned long long c = 0;
    for (int e = sg.y; e < sg.z; ++e) {
        int2 bi = a.blk[a.ent[e] & 0x7fffffff];
        __syncthreads();
        if ((int)threadIdx.x < bi.y) s_p[threadIdx.x] = a.pos[bi.x + threadIdx.x];
        __syncthreads();
        for (int j = 0; j < bi.y; ++j) {
            float4 q = s_p[j];
            float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            bool in;
            if (r2 < lo) in = true;
            else if (r2 >= hi) in = false;
            else {
                double ex = (double)px - (double)q.x, ey = (double)py - (double)q.y, ez = (double)pz - (double)q.z;
                in = ex * ex + ey * ey + ez * ez < rc2;
            }
            c += in ? 1 : 0;
        }
    }
    if (!valid) c = 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kT64 / 32; ++w) t += s_cnt[w];
        atomicAdd(cnt, t);
    }
}

}  // namespace

int64_t count_grid_pairs_launch(rbf_plan *P, const PairList &pl, const rbf_grid &g, const GridCache &gc,
                                cudaStream_t s) {
    int64_t nodes = g.dims[0] * g.dims[1] * g.dims[2];
    if (P->k <= 0.f) return nodes * P->n;
    MvArgs a = base_args(P, pl, nullptr, nullptr, nullptr);
    set_grid_args(a, g, gc);
    DevBuf<unsigned long long> c;
    c.alloc(1, s);
    c.zero(s);
    if (pl.nseg > 0) {
        k_count_grid_pairs<<<(unsigned)pl.nseg, kT64, 0, s>>>(a, P->rc2_64, c.p);
        RBF_LAUNCHED();
    }
    unsigned long long h = 0;
    RBF_CUDA(cudaMemcpyAsync(&h, c.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    return (int64_t)h;
}

namespace {
// Pairs the tensor-core product evaluates: per list entry, every quarter of 32 targets
// whose code is not 0 times the block's sources.  One warp per tile.
// tiles == nullptr: every tile has kChunk target slots (grid bricks)
__global__ void k_count_candidates(const int32_t *__restrict__ off, const int2 *__restrict__ ebi,
                                   const int2 *__restrict__ tiles, int64_t ntiles,
                                   unsigned long long *__restrict__ cnt) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    const int nt = tiles ? tiles[t].y : kChunk;
    unsigned long long c = 0;
    for (int e = off[t] + lane; e < off[t + 1]; e += 32) {
        const int w = ebi[e].y;
        for (int q = 0; q < 4; ++q) {
            const int tq = min(32, max(0, nt - 32 * q));
            if ((w >> (8 + 2 * q)) & 3) c += (unsigned long long)tq * (unsigned long long)(w & 0xff);
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0 && c) atomicAdd(cnt, c);
}
}  // namespace

int64_t count_candidates(rbf_plan *P, cudaStream_t s) { return count_candidates_list(P->pl, P->tiles.p, s); }

int64_t count_candidates_list(const PairList &pl, const int2 *tiles, cudaStream_t s) {
    DevBuf<unsigned long long> c;
    c.alloc(1, s);
    c.zero(s);
    if (pl.ntiles > 0 && pl.len > 0) {
        k_count_candidates<<<(unsigned)ceil_div(pl.ntiles * 32, 256), 256, 0, s>>>(pl.off.p, pl.ebi.p, tiles,
                                                                                 pl.ntiles, c.p);
        RBF_LAUNCHED();
    }
    unsigned long long h = 0;
    RBF_CUDA(cudaMemcpyAsync(&h, c.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    return (int64_t)h;
}

int64_t count_pairs(rbf_plan *P, cudaStream_t s) {
    if (P->pairs >= 0) return P->pairs;
    if (P->k <= 0.f) {
        P->pairs = P->n * P->n;
        return P->pairs;
    }
    DevBuf<unsigned long long> c;
    c.alloc(1, s);
    c.zero(s);
    if (P->pl.nseg > 0) {
        k_count_pairs<<<(unsigned)P->pl.nseg, kT64, 0, s>>>(P->pos.p, P->tiles.p, P->blk.p, P->pl.ent.p, P->pl.seg.p, P->n,
                                                           P->rc2_64, c.p);
        RBF_LAUNCHED();
    }
    unsigned long long h = 0;
    RBF_CUDA(cudaMemcpyAsync(&h, c.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    P->pairs = (int64_t)h;
    return P->pairs;
}
