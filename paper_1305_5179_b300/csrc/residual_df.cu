// True residual r = b - A~ x with float64-class accuracy on the float32 pipes.
//
// B300's FP64 units run at a small fraction of its FP32 rate, so the residual
// product (one per restart of the refinement loop) is evaluated in
// double-float arithmetic: every quantity is an unevaluated sum hi + lo of two
// float32, combined with the error-free transformations TwoSum (Knuth),
// Fast2Sum (Dekker; where the larger operand is known) and TwoProd (via FMA).
// Per pair:
//   d = p - q exactly (TwoSum per axis; p, q are float32),
//   r2 = |d|^2 to ~2^-46 relative (left unnormalised),
//   cut-off  r2 < (k sigma)^2 against a double-float constant,
//   t = r2 log2(e)/(2 sigma^2),
//   2^-t by the table-driven method of P. T. P. Tang (ACM TOMS 15(2), 1989):
//     t = e + j/1024 + f with |f| <= 1/2048, 2^-t = 2^-e 2^(-j/1024) exp(-f ln 2),
//     2^(-j/1024) from a 1024-entry double-float table built on the host,
//     exp(-g) - 1, |g| <= ln2/2048 + t 2^-23, as -g (double-float) plus
//     g^2/2 - g^3/6 in float32 of the rounded g (the dropped g^4/24 is below 1e-15;
//     the float32 rounding of g^2/2 below 4e-15),
//   product with x_j (double-float split of the float64 weight) and
//   accumulation of each block's <= 32 terms in double-float, added to a float64
//   accumulator once per block.
// Per-term relative error is of order 1e-14.  Pairs beyond the cut-off get a zero
// scale 2^-e, so their terms are exactly zero; every intermediate stays finite for
// t below 1e20.
#include <cmath>
#include <vector>

#include "batch.cuh"

namespace {

constexpr int kT = kChunk;   // one thread per target
constexpr int kTabBits = 10;
constexpr int kTab = 1 << kTabBits;

struct df {
    float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// The same sum and error as two_sum when |a| >= |b| (Dekker's Fast2Sum).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// two_sum of two non-negative numbers, ordered first (the sum is the same either way).
__device__ __forceinline__ df two_sum_pos(float a, float b) { return fast_two_sum(fmaxf(a, b), fminf(a, b)); }

__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

struct DfConst {
    float Ch, Cl;     // log2(e) / (2 sigma^2)
    float Rh, Rl;     // (k sigma)^2, or Rh = +inf when untruncated
    float Lh, Ll;     // ln 2
};

__device__ float2 d_tab[kTab];   // 2^(-j/1024) as (hi, lo)

// copies the table into shared memory; the caller synchronises the CTA afterwards
__device__ __forceinline__ void load_table(float2 *s_tab) {
    for (int j = threadIdx.x; j < kTab; j += blockDim.x) s_tab[j] = d_tab[j];
}

// sum over one staged block of w_j 2^(-t_ij) for the target (px, py, pz); called by
// every lane of a warp with the same cnt
__device__ __forceinline__ df block_terms(float px, float py, float pz, const float4 *__restrict__ sp,
                                          const float2 *__restrict__ sw, int cnt, const DfConst &k,
                                          const float2 *__restrict__ tab) {
    const float Lh = k.Lh, Ll = k.Ll;
    df acc = {0.f, 0.f};
    for (int j = 0; j < cnt; ++j) {
        const float4 q = sp[j];
        const float2 w = sw[j];
        const df dx = two_sum(px, -q.x), dy = two_sum(py, -q.y), dz = two_sum(pz, -q.z);
        // |d|^2 = sum dh^2 (exact products) + 2 sum dh dl (dl^2 < 2^-48 dh^2 is dropped)
        const df sx = two_prod(dx.h, dx.h), sy = two_prod(dy.h, dy.h), sz = two_prod(dz.h, dz.h);
        const float cr = __fmaf_rn(dx.h, dx.l, __fmaf_rn(dy.h, dy.l, __fmul_rn(dz.h, dz.l)));
        const df s = two_sum_pos(sx.h, sy.h);
        df r2 = two_sum_pos(s.h, sz.h);
        r2.l = __fadd_rn(__fadd_rn(r2.l, __fadd_rn(s.l, __fadd_rn(sx.l, sy.l))), __fmaf_rn(2.f, cr, sz.l));
        // r2 < R: (r2.h - Rh) is exact near the radius (Sterbenz) and decides the sign elsewhere
        const bool in = __fadd_rn(__fsub_rn(r2.h, k.Rh), __fsub_rn(r2.l, k.Rl)) < 0.f;
        // a source beyond the cut-off for every target of the warp adds nothing: skip its
        // exponential (the loop runs over the same sources on every lane, so the vote is uniform)
        if (!__any_sync(0xffffffffu, in)) continue;
        // t = r2 * C
        df t = two_prod(r2.h, k.Ch);
        t.l = __fadd_rn(t.l, __fmaf_rn(r2.h, k.Cl, __fmul_rn(r2.l, k.Ch)));
        // m = round(1024 t) by the 1.5 x 2^23 shift (exact below 2^22; t is clamped far above
        // where 2^-t underflows), then t = m / 1024 + fh exactly
        const float th = fminf(t.h, 2048.f);
        const float y = __fmaf_rn(th, (float)kTab, 12582912.f);
        const float mf = __fsub_rn(y, 12582912.f);
        const int m = __float_as_int(y) - 0x4B400000;
        const float fh = __fmaf_rn(mf, -1.f / kTab, th);
        // g = (fh + t.l) ln 2
        df g = two_prod(fh, Lh);
        g.l = __fadd_rn(g.l, __fmaf_rn(fh, Ll, __fmul_rn(t.l, Lh)));
        // exp(-g) - 1 = -g + g^2/2 - g^3/6 + ...; g.l holds t.l ln 2 and is not below ulp(g.h),
        // so the float32 terms take the rounded sum gs = g.h + g.l
        const float gs = __fadd_rn(g.h, g.l);
        const float g2 = __fmul_rn(gs, gs);
        const float rest = __fmul_rn(g2, __fmaf_rn(gs, -1.f / 6.f, 0.5f));
        df D = fast_two_sum(-g.h, rest);          // |g| >= g^2 / 2
        D.l = __fsub_rn(D.l, g.l);
        // E = T_j (1 + D)
        const float2 T = tab[m & (kTab - 1)];
        const df p = two_prod(T.x, D.h);
        df E = fast_two_sum(T.x, p.h);            // T in [1/2, 1], |p| < 3e-4
        E.l = __fadd_rn(E.l, __fadd_rn(p.l, __fmaf_rn(T.x, D.l, __fmaf_rn(T.y, D.h, T.y))));
        // 2^-e (zero from e = 127 on, and for a pair beyond the cut-off)
        const int e = min(m >> kTabBits, 127);
        const float sc = in ? __int_as_float((127 - e) << 23) : 0.f;
        E.h = __fmul_rn(E.h, sc);
        E.l = __fmul_rn(E.l, sc);
        // term = E * w, accumulated in double-float
        df P = two_prod(E.h, w.x);
        P.l = __fadd_rn(P.l, __fmaf_rn(E.h, w.y, __fmul_rn(E.l, w.x)));
        const df a2 = two_sum(acc.h, P.h);
        acc.h = a2.h;
        acc.l = __fadd_rn(acc.l, __fadd_rn(a2.l, P.l));
    }
    return acc;
}

// One segment of one problem: acc over the segment's blocks for target thread.  Warp
// w holds the tile's targets 32w .. 32w + 31 and walks the segment on its own: it
// skips a block whose pair-list code for that quarter says no pair is within the
// cut-off (those terms are zero) and stages the others in its own slice of shared
// memory (one source per lane), so warps never wait for each other.  s_p and s_w
// hold 32 entries per warp of the CTA.
__device__ __forceinline__ double resid_segment(const float4 *__restrict__ pos, const int2 tl, const double *__restrict__ x,
                                                const int2 *__restrict__ blk, const int32_t *__restrict__ ent,
                                                const int2 *__restrict__ ebi, const int4 sg, const DfConst &kc,
                                                float4 *s_p, float2 *s_w, const float2 *s_tab, bool &valid,
                                                int64_t &i) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter_shift = 8 + 2 * warp;
    float4 *wp = s_p + 32 * warp;
    float2 *ww = s_w + 32 * warp;
    i = (int64_t)tl.x + threadIdx.x;
    valid = (int)threadIdx.x < tl.y;
    float4 p = valid ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    double acc = 0.0;
    for (int e = sg.y; e < sg.z; ++e) {
        if (ebi && ((ebi[e].y >> quarter_shift) & 3) == 0) continue;
        const int2 bi = blk[ent[e] & 0x7fffffff];
        __syncwarp();
        if (lane < bi.y) {
            wp[lane] = pos[bi.x + lane];
            const double xv = x[bi.x + lane];
            const float xh = (float)xv;
            ww[lane] = make_float2(xh, (float)(xv - (double)xh));
        }
        __syncwarp();
        df a = block_terms(p.x, p.y, p.z, wp, ww, bi.y, kc, s_tab);
        acc += (double)a.h + (double)a.l;
    }
    return acc;
}

__global__ void __launch_bounds__(kT) k_resid_df(const float4 *__restrict__ pos, const int2 *__restrict__ tiles,
                                                 const double *__restrict__ x,
                                                 const int2 *__restrict__ blk, const int32_t *__restrict__ ent,
                                                 const int2 *__restrict__ ebi, const int4 *__restrict__ seg,
                                                 int64_t n, DfConst kc,
                                                 const float *__restrict__ b, double *__restrict__ out,
                                                 double *__restrict__ part) {
    __shared__ float4 s_p[kT];
    __shared__ float2 s_w[kT];
    __shared__ float2 s_tab[kTab];
    load_table(s_tab);
    __syncthreads();
    const int4 sg = seg[blockIdx.x];
    bool valid;
    int64_t i;
    double acc = resid_segment(pos, tiles[sg.x], x, blk, ent, ebi, sg, kc, s_p, s_w, s_tab, valid, i);
    if (sg.w) {
        if (valid) out[i] = (double)b[i] - acc;
    } else {
        part[(int64_t)blockIdx.x * kChunk + threadIdx.x] = acc;
    }
}

__global__ void k_reduce_resid_df(const int32_t *__restrict__ tile_seg, const int2 *__restrict__ tiles,
                                  const double *__restrict__ part, const float *__restrict__ b,
                                  double *__restrict__ out) {
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

// batched: one CTA per (problem, segment)
__global__ void __launch_bounds__(kT) k_resid_df_batched(const PlanView *__restrict__ views,
                                                         const int2 *__restrict__ items, float Lh, float Ll,
                                                         const float *__restrict__ bs, const double *__restrict__ xs,
                                                         double *__restrict__ rs, double *__restrict__ pool,
                                                         const int64_t *__restrict__ poff) {
    __shared__ float4 s_p[kT];
    __shared__ float2 s_w[kT];
    __shared__ float2 s_tab[kTab];
    load_table(s_tab);
    __syncthreads();
    const int2 it = items[blockIdx.x];
    const PlanView &v = views[it.x];
    const int4 sg = v.seg[it.y];
    DfConst kc;
    kc.Ch = v.Ch;
    kc.Cl = v.Cl;
    kc.Rh = v.Rh;
    kc.Rl = v.Rl;
    kc.Lh = Lh;
    kc.Ll = Ll;
    bool valid;
    int64_t i;
    double acc = resid_segment(v.pos, v.tiles[sg.x], xs + v.off, v.blk, v.ent, v.ebi, sg, kc, s_p, s_w, s_tab, valid,
                               i);
    if (sg.w) {
        if (valid) rs[v.off + i] = (double)bs[v.off + i] - acc;
    } else {
        pool[poff[it.x] + (int64_t)it.y * kChunk + threadIdx.x] = acc;
    }
}

__global__ void k_reduce_resid_df_batched(const PlanView *__restrict__ views, const int2 *__restrict__ splits,
                                          const double *__restrict__ pool, const int64_t *__restrict__ poff,
                                          const float *__restrict__ bs, double *__restrict__ rs) {
    const int2 it = splits[blockIdx.x];
    const PlanView &v = views[it.x];
    int s0 = v.tile_seg[it.y], s1 = v.tile_seg[it.y + 1];
    const int2 tl = v.tiles[it.y];
    for (int q = threadIdx.x; q < tl.y; q += blockDim.x) {
        double acc = 0.0;
        for (int sidx = s0; sidx < s1; ++sidx) acc += pool[poff[it.x] + (int64_t)sidx * kChunk + q];
        int64_t i = v.off + tl.x + q;
        rs[i] = (double)bs[i] - acc;
    }
}

inline void split(double v, float &h, float &l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

bool g_tab_ready[64] = {false};

void upload_table(int device, cudaStream_t s) {
    if (device >= 0 && device < 64 && g_tab_ready[device]) return;
    std::vector<float2> tab(kTab);
    for (int j = 0; j < kTab; ++j) split(std::exp2(-j / (double)kTab), tab[j].x, tab[j].y);
    RBF_CUDA(cudaMemcpyToSymbolAsync(d_tab, tab.data(), kTab * sizeof(float2), 0, cudaMemcpyHostToDevice, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    if (device >= 0 && device < 64) g_tab_ready[device] = true;
}

}  // namespace

void residual_df_prepare(int device, cudaStream_t s) { upload_table(device, s); }

void residual_df_batched(const PlanView *views, const int2 *items, int64_t nitems, const int2 *splits,
                         int64_t nsplits, const float *bs, const double *xs, double *rs, double *part_pool,
                         const int64_t *part_off, int device, cudaStream_t s) {
    upload_table(device, s);
    float Lh, Ll;
    split(0.6931471805599453, Lh, Ll);
    if (nitems > 0) {
        k_resid_df_batched<<<(unsigned)nitems, kT, 0, s>>>(views, items, Lh, Ll, bs, xs, rs, part_pool, part_off);
        RBF_LAUNCHED();
    }
    if (nsplits > 0) {
        k_reduce_resid_df_batched<<<(unsigned)nsplits, kChunk, 0, s>>>(views, splits, part_pool, part_off, bs, rs);
        RBF_LAUNCHED();
    }
}

void residual_binned_df(rbf_plan *P, const float *bs, const double *xs, double *rs, cudaStream_t s) {
    upload_table(P->ctx->device, s);
    const PairList &pl = P->pl;
    DfConst kc;
    split(1.4426950408889634 * P->inv2s2_64, kc.Ch, kc.Cl);
    split(0.6931471805599453, kc.Lh, kc.Ll);
    if (P->rc2_64 > 0.0) {
        split(P->rc2_64, kc.Rh, kc.Rl);
    } else {
        kc.Rh = INFINITY;
        kc.Rl = 0.f;
    }
    DevBuf<double> part;
    if (pl.any_split) part.alloc((size_t)pl.nseg * kChunk, s);
    if (pl.nseg > 0) {
        k_resid_df<<<(unsigned)pl.nseg, kT, 0, s>>>(P->pos.p, P->tiles.p, xs, P->blk.p, pl.ent.p, pl.ebi.p, pl.seg.p,
                                                    P->n, kc, bs, rs, part.p);
        RBF_LAUNCHED();
    }
    if (pl.any_split) {
        k_reduce_resid_df<<<(unsigned)pl.ntiles, kChunk, 0, s>>>(pl.tile_seg.p, P->tiles.p, part.p, bs, rs);
        RBF_LAUNCHED();
    }
}
