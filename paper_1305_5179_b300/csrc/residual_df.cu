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
// t below 1e20.  For one plan each pair's entry is evaluated once and serves both of
// its rows (the symmetric form below), in a batch within each problem.
#include <algorithm>
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

// Squared distance of a target and a source in double-float, and the cut-off test.
struct PairR2 {
    df r2;
    bool in;
};
__device__ __forceinline__ PairR2 pair_r2(float px, float py, float pz, const float4 q, const DfConst &k) {
    const df dx = two_sum(px, -q.x), dy = two_sum(py, -q.y), dz = two_sum(pz, -q.z);
    // |d|^2 = sum dh^2 (exact products) + 2 sum dh dl (dl^2 < 2^-48 dh^2 is dropped)
    const df sx = two_prod(dx.h, dx.h), sy = two_prod(dy.h, dy.h), sz = two_prod(dz.h, dz.h);
    const float cr = __fmaf_rn(dx.h, dx.l, __fmaf_rn(dy.h, dy.l, __fmul_rn(dz.h, dz.l)));
    const df s = two_sum_pos(sx.h, sy.h);
    df r2 = two_sum_pos(s.h, sz.h);
    r2.l = __fadd_rn(__fadd_rn(r2.l, __fadd_rn(s.l, __fadd_rn(sx.l, sy.l))), __fmaf_rn(2.f, cr, sz.l));
    // r2 < R: (r2.h - Rh) is exact near the radius (Sterbenz) and decides the sign elsewhere
    const bool in = __fadd_rn(__fsub_rn(r2.h, k.Rh), __fsub_rn(r2.l, k.Rl)) < 0.f;
    return {r2, in};
}

// The matrix entry 2^-t, t = r2 C, in double-float; exactly zero beyond the cut-off.
__device__ __forceinline__ df pair_exp(const PairR2 &pr, const DfConst &k, const float2 *__restrict__ tab) {
    const float Lh = k.Lh, Ll = k.Ll;
    const df r2 = pr.r2;
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
    const float sc = pr.in ? __int_as_float((127 - e) << 23) : 0.f;
    E.h = __fmul_rn(E.h, sc);
    E.l = __fmul_rn(E.l, sc);
    return E;
}

// E * w for a double-float weight w = (hi, lo), and acc += it, in double-float
__device__ __forceinline__ df times_w(const df E, const float2 w) {
    df P = two_prod(E.h, w.x);
    P.l = __fadd_rn(P.l, __fmaf_rn(E.h, w.y, __fmul_rn(E.l, w.x)));
    return P;
}
__device__ __forceinline__ void add_to(df &acc, const df P) {
    const df a2 = two_sum(acc.h, P.h);
    acc.h = a2.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(a2.l, P.l));
}

// ---------------------------------------------------------------- symmetric form
// A~ is symmetric, so one evaluation of a pair's entry serves both rows.  A pair (i, j),
// i in the CTA's tile T and j in a block of its list, is taken from this side when j's
// tile comes after T (both rows) or is T itself (this row only: the tile meets its own
// blocks from both sides), and skipped when j's tile comes before T (the other side
// takes it).  Every pair within the cut-off appears in both tiles' lists, so each is
// counted once per row.  Row j's share, sum_i a_ij x_i over this warp's 32 targets, is
// summed per source in double-float and added to a 128-bit fixed-point accumulator
// (units of 2^-80) with integer atomics: integer addition is exact, so the result does
// not depend on the order the CTAs run in.  Range: the signed 128-bit accumulator holds
// magnitudes below 2^47, and a row receives at most one share per (tile, warp), i.e.
// at most 4 ntiles shares.  Every share is therefore checked against
// lim = min(2^44, 2^46 / (4 ntiles)): a larger share raises kErrRange in the context's
// error word (the call reports RBF_ERR_RANGE) instead of wrapping silently.  Entries are
// at most 1, so lim bounds 32 x max |x_i| from above.  The truncation below 2^-80 costs
// at most 2^-80 per share.
constexpr int kFix = 80;

float fix_share_limit(int64_t ntiles) {
    const double lim = std::ldexp(1.0, 46) / (4.0 * (double)(ntiles > 0 ? ntiles : 1));
    return (float)std::min(lim, std::ldexp(1.0, 44));
}

// v 2^kFix as a signed 128-bit integer, truncated toward zero below 2^-kFix; shares of
// 2^44 and above saturate (see the range above)
__device__ __forceinline__ __int128 to_fix(float v) {
    const unsigned u = __float_as_uint(v);
    const int ex = (int)((u >> 23) & 0xffu);
    if (ex == 0) return 0;                              // zero, or below 2^-126
    const unsigned long long m = (u & 0x7fffffu) | 0x800000u;
    const int sh = ex - 150 + kFix;                    // v = m 2^(ex - 150)
    unsigned __int128 mag = 0;
    if (sh >= 0) mag = (unsigned __int128)m << (sh < 100 ? sh : 100);
    else if (sh > -24) mag = m >> (-sh);
    return (u >> 31) ? -(__int128)mag : (__int128)mag;
}

__device__ __forceinline__ void atomic_add_fix(unsigned long long *a, __int128 v) {
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
    const unsigned long long old = atomicAdd(a, lo);
    atomicAdd(a + 1, hi + (old + lo < old ? 1ull : 0ull));
}

// one segment: target-side sum returned; source-side sums added to fix_acc (2 words per
// centre, binned order).  Staging as resid_segment, plus each source's tile; qs is this
// warp's 16 x 33 scratch of per-pair source-side terms (16 sources at a time).
__device__ __forceinline__ double resid_segment_sym(const float4 *__restrict__ pos, const int2 tl, int64_t T,
                                                    const double *__restrict__ x, const int2 *__restrict__ blk,
                                                    const int32_t *__restrict__ ent, const int2 *__restrict__ ebi,
                                                    const int32_t *__restrict__ tile_of, const int4 sg,
                                                    const DfConst &kc, float4 *s_p, float2 *s_w, int *s_tj,
                                                    float2 (*qs)[33], const float2 *s_tab,
                                                    unsigned long long *__restrict__ fix_acc, float fix_lim,
                                                    unsigned *err, bool &valid, int64_t &i) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter_shift = 8 + 2 * warp;
    float4 *wp = s_p + 32 * warp;
    float2 *ww = s_w + 32 * warp;
    int *wt = s_tj + 32 * warp;
    i = (int64_t)tl.x + threadIdx.x;
    valid = (int)threadIdx.x < tl.y;
    const float4 p = valid ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float2 xi = make_float2(0.f, 0.f);                  // this target's weight (zero for an empty slot)
    if (valid) {
        const double xv = x[i];
        xi.x = (float)xv;
        xi.y = (float)(xv - (double)xi.x);
    }
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
            wt[lane] = tile_of[bi.x + lane];
        }
        __syncwarp();
        df a = {0.f, 0.f};
        // the block's sources in two halves of 16, so that the scratch holds 16 columns
        for (int h0 = 0; h0 < bi.y; h0 += 16) {
            const int h1 = min(h0 + 16, bi.y);
            unsigned symmask = 0;
            for (int j = h0; j < h1; ++j) {
                const int tj = wt[j];
                if (tj < T) continue;                   // the other tile takes this pair
                const float4 q = wp[j];
                const float2 w = ww[j];
                const PairR2 pr = pair_r2(p.x, p.y, p.z, q, kc);
                if (!__any_sync(0xffffffffu, pr.in)) continue;
                const df E = pair_exp(pr, kc, s_tab);
                add_to(a, times_w(E, w));
                if (tj > T) {                           // row j's term a_ij x_i
                    const df Q = times_w(E, xi);
                    qs[j - h0][lane] = make_float2(Q.h, Q.l);
                    symmask |= 1u << (j - h0);
                }
            }
            if (symmask) {
                // column c = lane & 15 summed over rows 16 (lane >> 4) .. + 15 by each half of
                // the warp, the halves combined by a shuffle; the first half holds the sums
                __syncwarp();
                const int c = lane & 15, r0 = (lane >> 4) * 16;
                df cs = {0.f, 0.f};
                if ((symmask >> c) & 1u)
                    for (int r = r0; r < r0 + 16; ++r) {
                        const float2 v = qs[c][r];
                        add_to(cs, df{v.x, v.y});
                    }
                const df other = {__shfl_down_sync(0xffffffffu, cs.h, 16), __shfl_down_sync(0xffffffffu, cs.l, 16)};
                if (lane < 16 && ((symmask >> c) & 1u)) {
                    add_to(cs, other);
                    if (fabsf(cs.h) < fix_lim)     // NaN fails too
                        atomic_add_fix(fix_acc + 2 * (bi.x + h0 + c), to_fix(cs.h) + to_fix(cs.l));
                    else if (err)
                        atomicOr(err, kErrRange);
                }
                __syncwarp();
            }
        }
        acc += (double)a.h + (double)a.l;
    }
    return acc;
}

__global__ void __launch_bounds__(kT) k_resid_df_sym(const float4 *__restrict__ pos, const int2 *__restrict__ tiles,
                                                     const double *__restrict__ x, const int2 *__restrict__ blk,
                                                     const int32_t *__restrict__ ent, const int2 *__restrict__ ebi,
                                                     const int4 *__restrict__ seg, const int32_t *__restrict__ tile_of,
                                                     DfConst kc, const float *__restrict__ b, double *__restrict__ out,
                                                     double *__restrict__ part, unsigned long long *__restrict__ fix_acc,
                                                     float fix_lim, unsigned *err) {
    __shared__ float4 s_p[kT];
    __shared__ float2 s_w[kT];
    __shared__ int s_tj[kT];
    __shared__ float2 s_q[kT / 32][16][33];
    __shared__ float2 s_tab[kTab];
    load_table(s_tab);
    __syncthreads();
    const int4 sg = seg[blockIdx.x];
    bool valid;
    int64_t i;
    double acc = resid_segment_sym(pos, tiles[sg.x], sg.x, x, blk, ent, ebi, tile_of, sg, kc, s_p, s_w, s_tj,
                                   s_q[threadIdx.x >> 5], s_tab, fix_acc, fix_lim, err, valid, i);
    if (sg.w) {
        if (valid) out[i] = (double)b[i] - acc;
    } else {
        part[(int64_t)blockIdx.x * kChunk + threadIdx.x] = acc;
    }
}

// batched: one CTA per (problem, segment), the symmetric form within each problem
__global__ void __launch_bounds__(kT) k_resid_df_sym_batched(const PlanView *__restrict__ views,
                                                             const int2 *__restrict__ items, float Lh, float Ll,
                                                             const float *__restrict__ bs, const double *__restrict__ xs,
                                                             double *__restrict__ rs, double *__restrict__ pool,
                                                             const int64_t *__restrict__ poff,
                                                             unsigned long long *__restrict__ fix, float fix_lim,
                                                             unsigned *err) {
    __shared__ float4 s_p[kT];
    __shared__ float2 s_w[kT];
    __shared__ int s_tj[kT];
    __shared__ float2 s_q[kT / 32][16][33];
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
    double acc = resid_segment_sym(v.pos, v.tiles[sg.x], sg.x, xs + v.off, v.blk, v.ent, v.ebi, v.tile_of, sg, kc,
                                   s_p, s_w, s_tj, s_q[threadIdx.x >> 5], s_tab, fix + 2 * v.off, fix_lim, err,
                                   valid, i);
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

// tile_of[i] = the tile holding binned position i
__global__ void k_tile_of(const int2 *__restrict__ tiles, int32_t *__restrict__ tile_of) {
    const int2 tl = tiles[blockIdx.x];
    for (int q = threadIdx.x; q < tl.y; q += blockDim.x) tile_of[tl.x + q] = (int32_t)blockIdx.x;
}

// out[j] -= the source-side sum of row j (fixed point)
__global__ void k_resid_fix_finish(const unsigned long long *__restrict__ fix_acc, int64_t n, double *__restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const unsigned long long lo = fix_acc[2 * j], hi = fix_acc[2 * j + 1];
    const double v = ((double)(long long)hi * 18446744073709551616.0 + (double)lo) * 0x1p-80;
    out[j] -= v;
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
                         const int64_t *part_off, unsigned long long *fix, int64_t ntotal, int64_t max_tiles,
                         unsigned *err, int device, cudaStream_t s) {
    upload_table(device, s);
    float Lh, Ll;
    split(0.6931471805599453, Lh, Ll);
    if (ntotal > 0) RBF_CUDA(cudaMemsetAsync(fix, 0, 2 * (size_t)ntotal * sizeof(unsigned long long), s));
    if (nitems > 0) {
        k_resid_df_sym_batched<<<(unsigned)nitems, kT, 0, s>>>(views, items, Lh, Ll, bs, xs, rs, part_pool, part_off,
                                                               fix, fix_share_limit(max_tiles), err);
        RBF_LAUNCHED();
    }
    if (nsplits > 0) {
        k_reduce_resid_df_batched<<<(unsigned)nsplits, kChunk, 0, s>>>(views, splits, part_pool, part_off, bs, rs);
        RBF_LAUNCHED();
    }
    if (ntotal > 0) {
        k_resid_fix_finish<<<(unsigned)ceil_div(ntotal, (int64_t)256), 256, 0, s>>>(fix, ntotal, rs);
        RBF_LAUNCHED();
    }
}

void tile_of_launch(const int2 *tiles, int64_t ntiles, int32_t *tile_of, cudaStream_t s) {
    if (ntiles <= 0) return;
    k_tile_of<<<(unsigned)ntiles, kChunk, 0, s>>>(tiles, tile_of);
    RBF_LAUNCHED();
}

void residual_binned_df(rbf_plan *P, const float *bs, const double *xs, double *rs, cudaStream_t s) {
    upload_table(P->ctx->device, s);
    // A plan with the symmetric sub-list walks it: it holds exactly the entries this kernel does
    // not skip (block in the same or a later tile), in the same order within each tile.
    const PairList &pl = P->sym_ready ? P->sym : P->pl;
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
    DevBuf<int32_t> tile_of_own;
    DevBuf<unsigned long long> fix;
    fix.alloc(2 * (size_t)P->n, s);
    fix.zero(s);
    const int32_t *tile_of = P->tile_of.p;
    if (!P->sym_ready) {
        tile_of_own.alloc(P->n, s);
        tile_of = tile_of_own.p;
        if (pl.ntiles > 0) {
            k_tile_of<<<(unsigned)pl.ntiles, kChunk, 0, s>>>(P->tiles.p, tile_of_own.p);
            RBF_LAUNCHED();
        }
    }
    if (pl.nseg > 0) {
        k_resid_df_sym<<<(unsigned)pl.nseg, kT, 0, s>>>(P->pos.p, P->tiles.p, xs, P->blk.p, pl.ent.p, pl.ebi.p,
                                                        pl.seg.p, tile_of, kc, bs, rs, part.p, fix.p,
                                                        fix_share_limit(pl.ntiles), ctx_error_word(P->ctx));
        RBF_LAUNCHED();
    }
    if (pl.any_split) {
        k_reduce_resid_df<<<(unsigned)pl.ntiles, kChunk, 0, s>>>(pl.tile_seg.p, P->tiles.p, part.p, bs, rs);
        RBF_LAUNCHED();
    }
    if (P->n > 0) {
        k_resid_fix_finish<<<(unsigned)ceil_div(P->n, (int64_t)256), 256, 0, s>>>(fix.p, P->n, rs);
        RBF_LAUNCHED();
    }
}
