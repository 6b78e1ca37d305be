// Batched solve of many independent problems (one plan each, e.g. many clouds of
// uneven size): flexible GMRES in lockstep over all problems with every step on
// the device, so that a whole solve is one CUDA graph.
//
//  * the product is one launch over all problems, (problem, segment) work items
//    longest first: with the tensor-core product one CTA per item, with the
//    CUDA-core product persistent CTAs that pull items from an atomic counter; so
//    small and large problems share the GPU without a launch per problem;
//  * the Arnoldi dot products and updates are segmented reductions over chunks of
//    <= kRange entries that never cross a problem boundary (float64, fixed order);
//  * the Hessenberg column, Givens rotations, residual estimate and the final
//    triangular solve run on the device, one thread per problem;
//  * the preconditioner is each plan's restricted additive Schwarz data, applied
//    by one warp per (problem, subdomain);
//  * the float64-class true residual uses the batched double-float kernel.
// The captured solve has a fixed number of steps.  With fixed_iterations every problem
// takes all of them (the paper's timing protocol of Table II); otherwise a problem stops
// at the tolerance (its estimate within a cycle, its true residual at a restart) and a
// per-problem flag makes every kernel skip its work from then on.  Every problem reports
// its own true residual and step count.  The subdomain size can be chosen by
// rbf_batch_autotune, which times short solves of the candidate sizes.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "batch.cuh"
#include "schwarz.cuh"
#include "product.cuh"

using rbfk::kWarps;
using rbfk::MvArgs;
using rbfk::Stage;

struct rbf_batch {
    rbf_ctx *ctx = nullptr;
    std::vector<rbf_plan *> plans;
    int64_t max_tiles = 0;          // largest tile count of a problem (the residual's share limit)
    int nb = 0;
    int64_t N = 0;
    std::vector<int64_t> off;
    PBuf<PlanView> views;
    std::vector<PlanView> hviews;
    PBuf<int2> seg_items, split_tiles, sub_items;
    int64_t nseg_items = 0, nsplit = 0, nsub_items = 0;
    PBuf<int4> chunks;            // (problem, global start, length, 0)
    PBuf<int32_t> chunk_off;      // nb + 1
    int64_t nchunks = 0;
    std::vector<PBuf<int4>> bseg;          // per problem: the batch's own segments
    std::vector<PBuf<int32_t>> btile_seg;  // per problem: segments of each tile
    PBuf<float> part_f;                    // product partial sums of split tiles, all problems
    PBuf<double> part_d;
    PBuf<int64_t> part_off_d;
    PBuf<unsigned int> counter;
    PBuf<int32_t> tile_of;                 // per binned position, its problem's tile
    PBuf<unsigned long long> fix;          // residual: fixed-point row accumulators (2 words each)
    int persistent_ctas = 0;
    bool tc = false;              // every plan takes the tensor-core product
    bool sz_valid = false;        // the plans hold a Schwarz set-up made with sz_p
    rbf_schwarz_params sz_p{};
    // solve state
    int m_alloc = 0;
    PBuf<float> bs, Z, w32;
    PBuf<double> V, w64, x, r, red, hA, hB, hN, hs, H, g, cs, sn, y, est, bn2, rn2, dtol;
    PBuf<int> act, kp, itp;       // per problem: still iterating; steps of this cycle; steps in all
    // captured solve, on a private stream ordered after and before the caller's
    cudaStream_t own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int g_m = -1, g_it = -1, g_pc = -1, g_act = -1;
    long long g_kernels = 0;      // kernel nodes of the captured solve
    ~rbf_batch() {
        if (own) cudaStreamSynchronize(own);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (own) cudaStreamDestroy(own);
    }
};

namespace {

constexpr int kThreads = 256;
constexpr int kRange = 8192;

// ------------------------------------------------------------------ product
__global__ void __launch_bounds__(kWarps * 32, RBF_MV_MINBLOCKS)
    k_bmatvec(const PlanView *__restrict__ views, const int2 *__restrict__ items, int nitems,
              unsigned int *__restrict__ counter, const float *__restrict__ z, float *__restrict__ y,
              const int *__restrict__ act) {
    __shared__ Stage s_st[kWarps];
    __shared__ float s_red[kWarps][kChunk];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int2 ci = items[it];
        if (act && !act[ci.x]) continue;   // the problem has met its tolerance
        const PlanView &v = views[ci.x];
        MvArgs a{};
        a.pos = v.pos;
        a.tiles = v.tiles;
        a.src = v.src;
        a.w = z + v.off;
        a.blk = v.blk;
        a.blk_c = v.blk_c;
        a.ent = v.ent;
        a.seg = v.seg;
        a.n = v.n;
        a.scl = v.scl;
        a.R = v.R;
        a.out = y + v.off;
        a.partial = v.partial;
        rbfk::product_segment<false>(a, v.seg[ci.y], ci.y, s_st, s_red);
    }
}

__global__ void k_breduce_split(const PlanView *__restrict__ views, const int2 *__restrict__ splits,
                                float *__restrict__ y, const int *__restrict__ act) {
    const int2 it = splits[blockIdx.x];
    if (act && !act[it.x]) return;
    const PlanView &v = views[it.x];
    const int s0 = v.tile_seg[it.y], s1 = v.tile_seg[it.y + 1];
    const int2 tl = v.tiles[it.y];
    for (int q = threadIdx.x; q < tl.y; q += blockDim.x) {
        float acc = 0.f;
        for (int sidx = s0; sidx < s1; ++sidx) acc += v.partial[(int64_t)sidx * kChunk + q];
        y[v.off + tl.x + q] = acc;
    }
}

// ------------------------------------------------------------------ Schwarz
template <bool kOne>   // kOne: every subdomain has at most 32 centres (one factor tile)
__global__ void __launch_bounds__(256) k_bschwarz_apply(const PlanView *__restrict__ views, const int2 *__restrict__ items,
                                                        int64_t nitems, const double *__restrict__ vin,
                                                        float *__restrict__ z, const int *__restrict__ act) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nitems) return;
    const int2 it = items[w];
    if (!act[it.x]) return;   // a whole warp's item: the warp leaves together
    const PlanView &v = views[it.x];
    const int B = v.B, core = v.core;
    const int64_t n = v.n;
    int64_t s = (int64_t)it.y * core, e = s + core < n ? s + core : n;
    int64_t d0 = s - (B - core) / 2;
    if (d0 > n - B) d0 = n - B;
    if (d0 < 0) d0 = 0;
    const float *L = v.L + (int64_t)it.y * B * B;
    const double *vv = vin + v.off;
    float *zz = z + v.off;
    constexpr int Q = 4;
    float yv[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        int k = lane + 32 * q;
        yv[q] = k < B ? (float)vv[d0 + k] : 0.f;
    }
    if (kOne) ras::solve_block32(L, B, yv[0], lane);
    else ras::solve_block(L, B, yv, lane);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        int k = lane + 32 * q;
        if (k >= B) continue;
        int64_t gi = d0 + k;
        if (v.restricted) {
            if (gi >= s && gi < e) zz[gi] = yv[q];
        } else {
            atomicAdd(&zz[gi], yv[q]);
        }
    }
}

// ------------------------------------------------------------------ segmented vector work
__device__ double cta_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
    return t;
}

// red[k * nchunks + c] = sum over chunk c of V[k][i] w[i]
template <typename Tw>
__global__ void __launch_bounds__(kThreads) k_bmdot(const double *__restrict__ V, int64_t ldv, int nv,
                                                    const Tw *__restrict__ w, const int4 *__restrict__ chunks,
                                                    int64_t nchunks, double *__restrict__ red,
                                                    const int *__restrict__ act) {
    __shared__ double sh[kThreads / 32];
    const int4 c = chunks[blockIdx.x];
    if (act && !act[c.x]) return;   // problem done: its sums are not read
    for (int k = 0; k < nv; ++k) {
        const double *vk = V + k * ldv;
        double s = 0.0;
        for (int i = threadIdx.x; i < c.z; i += kThreads) s += vk[c.y + i] * (double)w[c.y + i];
        double t = cta_sum(s, sh);
        if (threadIdx.x == 0) red[(int64_t)k * nchunks + blockIdx.x] = t;
    }
}

// out[p * stride + k] = sum over problem p's chunks of red[k * nchunks + c]; grid (nb, nv)
__global__ void k_bmdot_final(const double *__restrict__ red, int64_t nchunks, const int32_t *__restrict__ chunk_off,
                              double *__restrict__ out, int stride, const int *__restrict__ act) {
    __shared__ double sh[kThreads / 32];
    const int p = blockIdx.x, k = blockIdx.y;
    if (act && !act[p]) return;
    double s = 0.0;
    for (int c = chunk_off[p] + threadIdx.x; c < chunk_off[p + 1]; c += kThreads) s += red[(int64_t)k * nchunks + c];
    double t = cta_sum(s, sh);
    if (threadIdx.x == 0) out[(int64_t)p * stride + k] = t;
}

// wout = win - V h(problem); red[c] = sum over chunk of wout^2 when red != null
template <typename Tw>
__global__ void __launch_bounds__(kThreads) k_bmaxpy(const double *__restrict__ V, int64_t ldv, int nv,
                                                     const double *__restrict__ h, int stride,
                                                     const Tw *__restrict__ win, double *__restrict__ wout,
                                                     const int4 *__restrict__ chunks, double *__restrict__ red,
                                                     const int *__restrict__ act) {
    __shared__ double sh[kThreads / 32];
    __shared__ double hs[72];
    const int4 c = chunks[blockIdx.x];
    if (!act[c.x]) return;
    for (int k = threadIdx.x; k < nv; k += kThreads) hs[k] = h[(int64_t)c.x * stride + k];
    __syncthreads();
    double sq = 0.0;
    for (int i = threadIdx.x; i < c.z; i += kThreads) {
        const int64_t gi = c.y + i;
        double v = (double)win[gi];
        for (int k = 0; k < nv; ++k) v -= hs[k] * V[k * ldv + gi];
        wout[gi] = v;
        sq += v * v;
    }
    if (red) {
        double t = cta_sum(sq, sh);
        if (threadIdx.x == 0) red[blockIdx.x] = t;
    }
}

// dst = src / scale(problem) (0 where the scale is 0)
__global__ void k_bscale(const double *__restrict__ src, const double *__restrict__ scale,
                         double *__restrict__ dst, const int4 *__restrict__ chunks, const int *__restrict__ act) {
    __shared__ double s_inv;    // one float64 division per CTA
    const int4 c = chunks[blockIdx.x];
    if (!act[c.x]) return;
    if (threadIdx.x == 0) {
        const double sv = scale[c.x];
        s_inv = sv > 0.0 ? 1.0 / sv : 0.0;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int i = threadIdx.x; i < c.z; i += blockDim.x) dst[c.y + i] = src[c.y + i] * inv;
}

__global__ void k_bupdate_x(double *__restrict__ x, const float *__restrict__ Z, int64_t ldz,
                            const int *__restrict__ kp, const double *__restrict__ y, int ystride,
                            const int4 *__restrict__ chunks) {
    __shared__ double ys[72];
    const int4 c = chunks[blockIdx.x];
    const int k = kp[c.x];   // the steps this problem took in the cycle (0: none)
    if (k == 0) return;
    for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[(int64_t)c.x * ystride + j];
    __syncthreads();
    for (int i = threadIdx.x; i < c.z; i += blockDim.x) {
        const int64_t gi = c.y + i;
        double v = x[gi];
        for (int j = 0; j < k; ++j) v += ys[j] * (double)Z[j * ldz + gi];
        x[gi] = v;
    }
}

__global__ void k_bcast(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void k_bto64(const float *__restrict__ a, double *__restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

__global__ void k_bset(double *__restrict__ a, double v) { *a = v; }

__global__ void k_bzero(double *__restrict__ a, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 0.0;
}

// per problem: beta = sqrt(norm^2); restart the Givens state; the problem iterates in this
// cycle unless its residual already meets the tolerance (*tol < 0: every problem iterates)
__global__ void k_bstart(const double *__restrict__ nrm2, double *__restrict__ beta, double *__restrict__ g,
                         double *__restrict__ H, int m, int nb, const double *__restrict__ bn2,
                         const double *__restrict__ tol, int *__restrict__ act, int *__restrict__ kp) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nb) return;
    const double b = sqrt(nrm2[p]);
    beta[p] = b;
    const double t = *tol;
    act[p] = (t < 0.0 || b > t * sqrt(bn2[p])) && b > 0.0 ? 1 : 0;
    kp[p] = 0;
    for (int i = 0; i <= m; ++i) g[(int64_t)p * (m + 1) + i] = 0.0;
    g[(int64_t)p * (m + 1)] = b;
    for (int i = 0; i < (m + 1) * m; ++i) H[(int64_t)p * (m + 1) * m + i] = 0.0;
}

// per problem: column j of H from the two Gram-Schmidt passes, Givens rotations, estimate
__global__ void k_bgivens(const double *__restrict__ hA, const double *__restrict__ hB, const double *__restrict__ hN,
                          int stride, int j, int m, double *__restrict__ H, double *__restrict__ cs,
                          double *__restrict__ sn, double *__restrict__ g, double *__restrict__ hscale,
                          const double *__restrict__ bn2, double *__restrict__ est, int nb,
                          const double *__restrict__ tol, int *__restrict__ act, int *__restrict__ kp) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nb || !act[p]) return;
    double *Hp = H + (int64_t)p * (m + 1) * m;
    double *cp = cs + (int64_t)p * m, *sp = sn + (int64_t)p * m, *gp = g + (int64_t)p * (m + 1);
    for (int i = 0; i <= j; ++i) Hp[i * m + j] = hA[(int64_t)p * stride + i] + hB[(int64_t)p * stride + i];
    const double hn = sqrt(hN[p]);
    Hp[(j + 1) * m + j] = hn;
    hscale[p] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = cp[i] * Hp[i * m + j] + sp[i] * Hp[(i + 1) * m + j];
        Hp[(i + 1) * m + j] = -sp[i] * Hp[i * m + j] + cp[i] * Hp[(i + 1) * m + j];
        Hp[i * m + j] = t;
    }
    const double a = Hp[j * m + j], b = Hp[(j + 1) * m + j];
    const double rho = hypot(a, b);
    cp[j] = rho > 0.0 ? a / rho : 1.0;
    sp[j] = rho > 0.0 ? b / rho : 0.0;
    Hp[j * m + j] = rho;
    Hp[(j + 1) * m + j] = 0.0;
    gp[j + 1] = -sp[j] * gp[j];
    gp[j] = cp[j] * gp[j];
    const double bn = sqrt(bn2[p]);
    est[p] = bn > 0.0 ? fabs(gp[j + 1]) / bn : 0.0;
    kp[p] = j + 1;
    // the estimate met the tolerance (or the Krylov space holds the solution): this problem
    // takes no more steps in the cycle
    if ((*tol >= 0.0 && est[p] <= *tol) || hn == 0.0) act[p] = 0;
}

// per problem: y = R^-1 g (k x k upper triangle of the rotated H)
__global__ void k_bbacksolve(const double *__restrict__ H, const double *__restrict__ g, const int *__restrict__ kp,
                             int m, double *__restrict__ y, int nb, int *__restrict__ itp) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nb) return;
    const int k = kp[p];
    itp[p] += k;
    const double *Hp = H + (int64_t)p * (m + 1) * m;
    const double *gp = g + (int64_t)p * (m + 1);
    double *yp = y + (int64_t)p * m;
    for (int i = k - 1; i >= 0; --i) {
        double t = gp[i];
        for (int c = i + 1; c < k; ++c) t -= Hp[i * m + c] * yp[c];
        yp[i] = Hp[i * m + i] != 0.0 ? t / Hp[i * m + i] : 0.0;
    }
}

// caller order <-> binned order, per problem
__global__ void k_bgather_in(const PlanView *__restrict__ views, const int4 *__restrict__ chunks,
                             const float *__restrict__ in, float *__restrict__ out) {
    const int4 c = chunks[blockIdx.x];
    const PlanView &v = views[c.x];
    for (int i = threadIdx.x; i < c.z; i += blockDim.x) {
        const int64_t p = c.y + i - v.off;
        out[c.y + i] = in[v.off + v.perm[p]];
    }
}

__global__ void k_bscatter_out(const PlanView *__restrict__ views, const int4 *__restrict__ chunks,
                               const double *__restrict__ in, double *__restrict__ out) {
    const int4 c = chunks[blockIdx.x];
    const PlanView &v = views[c.x];
    for (int i = threadIdx.x; i < c.z; i += blockDim.x) {
        const int64_t p = c.y + i - v.off;
        out[v.off + v.perm[p]] = in[c.y + i];
    }
}

__global__ void k_bscatter_out_f32(const PlanView *__restrict__ views, const int4 *__restrict__ chunks,
                                   const float *__restrict__ in, float *__restrict__ out) {
    const int4 c = chunks[blockIdx.x];
    const PlanView &v = views[c.x];
    for (int i = threadIdx.x; i < c.z; i += blockDim.x) {
        const int64_t p = c.y + i - v.off;
        out[v.off + v.perm[p]] = in[c.y + i];
    }
}

inline unsigned g1(int64_t n) { return (unsigned)std::max<int64_t>(1, ceil_div(n, kThreads)); }

}  // namespace

// ------------------------------------------------------------------ host side
static void batch_refresh_views(rbf_batch *Bt, cudaStream_t s) {
    // the captured solve bakes in the subdomain list and its length: capture again
    if (Bt->gexec) {
        cudaGraphExecDestroy(Bt->gexec);
        Bt->gexec = nullptr;
    }
    for (int b = 0; b < Bt->nb; ++b) {
        rbf_plan *P = Bt->plans[b];
        PlanView &v = Bt->hviews[b];
        v.L = P->sz.ready ? P->sz.L.p : nullptr;
        v.core = P->sz.core;
        v.B = P->sz.block;
        v.restricted = P->sz.restricted;
        v.nsub = P->sz.ready ? P->sz.nblocks : 0;
    }
    RBF_CUDA(cudaMemcpyAsync(Bt->views.p, Bt->hviews.data(), Bt->nb * sizeof(PlanView), cudaMemcpyHostToDevice, s));
    // (problem, subdomain) items of the Schwarz apply
    std::vector<int2> sub;
    for (int b = 0; b < Bt->nb; ++b)
        for (int64_t k = 0; k < Bt->hviews[b].nsub; ++k) sub.push_back(make_int2(b, (int)k));
    Bt->nsub_items = (int64_t)sub.size();
    Bt->sub_items.alloc(std::max<size_t>(sub.size(), 1), s);
    if (!sub.empty())
        RBF_CUDA(cudaMemcpyAsync(Bt->sub_items.p, sub.data(), sub.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    RBF_CUDA(cudaStreamSynchronize(s));
}

rbf_batch *batch_create(rbf_ctx *ctx, rbf_plan *const *plans, int nplans, cudaStream_t s) {
    RBF_CHECK(plans && nplans > 0, RBF_ERR_INVALID, "empty batch");
    rbf_batch *Bt = new rbf_batch();
    try {
        Bt->ctx = ctx;
        Bt->nb = nplans;
        Bt->plans.assign(plans, plans + nplans);
        Bt->off.resize(nplans + 1, 0);
        int64_t total_len = 0, total_tiles = 0;
        for (int b = 0; b < nplans; ++b) {
            RBF_CHECK(plans[b] && plans[b]->ctx == ctx, RBF_ERR_INVALID, "plan %d is null or from another context", b);
            RBF_CHECK(plans[b]->kernel == RBF_KERNEL_GAUSSIAN, RBF_ERR_UNSUPPORTED,
                      "plan %d: the batched solve takes Gaussian plans only", b);
            Bt->off[b + 1] = Bt->off[b] + plans[b]->n;
            total_len += plans[b]->pl.len;
            total_tiles += plans[b]->pl.ntiles;
            Bt->max_tiles = std::max<int64_t>(Bt->max_tiles, plans[b]->pl.ntiles);
        }
        Bt->N = Bt->off[nplans];
        RBF_CHECK(Bt->N < (1LL << 31), RBF_ERR_UNSUPPORTED, "batch of %lld centres (limit 2^31)", (long long)Bt->N);
        // the residual's symmetric form: each problem's tile of every binned position, and
        // the fixed-point row accumulators
        Bt->tile_of.alloc(std::max<int64_t>(Bt->N, 1), s);
        Bt->fix.alloc(2 * std::max<int64_t>(Bt->N, 1), s);
        for (int b = 0; b < nplans; ++b)
            tile_of_launch(plans[b]->tiles.p, plans[b]->pl.ntiles, Bt->tile_of.p + Bt->off[b], s);
        // one segment length for the whole batch: the persistent product balances across problems
        const int64_t seglen = std::max<int64_t>(64, 2 * ceil_div(std::max<int64_t>(total_len, 1),
                                                                  std::max<int64_t>(total_tiles, 1)));
        Bt->hviews.resize(nplans);
        std::vector<std::pair<int, int2>> items;   // (length, (problem, segment))
        std::vector<int2> splits;
        std::vector<int64_t> poff(nplans + 1, 0);
        Bt->bseg.resize(nplans);
        Bt->btile_seg.resize(nplans);
        std::vector<int64_t> nsegs(nplans);
        std::vector<bool> splitv(nplans);
        for (int b = 0; b < nplans; ++b) {
            rbf_plan *P = plans[b];
            int64_t ns = 0;
            bool sp = false;
            segment_into(P, P->pl, seglen, Bt->bseg[b], Bt->btile_seg[b], ns, sp, s);
            nsegs[b] = ns;
            splitv[b] = sp;
            std::vector<int4> seg(ns);
            std::vector<int32_t> ts(P->pl.ntiles + 1);
            if (ns) RBF_CUDA(cudaMemcpyAsync(seg.data(), Bt->bseg[b].p, ns * sizeof(int4), cudaMemcpyDeviceToHost, s));
            RBF_CUDA(cudaMemcpyAsync(ts.data(), Bt->btile_seg[b].p, ts.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                     s));
            RBF_CUDA(cudaStreamSynchronize(s));
            for (int k = 0; k < (int)seg.size(); ++k) items.push_back({seg[k].z - seg[k].y, make_int2(b, k)});
            for (int64_t t = 0; t < P->pl.ntiles; ++t)
                if (ts[t + 1] - ts[t] > 1) splits.push_back(make_int2(b, (int)t));
            poff[b + 1] = poff[b] + (sp ? ns * (int64_t)kChunk : 0);
        }
        Bt->part_f.alloc(std::max<int64_t>(poff[nplans], 1), s);
        for (int b = 0; b < nplans; ++b) {
            rbf_plan *P = plans[b];
            PlanView &v = Bt->hviews[b];
            v = PlanView{};
            v.pos = P->pos.p;
            v.src = P->src.p;
            v.blk_c = P->blk_c.p;
            v.tiles = P->tiles.p;
            v.blk = P->blk.p;
            v.ent = P->pl.ent.p;
            v.ebi = P->pl.ebi.p;
            v.seg = Bt->bseg[b].p;
            v.tile_seg = Bt->btile_seg[b].p;
            v.perm = P->perm.p;
            v.tile_of = Bt->tile_of.p + Bt->off[b];
            v.partial = splitv[b] ? Bt->part_f.p + poff[b] : nullptr;
            v.n = P->n;
            v.off = Bt->off[b];
            v.nseg = (int)nsegs[b];
            v.ntiles = (int)P->pl.ntiles;
            v.any_split = splitv[b] ? 1 : 0;
            v.scl = P->scl;
            v.R = P->R;
            double C = 1.4426950408889634 * P->inv2s2_64;
            v.Ch = (float)C;
            v.Cl = (float)(C - (double)v.Ch);
            if (P->rc2_64 > 0.0) {
                v.Rh = (float)P->rc2_64;
                v.Rl = (float)(P->rc2_64 - (double)v.Rh);
            } else {
                v.Rh = INFINITY;
                v.Rl = 0.f;
            }
        }
        // longest work first: the atomic queue then ends on short items
        std::stable_sort(items.begin(), items.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
        std::vector<int2> it2(items.size());
        for (size_t k = 0; k < items.size(); ++k) it2[k] = items[k].second;
        Bt->nseg_items = (int64_t)it2.size();
        Bt->seg_items.alloc(std::max<size_t>(it2.size(), 1), s);
        if (!it2.empty())
            RBF_CUDA(cudaMemcpyAsync(Bt->seg_items.p, it2.data(), it2.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        Bt->nsplit = (int64_t)splits.size();
        Bt->split_tiles.alloc(std::max<size_t>(splits.size(), 1), s);
        if (!splits.empty())
            RBF_CUDA(cudaMemcpyAsync(Bt->split_tiles.p, splits.data(), splits.size() * sizeof(int2),
                                     cudaMemcpyHostToDevice, s));
        Bt->part_d.alloc(std::max<int64_t>(poff[nplans], 1), s);
        Bt->part_off_d.alloc(nplans + 1, s);
        RBF_CUDA(cudaMemcpyAsync(Bt->part_off_d.p, poff.data(), poff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        // element chunks that never cross a problem
        std::vector<int4> ch;
        std::vector<int32_t> choff(nplans + 1, 0);
        for (int b = 0; b < nplans; ++b) {
            for (int64_t q = 0; q < plans[b]->n; q += kRange)
                ch.push_back(make_int4(b, (int)(Bt->off[b] + q), (int)std::min<int64_t>(kRange, plans[b]->n - q), 0));
            choff[b + 1] = (int32_t)ch.size();
        }
        Bt->nchunks = (int64_t)ch.size();
        Bt->chunks.alloc(ch.size(), s);
        RBF_CUDA(cudaMemcpyAsync(Bt->chunks.p, ch.data(), ch.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
        Bt->chunk_off.alloc(nplans + 1, s);
        RBF_CUDA(cudaMemcpyAsync(Bt->chunk_off.p, choff.data(), choff.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        Bt->views.alloc(nplans, s);
        Bt->counter.alloc(1, s);
        RBF_CUDA(cudaStreamCreateWithFlags(&Bt->own, cudaStreamNonBlocking));
        RBF_CUDA(cudaEventCreateWithFlags(&Bt->ev_in, cudaEventDisableTiming));
        RBF_CUDA(cudaEventCreateWithFlags(&Bt->ev_out, cudaEventDisableTiming));
        int per_sm = 0;
        RBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bmatvec, kWarps * 32, 0));
        Bt->persistent_ctas = std::max(1, per_sm) * ctx->num_sms;
        residual_df_prepare(ctx->device, s);
        Bt->tc = true;
        for (int b = 0; b < nplans; ++b) Bt->tc = Bt->tc && plans[b]->product == RBF_PRODUCT_TC;
        if (Bt->tc) product_tc_prepare(ctx->device);
        batch_refresh_views(Bt, s);
    } catch (...) {
        delete Bt;
        throw;
    }
    return Bt;
}

static void batch_alloc(rbf_batch *Bt, int m, cudaStream_t s) {
    if (Bt->m_alloc >= m) return;
    const int64_t N = Bt->N, nb = Bt->nb;
    Bt->bs.alloc(N, s);
    Bt->Z.alloc((size_t)m * N, s);
    Bt->w32.alloc(N, s);
    Bt->V.alloc((size_t)(m + 1) * N, s);
    Bt->w64.alloc(N, s);
    Bt->x.alloc(N, s);
    Bt->r.alloc(N, s);
    Bt->red.alloc((size_t)(m + 1) * Bt->nchunks, s);
    Bt->hA.alloc((size_t)nb * (m + 1), s);
    Bt->hB.alloc((size_t)nb * (m + 1), s);
    Bt->hN.alloc(nb, s);
    Bt->hs.alloc(nb, s);
    Bt->H.alloc((size_t)nb * (m + 1) * m, s);
    Bt->g.alloc((size_t)nb * (m + 1), s);
    Bt->cs.alloc((size_t)nb * m, s);
    Bt->sn.alloc((size_t)nb * m, s);
    Bt->y.alloc((size_t)nb * m, s);
    Bt->est.alloc(nb, s);
    Bt->bn2.alloc(nb, s);
    Bt->rn2.alloc(nb, s);
    Bt->dtol.alloc(1, s);
    Bt->act.alloc(nb, s);
    Bt->kp.alloc(nb, s);
    Bt->itp.alloc(nb, s);
    Bt->m_alloc = m;
    if (Bt->gexec) {
        cudaGraphExecDestroy(Bt->gexec);
        Bt->gexec = nullptr;
    }
}

// problems whose act flag is 0 are skipped (their y rows are left as they were)
void batch_matvec_binned(rbf_batch *Bt, const float *z, float *y, cudaStream_t s, const int *act) {
    if (Bt->tc) {
        product_tc_batched_launch(Bt->views.p, Bt->seg_items.p, Bt->nseg_items, z, y, ctx_error_word(Bt->ctx),
                                  Bt->ctx->device, s, act);
    } else {
        RBF_CUDA(cudaMemsetAsync(Bt->counter.p, 0, sizeof(unsigned int), s));
        const int grid = (int)std::min<int64_t>(Bt->persistent_ctas, std::max<int64_t>(Bt->nseg_items, 1));
        k_bmatvec<<<grid, kWarps * 32, 0, s>>>(Bt->views.p, Bt->seg_items.p, (int)Bt->nseg_items, Bt->counter.p, z,
                                               y, act);
        RBF_LAUNCHED();
    }
    if (Bt->nsplit > 0) {
        k_breduce_split<<<(unsigned)Bt->nsplit, kChunk, 0, s>>>(Bt->views.p, Bt->split_tiles.p, y, act);
        RBF_LAUNCHED();
    }
}

// segmented norms^2 of a float64 vector -> out[problem]
static void batch_norm2(rbf_batch *Bt, const double *v, double *out, cudaStream_t s) {
    k_bmdot<double><<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(v, 0, 1, v, Bt->chunks.p, Bt->nchunks, Bt->red.p,
                                                               nullptr);
    RBF_LAUNCHED();
    k_bmdot_final<<<dim3(Bt->nb, 1), kThreads, 0, s>>>(Bt->red.p, Bt->nchunks, Bt->chunk_off.p, out, 1, nullptr);
    RBF_LAUNCHED();
}

// The whole solve on the stream (no host synchronisation): input Bt->bs (binned) and the
// tolerance *Bt->dtol (< 0: every problem takes every step), output Bt->x, Bt->rn2,
// Bt->bn2, Bt->est, Bt->itp.  The captured sequence has max_it steps; a problem that meets
// the tolerance (its Givens estimate within a cycle, its true residual at a restart) takes
// no further steps: the kernels skip its items, chunks and subdomains.
static void batch_solve_body(rbf_batch *Bt, int m, int max_it, bool precond, cudaStream_t s) {
    const int64_t N = Bt->N;
    const int nb = Bt->nb;
    const unsigned nbg = (unsigned)ceil_div(nb, 128);
    k_bto64<<<g1(N), kThreads, 0, s>>>(Bt->bs.p, Bt->r.p, N);   // x0 = 0: r0 = b
    RBF_LAUNCHED();
    k_bzero<<<g1(N), kThreads, 0, s>>>(Bt->x.p, N);
    RBF_LAUNCHED();
    RBF_CUDA(cudaMemsetAsync(Bt->itp.p, 0, nb * sizeof(int), s));
    batch_norm2(Bt, Bt->r.p, Bt->bn2.p, s);
    const int *act = Bt->act.p;
    int it = 0;
    bool first = true;
    while (it < max_it) {
        if (!first) {
            residual_df_batched(Bt->views.p, Bt->seg_items.p, Bt->nseg_items, Bt->split_tiles.p, Bt->nsplit, Bt->bs.p,
                                Bt->x.p, Bt->r.p, Bt->part_d.p, Bt->part_off_d.p, Bt->fix.p, Bt->N,
                                Bt->max_tiles, ctx_error_word(Bt->ctx), Bt->ctx->device, s);
        }
        first = false;
        batch_norm2(Bt, Bt->r.p, Bt->hN.p, s);
        k_bstart<<<nbg, 128, 0, s>>>(Bt->hN.p, Bt->hs.p, Bt->g.p, Bt->H.p, m, nb, Bt->bn2.p, Bt->dtol.p, Bt->act.p,
                                     Bt->kp.p);
        RBF_LAUNCHED();
        k_bscale<<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->r.p, Bt->hs.p, Bt->V.p, Bt->chunks.p, act);
        RBF_LAUNCHED();
        const int steps = std::min(m, max_it - it);
        for (int j = 0; j < steps; ++j) {
            double *Vj = Bt->V.p + (size_t)j * N;
            float *Zj = Bt->Z.p + (size_t)j * N;
            if (precond) {
                RBF_CUDA(cudaMemsetAsync(Zj, 0, N * sizeof(float), s));   // additive subdomains accumulate
                if (Bt->sz_p.block <= 32)
                    k_bschwarz_apply<true><<<(unsigned)ceil_div(Bt->nsub_items * 32, 256), 256, 0, s>>>(
                        Bt->views.p, Bt->sub_items.p, Bt->nsub_items, Vj, Zj, act);
                else
                    k_bschwarz_apply<false><<<(unsigned)ceil_div(Bt->nsub_items * 32, 256), 256, 0, s>>>(
                        Bt->views.p, Bt->sub_items.p, Bt->nsub_items, Vj, Zj, act);
                RBF_LAUNCHED();
            } else {
                k_bcast<<<g1(N), kThreads, 0, s>>>(Vj, Zj, N);
                RBF_LAUNCHED();
            }
            batch_matvec_binned(Bt, Zj, Bt->w32.p, s, act);
            const int nv = j + 1, st = m + 1;
            k_bmdot<float><<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->V.p, N, nv, Bt->w32.p, Bt->chunks.p,
                                                                      Bt->nchunks, Bt->red.p, act);
            RBF_LAUNCHED();
            k_bmdot_final<<<dim3(nb, nv), kThreads, 0, s>>>(Bt->red.p, Bt->nchunks, Bt->chunk_off.p, Bt->hA.p, st,
                                                            act);
            RBF_LAUNCHED();
            k_bmaxpy<float><<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->V.p, N, nv, Bt->hA.p, st, Bt->w32.p,
                                                                       Bt->w64.p, Bt->chunks.p, nullptr, act);
            RBF_LAUNCHED();
            k_bmdot<double><<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->V.p, N, nv, Bt->w64.p, Bt->chunks.p,
                                                                       Bt->nchunks, Bt->red.p, act);
            RBF_LAUNCHED();
            k_bmdot_final<<<dim3(nb, nv), kThreads, 0, s>>>(Bt->red.p, Bt->nchunks, Bt->chunk_off.p, Bt->hB.p, st,
                                                            act);
            RBF_LAUNCHED();
            k_bmaxpy<double><<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->V.p, N, nv, Bt->hB.p, st, Bt->w64.p,
                                                                        Bt->w64.p, Bt->chunks.p, Bt->red.p, act);
            RBF_LAUNCHED();
            k_bmdot_final<<<dim3(nb, 1), kThreads, 0, s>>>(Bt->red.p, Bt->nchunks, Bt->chunk_off.p, Bt->hN.p, 1,
                                                           act);
            RBF_LAUNCHED();
            k_bgivens<<<nbg, 128, 0, s>>>(Bt->hA.p, Bt->hB.p, Bt->hN.p, st, j, m, Bt->H.p, Bt->cs.p, Bt->sn.p,
                                          Bt->g.p, Bt->hs.p, Bt->bn2.p, Bt->est.p, nb, Bt->dtol.p, Bt->act.p,
                                          Bt->kp.p);
            RBF_LAUNCHED();
            k_bscale<<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->w64.p, Bt->hs.p, Bt->V.p + (size_t)(j + 1) * N,
                                                                 Bt->chunks.p, act);
            RBF_LAUNCHED();
        }
        k_bbacksolve<<<nbg, 128, 0, s>>>(Bt->H.p, Bt->g.p, Bt->kp.p, m, Bt->y.p, nb, Bt->itp.p);
        RBF_LAUNCHED();
        k_bupdate_x<<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->x.p, Bt->Z.p, N, Bt->kp.p, Bt->y.p, m,
                                                                Bt->chunks.p);
        RBF_LAUNCHED();
        it += steps;
    }
    residual_df_batched(Bt->views.p, Bt->seg_items.p, Bt->nseg_items, Bt->split_tiles.p, Bt->nsplit, Bt->bs.p,
                        Bt->x.p, Bt->r.p, Bt->part_d.p, Bt->part_off_d.p, Bt->fix.p, Bt->N, Bt->max_tiles,
                        ctx_error_word(Bt->ctx), Bt->ctx->device, s);
    batch_norm2(Bt, Bt->r.p, Bt->rn2.p, s);
}

rbf_status batch_solve(rbf_batch *Bt, const float *b, const rbf_solve_params &p, double *x, rbf_report *reps,
                       rbf_batch_stats *stats, cudaStream_t s) {
    const int m = p.m > 0 ? p.m : 50;
    const int max_it = p.max_it > 0 ? p.max_it : 500;
    RBF_CHECK(m <= 64, RBF_ERR_UNSUPPORTED, "batched restart length %d > 64", m);
    RBF_CHECK(p.precond == RBF_PRECOND_NONE || p.precond == RBF_PRECOND_SCHWARZ, RBF_ERR_INVALID, "unknown preconditioner");
    RBF_CHECK(!p.assembled, RBF_ERR_UNSUPPORTED, "the batched solve has no assembled operator");
    const bool pc = p.precond == RBF_PRECOND_SCHWARZ;
    cudaEvent_t e0, e1, e2;
    RBF_CUDA(cudaEventCreate(&e0));
    RBF_CUDA(cudaEventCreate(&e1));
    RBF_CUDA(cudaEventCreate(&e2));
    rbf_batch_stats st{};
    try {
        RBF_CUDA(cudaEventRecord(e0, s));
        int failed = 0;
        const rbf_schwarz_params &q = p.schwarz;
        const bool same = Bt->sz_valid && Bt->sz_p.core == q.core && Bt->sz_p.block == q.block &&
                          Bt->sz_p.shift == q.shift && Bt->sz_p.restricted == q.restricted &&
                          Bt->sz_p.escalate == q.escalate;
        if (pc && !same) {
            for (auto *P : Bt->plans) {
                int64_t f = 0;
                schwarz_setup(P, p.schwarz, &f, s);
                failed += (int)f;
            }
            Bt->sz_p = q;
            Bt->sz_valid = true;
            batch_refresh_views(Bt, s);
        }
        RBF_CHECK(!pc || Bt->nsub_items > 0, RBF_ERR_INVALID, "Schwarz preconditioner not set up");
        batch_alloc(Bt, m, s);
        // the tolerance the captured solve reads (a graph replay needs no new capture for it)
        const double tol = p.fixed_iterations ? -1.0 : (p.tol > 0 ? p.tol : 1e-6);
        k_bset<<<1, 1, 0, s>>>(Bt->dtol.p, tol);
        RBF_LAUNCHED();
        RBF_CUDA(cudaEventRecord(e1, s));
        k_bgather_in<<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->views.p, Bt->chunks.p, b, Bt->bs.p);
        RBF_LAUNCHED();
        const bool recapture = !Bt->gexec || Bt->g_m != m || Bt->g_it != max_it || Bt->g_pc != (int)pc;
        // the graph is captured and launched on the batch's own stream (a legacy default stream
        // cannot be captured), ordered after the caller's stream and before its next work
        RBF_CUDA(cudaEventRecord(Bt->ev_in, s));
        RBF_CUDA(cudaStreamWaitEvent(Bt->own, Bt->ev_in, 0));
        if (recapture) {
            if (Bt->gexec) {
                cudaGraphExecDestroy(Bt->gexec);
                Bt->gexec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            RBF_CUDA(cudaStreamBeginCapture(Bt->own, cudaStreamCaptureModeThreadLocal));
            try {
                batch_solve_body(Bt, m, max_it, pc, Bt->own);
            } catch (...) {
                cudaStreamEndCapture(Bt->own, &graph);
                if (graph) cudaGraphDestroy(graph);
                throw;
            }
            RBF_CUDA(cudaStreamEndCapture(Bt->own, &graph));
            size_t nodes = 0;
            cudaGraphGetNodes(graph, nullptr, &nodes);
            st.graph_nodes = (int64_t)nodes;
            std::vector<cudaGraphNode_t> nv(nodes);
            cudaGraphGetNodes(graph, nv.data(), &nodes);
            Bt->g_kernels = 0;
            for (auto nd : nv) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++Bt->g_kernels;
            }
            cudaError_t ei = cudaGraphInstantiate(&Bt->gexec, graph, 0);
            cudaGraphDestroy(graph);
            RBF_CUDA(ei);
            Bt->g_m = m;
            Bt->g_it = max_it;
            Bt->g_pc = (int)pc;
        }
        RBF_CUDA(cudaGraphLaunch(Bt->gexec, Bt->own));
        rbf_count_launches(Bt->g_kernels);
        RBF_CUDA(cudaEventRecord(Bt->ev_out, Bt->own));
        RBF_CUDA(cudaStreamWaitEvent(s, Bt->ev_out, 0));
        k_bscatter_out<<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->views.p, Bt->chunks.p, Bt->x.p, x);
        RBF_LAUNCHED();
        RBF_CUDA(cudaEventRecord(e2, s));
        std::vector<double> rn(Bt->nb), bn(Bt->nb), es(Bt->nb);
        std::vector<int> itp(Bt->nb);
        RBF_CUDA(cudaMemcpyAsync(itp.data(), Bt->itp.p, Bt->nb * sizeof(int), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(cudaMemcpyAsync(rn.data(), Bt->rn2.p, Bt->nb * sizeof(double), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(cudaMemcpyAsync(bn.data(), Bt->bn2.p, Bt->nb * sizeof(double), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(cudaMemcpyAsync(es.data(), Bt->est.p, Bt->nb * sizeof(double), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(cudaStreamSynchronize(s));
        ctx_check_device_error(Bt->ctx);     // a tensor-core product that gave up on a wait
        float msa = 0, msb = 0;
        cudaEventElapsedTime(&msa, e0, e1);
        cudaEventElapsedTime(&msb, e1, e2);
        st.ms_setup = msa;
        st.ms_solve = msb;
        st.recaptured = recapture ? 1 : 0;
        st.persistent_ctas = Bt->persistent_ctas;
        st.work_items = Bt->nseg_items;
        int nconv = 0;
        double worst = 0;
        for (int b2 = 0; b2 < Bt->nb; ++b2) {
            double rel = bn[b2] > 0 ? std::sqrt(rn[b2] / bn[b2]) : 0.0;
            worst = std::max(worst, rel);
            nconv += rel <= (p.tol > 0 ? p.tol : 1e-6);
            if (reps) {
                rbf_report R{};
                R.iterations = itp[b2];
                R.restarts = (int)ceil_div(max_it, m);
                R.residual_true = rel;
                R.residual_estimate = es[b2];
                R.converged = rel <= (p.tol > 0 ? p.tol : 1e-6);
                R.precond_failed_blocks = 0;
                R.ms_solve = msb;
                R.matvec_launches = itp[b2];
                reps[b2] = R;
            }
        }
        st.converged = nconv;
        st.worst_residual = worst;
        st.precond_failed_blocks = failed;
        if (stats) *stats = st;
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    return RBF_OK;
}

int batch_autotune(rbf_batch *Bt, const float *b, const rbf_solve_params &p, const int *cands, int ncand,
                   double *scores, cudaStream_t s) {
    // short fixed solves of each candidate subdomain size (block Jacobi: core = block, the
    // caller's shift), scored by decades of residual reduction per millisecond
    DevBuf<double> xdev;
    xdev.alloc(Bt->N, s);
    int best = -1;
    double best_score = -1e300;
    for (int c = 0; c < ncand; ++c) {
        rbf_solve_params q = p;
        q.precond = RBF_PRECOND_SCHWARZ;
        q.schwarz.block = cands[c];
        q.schwarz.core = cands[c];
        q.m = std::min(p.m > 0 ? p.m : 20, 20);
        q.max_it = q.m;
        q.fixed_iterations = 1;   // every candidate takes the same steps
        Bt->sz_valid = false;   // force set-up
        rbf_batch_stats st{};
        batch_solve(Bt, b, q, xdev.p, nullptr, &st, s);          // set-up + capture
        batch_solve(Bt, b, q, xdev.p, nullptr, &st, s);          // timed replay
        const double ms = st.ms_solve + 1e-3;
        const double red = st.worst_residual > 0 ? -std::log10(st.worst_residual) : 16.0;
        const double score = red / ms;
        if (scores) scores[c] = score;
        if (score > best_score) {
            best_score = score;
            best = cands[c];
        }
    }
    Bt->sz_valid = false;
    return best;
}

int64_t batch_size(const rbf_batch *Bt) { return Bt->N; }
void batch_destroy(rbf_batch *Bt) { delete Bt; }
rbf_ctx *batch_ctx(rbf_batch *Bt) { return Bt->ctx; }

void batch_gather_f32(rbf_batch *Bt, const float *in, float *out, cudaStream_t s) {
    k_bgather_in<<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->views.p, Bt->chunks.p, in, out);
    RBF_LAUNCHED();
}

void batch_scatter_f32(rbf_batch *Bt, const float *in, float *out, cudaStream_t s) {
    k_bscatter_out_f32<<<(unsigned)Bt->nchunks, kThreads, 0, s>>>(Bt->views.p, Bt->chunks.p, in, out);
    RBF_LAUNCHED();
}
