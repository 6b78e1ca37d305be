// The float32 Gaussian product over one segment of a tile's pair list (shared by
// the per-plan kernel in matvec.cu and the batched persistent kernel in
// batch.cu).  See matvec.cu for the formulation.
#pragma once
#include "plan.cuh"

namespace rbfk {

constexpr int kWarps = 4;
#ifndef RBF_MV_MINBLOCKS
#define RBF_MV_MINBLOCKS 4
#endif

typedef unsigned long long f2;      // two float32 in one 64-bit register pair

__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &a, float &b) { asm("mov.b64 {%0,%1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

struct MvArgs {
    const float4 *pos;   // binned positions (targets, sorted mode)
    const int2 *tiles;   // target tiles (start, count) in sorted mode
    const float4 *src;
    const float *w;      // binned weights
    const int2 *blk;
    const float4 *blk_c; // (centre, overflow guard U_B = (32 / r_B)^2 in scaled units)
    const int32_t *ent;
    const int2 *ebi;     // per entry (block start, count | cut-off flag)
    const int4 *seg;
    int64_t n;
    float scl, R;
    float *out;          // y (binned) or grid f, for tiles with a single segment
    float *partial;      // [seg][kChunk] partial sums of split tiles
    float *colpart;      // symmetric form: [entry][kBlk] transposed sums of upper entries
    // grid targets: bricks of 2^blog[0] x 2^blog[1] x 2^blog[2] = 128 nodes (bdim[d] bricks along
    // axis d), each cut into four quarters of 2^qlog[0] x 2^qlog[1] x 2^qlog[2] = 32 nodes
    float glo[3], gstep[3];
    int gdim[3];
    int bdim[3];
    int blog[3], qlog[3];
    // inverse multiquadric plans (direct kernel): 1 / sigma^2, beta, squared cut-off (k sigma)^2
    float imq_ic, imq_beta, rc2f;
};

// Target slot q (0..kChunk-1) of tile t: coordinates and validity.
template <bool kGrid>
__device__ __forceinline__ bool target_xyz(const MvArgs &a, int64_t t, int q, float &x, float &y, float &z,
                                           int64_t &outidx) {
    if (!kGrid) {
        const int2 tl = a.tiles[t];
        int64_t i = (int64_t)tl.x + q;
        if (q < tl.y) {
            float4 p = a.pos[i];
            x = p.x; y = p.y; z = p.z;
            outidx = i;
            return true;
        }
        x = y = z = 0.f;
        outidx = -1;
        return false;
    } else {
        // brick t; quarter u = q / 32 is a compact block of the brick (x fastest among the
        // quarters and among the 32 nodes of a quarter), so that the quarter box tests of the
        // pair list are tight
        int64_t bx = t % a.bdim[0], by = (t / a.bdim[0]) % a.bdim[1], bz = t / ((int64_t)a.bdim[0] * a.bdim[1]);
        const int u = q >> 5, l = q & 31;
        const int nx = a.blog[0] - a.qlog[0], ny = a.blog[1] - a.qlog[1];   // log2 quarters along x, y
        const int ux = u & ((1 << nx) - 1), uy = (u >> nx) & ((1 << ny) - 1), uz = u >> (nx + ny);
        const int lx = l & ((1 << a.qlog[0]) - 1), ly = (l >> a.qlog[0]) & ((1 << a.qlog[1]) - 1),
                  lz = l >> (a.qlog[0] + a.qlog[1]);
        int ix = ((int)bx << a.blog[0]) + (ux << a.qlog[0]) + lx, iy = ((int)by << a.blog[1]) + (uy << a.qlog[1]) + ly,
            iz = ((int)bz << a.blog[2]) + (uz << a.qlog[2]) + lz;
        bool v = ix < a.gdim[0] && iy < a.gdim[1] && iz < a.gdim[2];
        x = fmaf((float)ix, a.gstep[0], a.glo[0]);
        y = fmaf((float)iy, a.gstep[1], a.glo[1]);
        z = fmaf((float)iz, a.gstep[2], a.glo[2]);
        outidx = v ? ((int64_t)iz * a.gdim[1] + iy) * a.gdim[0] + ix : -1;
        return v;
    }
}

__device__ __forceinline__ float set_gt(float a, float b) {
    float r;
    asm("set.gt.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));   // 1.0f if a > b else 0.0f
    return r;
}

constexpr int kTpl = kChunk / 32;   // targets per lane

struct Stage {            // one block of sources, structure of arrays (2 s_x, 2 s_y, 2 s_z, b, w)
    float4 x[kBlk / 4], y[kBlk / 4], z[kBlk / 4], b[kBlk / 4], w[kBlk / 4];
};

// p[t] = (sum over even j, sum over odd j) of w_j 2^(arg_tj), arg = d_t.(2 s_j) - |s_j|^2 (- shift_t);
// masked: only terms with arg > thr_t.  Sources are paired in the f32x2 operands, targets broadcast.
template <bool kMasked, bool kShift>
__device__ __forceinline__ void block_sum(const Stage &st, int cnt4, const f2 (&DX)[kTpl], const f2 (&DY)[kTpl],
                                          const f2 (&DZ)[kTpl], const float (&TH)[kTpl], const float (&SH)[kTpl],
                                          f2 (&P)[kTpl]) {
#pragma unroll
    for (int t = 0; t < kTpl; ++t) P[t] = 0ull;
#pragma unroll 1
    for (int q = 0; q < cnt4; ++q) {            // four sources per step: two f32x2 pairs
        const float4 X = st.x[q], Y = st.y[q], Z = st.z[q], B = st.b[q], W = st.w[q];
        const f2 X0 = pk(X.x, X.y), X1 = pk(X.z, X.w), Y0 = pk(Y.x, Y.y), Y1 = pk(Y.z, Y.w);
        const f2 Z0 = pk(Z.x, Z.y), Z1 = pk(Z.z, Z.w), B0 = pk(B.x, B.y), B1 = pk(B.z, B.w);
        const f2 W0 = pk(W.x, W.y), W1 = pk(W.z, W.w);
#pragma unroll
        for (int t = 0; t < kTpl; ++t) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const f2 Xs = h ? X1 : X0, Ys = h ? Y1 : Y0, Zs = h ? Z1 : Z0, Ws = h ? W1 : W0;
                const f2 c0 = kShift ? sub2(h ? B1 : B0, pk(SH[t], SH[t])) : (h ? B1 : B0);
                const f2 arg = fma2(DX[t], Xs, fma2(DY[t], Ys, fma2(DZ[t], Zs, c0)));
                float a0, a1;
                upk(arg, a0, a1);
                f2 E = pk(ex2_approx(a0), ex2_approx(a1));
                if (kMasked) E = mul2(E, pk(set_gt(a0, TH[t]), set_gt(a1, TH[t])));
                P[t] = fma2(Ws, E, P[t]);
            }
        }
    }
}

// One segment (tile, entries [sg.y, sg.z)) of the product; `slot` indexes the
// partial-sum row of split tiles.  Called by every thread of a 128-thread CTA.
template <bool kGrid>
__device__ __forceinline__ void product_segment(const MvArgs &a, const int4 sg, int64_t slot, Stage (&s_st)[kWarps],
                                                float (&s_red)[kWarps][kChunk]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t = sg.x;

    // targets lane + 32 u
    float tx[kTpl], ty[kTpl], tz[kTpl], acc[kTpl];
#pragma unroll
    for (int u = 0; u < kTpl; ++u) {
        int64_t oi;
        target_xyz<kGrid>(a, t, lane + 32 * u, tx[u], ty[u], tz[u], oi);
        acc[u] = 0.f;
    }
    Stage &st = s_st[warp];
    float *sx = reinterpret_cast<float *>(st.x), *sy = reinterpret_cast<float *>(st.y),
          *sz = reinterpret_cast<float *>(st.z), *sb = reinterpret_cast<float *>(st.b),
          *swt = reinterpret_cast<float *>(st.w);
    int e = sg.y + warp;
    int ent = 0;
    int2 bi = make_int2(0, 0);
    float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
    float wv = 0.f;
    if (e < sg.z) {
        ent = a.ent[e];
        bi = a.blk[ent & 0x7fffffff];
        if (lane < bi.y) {
            sv = a.src[bi.x + lane];
            wv = a.w[bi.x + lane];
        }
    }
    for (; e < sg.z; e += kWarps) {
        const bool masked = ent < 0;
        const int b = ent & 0x7fffffff;
        const int cnt4 = (bi.y + 3) >> 2;
        const float4 c = a.blk_c[b];
        sx[lane] = sv.x;
        sy[lane] = sv.y;
        sz[lane] = sv.z;
        sb[lane] = sv.w;
        swt[lane] = wv;      // zero past the block's count: padded terms vanish
        __syncwarp();
        const int en = e + kWarps;
        if (en < sg.z) {
            ent = a.ent[en];
            bi = a.blk[ent & 0x7fffffff];
            sv = make_float4(0.f, 0.f, 0.f, 0.f);
            wv = 0.f;
            if (lane < bi.y) {
                sv = a.src[bi.x + lane];
                wv = a.w[bi.x + lane];
            }
        }
        f2 DX[kTpl], DY[kTpl], DZ[kTpl], P[kTpl];
        float TH[kTpl], SH[kTpl], D2[kTpl], ea[kTpl];
        bool unsafe = false;
#pragma unroll
        for (int u = 0; u < kTpl; ++u) {
            const float dx = (tx[u] - c.x) * a.scl, dy = (ty[u] - c.y) * a.scl, dz = (tz[u] - c.z) * a.scl;
            DX[u] = pk(dx, dx);
            DY[u] = pk(dy, dy);
            DZ[u] = pk(dz, dz);
            D2[u] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            TH[u] = D2[u] - a.R;
            unsafe |= D2[u] > c.w;
        }
        unsafe = __any_sync(0xffffffffu, unsafe);
        if (!unsafe) {
#pragma unroll
            for (int u = 0; u < kTpl; ++u) ea[u] = ex2_approx(-D2[u]);
            if (masked)
                block_sum<true, false>(st, cnt4, DX, DY, DZ, TH, SH, P);
            else
                block_sum<false, false>(st, cnt4, DX, DY, DZ, TH, SH, P);
        } else {
            // shift c = 2 |d| r_B with r_B = 32 / sqrt(U_B): the inner exponent is never positive
            const float rB = c.w < INFINITY ? 32.f * rsqrtf(c.w) : 0.f;
#pragma unroll
            for (int u = 0; u < kTpl; ++u) {
                const float cs = 2.f * sqrtf(D2[u]) * rB;
                SH[u] = cs;
                ea[u] = ex2_approx(cs - D2[u]);
                TH[u] -= cs;
            }
            block_sum<true, true>(st, cnt4, DX, DY, DZ, TH, SH, P);
        }
#pragma unroll
        for (int u = 0; u < kTpl; ++u) {
            float p0, p1;
            upk(P[u], p0, p1);
            acc[u] = fmaf(ea[u], p0 + p1, acc[u]);
        }
        __syncwarp();
    }
#pragma unroll
    for (int u = 0; u < kTpl; ++u) s_red[warp][lane + 32 * u] = acc[u];
    __syncthreads();
    for (int q = threadIdx.x; q < kChunk; q += kWarps * 32) {
        float v = ((s_red[0][q] + s_red[1][q]) + s_red[2][q]) + s_red[3][q];
        if (sg.w) {
            float x, y, z;
            int64_t oi;
            if (target_xyz<kGrid>(a, t, q, x, y, z, oi)) a.out[oi] = v;
        } else {
            a.partial[slot * kChunk + q] = v;
        }
    }
}


}  // namespace rbfk

// product_tc.cu: the same product with the exponents from tcgen05.mma (pl.nseg CTAs).
void product_tc_launch(const rbf_plan *P, const PairList &pl, const rbfk::MvArgs &a, bool grid, cudaStream_t s);
// The symmetric form over P->sym (a.seg, a.ent, a.ebi from P->sym, a.colpart = P->colpart),
// then, after the split tiles' segments are reduced, the gather of the transposed sums.
void product_tc_sym_launch(const rbf_plan *P, const rbfk::MvArgs &a, cudaStream_t s);
void product_tc_sym_gather(const rbf_plan *P, float *ys, cudaStream_t s);
