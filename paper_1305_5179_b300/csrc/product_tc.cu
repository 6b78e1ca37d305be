// Tensor-core form of the float32 Gaussian product (Sec. III.A, Eq. matrixEntries;
// the grid evaluation of Eq. matxvet uses the same kernel with grid targets).
//
// For a target tile T (128 targets, one TMEM lane each) and a source block B
// (32 sources), the exponent of every pair is a rank-4 contraction: with the
// tile centre c_T, u_i = (x_i - c_T) scl and v_j = (x_j - c_T) scl (scaled
// units, phi = 2^(-|u - v|^2)),
//      -|u_i - v_j|^2 = u_i . (2 v_j) - |v_j|^2 - |u_i|^2.
// Each factor is split into a tf32 head and a tf32 tail (h + l, 22 significant
// bits), and the products h.h + h.l + l.h together with the two squared norms
// (head + tail each) form K = 13 of a K = 16 tf32 contraction:
//      A_i = [hx hx lx hy | hy ly hz hz | lz 1 1 ph | pl 0 0 0]
//      B_j = [Hx Lx Hx Hy | Ly Hy Hz Lz | Hz qh ql 1 | 1 0 0 0]
// (h, l of u_i; H, L of 2 v_j; p = -|u_i|^2, q = -|v_j|^2).  Two
// tcgen05.mma (M = 128, N = 32, K = 8) write the 128 x 32 exponents to tensor
// memory; the CUDA cores then only evaluate MUFU.EX2 and the weighted sum.  The
// exponent is never positive, so no overflow guard is needed.
//
// CTA = one segment of a tile's pair list, 6 warps.  Warps 4 and 5 (producers,
// alternate blocks) build the B operand of a block in shared memory (one source
// per lane) and issue its MMAs into one of 4 TMEM stages of 32 columns; warps 0-3
// (consumers) each
// own 32 targets (TMEM lanes 32w..32w+31), read their 32 x 32 exponents,
// and accumulate z_j 2^t over the segment.  The pair list carries, per block, a
// 2-bit code for each quarter of 32 targets (box tests on the quarter's box, refined
// pair by pair): a consumer skips a block its quarter cannot reach and sums the pairs
// of the others; in a combination that straddles the cut-off it tests each pair
// against it when the cut-off entry e^(-k^2/2) = 2^-R is at least 2^-24, and otherwise
// (k >= 5.77, e.g. the scan configurations' k = 6) sums every pair: those beyond the
// cut-off carry entries below float32's resolution of the unit diagonal and below the
// truncation bound itself.  A producer issues no MMA for a block no quarter reaches.  full[s] completes when the stage's
// MMAs have finished and the producer has written its weights; empty[s] when
// all four consumers have read it.  Every wait is bounded (1 s); on expiry the
// kernel raises the context's device error word and returns after freeing its
// tensor memory.
#include <cmath>

#include "batch.cuh"
#include "plan.cuh"
#include "product.cuh"
#include "tcgen05.cuh"

namespace {

using namespace rbfk;

constexpr int kStages = 4;
constexpr int kCons = 4;                       // consumer warps, one per 32 TMEM lanes
constexpr int kProd = 2;                       // producer warps, alternate blocks
constexpr int kThreadsTc = (kCons + kProd) * 32;
constexpr uint32_t kLbo = 128;                 // next 16-byte K chunk of the same 8 rows
constexpr uint32_t kSbo = 512;                 // next group of 8 rows (4 chunks of 128 bytes)
constexpr int kABytes = kChunk / 8 * kSbo;     // 8 KB
constexpr int kBBytes = kBlk / 8 * kSbo;       // 2 KB
constexpr uint32_t kIdesc = tc5::idesc_tf32(kChunk, kBlk);
constexpr uint32_t kTmemCols = kStages * kBlk;
// Shared memory per CTA is padded so that at most 4 CTAs share an SM: 4 x 128 TMEM
// columns fill the 512 an SM has, so no CTA ever waits in tcgen05.alloc.
constexpr int kSmemTc = 56 * 1024;
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr int kL = 128;     // pair-list entries staged per chunk (4 per producer lane)
constexpr int kR = 8;       // depth of the cp.async ring of raw source data
static_assert(kL > kR && kL % 32 == 0, "staging depths");

constexpr int kTr = 36;     // row stride (floats) of a consumer warp's transpose tile

struct TcSmem {
    uint8_t a[kABytes];
    uint8_t b[kStages][kBBytes];
    float tr[kCons][kBlk][kTr];          // symmetric form: [source][target lane] exponentials
    float zt[kCons][32];                 // symmetric form: the warp's own target weights
    float col[kStages][kCons][kBlk];     // symmetric form: each warp's transposed partial sums
    float4 rpos[kProd][kR][kBlk];
    float rz[kProd][kR][kBlk];
    float z[kStages][kBlk];
    int2 lst[kProd][2][kL];
    int flag[kStages];
    uint64_t full[kStages];
    uint64_t empty[kStages];
    float box[kCons][6];
    uint32_t tmem;
    int abort;
};
static_assert(sizeof(TcSmem) <= kSmemTc, "shared memory layout");

// Two exponentials / two cut-off masks (1.0 or 0.0) written straight into a register pair.
__device__ __forceinline__ f2 ex2_pair(float a, float b) {
    f2 r;
    asm("{\n\t.reg .f32 lo, hi;\n\tex2.approx.ftz.f32 lo, %1;\n\tex2.approx.ftz.f32 hi, %2;\n\t"
        "mov.b64 %0, {lo, hi};\n\t}"
        : "=l"(r)
        : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ f2 gt_pair(float a, float b, float thr) {
    f2 r;
    asm("{\n\t.reg .f32 lo, hi;\n\tset.gt.f32.f32 lo, %1, %3;\n\tset.gt.f32.f32 hi, %2, %3;\n\t"
        "mov.b64 %0, {lo, hi};\n\t}"
        : "=l"(r)
        : "f"(a), "f"(b), "f"(thr));
    return r;
}

__device__ __forceinline__ uint32_t core_off(int row, int chunk) {
    return (uint32_t)((row >> 3) * kSbo + chunk * kLbo + (row & 7) * 16);
}

__device__ __forceinline__ void put4(uint8_t *base, int row, int chunk, float x, float y, float z, float w) {
    *reinterpret_cast<float4 *>(base + core_off(row, chunk)) = make_float4(x, y, z, w);
}

// the exponentials of targets lane x sources 4g .. 4g + 3 into column `lane` of the tile
__device__ __forceinline__ void put_t(float *tcol, int g, f2 e0, f2 e1) {
    float x0, x1, x2, x3;
    upk(e0, x0, x1);
    upk(e1, x2, x3);
    tcol[(4 * g) * kTr] = x0;
    tcol[(4 * g + 1) * kTr] = x1;
    tcol[(4 * g + 2) * kTr] = x2;
    tcol[(4 * g + 3) * kTr] = x3;
}

// Symmetric form: the transposed sums of the block that used stage s (entry e of the list),
// the four consumer warps' partials added in a fixed order; nothing for a diagonal entry.
__device__ __forceinline__ void combine_columns(const MvArgs &a, TcSmem &S, int s, int64_t e, int lane) {
    if ((S.flag[s] >> 16) & 1) {
        const float v = ((S.col[s][0][lane] + S.col[s][1][lane]) + S.col[s][2][lane]) + S.col[s][3][lane];
        a.colpart[e * kBlk + lane] = v;
    }
}

__device__ __forceinline__ void raise_error(TcSmem &S, unsigned *err) {
    *(volatile int *)&S.abort = 1;
    if (err) atomicOr(err, 1u);
}

// One segment sg of a pair list; `slot` indexes its row of partial sums when its tile
// has more than one segment.  Run by a whole CTA of kThreadsTc threads.
// kScalar: the summed combinations accumulate in eight scalar sums (one FMA per pair)
// instead of four packed pairs; measured faster for the single-plan product and slower
// for the batched one (one more live register set where that kernel already spills).
template <bool kGrid, bool kSym = false, bool kScalar = false>
__device__ __forceinline__ void product_tc_body(const MvArgs &a, const int4 sg, int64_t slot, unsigned *err) {
    static_assert(!(kGrid && kSym), "grid targets carry no weights: the symmetric form is for products");
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = sg.x;
    const int nb = sg.z - sg.y;

    if (warp == kCons) {
        tc5::tmem_alloc(&S.tmem, kTmemCols);
        tc5::tmem_relinquish();
        for (int s = 0; s < kStages; ++s) put4(S.b[s], lane, 3, 1.f, 0.f, 0.f, 0.f);   // constant chunk of B
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc5::mbar_init(&S.full[s], 2);        // tcgen05.commit + the producer's own arrival
            tc5::mbar_init(&S.empty[s], kCons);
        }
        S.abort = 0;
        tc5::mbar_init_fence();
    }
    float tx = 0.f, ty = 0.f, tz = 0.f;
    int64_t oi = -1;
    bool valid = false;
    if (warp < kCons) {
        valid = target_xyz<kGrid>(a, t, threadIdx.x, tx, ty, tz, oi);
        float b6[6] = {valid ? tx : INFINITY,  valid ? ty : INFINITY,  valid ? tz : INFINITY,
                       valid ? tx : -INFINITY, valid ? ty : -INFINITY, valid ? tz : -INFINITY};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                b6[d] = fminf(b6[d], __shfl_xor_sync(0xffffffffu, b6[d], o));
                b6[d + 3] = fmaxf(b6[d + 3], __shfl_xor_sync(0xffffffffu, b6[d + 3], o));
            }
        }
        if (lane == 0)
            for (int d = 0; d < 6; ++d) S.box[warp][d] = b6[d];
        if (kSym) S.zt[warp][lane] = valid ? a.w[oi] : 0.f;
    }
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tmem = S.tmem;

    // tile centre: centre of the targets' bounding box (the frame of u and v)
    float c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float lo = fminf(fminf(S.box[0][d], S.box[1][d]), fminf(S.box[2][d], S.box[3][d]));
        float hi = fmaxf(fmaxf(S.box[0][d + 3], S.box[1][d + 3]), fmaxf(S.box[2][d + 3], S.box[3][d + 3]));
        c[d] = lo <= hi ? 0.5f * (lo + hi) : 0.f;
    }

    if (warp < kCons) {   // A row of this thread's target (zero row for an empty slot)
        const int r = threadIdx.x;
        if (valid) {
            const float ux = (tx - c[0]) * a.scl, uy = (ty - c[1]) * a.scl, uz = (tz - c[2]) * a.scl;
            const float p = -fmaf(ux, ux, fmaf(uy, uy, uz * uz));
            const float hx = tc5::to_tf32(ux), hy = tc5::to_tf32(uy), hz = tc5::to_tf32(uz);
            const float lx = tc5::to_tf32(ux - hx), ly = tc5::to_tf32(uy - hy), lz = tc5::to_tf32(uz - hz);
            const float ph = tc5::to_tf32(p), pl = tc5::to_tf32(p - ph);
            put4(S.a, r, 0, hx, hx, lx, hy);
            put4(S.a, r, 1, hy, ly, hz, hz);
            put4(S.a, r, 2, lz, 1.f, 1.f, ph);
            put4(S.a, r, 3, pl, 0.f, 0.f, 0.f);
        } else {
            for (int k = 0; k < 4; ++k) put4(S.a, r, k, 0.f, 0.f, 0.f, 0.f);
        }
    }
    tc5::fence_async_smem();
    __syncthreads();

    if (warp >= kCons) {
        // ------------------------------------------------------------ producers
        // Producer warp p handles blocks p, p + kProd, ...  Its entries (block start,
        // count | flag) are staged kL at a time in shared memory (the next chunk waits
        // in registers), and each block's sources and weights are copied kR - 1 of its
        // blocks ahead into a ring with cp.async, so the build never waits on a global load.
        const int pw = warp - kCons;
        const int my_nb = nb > pw ? (nb - pw + kProd - 1) / kProd : 0;
        const float s2 = 2.f * a.scl;
        // descriptors: A's two K halves are fixed; a B stage's differ from stage 0's only in
        // the start address field (address >> 4, added without carry out of the field)
        const uint64_t da0 = tc5::smem_desc(tc5::smem_u32(S.a), kLbo, kSbo);
        const uint64_t da1 = tc5::smem_desc(tc5::smem_u32(S.a) + 2 * kLbo, kLbo, kSbo);
        const uint64_t db0 = tc5::smem_desc(tc5::smem_u32(S.b[0]), kLbo, kSbo);
        const uint32_t row_off = core_off(lane, 0);   // this lane's B row within a stage
        const float4 *pos_l = a.pos + lane;
        const float *w_l = a.w + lane;
        const int2 *ebi = a.ebi + sg.y + pw;
        int2 nx[kL / 32];
        auto fetch = [&](int ch) {
#pragma unroll
            for (int i = 0; i < kL / 32; ++i) {
                const int j = ch * kL + lane + 32 * i;
                nx[i] = j < my_nb ? ebi[(int64_t)j * kProd] : make_int2(0, 0);
            }
        };
        auto stash = [&](int ch) {
#pragma unroll
            for (int i = 0; i < kL / 32; ++i) S.lst[pw][ch & 1][lane + 32 * i] = nx[i];
        };
        auto issue = [&](int pj) {
            if (pj < my_nb) {
                const int2 e = S.lst[pw][(pj / kL) & 1][pj % kL];
                if (lane < (e.y & 0xff)) {
                    tc5::cp_async16(&S.rpos[pw][pj % kR][lane], pos_l + e.x);
                    tc5::cp_async4(&S.rz[pw][pj % kR][lane], w_l + e.x);
                }
            }
            tc5::cp_async_commit();
        };
        fetch(0);
        stash(0);
        fetch(1);
        __syncwarp();
        for (int pj = 0; pj < kR - 1; ++pj) issue(pj);
        int issued = -1;
        for (int j = 0; j < my_nb; ++j) {
            const int b = pw + kProd * j;
            const int s = b % kStages;
            const uint32_t k = (uint32_t)(b / kStages);
            if (j % kL == kL - kR) {      // chunk j/kL + 1 is needed from the next issue on
                stash(j / kL + 1);
                __syncwarp();
                fetch(j / kL + 2);
            }
            issue(j + kR - 1);
            tc5::cp_async_wait<kR - 1>();   // this lane's copies of block j have landed
            const int2 e = S.lst[pw][(j / kL) & 1][j % kL];
            float4 cp = make_float4(c[0], c[1], c[2], 0.f);
            float cz = 0.f;
            if (lane < (e.y & 0xff)) {
                cp = S.rpos[pw][j % kR][lane];
                cz = S.rz[pw][j % kR][lane];
            }
            if (b >= kStages && !tc5::mbar_wait(&S.empty[s], (k - 1) & 1u, &S.abort, kWaitNs)) {
                raise_error(S, err);
                break;
            }
            if (kSym && b >= kStages) {
                // block b - kStages (this producer's) left its consumers' transposed partials here
                combine_columns(a, S, s, sg.y + b - kStages, lane);
                __syncwarp();      // every lane has read the old flag before it is replaced
            }
            if (lane == 0) S.flag[s] = e.y;
            if (((e.y >> 8) & 0xff) == 0) {   // no quarter of the tile meets this block: no MMA
                __syncwarp();
                if (lane == 0) {
                    tc5::mbar_arrive(&S.full[s]);
                    tc5::mbar_arrive(&S.full[s]);
                }
                __syncwarp();
                continue;
            }
            const float wx = (cp.x - c[0]) * s2, wy = (cp.y - c[1]) * s2, wz = (cp.z - c[2]) * s2;
            const float q = -0.25f * fmaf(wx, wx, fmaf(wy, wy, wz * wz));
            const float Hx = tc5::to_tf32(wx), Hy = tc5::to_tf32(wy), Hz = tc5::to_tf32(wz);
            const float Lx = tc5::to_tf32(wx - Hx), Ly = tc5::to_tf32(wy - Hy), Lz = tc5::to_tf32(wz - Hz);
            const float qh = tc5::to_tf32(q), ql = tc5::to_tf32(q - qh);
            uint8_t *Bs = S.b[s] + row_off;
            *reinterpret_cast<float4 *>(Bs) = make_float4(Hx, Lx, Hx, Hy);
            *reinterpret_cast<float4 *>(Bs + kLbo) = make_float4(Ly, Hy, Hz, Lz);
            *reinterpret_cast<float4 *>(Bs + 2 * kLbo) = make_float4(Hz, qh, ql, 1.f);
            S.z[s][lane] = cz;      // zero past the block's count: padded sources vanish
            tc5::fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                tc5::fence_after_sync();
                const uint64_t db = db0 + (uint64_t)((s * kBBytes) >> 4);
                const uint32_t d = tmem + (uint32_t)(s * kBlk);
                tc5::mma_tf32(d, da0, db, kIdesc, 0u);
                tc5::mma_tf32(d, da1, db + ((2 * kLbo) >> 4), kIdesc, 1u);
                tc5::mma_commit(&S.full[s]);
                tc5::mbar_arrive(&S.full[s]);
            }
            issued = b;
            __syncwarp();
        }
        if (kSym && !*(volatile int *)&S.abort) {
            // this producer's last blocks: their stages are not reused, so wait for their
            // consumers here and combine
            for (int jj = my_nb > 2 ? my_nb - 2 : 0; jj < my_nb; ++jj) {
                const int b = pw + kProd * jj;
                if (b + kStages < nb) continue;
                const int s = b % kStages;
                if (!tc5::mbar_wait(&S.empty[s], (uint32_t)(b / kStages) & 1u, &S.abort, kWaitNs)) {
                    raise_error(S, err);
                    break;
                }
                combine_columns(a, S, s, sg.y + b, lane);
            }
        }
        tc5::cp_async_wait_all();
        if (issued >= 0 && lane == 0 && *(volatile int *)&S.abort) {
            // let the MMAs already issued finish before the tensor memory is released
            const int s = issued % kStages;
            const uint32_t par = (uint32_t)(issued / kStages) & 1u;
            const uint64_t t0 = tc5::global_ns();
            while (!tc5::mbar_try_wait(&S.full[s], par) && tc5::global_ns() - t0 < kWaitNs / 10) {
            }
        }
    } else {
        // ------------------------------------------------------------ consumers
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        const float thr = -a.R;      // in the cut-off iff -|u - v|^2 > -R
        // entries beyond the cut-off are below 2^-R: with R >= 24 (k >= 5.77) they are below
        // float32's resolution of the unit diagonal and are summed instead of tested
        const bool mask = a.R < 24.f;
        f2 acc[4] = {0ull, 0ull, 0ull, 0ull};
        float sac[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // kScalar sums
        float gtot = 0.f, gcomp = 0.f;   // grid targets: compensated total of the per-block sums
        for (int b = 0; b < nb; ++b) {
            const int s = b % kStages;
            const uint32_t k = (uint32_t)(b / kStages);
            if (!tc5::mbar_wait(&S.full[s], k & 1u, &S.abort, kWaitNs)) {
                raise_error(S, err);
                break;
            }
            const int code = (S.flag[s] >> (8 + 2 * warp)) & 3;   // this warp's quarter vs the block
            const bool upper = kSym && ((S.flag[s] >> 16) & 1);
            if (code == 0) {
                if (upper) S.col[s][warp][lane] = 0.f;       // the quarter meets no source of the block
                __syncwarp();
                if (lane == 0) tc5::mbar_arrive(&S.empty[s]);
                continue;
            }
            tc5::fence_after_sync();
            float tv[32];
            tc5::tmem_ld_32x32(trow + (uint32_t)(s * kBlk), tv);
            const float4 *zz = reinterpret_cast<const float4 *>(S.z[s]);
            float *tcol = &S.tr[warp][0][lane];             // column `lane` of the transpose tile
            if (kScalar && !kSym && (code == 2 || !mask)) {
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    const float4 Z = zz[g];
                    sac[(4 * g) & 7] = fmaf(ex2_approx(tv[4 * g]), Z.x, sac[(4 * g) & 7]);
                    sac[(4 * g + 1) & 7] = fmaf(ex2_approx(tv[4 * g + 1]), Z.y, sac[(4 * g + 1) & 7]);
                    sac[(4 * g + 2) & 7] = fmaf(ex2_approx(tv[4 * g + 2]), Z.z, sac[(4 * g + 2) & 7]);
                    sac[(4 * g + 3) & 7] = fmaf(ex2_approx(tv[4 * g + 3]), Z.w, sac[(4 * g + 3) & 7]);
                }
                if (kGrid) {
                    // A grid node far from the data sums thousands of terms whose weights
                    // cancel: each block's 32 terms are summed on their own and added to the
                    // node's total with a compensated (Kahan) addition, so that the rounding
                    // of the long sum is that of one addition.
                    const float bs = ((sac[0] + sac[1]) + (sac[2] + sac[3])) + ((sac[4] + sac[5]) + (sac[6] + sac[7]));
                    const float yk = bs - gcomp;
                    const float tk = gtot + yk;
                    gcomp = (tk - gtot) - yk;
                    gtot = tk;
#pragma unroll
                    for (int q = 0; q < 8; ++q) sac[q] = 0.f;
                }
            } else if (code == 2 || !mask) {
                // every pair summed: inside the cut-off, or (mask off) beyond it with an entry
                // below 2^-24 (see the top of the file)
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    const float4 Z = zz[g];
                    const f2 e0 = ex2_pair(tv[4 * g], tv[4 * g + 1]);
                    const f2 e1 = ex2_pair(tv[4 * g + 2], tv[4 * g + 3]);
                    acc[2 * (g & 1)] = fma2(e0, pk(Z.x, Z.y), acc[2 * (g & 1)]);
                    acc[2 * (g & 1) + 1] = fma2(e1, pk(Z.z, Z.w), acc[2 * (g & 1) + 1]);
                    if (upper) put_t(tcol, g, e0, e1);
                }
            } else {
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    const float4 Z = zz[g];
                    const float t0 = tv[4 * g], t1 = tv[4 * g + 1], t2 = tv[4 * g + 2], t3 = tv[4 * g + 3];
                    const f2 m0 = gt_pair(t0, t1, thr), m1 = gt_pair(t2, t3, thr);
                    const f2 e0 = mul2(ex2_pair(t0, t1), m0), e1 = mul2(ex2_pair(t2, t3), m1);
                    acc[2 * (g & 1)] = fma2(e0, pk(Z.x, Z.y), acc[2 * (g & 1)]);
                    acc[2 * (g & 1) + 1] = fma2(e1, pk(Z.z, Z.w), acc[2 * (g & 1) + 1]);
                    if (upper) put_t(tcol, g, e0, e1);
                }
            }
            if (upper) {
                // source `lane` of the block: sum over this warp's 32 targets of a_ij z_i
                __syncwarp();
                const float4 *row = reinterpret_cast<const float4 *>(&S.tr[warp][lane][0]);
                const float4 *zw = reinterpret_cast<const float4 *>(S.zt[warp]);
                f2 ca = 0ull, cb = 0ull;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 R = row[q], Zi = zw[q];
                    ca = fma2(pk(R.x, R.y), pk(Zi.x, Zi.y), ca);
                    cb = fma2(pk(R.z, R.w), pk(Zi.z, Zi.w), cb);
                }
                float c0, c1, c2, c3;
                upk(ca, c0, c1);
                upk(cb, c2, c3);
                S.col[s][warp][lane] = (c0 + c1) + (c2 + c3);
                __syncwarp();       // the tile is rewritten by the next block
            }
            tc5::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc5::mbar_arrive(&S.empty[s]);
        }
        float v[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) upk(acc[i], v[2 * i], v[2 * i + 1]);
        const float y = (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) +
                        ((((sac[0] + sac[1]) + (sac[2] + sac[3])) + ((sac[4] + sac[5]) + (sac[6] + sac[7]))) + gtot);
        if (sg.w) {
            if (valid) a.out[oi] = y;
        } else {
            a.partial[slot * kChunk + threadIdx.x] = y;
        }
    }

    tc5::fence_before_sync();
    __syncthreads();
    if (warp == kCons) {
        tc5::fence_after_sync();
        tc5::tmem_dealloc(tmem, kTmemCols);
    }
}

template <bool kGrid>
__global__ void __launch_bounds__(kThreadsTc, 4) k_product_tc(MvArgs a, unsigned *err) {
    product_tc_body<kGrid, false, true>(a, a.seg[blockIdx.x], blockIdx.x, err);
}

// the symmetric form over rbf_plan::sym (row sums as above, transposed sums per entry)
__global__ void __launch_bounds__(kThreadsTc, 4) k_product_tc_sym(MvArgs a, unsigned *err) {
    product_tc_body<false, true>(a, a.seg[blockIdx.x], blockIdx.x, err);
}

// y[source] += the transposed sums of its block over the block's upper entries, in the
// entries' order (one warp per block)
__global__ void k_sym_gather(const int2 *__restrict__ blk, int64_t nblk, const int32_t *__restrict__ bstart,
                             const int32_t *__restrict__ bend, const int32_t *__restrict__ src,
                             const float *__restrict__ colpart, float *__restrict__ y) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nblk) return;
    const int s0 = bstart[b], s1 = bend[b];
    if (s1 <= s0) return;
    float acc = 0.f;
    for (int q = s0; q < s1; ++q) acc += colpart[(int64_t)src[q] * kBlk + lane];
    const int2 bl = blk[b];
    if (lane < bl.y) y[bl.x + lane] += acc;
}

// Many problems at once: CTA = one (problem, segment) item of a batch.
__global__ void __launch_bounds__(kThreadsTc, 4) k_bproduct_tc(const PlanView *__restrict__ views,
                                                              const int2 *__restrict__ items,
                                                              const float *__restrict__ z, float *__restrict__ y,
                                                              unsigned *err, const int *__restrict__ act) {
    const int2 ci = items[blockIdx.x];
    if (act && !act[ci.x]) return;   // the problem has met its tolerance (uniform over the CTA)
    const PlanView &v = views[ci.x];
    MvArgs a{};
    a.pos = v.pos;
    a.tiles = v.tiles;
    a.src = v.src;
    a.w = z + v.off;
    a.blk = v.blk;
    a.blk_c = v.blk_c;
    a.ent = v.ent;
    a.ebi = v.ebi;
    a.seg = v.seg;
    a.n = v.n;
    a.scl = v.scl;
    a.R = v.R;
    a.out = y + v.off;
    a.partial = v.partial;
    product_tc_body<false>(a, v.seg[ci.y], ci.y, err);
}

template <bool kGrid>
void set_smem_attr(int device) {
    static bool done[64] = {};
    if (device >= 0 && device < 64 && !done[device]) {
        RBF_CUDA(cudaFuncSetAttribute(k_product_tc<kGrid>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTc));
        done[device] = true;
    }
}

}  // namespace

void product_tc_prepare(int device) {
    set_smem_attr<false>(device);
    set_smem_attr<true>(device);
    static bool done_sym[64] = {};
    if (device >= 0 && device < 64 && !done_sym[device]) {
        RBF_CUDA(cudaFuncSetAttribute(k_product_tc_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTc));
        done_sym[device] = true;
    }
    static bool done[64] = {};
    if (device >= 0 && device < 64 && !done[device]) {
        RBF_CUDA(cudaFuncSetAttribute(k_bproduct_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTc));
        done[device] = true;
    }
}

void product_tc_batched_launch(const PlanView *views, const int2 *items, int64_t nitems, const float *z, float *y,
                               unsigned *err, int device, cudaStream_t s, const int *act) {
    if (nitems <= 0) return;
    product_tc_prepare(device);
    k_bproduct_tc<<<(unsigned)nitems, kThreadsTc, kSmemTc, s>>>(views, items, z, y, err, act);
    RBF_LAUNCHED();
}

// The product over a pair list with the tensor-core exponent (see the top of this file).
void product_tc_launch(const rbf_plan *P, const PairList &pl, const rbfk::MvArgs &a, bool grid, cudaStream_t s) {
    if (pl.nseg <= 0) return;
    unsigned *err = ctx_error_word(P->ctx);
    if (grid) {
        set_smem_attr<true>(P->ctx->device);
        k_product_tc<true><<<(unsigned)pl.nseg, kThreadsTc, kSmemTc, s>>>(a, err);
    } else {
        set_smem_attr<false>(P->ctx->device);
        k_product_tc<false><<<(unsigned)pl.nseg, kThreadsTc, kSmemTc, s>>>(a, err);
    }
    RBF_LAUNCHED();
}

// The symmetric product over P->sym (see rbf_plan::sym): the kernel writes each tile's row
// sums (or its segments' partial sums) and the upper entries' transposed sums; after the
// segments are reduced, the gather adds the transposed sums to the sources' rows.
void product_tc_sym_launch(const rbf_plan *P, const rbfk::MvArgs &a, cudaStream_t s) {
    if (P->sym.nseg <= 0) return;
    product_tc_prepare(P->ctx->device);
    k_product_tc_sym<<<(unsigned)P->sym.nseg, kThreadsTc, kSmemTc, s>>>(a, ctx_error_word(P->ctx));
    RBF_LAUNCHED();
}

void product_tc_sym_gather(const rbf_plan *P, float *ys, cudaStream_t s) {
    if (P->nblk <= 0 || P->sym_upper <= 0) return;
    k_sym_gather<<<(unsigned)ceil_div(P->nblk * 32, 256), 256, 0, s>>>(P->blk.p, P->nblk, P->sym_bstart.p,
                                                                        P->sym_bend.p, P->sym_src.p, P->colpart.p, ys);
    RBF_LAUNCHED();
}
