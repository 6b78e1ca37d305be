// Assembled truncated matrix (Algorithm 2) and its sparse product.
//
// The paper's GPU solve built the interpolation matrix entry by entry (for each
// subdomain, each of its points, each point of the truncation area: A_ij =
// phi(|x_i - x_j|)) and handed it to a library sparse product (CSR and related
// formats, Sec. III.B).  Here the same matrix is built from the plan's pair list,
// in the plan's binned order, as CSR with float32 values and int32 columns:
//
//   1. count: one thread per target row and segment of its tile's source blocks;
//   2. rows: per tile, the segments' counts become per-segment offsets inside the
//      row, and row lengths are padded to a multiple of 4 entries (so every row
//      starts on a 16-byte boundary and the product reads 4 entries per load);
//   3. row_ptr: exclusive int64 scan of the padded lengths;
//   4. fill: a warp per quarter (32 rows) of a tile; for each source block the
//      lanes test the 32 sources against one row at a time, and the sources within
//      the cut-off are written contiguously (ballot, population count);
//   5. padding: entries (column = the row itself, value 0) after each row's last one.
//
// Stored entries: pairs with |x_i - x_j| < k sigma, decided in float32 and
// repeated in float64 within 1e-5 (relative) of the cut-off, the decision of the
// pair count; for an untruncated Gaussian plan, pairs closer than 13 sigma (every
// other entry is below exp(-84.5) < 2.2e-37), for an untruncated inverse
// multiquadric plan every pair.  Values exp(-|x_i - x_j|^2 / (2 sigma^2)), or
// (1 + |x_i - x_j|^2 / sigma^2)^-beta, from the float32 squared distance through
// ex2.approx (and lg2.approx); columns of a row appear in the order of the tile's
// source blocks, ascending within a block.
//
// The product (one warp per row, 16-byte streaming loads of columns and values,
// z gathered through L1) moves 8 bytes per stored entry from HBM; the matrix-free
// product moves none.
#include <algorithm>
#include <cmath>

#include "plan.cuh"

namespace {

constexpr int kT = kChunk;            // threads of the count and fill kernels (one per tile row)
constexpr int kSpmvWarps = 8;

struct Cut {
    double rc2;        // float64 squared cut-off
    float lo, hi;      // float32 band around it where the test is repeated in float64
    float c;           // Gaussian: log2(e) / (2 sigma^2); inverse multiquadric: 1 / sigma^2
    float beta;        // inverse multiquadric exponent (0: Gaussian)
};

__device__ __forceinline__ float entry(const Cut &k, float r2) {
    return k.beta > 0.f ? ex2_approx(-k.beta * __log2f(fmaf(r2, k.c, 1.f))) : ex2_approx(-(r2 * k.c));
}

__device__ __forceinline__ bool within(const Cut &k, float px, float py, float pz, float qx, float qy, float qz,
                                       float &r2) {
    const float dx = px - qx, dy = py - qy, dz = pz - qz;
    r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 < k.lo) return true;
    if (r2 >= k.hi) return false;
    // explicit roundings (no contraction), so that the count and fill passes decide alike
    const double ex = (double)px - (double)qx, ey = (double)py - (double)qy, ez = (double)pz - (double)qz;
    return __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) < k.rc2;
}

// 1. per (segment, row of its tile): entries within the cut-off.
__global__ void __launch_bounds__(kT) k_asm_count(const float4 *__restrict__ pos, const int2 *__restrict__ tiles,
                                                  const int2 *__restrict__ ebi, const int4 *__restrict__ seg, Cut cut,
                                                  int32_t *__restrict__ cnt_seg) {
    __shared__ float4 s_p[kBlk];
    const int4 sg = seg[blockIdx.x];
    const int2 tl = tiles[sg.x];
    const bool valid = (int)threadIdx.x < tl.y;
    const float4 p = valid ? pos[(int64_t)tl.x + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int quarter_shift = 8 + 2 * (int)(threadIdx.x >> 5);
    int c = 0;
    for (int e = sg.y; e < sg.z; ++e) {
        const int2 bi = ebi[e];
        const int cntb = bi.y & 0xff;
        __syncthreads();
        if ((int)threadIdx.x < cntb) s_p[threadIdx.x] = pos[bi.x + threadIdx.x];
        __syncthreads();
        if (((bi.y >> quarter_shift) & 3) == 0) continue;   // no source of the block reaches this quarter
        for (int j = 0; j < cntb; ++j) {
            const float4 q = s_p[j];
            float r2;
            c += within(cut, p.x, p.y, p.z, q.x, q.y, q.z, r2) ? 1 : 0;
        }
    }
    cnt_seg[(int64_t)blockIdx.x * kT + threadIdx.x] = valid ? c : 0;
}

// 2. per tile row: segment counts -> offsets inside the row; row length and its padding;
// the unpadded total is added to *total.
__global__ void __launch_bounds__(kT) k_asm_rows(const int2 *__restrict__ tiles, const int32_t *__restrict__ tile_seg,
                                                 int32_t *__restrict__ cnt_seg, int32_t *__restrict__ rowcnt,
                                                 int64_t *__restrict__ rowlen, unsigned long long *__restrict__ total) {
    const int64_t t = blockIdx.x;
    const int2 tl = tiles[t];
    const int q = threadIdx.x;
    int run = 0;
    if (q < tl.y) {
        for (int s = tile_seg[t]; s < tile_seg[t + 1]; ++s) {
            const int v = cnt_seg[(int64_t)s * kT + q];
            cnt_seg[(int64_t)s * kT + q] = run;
            run += v;
        }
        const int64_t i = (int64_t)tl.x + q;
        rowcnt[i] = run;
        rowlen[i] = (int64_t)((run + 3) & ~3);
    }
    unsigned long long r = (unsigned long long)run;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if ((q & 31) == 0 && r) atomicAdd(total, r);
}

// 4. fill.  Warp w of a segment's CTA owns rows 32 w .. 32 w + 31 of the tile; lane r
// keeps the next free position of row r and the end of the segment's part of the row
// (the next segment's offset, or the row's count for the tile's last segment).  No
// write goes past that end; a row whose part does not end exactly there (which would
// mean the two passes decided differently) sets *err.
__global__ void __launch_bounds__(kT) k_asm_fill(const float4 *__restrict__ pos, const int2 *__restrict__ tiles,
                                                 const int2 *__restrict__ ebi, const int4 *__restrict__ seg,
                                                 const int32_t *__restrict__ tile_seg, Cut cut,
                                                 const int32_t *__restrict__ seg_off,
                                                 const int32_t *__restrict__ rowcnt,
                                                 const int64_t *__restrict__ row_ptr, int32_t *__restrict__ col,
                                                 float *__restrict__ val, unsigned *__restrict__ err) {
    const int4 sg = seg[blockIdx.x];
    const int2 tl = tiles[sg.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nrows = min(32, tl.y - 32 * w);   // rows of this warp's quarter
    if (nrows <= 0) return;
    const int64_t i = (int64_t)tl.x + 32 * w + lane;
    const bool last = (int)blockIdx.x + 1 == tile_seg[sg.x + 1];
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    int64_t next = 0, end = 0;
    if (lane < nrows) {
        t = pos[i];
        next = row_ptr[i] + seg_off[(int64_t)blockIdx.x * kT + threadIdx.x];
        end = row_ptr[i] + (last ? rowcnt[i] : seg_off[(int64_t)(blockIdx.x + 1) * kT + threadIdx.x]);
    }
    const int quarter_shift = 8 + 2 * w;
    const unsigned lt = (1u << lane) - 1u;
    for (int e = sg.y; e < sg.z; ++e) {
        const int2 bi = ebi[e];
        if (((bi.y >> quarter_shift) & 3) == 0) continue;
        const int cntb = bi.y & 0xff;
        const bool have = lane < cntb;
        const float4 q = have ? pos[bi.x + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int r = 0; r < nrows; ++r) {
            const float tx = __shfl_sync(0xffffffffu, t.x, r);
            const float ty = __shfl_sync(0xffffffffu, t.y, r);
            const float tz = __shfl_sync(0xffffffffu, t.z, r);
            float r2;
            const bool in = have && within(cut, tx, ty, tz, q.x, q.y, q.z, r2);
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (m == 0u) continue;
            const int64_t base = __shfl_sync(0xffffffffu, next, r);
            const int64_t lim = __shfl_sync(0xffffffffu, end, r);
            if (in) {
                const int64_t at = base + __popc(m & lt);
                if (at < lim) {
                    __stcs(col + at, bi.x + lane);
                    __stcs(val + at, entry(cut, r2));
                }
            }
            if (lane == r) next += __popc(m);
        }
    }
    if (lane < nrows && next != end) atomicOr(err, 1u);
}

// 5. padding entries of each row: column = the row, value 0.
__global__ void k_asm_pad(const int32_t *__restrict__ rowcnt, const int64_t *__restrict__ row_ptr, int64_t n,
                          int32_t *__restrict__ col, float *__restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t a = row_ptr[i] + rowcnt[i]; a < row_ptr[i + 1]; ++a) {
        col[a] = (int32_t)i;
        val[a] = 0.f;
    }
}

// y = A z through the CSR (binned order).  One warp per row; entry runs are 16-byte aligned.
__global__ void __launch_bounds__(kSpmvWarps * 32) k_spmv_csr(const int64_t *__restrict__ row_ptr,
                                                             const int4 *__restrict__ col4,
                                                             const float4 *__restrict__ val4,
                                                             const float *__restrict__ z, int64_t n,
                                                             float *__restrict__ y) {
    const int64_t row = (int64_t)blockIdx.x * kSpmvWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    int64_t k = (row_ptr[row] >> 2) + lane;
    const int64_t kend = row_ptr[row + 1] >> 2;
    float acc0 = 0.f, acc1 = 0.f;
    for (; k + 32 < kend; k += 64) {
        const int4 c0 = __ldcs(col4 + k), c1 = __ldcs(col4 + k + 32);
        const float4 v0 = __ldcs(val4 + k), v1 = __ldcs(val4 + k + 32);
        acc0 = fmaf(v0.x, __ldg(z + c0.x), acc0);
        acc1 = fmaf(v0.y, __ldg(z + c0.y), acc1);
        acc0 = fmaf(v0.z, __ldg(z + c0.z), acc0);
        acc1 = fmaf(v0.w, __ldg(z + c0.w), acc1);
        acc0 = fmaf(v1.x, __ldg(z + c1.x), acc0);
        acc1 = fmaf(v1.y, __ldg(z + c1.y), acc1);
        acc0 = fmaf(v1.z, __ldg(z + c1.z), acc0);
        acc1 = fmaf(v1.w, __ldg(z + c1.w), acc1);
    }
    if (k < kend) {
        const int4 c0 = __ldcs(col4 + k);
        const float4 v0 = __ldcs(val4 + k);
        acc0 = fmaf(v0.x, __ldg(z + c0.x), acc0);
        acc1 = fmaf(v0.y, __ldg(z + c0.y), acc1);
        acc0 = fmaf(v0.z, __ldg(z + c0.z), acc0);
        acc1 = fmaf(v0.w, __ldg(z + c0.w), acc1);
    }
    float acc = acc0 + acc1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[row] = acc;
}

Cut make_cut(const rbf_plan *P) {
    Cut k;
    const double s = (double)P->sigma;
    const bool imq = P->kernel == RBF_KERNEL_IMQ;
    k.rc2 = P->rc2_64 > 0.0 ? P->rc2_64 : imq ? (double)INFINITY : (13.0 * s) * (13.0 * s);
    const float f = (float)k.rc2;
    k.lo = f * (1.f - 1e-5f);
    k.hi = f * (1.f + 1e-5f);
    k.c = imq ? (float)(1.0 / (s * s)) : (float)(1.4426950408889634 / (2.0 * s * s));
    k.beta = imq ? P->beta : 0.f;
    return k;
}

}  // namespace

void assemble_csr(rbf_plan *P, int64_t max_bytes, int64_t *nnz_out, int64_t *stored_out, cudaStream_t s) {
    CsrData &M = P->csr;
    M.release();
    const PairList &pl = P->pl;
    const int64_t n = P->n;
    const Cut cut = make_cut(P);
    DevBuf<int32_t> cnt_seg, rowcnt;
    DevBuf<int64_t> rowlen;
    PBuf<int64_t> row_ptr;   // kept by the plan on success
    DevBuf<unsigned long long> total;
    cnt_seg.alloc((size_t)std::max<int64_t>(pl.nseg, 1) * kT, s);
    rowcnt.alloc(n, s);
    rowlen.alloc(n, s);
    row_ptr.alloc(n + 1, s);
    total.alloc(1, s);
    total.zero(s);
    if (pl.nseg > 0) {
        k_asm_count<<<(unsigned)pl.nseg, kT, 0, s>>>(P->pos.p, P->tiles.p, pl.ebi.p, pl.seg.p, cut, cnt_seg.p);
        RBF_LAUNCHED();
    }
    if (pl.ntiles > 0) {
        k_asm_rows<<<(unsigned)pl.ntiles, kT, 0, s>>>(P->tiles.p, pl.tile_seg.p, cnt_seg.p, rowcnt.p, rowlen.p,
                                                      total.p);
        RBF_LAUNCHED();
    }
    scan_exclusive_i64(rowlen.p, row_ptr.p, n, s);
    // algorithmic entries (the unpadded total) and stored entries (row_ptr[n])
    int64_t nnz = 0, stored = 0;
    RBF_CUDA(cudaMemcpyAsync(&nnz, total.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaMemcpyAsync(&stored, row_ptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    *nnz_out = nnz;
    *stored_out = stored;
    const double bytes = (double)stored * 8.0 + (double)(n + 1) * 8.0;
    RBF_CHECK(max_bytes <= 0 || bytes <= (double)max_bytes, RBF_ERR_OOM,
              "assembled matrix needs %.3g bytes (%lld stored entries), above the limit of %lld", bytes,
              (long long)stored, (long long)max_bytes);
    size_t free_b = 0, total_b = 0;
    RBF_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double reserve = 2.0 * 1024.0 * 1024.0 * 1024.0;
    RBF_CHECK(bytes + reserve <= (double)free_b, RBF_ERR_OOM,
              "assembled matrix needs %.3g bytes (%lld stored entries); %.3g bytes free on the device", bytes,
              (long long)stored, (double)free_b);
    RBF_CHECK(stored < ((int64_t)1 << 62), RBF_ERR_UNSUPPORTED, "too many entries");
    M.col.alloc((size_t)std::max<int64_t>(stored, 4), s);
    M.val.alloc((size_t)std::max<int64_t>(stored, 4), s);
    M.row_ptr = std::move(row_ptr);
    DevBuf<unsigned> err;
    err.alloc(1, s);
    err.zero(s);
    if (pl.nseg > 0) {
        k_asm_fill<<<(unsigned)pl.nseg, kT, 0, s>>>(P->pos.p, P->tiles.p, pl.ebi.p, pl.seg.p, pl.tile_seg.p, cut,
                                                    cnt_seg.p, rowcnt.p, M.row_ptr.p, M.col.p, M.val.p, err.p);
        RBF_LAUNCHED();
    }
    if (n > 0) {
        k_asm_pad<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(rowcnt.p, M.row_ptr.p, n, M.col.p, M.val.p);
        RBF_LAUNCHED();
    }
    unsigned herr = 0;
    RBF_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(herr), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        M.release();
        rbf_fail(RBF_ERR_CUDA, "assembly: the fill pass found other entries than the count pass");
    }
    M.nnz = nnz;
    M.stored = stored;
    M.ready = true;
}

void spmv_binned(rbf_plan *P, const float *zs, float *ys, cudaStream_t s) {
    const CsrData &M = P->csr;
    RBF_CHECK(M.ready, RBF_ERR_INVALID, "the plan has no assembled matrix (call rbf_plan_assemble first)");
    if (P->n == 0) return;
    k_spmv_csr<<<(unsigned)ceil_div(P->n, kSpmvWarps), kSpmvWarps * 32, 0, s>>>(
        M.row_ptr.p, reinterpret_cast<const int4 *>(M.col.p), reinterpret_cast<const float4 *>(M.val.p), zs, P->n,
        ys);
    RBF_LAUNCHED();
}
