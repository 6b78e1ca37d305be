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

// Runs of at most `len` consecutive binned centres counted from each cell start:
// source blocks (32), target tiles (128) and k-d chunks (4096) are such runs.
__global__ void k_cell_nruns(const int32_t *__restrict__ start, const int32_t *__restrict__ end, int64_t ncells,
                             int len, int32_t *__restrict__ nr) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int m = end[c] - start[c];
    nr[c] = (m + len - 1) / len;
}

__global__ void k_fill_runs(const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                            const int32_t *__restrict__ cell_run, int64_t ncells, int len, int2 *__restrict__ run) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int s = start[c], m = end[c] - s, r0 = cell_run[c];
    for (int k = 0; k * len < m; ++k) run[r0 + k] = make_int2(s + k * len, min(len, m - k * len));
}

// k-d refinement of one run of <= kKdMax centres of a cell: recursive splits
// along the axis of the largest float32 extent (first of x, y, z on ties); the
// left part takes the u * ceil(ceil(len/u)/2) smallest coordinates (u = kChunk
// above kChunk centres, kBlk below; ties keep the current order), so runs of
// kChunk and kBlk counted from the run start are subtrees.  Every level is one
// bitonic sort of (segment, coordinate, position) keys in shared memory.
constexpr int kKdMax = 4096;
constexpr int kKdThreads = 512;
constexpr int kKdMaxSeg = kKdMax / kBlk + 8;

__device__ __forceinline__ uint32_t ordered_bits(float v) {
    uint32_t u = __float_as_uint(v + 0.0f);   // -0 -> +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void __launch_bounds__(kKdThreads) k_kd_refine(const int2 *__restrict__ chunks, float4 *__restrict__ pos,
                                                          int32_t *__restrict__ perm, uint32_t *__restrict__ keys) {
    extern __shared__ unsigned long long kd_sm[];
    unsigned long long *skey = kd_sm;                         // kKdMax
    float *sx = reinterpret_cast<float *>(skey + kKdMax);     // kKdMax each
    float *sy = sx + kKdMax;
    float *sz = sy + kKdMax;
    uint16_t *ord = reinterpret_cast<uint16_t *>(sz + kKdMax);
    uint16_t *ord2 = ord + kKdMax;
    __shared__ int2 seg[kKdMaxSeg];
    __shared__ int segaxis[kKdMaxSeg];
    __shared__ int nseg, busy;

    const int2 ch = chunks[blockIdx.x];
    const int s0 = ch.x, m = ch.y;
    if (m <= kBlk) return;   // a single leaf: nothing to reorder
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = kKdThreads / 32;
    for (int i = tid; i < m; i += kKdThreads) {
        float4 p = pos[s0 + i];
        sx[i] = p.x;
        sy[i] = p.y;
        sz[i] = p.z;
        ord[i] = (uint16_t)i;
    }
    int M = 1;
    while (M < m) M <<= 1;
    if (tid == 0) {
        nseg = 1;
        seg[0] = make_int2(0, m);
    }
    __syncthreads();
    for (int level = 0; level < 32; ++level) {
        if (tid == 0) {
            int b = 0;
            for (int g = 0; g < nseg; ++g) b |= seg[g].y > kBlk;
            busy = b;
        }
        __syncthreads();
        if (!busy) break;
        // axis of every segment that is still split
        for (int g = warp; g < nseg; g += nwarp) {
            int2 sgm = seg[g];
            int ax = -1;
            if (sgm.y > kBlk) {
                float mn0 = INFINITY, mn1 = INFINITY, mn2 = INFINITY, mx0 = -INFINITY, mx1 = -INFINITY, mx2 = -INFINITY;
                for (int i = sgm.x + lane; i < sgm.x + sgm.y; i += 32) {
                    int o = ord[i];
                    mn0 = fminf(mn0, sx[o]); mx0 = fmaxf(mx0, sx[o]);
                    mn1 = fminf(mn1, sy[o]); mx1 = fmaxf(mx1, sy[o]);
                    mn2 = fminf(mn2, sz[o]); mx2 = fmaxf(mx2, sz[o]);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    mn0 = fminf(mn0, __shfl_xor_sync(0xffffffffu, mn0, o));
                    mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
                    mn1 = fminf(mn1, __shfl_xor_sync(0xffffffffu, mn1, o));
                    mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
                    mn2 = fminf(mn2, __shfl_xor_sync(0xffffffffu, mn2, o));
                    mx2 = fmaxf(mx2, __shfl_xor_sync(0xffffffffu, mx2, o));
                }
                float e0 = __fsub_rn(mx0, mn0), e1 = __fsub_rn(mx1, mn1), e2 = __fsub_rn(mx2, mn2);
                ax = 0;
                float best = e0;
                if (e1 > best) { ax = 1; best = e1; }
                if (e2 > best) ax = 2;
            }
            if (lane == 0) segaxis[g] = ax;
        }
        __syncthreads();
        // keys (segment, coordinate, position); positions past m sort last
        for (int g = warp; g < nseg; g += nwarp) {
            int2 sgm = seg[g];
            int ax = segaxis[g];
            const float *col = ax == 0 ? sx : (ax == 1 ? sy : sz);
            for (int i = sgm.x + lane; i < sgm.x + sgm.y; i += 32) {
                unsigned long long cb = ax >= 0 ? ordered_bits(col[ord[i]]) : 0u;
                skey[i] = ((unsigned long long)g << 44) | (cb << 12) | (unsigned long long)i;
            }
        }
        for (int i = m + tid; i < M; i += kKdThreads) skey[i] = ~0ull;
        __syncthreads();
        for (int k = 2; k <= M; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < M; i += kKdThreads) {
                    int ixj = i ^ j;
                    if (ixj > i) {
                        unsigned long long a = skey[i], b = skey[ixj];
                        bool up = (i & k) == 0;
                        if ((a > b) == up) {
                            skey[i] = b;
                            skey[ixj] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = tid; i < m; i += kKdThreads) ord2[i] = ord[skey[i] & 0xfffu];
        __syncthreads();
        for (int i = tid; i < m; i += kKdThreads) ord[i] = ord2[i];
        if (tid == 0) {
            int2 tmp[kKdMaxSeg];
            int nn = 0;
            for (int g = 0; g < nseg; ++g) {
                int2 sgm = seg[g];
                if (sgm.y > kBlk) {
                    int u = sgm.y > kChunk ? kChunk : kBlk;
                    int left = u * ((((sgm.y + u - 1) / u) + 1) / 2);
                    tmp[nn++] = make_int2(sgm.x, left);
                    tmp[nn++] = make_int2(sgm.x + left, sgm.y - left);
                } else {
                    tmp[nn++] = sgm;
                }
            }
            for (int g = 0; g < nn; ++g) seg[g] = tmp[g];
            nseg = nn;
        }
        __syncthreads();
    }
    // apply the order to the binned arrays (read everything, then write)
    float4 pv[kKdMax / kKdThreads];
    int32_t iv[kKdMax / kKdThreads];
    uint32_t kv[kKdMax / kKdThreads];
    for (int r = 0; r < kKdMax / kKdThreads; ++r) {
        int i = tid + r * kKdThreads;
        if (i < m) {
            int o = ord[i];
            pv[r] = pos[s0 + o];
            iv[r] = perm[s0 + o];
            kv[r] = keys[s0 + o];
        }
    }
    __syncthreads();
    for (int r = 0; r < kKdMax / kKdThreads; ++r) {
        int i = tid + r * kKdThreads;
        if (i < m) {
            pos[s0 + i] = pv[r];
            perm[s0 + i] = iv[r];
            keys[s0 + i] = kv[r];
        }
    }
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

// One warp per target tile (a run of <= kChunk binned centres): its box, and the
// boxes of its four quarters of 32 targets (an empty quarter gets lo > hi).
__global__ void k_chunk_boxes(const float4 *__restrict__ pos, const int2 *__restrict__ tiles, int64_t nchk,
                              float4 *__restrict__ lo, float4 *__restrict__ hi, float4 *__restrict__ qlo,
                              float4 *__restrict__ qhi) {
    int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (t >= nchk) return;
    const int2 tl = tiles[t];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int u = 0; u < kChunk / 32; ++u) {
        const int q = lane + 32 * u;
        float a[3] = {INFINITY, INFINITY, INFINITY}, b[3] = {-INFINITY, -INFINITY, -INFINITY};
        if (q < tl.y) {
            float4 p = pos[tl.x + q];
            a[0] = b[0] = p.x; a[1] = b[1] = p.y; a[2] = b[2] = p.z;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d)
            for (int o = 16; o > 0; o >>= 1) {
                a[d] = fminf(a[d], __shfl_xor_sync(0xffffffffu, a[d], o));
                b[d] = fmaxf(b[d], __shfl_xor_sync(0xffffffffu, b[d], o));
            }
        if (lane == 0) {
            qlo[4 * t + u] = make_float4(a[0], a[1], a[2], 0.f);
            qhi[4 * t + u] = make_float4(b[0], b[1], b[2], 0.f);
        }
        for (int d = 0; d < 3; ++d) {
            mn[d] = fminf(mn[d], a[d]);
            mx[d] = fmaxf(mx[d], b[d]);
        }
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
    ns[t] = c > 0 ? (int32_t)((c - 1) / seglen + 1) : 0;   // empty tiles have no segment
}

__global__ void k_seg_fill(const int32_t *__restrict__ off, const int32_t *__restrict__ tseg, int64_t ntiles,
                           int seglen, int4 *__restrict__ seg) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int64_t e0 = off[t], e1 = off[t + 1];
    int s0 = tseg[t];
    int single = (tseg[t + 1] - s0) == 1;
    for (int64_t k = 0; e0 + k * seglen < e1; ++k) {
        int64_t a = e0 + k * seglen, b = a + seglen < e1 ? a + seglen : e1;
        seg[s0 + k] = make_int4((int)t, (int)a, (int)b, single);
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

namespace {
// Per entry, for the tensor-core product: its block (start, count) and, for each
// quarter u of 32 targets of the tile, a 2-bit code at bit 8 + 2u of the count word:
// 0 = no pair of the quarter and the block within the cut-off, 1 = pair-wise test
// needed, 2 = every pair within it (the box tests of the tile list, on the quarter's
// box).  Bit 31 keeps the tile's own flag.  One warp per tile.
__global__ void k_pl_expand(CellGridArgs g, const int32_t *__restrict__ off, int64_t ntiles,
                            const int32_t *__restrict__ ent, const int2 *__restrict__ blk,
                            const float4 *__restrict__ blo, const float4 *__restrict__ bhi,
                            const float4 *__restrict__ qlo, const float4 *__restrict__ qhi, int2 *__restrict__ ebi) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    float4 ql[4], qh[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        ql[u] = qlo[4 * t + u];
        qh[u] = qhi[4 * t + u];
    }
    for (int e = off[t] + lane; e < off[t + 1]; e += 32) {
        const int v = ent[e];
        const int b = v & 0x7fffffff;
        const int2 bi = blk[b];
        const float4 l = blo[b], h = bhi[b];
        int codes = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!(ql[u].x <= qh[u].x)) continue;          // empty quarter
            const float gx = fmaxf(0.f, fmaxf(l.x - qh[u].x, ql[u].x - h.x));
            const float gy = fmaxf(0.f, fmaxf(l.y - qh[u].y, ql[u].y - h.y));
            const float gz = fmaxf(0.f, fmaxf(l.z - qh[u].z, ql[u].z - h.z));
            if (!(gx * gx + gy * gy + gz * gz < g.keep2)) continue;
            int c = 1;
            if (g.dense) {
                c = 2;
            } else {
                const float mx = fmaxf(h.x - ql[u].x, qh[u].x - l.x);
                const float my = fmaxf(h.y - ql[u].y, qh[u].y - l.y);
                const float mz = fmaxf(h.z - ql[u].z, qh[u].z - l.z);
                if (mx * mx + my * my + mz * mz < g.full2) c = 2;
            }
            codes |= c << (2 * u);
        }
        ebi[e] = make_int2(bi.x, bi.y | (codes << 8) | (v & (int)0x80000000));
    }
}
}  // namespace

namespace {
// Exact quarter codes for the plan's own tiles.  The box tests leave a (quarter, block)
// undecided (code 1) when the boxes straddle the cut-off; here the smallest and largest
// squared distance between the quarter's targets and the block's sources decide it: 0
// when every pair lies beyond rc^2 (1 + 1e-5), 2 when every pair lies within rc^2 (1 - 1e-5),
// else 1.  The margins exceed the float32 distance error and the tensor-core exponent's,
// so a pair's contribution does not change: only the work to find it does.  The pairwise
// loop stops as soon as the warp has seen a pair inside and a pair outside (the quarter
// stays undecided), so only quarters that turn out uniform pay the full 32 x 32 test.
// One warp per tile; the tile's targets are staged in shared memory.
constexpr int kRefWarps = 8;
__global__ void __launch_bounds__(kRefWarps * 32) k_pl_refine(const float4 *__restrict__ pos,
                                                              const int2 *__restrict__ tiles,
                                                              const int32_t *__restrict__ off, int64_t ntiles,
                                                              float lo2, float hi2, int2 *__restrict__ ebi) {
    __shared__ float4 s_t[kRefWarps][kChunk];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * kRefWarps + warp;
    if (t >= ntiles) return;
    const int2 tl = tiles[t];
    for (int q = lane; q < kChunk; q += 32)
        s_t[warp][q] = q < tl.y ? pos[tl.x + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    for (int e = off[t]; e < off[t + 1]; ++e) {
        const int2 w = ebi[e];
        const int codes = (w.y >> 8) & 0xff;
        if (((codes & 0x55) & ~(codes >> 1)) == 0) continue;     // no quarter with code 1
        const int cnt = w.y & 0xff;
        const float4 src = lane < cnt ? pos[w.x + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        int nc = codes;
        for (int q = 0; q < 4; ++q) {
            if (((codes >> (2 * q)) & 3) != 1) continue;
            const int nq = min(32, tl.y - 32 * q);
            float mn = INFINITY, mx = 0.f;
            bool mixed = false;
            for (int r0 = 0; r0 < nq && !mixed; r0 += 8) {
                for (int r = r0; r < min(nq, r0 + 8); ++r) {
                    const float4 p = s_t[warp][32 * q + r];
                    const float dx = p.x - src.x, dy = p.y - src.y, dz = p.z - src.z;
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (lane < cnt) {
                        mn = fminf(mn, d2);
                        mx = fmaxf(mx, d2);
                    }
                }
                mixed = __any_sync(0xffffffffu, mn <= hi2) && __any_sync(0xffffffffu, mx >= lo2);
            }
            if (mixed) continue;     // stays 1
            for (int o = 16; o > 0; o >>= 1) {
                mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            const int c = mn > hi2 ? 0 : (mx < lo2 ? 2 : 1);
            nc = (nc & ~(3 << (2 * q))) | (c << (2 * q));
        }
        if (lane == 0 && nc != codes) ebi[e].y = (w.y & ~(0xff << 8)) | (nc << 8);
        __syncwarp();
    }
}
}  // namespace

// ------------------------------------------------------------------ symmetric sub-list
namespace {

__global__ void k_tile_of_pos(const int2 *__restrict__ tiles, int32_t *__restrict__ tile_of) {
    const int2 tl = tiles[blockIdx.x];
    for (int q = threadIdx.x; q < tl.y; q += blockDim.x) tile_of[tl.x + q] = (int32_t)blockIdx.x;
}

__device__ __forceinline__ int entry_tile(const int32_t *__restrict__ ent, const int2 *__restrict__ blk,
                                          const int32_t *__restrict__ tile_of, int64_t e) {
    return tile_of[blk[ent[e] & 0x7fffffff].x];
}

// one warp per tile: entries of tile t whose block lies in tile t or a later one
__global__ void k_sym_count(const int32_t *__restrict__ off, int64_t ntiles, const int32_t *__restrict__ ent,
                            const int2 *__restrict__ blk, const int32_t *__restrict__ tile_of,
                            int32_t *__restrict__ cnt) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    int c = 0;
    for (int64_t e0 = off[t]; e0 < off[t + 1]; e0 += 32) {
        const int64_t e = e0 + lane;
        const bool keep = e < off[t + 1] && entry_tile(ent, blk, tile_of, e) >= t;
        c += __popc(__ballot_sync(0xffffffffu, keep));
    }
    if (lane == 0) cnt[t] = c;
}

// the kept entries in their order; upper ones flagged in bit 16 of ebi.y
__global__ void k_sym_fill(const int32_t *__restrict__ off, int64_t ntiles, const int32_t *__restrict__ ent,
                           const int2 *__restrict__ ebi, const int2 *__restrict__ blk,
                           const int32_t *__restrict__ tile_of, const int32_t *__restrict__ soff,
                           int32_t *__restrict__ sent, int2 *__restrict__ sebi) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    int64_t w = soff[t];
    for (int64_t e0 = off[t]; e0 < off[t + 1]; e0 += 32) {
        const int64_t e = e0 + lane;
        const int tb = e < off[t + 1] ? entry_tile(ent, blk, tile_of, e) : -1;
        const bool keep = tb >= t;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int64_t d = w + __popc(m & ((1u << lane) - 1u));
            sent[d] = ent[e];
            int2 v = ebi[e];
            if (tb > t) v.y |= 1 << 16;
            sebi[d] = v;
        }
        w += __popc(m);
    }
}

// sort keys: the block of an upper entry, or nblk (sorts after every block) otherwise
__global__ void k_sym_keys(const int32_t *__restrict__ sent, const int2 *__restrict__ sebi, int64_t len,
                           uint32_t nblk, uint32_t *__restrict__ keys, int32_t *__restrict__ vals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    keys[e] = (sebi[e].y >> 16) & 1 ? (uint32_t)(sent[e] & 0x7fffffff) : nblk;
    vals[e] = (int32_t)e;
}

}  // namespace

void build_symmetric(rbf_plan *P, cudaStream_t s) {
    const PairList &pl = P->pl;
    PairList &sy = P->sym;
    const int64_t nt = pl.ntiles;
    P->tile_of.alloc(std::max<int64_t>(P->n, 1), s);
    if (nt > 0) {
        k_tile_of_pos<<<(unsigned)nt, kChunk, 0, s>>>(P->tiles.p, P->tile_of.p);
        RBF_LAUNCHED();
    }
    sy.ntiles = nt;
    sy.off.alloc(nt + 1, s);
    DevBuf<int32_t> cnt;
    cnt.alloc(std::max<int64_t>(nt, 1), s);
    const unsigned wgrid = grid_for(nt * 32);
    if (nt > 0) {
        k_sym_count<<<wgrid, kThreads, 0, s>>>(pl.off.p, nt, pl.ent.p, P->blk.p, P->tile_of.p, cnt.p);
        RBF_LAUNCHED();
    }
    scan_exclusive_i32(cnt.p, sy.off.p, nt, s);
    int32_t len = 0;
    RBF_CUDA(cudaMemcpyAsync(&len, sy.off.p + nt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    sy.len = len;
    sy.ent.alloc(std::max<int64_t>(len, 1), s);
    sy.ebi.alloc(std::max<int64_t>(len, 1), s);
    if (nt > 0) {
        k_sym_fill<<<wgrid, kThreads, 0, s>>>(pl.off.p, nt, pl.ent.p, pl.ebi.p, P->blk.p, P->tile_of.p, sy.off.p,
                                              sy.ent.p, sy.ebi.p);
        RBF_LAUNCHED();
    }
    // segments by the rule of the full list
    int64_t want = 8LL * P->ctx->num_sms;
    int64_t seglen = len > 0 ? std::max<int64_t>(64, 2 * ceil_div((int64_t)len, std::max<int64_t>(nt, 1))) : 1;
    if (nt < want && len > 0) seglen = std::min<int64_t>(seglen, std::max<int64_t>(8, ceil_div((int64_t)len, want)));
    segment_pairlist(P, sy, seglen, s);
    // upper entries ordered by block (stable: entry order within a block), with per-block ranges
    const int64_t nblk = P->nblk;
    DevBuf<uint32_t> keys;
    DevBuf<int32_t> vals;
    keys.alloc(std::max<int64_t>(len, 1), s);
    vals.alloc(std::max<int64_t>(len, 1), s);
    if (len > 0) {
        k_sym_keys<<<grid_for(len), kThreads, 0, s>>>(sy.ent.p, sy.ebi.p, len, (uint32_t)nblk, keys.p, vals.p);
        RBF_LAUNCHED();
    }
    int bits = 1;
    while ((1LL << bits) <= nblk) ++bits;
    radix_sort_pairs(keys.p, vals.p, len, bits, s);
    P->sym_bstart.alloc(nblk + 1, s);
    P->sym_bend.alloc(nblk + 1, s);
    P->sym_bstart.zero(s);
    P->sym_bend.zero(s);
    if (len > 0) {
        k_cell_ranges<<<grid_for(len), kThreads, 0, s>>>(keys.p, len, 0, P->sym_bstart.p, P->sym_bend.p);
        RBF_LAUNCHED();
    }
    int32_t upper = 0;     // the upper entries are the ones before the first key nblk
    if (len > 0) {
        RBF_CUDA(cudaMemcpyAsync(&upper, P->sym_bstart.p + nblk, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        int32_t end_n = 0;
        RBF_CUDA(cudaMemcpyAsync(&end_n, P->sym_bend.p + nblk, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(cudaStreamSynchronize(s));
        if (end_n == 0) upper = len;   // no diagonal entry at all
    }
    P->sym_upper = upper;
    P->sym_src.alloc(std::max<int64_t>(upper, 1), s);
    if (upper > 0)
        RBF_CUDA(cudaMemcpyAsync(P->sym_src.p, vals.p, (size_t)upper * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    P->colpart.alloc((size_t)std::max<int64_t>(len, 1) * kBlk, s);
    RBF_CUDA(cudaStreamSynchronize(s));    // keys and vals are freed on return
    P->sym_ready = true;
}

void build_pairlist(rbf_plan *P, const float4 *tlo, const float4 *thi, const float4 *qlo, const float4 *qhi,
                    int64_t ntiles, PairList &pl, cudaStream_t s) {
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
    pl.ebi.alloc(std::max<int64_t>(len, 1), s);
    if (len > 0) {
        k_pl_expand<<<wgrid, kThreads, 0, s>>>(g, pl.off.p, ntiles, pl.ent.p, P->blk.p, P->blk_lo.p, P->blk_hi.p, qlo,
                                               qhi, pl.ebi.p);
        RBF_LAUNCHED();
    }

    // segments: enough independent work items to fill every SM several times, and no
    // segment much longer than the average tile (a tile whose box straddles a jump of
    // the Morton order can collect many blocks; splitting it keeps the SMs balanced)
    int64_t want = 8LL * P->ctx->num_sms;
    int64_t seglen = len > 0 ? std::max<int64_t>(64, 2 * ceil_div(len, std::max<int64_t>(ntiles, 1))) : 1;
    if (ntiles < want && len > 0) seglen = std::min<int64_t>(seglen, std::max<int64_t>(8, ceil_div(len, want)));
    segment_pairlist(P, pl, seglen, s);
}

void segment_into(rbf_plan *P, const PairList &pl, int64_t seglen, PBuf<int4> &seg, PBuf<int32_t> &tile_seg,
                  int64_t &nseg_out, bool &any_split, cudaStream_t s) {
    const int64_t ntiles = pl.ntiles;
    const int sl = (int)std::max<int64_t>(1, std::min<int64_t>(seglen, INT_MAX / 2));
    DevBuf<int32_t> cnt;
    cnt.alloc(std::max<int64_t>(ntiles, 1), s);
    tile_seg.alloc(ntiles + 1, s);
    k_seg_count<<<grid_for(ntiles), kThreads, 0, s>>>(pl.off.p, ntiles, sl, cnt.p);
    RBF_LAUNCHED();
    scan_exclusive_i32(cnt.p, tile_seg.p, ntiles, s);
    int32_t nseg = 0;
    RBF_CUDA(cudaMemcpyAsync(&nseg, tile_seg.p + ntiles, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    nseg_out = nseg;
    seg.alloc(std::max<int64_t>(nseg, 1), s);
    k_seg_fill<<<grid_for(ntiles), kThreads, 0, s>>>(pl.off.p, tile_seg.p, ntiles, sl, seg.p);
    RBF_LAUNCHED();
    // a split exists iff there are more segments than non-empty tiles
    std::vector<int32_t> offs(ntiles + 1);
    RBF_CUDA(cudaMemcpyAsync(offs.data(), pl.off.p, (ntiles + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    int64_t nonempty = 0;
    for (int64_t t = 0; t < ntiles; ++t) nonempty += offs[t + 1] > offs[t];
    any_split = nseg > nonempty;
}

void segment_pairlist(rbf_plan *P, PairList &pl, int64_t seglen, cudaStream_t s) {
    pl.seglen = (int)std::max<int64_t>(1, std::min<int64_t>(seglen, INT_MAX / 2));
    segment_into(P, pl, seglen, pl.seg, pl.tile_seg, pl.nseg, pl.any_split, s);
}

// Runs of <= len centres per cell -> run list (and the per-cell run offsets if asked).
static int64_t build_runs(rbf_plan *P, int len, PBuf<int2> &runs, PBuf<int32_t> *cell_run_out, cudaStream_t s) {
    DevBuf<int32_t> nr;
    nr.alloc(P->ncells, s);
    k_cell_nruns<<<grid_for(P->ncells), kThreads, 0, s>>>(P->cell_start.p, P->cell_end.p, P->ncells, len, nr.p);
    RBF_LAUNCHED();
    PBuf<int32_t> local;
    PBuf<int32_t> &cr = cell_run_out ? *cell_run_out : local;
    cr.alloc(P->ncells + 1, s);
    scan_exclusive_i32(nr.p, cr.p, P->ncells, s);
    int32_t total = 0;
    RBF_CUDA(cudaMemcpyAsync(&total, cr.p + P->ncells, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(cudaStreamSynchronize(s));
    runs.alloc(std::max<int32_t>(total, 1), s);
    k_fill_runs<<<grid_for(P->ncells), kThreads, 0, s>>>(P->cell_start.p, P->cell_end.p, cr.p, P->ncells, len, runs.p);
    RBF_LAUNCHED();
    if (!cell_run_out) RBF_CUDA(cudaStreamSynchronize(s));   // `local` is freed on return
    return total;
}

void plan_sorted_copy(const rbf_plan *P, const float4 *pts, int64_t m, float4 *sorted, cudaStream_t s) {
    DevBuf<uint32_t> keys;
    DevBuf<int32_t> order;
    keys.alloc(m, s);
    order.alloc(m, s);
    k_keys<<<grid_for(m), kThreads, 0, s>>>(pts, m, P->lo[0], P->lo[1], P->lo[2], P->inv,
                                            (uint32_t)((1 << P->nbits) - 1), keys.p, order.p);
    RBF_LAUNCHED();
    radix_sort_pairs(keys.p, order.p, m, 3 * P->nbits, s);
    k_gather_pos<<<grid_for(m), kThreads, 0, s>>>(pts, order.p, m, sorted);
    RBF_LAUNCHED();
}

void plan_build(rbf_plan *P, const float4 *centers, cudaStream_t s, bool binning_only) {
    const int64_t n = P->n;
    bool finite = bbox_host((const float *)centers, n, 4, P->lo, P->hi, s);
    RBF_CHECK(finite, RBF_ERR_INVALID, "non-finite centre coordinate");
    float ext[3];
    for (int d = 0; d < 3; ++d) ext[d] = P->hi[d] - P->lo[d];
    double hc;
    if (P->cell_edge > 0.f) {
        hc = (double)P->cell_edge;
    } else if (P->k > 0.f) {
        hc = (double)P->k * (double)P->sigma / (double)P->cells_per_cutoff;
    } else if (P->kernel == RBF_KERNEL_IMQ) {
        // untruncated inverse multiquadric: every pair is evaluated, 8 cells per axis suffice
        double m = std::max({(double)ext[0], (double)ext[1], (double)ext[2]});
        hc = m > 0 ? m / 8.0 : 1.0;
    } else {
        // untruncated: cells of at most 3 sigma keep blocks compact in scaled units, at least
        // max(ext)/128 keeps the fine grid within 1024 cells per axis
        double m = std::max({(double)ext[0], (double)ext[1], (double)ext[2]});
        hc = m > 0 ? std::max(std::min(m / 8.0, 3.0 * (double)P->sigma), m / 128.0) : 1.0;
    }
    P->hc = hc;
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
    } else if (P->kernel == RBF_KERNEL_IMQ) {
        // untruncated inverse multiquadric: an infinite culling radius keeps every block for
        // every target, grid nodes outside the centres' box included (the cell ranges clamp
        // before converting to integers)
        P->rc = INFINITY;
        P->rc2_64 = 0.0;
        P->R = INFINITY;
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
    if (binning_only) return;

    // 3: k-d refinement inside each cell (runs of <= kKdMax), then source blocks,
    //    target tiles and their boxes
    PBuf<int2> chunks;
    int64_t nkd = build_runs(P, kKdMax, chunks, nullptr, s);
    if (nkd > 0) {
        size_t smem = (size_t)kKdMax * (8 + 4 * 3 + 2 * 2);
        RBF_CUDA(cudaFuncSetAttribute(k_kd_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_kd_refine<<<(unsigned)nkd, kKdThreads, smem, s>>>(chunks.p, P->pos.p, P->perm.p, P->keys.p);
        RBF_LAUNCHED();
    }
    P->nblk = build_runs(P, kBlk, P->blk, &P->cell_blk, s);
    const int64_t nblk = P->nblk;
    P->blk_c.alloc(nblk, s);
    P->blk_lo.alloc(nblk, s);
    P->blk_hi.alloc(nblk, s);
    P->src.alloc(n, s);
    k_block_geom<<<grid_for(nblk * 32), kThreads, 0, s>>>(P->pos.p, P->blk.p, nblk, P->scl, P->blk_c.p, P->blk_lo.p,
                                                          P->blk_hi.p, P->src.p);
    RBF_LAUNCHED();

    // 4: target tiles and the pair list
    P->nchk = build_runs(P, kChunk, P->tiles, nullptr, s);
    P->chk_lo.alloc(P->nchk, s);
    P->chk_hi.alloc(P->nchk, s);
    DevBuf<float4> qlo, qhi;
    qlo.alloc(4 * P->nchk, s);
    qhi.alloc(4 * P->nchk, s);
    k_chunk_boxes<<<grid_for(P->nchk * 32), kThreads, 0, s>>>(P->pos.p, P->tiles.p, P->nchk, P->chk_lo.p,
                                                              P->chk_hi.p, qlo.p, qhi.p);
    RBF_LAUNCHED();
    build_pairlist(P, P->chk_lo.p, P->chk_hi.p, qlo.p, qhi.p, P->nchk, P->pl, s);
    if (P->k > 0.f && P->pl.len > 0) {
        const float rc2 = P->rc * P->rc;
        k_pl_refine<<<(unsigned)ceil_div(P->nchk, kRefWarps), kRefWarps * 32, 0, s>>>(
            P->pos.p, P->tiles.p, P->pl.off.p, P->nchk, rc2 * (1.f - 1e-5f), rc2 * (1.f + 1e-5f), P->pl.ebi.p);
        RBF_LAUNCHED();
    }
    // 5: the symmetric form of the tensor-core Gaussian product, for short lists.  Evaluating
    //    each pair once halves the MMAs and the exponentials but adds a shared-memory
    //    transpose per (warp, upper block) for the transposed sums.  Measured on B300: with
    //    39 entries per tile (the 3M-centre sphere at sigma = the spacing) the symmetric
    //    product takes 2.03 ms against 2.28; with 508 (the C2 torus) 9.92 ms against 9.43,
    //    where the transpose keeps the shared-memory pipe 91% busy.  So short lists only.
    if (P->product == RBF_PRODUCT_TC && P->kernel == RBF_KERNEL_GAUSSIAN &&
        P->pl.len < (int64_t)kSymMaxEntriesPerTile * P->pl.ntiles)
        build_symmetric(P, s);
}
