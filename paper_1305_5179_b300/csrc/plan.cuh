// The matrix-free operator over a fixed set of centres (internal).
#pragma once
#include "common.cuh"

constexpr int kBlk = 32;      // sources per block (one warp stages one block)
constexpr int kChunk = 128;   // targets per tile (4 per lane of a warp, as 2 packed pairs)
constexpr int kSymMaxEntriesPerTile = 128;   // the symmetric product is used below this mean list length

// A list of (target tile, source block) work: entries of a tile are contiguous,
// split into segments (one CTA each) when there are too few tiles to fill the GPU.
// A tile whose list is longer than the segment length is split over several
// CTAs (segments); a tile with a single segment writes its outputs directly,
// the others write partial sums that a second kernel adds in segment order.
struct PairList {
    int64_t ntiles = 0;
    int64_t len = 0;
    int64_t nseg = 0;
    int seglen = 0;
    bool any_split = false;      // some tile has more than one segment
    PBuf<int32_t> off;           // ntiles + 1
    PBuf<int32_t> ent;           // len; bit 31 set = pair-wise cut-off test needed
    PBuf<int2> ebi;              // len; (start, count | 2-bit codes of the tile's target quarters << 8
                                 //       | bit 31 of ent) of the entry's block
    PBuf<int4> seg;              // (tile, e0, e1, 1 if the tile has this one segment only)
    PBuf<int32_t> tile_seg;      // ntiles + 1: segments of tile t are [tile_seg[t], tile_seg[t+1])
};

struct SchwarzData {
    bool ready = false;
    int core = 0, block = 0, restricted = 1;
    float shift = 0.f;
    int64_t nblocks = 0;
    PBuf<float> L;               // nblocks x block x block, row-major lower factor
    PBuf<float> shift_used;      // nblocks
    PBuf<int32_t> failed;        // nblocks (1 = factorisation failed, block acts as identity)
};

struct GridCache {
    bool valid = false;
    rbf_grid g{};
    int64_t bricks[3] = {0, 0, 0};
    int blog[3] = {3, 2, 2};     // brick of 2^blog nodes per axis (128 in all)
    int qlog[3] = {2, 1, 2};     // its quarters of 2^qlog nodes per axis (32 in all)
    PairList pl;
};

// Assembled truncated matrix (CSR in binned order, rows padded to multiples of 4 entries).
struct CsrData {
    bool ready = false;
    int64_t nnz = 0;             // entries within the cut-off
    int64_t stored = 0;          // with the padding (row_ptr[n])
    PBuf<int64_t> row_ptr;       // n + 1
    PBuf<int32_t> col;           // stored
    PBuf<float> val;             // stored
    void release() {
        ready = false;
        nnz = stored = 0;
        row_ptr.release();
        col.release();
        val.release();
    }
};

struct rbf_plan {
    rbf_ctx *ctx = nullptr;
    int device = 0;               // the context's device (release does not read the context)
    int64_t n = 0;
    float sigma = 0.f, k = 0.f;
    int cells_per_cutoff = 1, levels = 3, nbits = 0;
    int product = RBF_PRODUCT_TC;   // kernel of the float32 product and grid evaluation
    int kernel = RBF_KERNEL_GAUSSIAN;
    float beta = 0.f;               // inverse multiquadric exponent
    float cell_edge = 0.f;          // requested cell edge (0: the default rule)
    double hc = 0.0;                // cell edge used
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    float inv = 0.f;          // fine cells per unit length
    int cdim = 0;             // cells per axis in the cell table (2^(nbits - levels))
    float rc = 0.f;           // cut-off radius used for box culling (k sigma, or the dense zero radius)
    float scl = 0.f;          // sqrt(log2(e) / (2 sigma^2)): scaled units where phi = 2^(-|d|^2)
    float R = 0.f;            // scaled squared cut-off (k^2 log2(e) / 2), +inf when untruncated
    double rc2_64 = 0.0;      // (k sigma)^2 in double, 0 = untruncated
    double inv2s2_64 = 0.0;   // 1 / (2 sigma^2) in double
    int64_t ncells = 0, nblk = 0, nchk = 0;
    int64_t pairs = -1;       // algorithmic pairs, once counted

    PBuf<int32_t> perm;        // binned position -> caller index
    PBuf<uint32_t> keys;       // sorted Morton keys
    PBuf<int32_t> cell_start, cell_end;
    PBuf<int32_t> cell_blk;    // ncells + 1: blocks of cell c are [cell_blk[c], cell_blk[c+1])
    PBuf<float4> pos;          // binned positions (x, y, z, 0)
    PBuf<int2> blk;            // (start, count)
    PBuf<float4> blk_c;        // block centre (x, y, z) and overflow guard (32 / scaled radius)^2
    PBuf<float4> blk_lo, blk_hi;
    PBuf<float4> src;          // per binned source: (2 s_x, 2 s_y, 2 s_z, -|s|^2), s = scaled offset to its block centre
    PBuf<int2> tiles;            // target tiles: (start, count), runs of <= kChunk per cell
    PBuf<float4> chk_lo, chk_hi;
    PairList pl;
    // Symmetric form of the product (tensor-core Gaussian plans whose pair list averages
    // fewer than kSymMaxEntriesPerTile entries per tile): the entries (T, b) of pl
    // whose block lies in tile T itself ("diagonal": T's rows only) or in a later tile
    // ("upper", ebi.y bit 16: T's rows and, transposed, the block's rows); entries whose
    // block lies in an earlier tile are left out - the other side takes them.
    bool sym_ready = false;
    PairList sym;
    PBuf<int32_t> tile_of;       // n: tile holding binned position i
    int64_t sym_upper = 0;       // upper entries
    PBuf<int32_t> sym_src;       // sym_upper: upper entry indices ordered by block (stable)
    PBuf<int32_t> sym_bstart, sym_bend;   // nblk + 1: block b's upper entries [start, end) in sym_src
    PBuf<float> colpart;         // sym.len x kBlk: per upper entry, the block's transposed partial sums

    // work vectors (binned order)
    PBuf<float> zs, ys;
    PBuf<float> partial;
    PBuf<double> xd, rd;

    SchwarzData sz;
    GridCache grid;
    CsrData csr;
    // learned preconditioner work space
    PBuf<float> mlp_x, mlp_y, mlp_n;
    PBuf<int32_t> mlp_bad;
};

// plan.cu
// binning_only: stop after the sorted positions and the cell table (no blocks, tiles
// or pair list).
void plan_build(rbf_plan *P, const float4 *centers, cudaStream_t s, bool binning_only = false);
// Copy of m points (float4, w cleared) in the order of their keys on the plan's grid
// (points outside the grid clamp to its border cells).
void plan_sorted_copy(const rbf_plan *P, const float4 *pts, int64_t m, float4 *sorted, cudaStream_t s);
// Pair list of target tiles given by boxes (lo, hi per tile; qlo, qhi per quarter of
// 32 targets, 4 per tile) against the plan's source blocks.
void build_pairlist(rbf_plan *P, const float4 *tlo, const float4 *thi, const float4 *qlo, const float4 *qhi,
                    int64_t ntiles, PairList &pl, cudaStream_t s);
// (Re)cut a built pair list into segments of at most seglen entries.
void segment_pairlist(rbf_plan *P, PairList &pl, int64_t seglen, cudaStream_t s);
// The same cut into caller-owned arrays (the pair list itself is not modified).
void segment_into(rbf_plan *P, const PairList &pl, int64_t seglen, PBuf<int4> &seg, PBuf<int32_t> &tile_seg,
                  int64_t &nseg, bool &any_split, cudaStream_t s);
void permute_to_binned_f32(const rbf_plan *P, const float *in, float *out, cudaStream_t s);
void permute_to_binned_f64_to_f32(const rbf_plan *P, const double *in, float *out, cudaStream_t s);
void permute_to_binned_f64(const rbf_plan *P, const double *in, double *out, cudaStream_t s);
void permute_from_binned_f32(const rbf_plan *P, const float *in, float *out, cudaStream_t s);
void permute_from_binned_f64(const rbf_plan *P, const double *in, double *out, cudaStream_t s);

// plan.cu: the symmetric sub-list of P->pl (see rbf_plan::sym); called by plan_build.
void build_symmetric(rbf_plan *P, cudaStream_t s);

// matvec.cu
void matvec_binned(rbf_plan *P, const float *zs, float *ys, cudaStream_t s);
// Algorithmic pair count (cached on the plan).
int64_t count_pairs(rbf_plan *P, cudaStream_t s);
// Pairs the tensor-core product evaluates (see rbf_count_candidate_pairs).
int64_t count_candidates(rbf_plan *P, cudaStream_t s);
// the same over any pair list; tiles == nullptr counts kChunk slots per tile (grid bricks)
int64_t count_candidates_list(const PairList &pl, const int2 *tiles, cudaStream_t s);
// r = b - A~ x in float64 (binned order); counts pairs when cnt != nullptr (device int64).
void residual_binned_f64(rbf_plan *P, const float *bs, const double *xs, double *rs,
                         unsigned long long *cnt, cudaStream_t s);
// residual_df.cu: the same residual in double-float arithmetic on the float32 pipes.
void residual_binned_df(rbf_plan *P, const float *bs, const double *xs, double *rs, cudaStream_t s);
// dispatch on rbf_residual_mode
// (inverse multiquadric plans always take the float64 kernel)
inline void residual_binned(rbf_plan *P, int mode, const float *bs, const double *xs, double *rs, cudaStream_t s) {
    if (mode == RBF_RESIDUAL_F64 || P->kernel == RBF_KERNEL_IMQ)
        residual_binned_f64(P, bs, xs, rs, nullptr, s);
    else
        residual_binned_df(P, bs, xs, rs, s);
}

// schwarz.cu
void schwarz_setup(rbf_plan *P, const rbf_schwarz_params &p, int64_t *failed_host, cudaStream_t s);
// z = M^-1 v, binned order; v given as float64 (vd) or float32 (vf), exactly one non-null.
void schwarz_apply_binned(rbf_plan *P, const double *vd, const float *vf, float *z, cudaStream_t s);

// assemble.cu: the truncated matrix as CSR (Algorithm 2) and its product.  Sets *nnz and
// *stored before any size check fails (RBF_ERR_OOM when the matrix exceeds max_bytes > 0
// or the device's free memory less 2 GiB).
void assemble_csr(rbf_plan *P, int64_t max_bytes, int64_t *nnz, int64_t *stored, cudaStream_t s);
void spmv_binned(rbf_plan *P, const float *zs, float *ys, cudaStream_t s);

// grid.cu
void eval_grid(rbf_plan *P, const double *weights, const rbf_grid &g, float *f, cudaStream_t s);
int64_t count_grid_pairs(rbf_plan *P, const rbf_grid &g, cudaStream_t s);
int64_t count_grid_candidates(rbf_plan *P, const rbf_grid &g, cudaStream_t s);

// batch.cu
rbf_batch *batch_create(rbf_ctx *ctx, rbf_plan *const *plans, int nplans, cudaStream_t s);
// act (device, one flag per problem, or null): problems whose flag is 0 are skipped
void batch_matvec_binned(rbf_batch *Bt, const float *z, float *y, cudaStream_t s, const int *act = nullptr);
rbf_status batch_solve(rbf_batch *Bt, const float *b, const rbf_solve_params &p, double *x, rbf_report *reps,
                       rbf_batch_stats *stats, cudaStream_t s);
int batch_autotune(rbf_batch *Bt, const float *b, const rbf_solve_params &p, const int *cands, int ncand,
                   double *scores, cudaStream_t s);
int64_t batch_size(const rbf_batch *Bt);
void batch_destroy(rbf_batch *Bt);
rbf_ctx *batch_ctx(rbf_batch *Bt);
void batch_gather_f32(rbf_batch *Bt, const float *in, float *out, cudaStream_t s);
void batch_scatter_f32(rbf_batch *Bt, const float *in, float *out, cudaStream_t s);

// mlp.cu
int64_t mlp_nparams();
rbf_mlp *mlp_create(rbf_ctx *ctx, const float *host_params, cudaStream_t s);
void mlp_destroy(rbf_mlp *M);
rbf_ctx *mlp_ctx(rbf_mlp *M);
void mlp_get_params(rbf_mlp *M, float *host, cudaStream_t s);
void mlp_get_grad(rbf_mlp *M, float *host, cudaStream_t s);
void mlp_forward(rbf_mlp *M, const float *X, int64_t rows, float *Y, int bf16, cudaStream_t s);
double mlp_loss_grad(rbf_mlp *M, const float *X, const float *T, int rows, bool want_grad, cudaStream_t s);
void mlp_adam_step(rbf_mlp *M, float lr, cudaStream_t s);
int64_t mlp_make_data(rbf_plan *P, float lambda, const int32_t *block_ids, const float *R, int64_t ns, float *X,
                      float *Y, cudaStream_t s);
int64_t mlp_apply(rbf_mlp *M, rbf_plan *P, float lambda, int core, const double *vd, float *z, cudaStream_t s);

// isosurface.cu: returns the triangle count; writes the triangles when tri != nullptr
// and capacity is enough
int64_t isosurface(rbf_ctx *ctx, const float *f, const rbf_grid &g, float iso, const float4 *pts, int64_t npts,
                   float band, float *tri, int64_t capacity, cudaStream_t s);

// density.cu
void density_measures(rbf_ctx *ctx, const float4 *pts, int64_t n, const float4 *probes, int64_t m, float cell,
                      float *nn, rbf_density *out, cudaStream_t s);

// fgmres.cu
rbf_status fgmres_solve(rbf_plan *P, const float *b_caller, const rbf_solve_params &p, double *x_caller,
                        rbf_report *rep, cudaStream_t s);
