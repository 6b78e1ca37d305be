// Device-side view of one plan inside a batch (internal).
#pragma once
#include "plan.cuh"

struct PlanView {
    // operator
    const float4 *pos;
    const float4 *src;
    const float4 *blk_c;
    const int2 *tiles;
    const int2 *blk;
    const int32_t *ent;
    const int2 *ebi;       // per entry (block start, count | quarter codes << 8)
    const int4 *seg;
    const int32_t *tile_seg;
    const int32_t *perm;
    const int32_t *tile_of;  // tile of each binned position (this problem's own tile numbers)
    float *partial;        // nseg x kChunk partial sums (split tiles only), or null
    int64_t n;             // centres of this problem
    int64_t off;           // offset of this problem in the concatenated vectors
    int nseg, ntiles, any_split;
    float scl, R;
    // double-float residual constants
    float Ch, Cl, Rh, Rl;
    // restricted additive Schwarz (L == null: no preconditioner data)
    const float *L;
    int core, B, restricted;
    int64_t nsub;
};

// Tensor-core product of every problem of a batch (product_tc.cu): one CTA per
// (problem, segment) item; split tiles' partial sums go to each view's `partial`.  act
// (device, one flag per problem, or null): items of problems whose flag is 0 are skipped.
void product_tc_batched_launch(const PlanView *views, const int2 *items, int64_t nitems, const float *z, float *y,
                               unsigned *err, int device, cudaStream_t s, const int *act = nullptr);
// Sets the product kernels' shared-memory attribute on `device` (call before any capture).
void product_tc_prepare(int device);

// Uploads the exp2 table once per device (synchronises; call before any capture).
void residual_df_prepare(int device, cudaStream_t s);

// r = b - A~ x for every problem of a batch (double-float, each pair evaluated once for
// both rows), vectors concatenated in binned order.  items: (problem, segment) pairs;
// splits: (problem, tile) pairs of split tiles; fix: 2 x ntotal words of fixed-point
// accumulator, zeroed here on the stream.  (residual_df.cu)
void residual_df_batched(const PlanView *views, const int2 *items, int64_t nitems, const int2 *splits,
                         int64_t nsplits, const float *bs, const double *xs, double *rs, double *part_pool,
                         const int64_t *part_off, unsigned long long *fix, int64_t ntotal, int64_t max_tiles,
                         unsigned *err, int device, cudaStream_t s);
// tile_of[i] = the tile holding binned position i (tiles of one plan)
void tile_of_launch(const int2 *tiles, int64_t ntiles, int32_t *tile_of, cudaStream_t s);
