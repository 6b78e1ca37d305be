// Local solve of one restricted additive Schwarz subdomain (Sec. III.A, RASM):
// (L L^T) x = v for a B x B lower Cholesky factor L (row-major, zeros above the
// diagonal), B <= 128, by one warp of a 256-thread CTA (internal header).
//
// The factor is taken in tiles of 32 x 32, each staged in shared memory with
// coalesced loads (row i of the tile by the 32 lanes at once).  A diagonal tile is
// solved one column per step: the pivot lane scales by its reciprocal pivot, a
// shuffle broadcasts the value, the other lanes update; the tiles below (forward)
// or beside (backward) it are then applied as products.  Forward lanes read the
// staged tile by rows, backward lanes by columns (a padded row of 33 keeps both
// free of bank conflicts).  Lane l holds the entries l, 32 + l, 64 + l, 96 + l of
// the right-hand side and, on return, of the solution.
#pragma once

namespace ras {

constexpr int kTiles = 4;        // B <= 128
constexpr int kWarpsPerCta = 8;  // the apply kernels run 256-thread CTAs

// sm[i][j] = L[r0 + i][c0 + j] (0 outside B x B)
__device__ __forceinline__ void stage(const float *__restrict__ L, int B, int r0, int c0, float (*sm)[33], int lane) {
    const int col = c0 + lane;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
        const int row = r0 + i;
        sm[i][lane] = (row < B && col < B) ? L[(int64_t)row * B + col] : 0.f;
    }
    __syncwarp();
}

// B <= 32: the factor is one tile, staged once (all 32 row loads in flight) and used by
// both sweeps; the same operations in the same order as the general form below, with the
// loops fully unrolled (the apply kernels run it as a separate instantiation, so that its
// registers do not lower the general form's occupancy).
__device__ __forceinline__ void solve_block32(const float *__restrict__ L, int B, float &y, int lane,
                                              float (*sm)[33]) {
    float r[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) r[i] = (i < B && lane < B) ? L[(int64_t)i * B + lane] : 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) sm[i][lane] = r[i];
    __syncwarp();
    const float inv = lane < B ? 1.f / sm[lane][lane] : 0.f;   // this lane's pivot
    float s = lane < B ? y : 0.f;
#pragma unroll
    for (int c = 0; c < 32; ++c) {                       // forward: L w = v
        const float wc = __shfl_sync(0xffffffffu, s * inv, c);
        if (lane == c) s = wc;
        else if (lane > c) s = fmaf(-sm[lane][c], wc, s);
    }
#pragma unroll
    for (int c = 31; c >= 0; --c) {                      // backward: L^T x = w
        const float xc = __shfl_sync(0xffffffffu, s * inv, c);
        if (lane == c) s = xc;
        else if (lane < c) s = fmaf(-sm[c][lane], xc, s);
    }
    y = s;
    __syncwarp();
}

__device__ __forceinline__ void solve_block32(const float *__restrict__ L, int B, float &y, int lane) {
    __shared__ float s_tile1[kWarpsPerCta][32][33];
    solve_block32(L, B, y, lane, s_tile1[threadIdx.x >> 5]);
}

__device__ __forceinline__ void solve_block(const float *__restrict__ L, int B, float (&y)[kTiles], int lane) {
    __shared__ float s_tile[kWarpsPerCta][32][33];
    float(*sm)[33] = s_tile[threadIdx.x >> 5];
    const int T = (B + 31) >> 5;
    // forward: L w = v
#pragma unroll
    for (int t = 0; t < kTiles; ++t) {
        if (t >= T) break;
        const int r = 32 * t + lane;
        const float inv = r < B ? 1.f / L[(int64_t)r * B + r] : 0.f;   // this lane's pivot
        stage(L, B, 32 * t, 32 * t, sm, lane);
        float s = y[t];
        for (int c = 0; c < 32 && 32 * t + c < B; ++c) {
            const float wc = __shfl_sync(0xffffffffu, s * inv, c);     // pivot lane c
            if (lane == c) s = wc;
            else if (lane > c) s = fmaf(-sm[lane][c], wc, s);
        }
        y[t] = s;
        __syncwarp();
#pragma unroll
        for (int u = t + 1; u < kTiles; ++u) {
            if (u >= T) break;
            stage(L, B, 32 * u, 32 * t, sm, lane);
            float acc = 0.f;
#pragma unroll 8
            for (int c = 0; c < 32; ++c) acc = fmaf(sm[lane][c], __shfl_sync(0xffffffffu, s, c), acc);
            y[u] -= acc;
            __syncwarp();
        }
    }
    // backward: L^T x = w
#pragma unroll
    for (int t = kTiles - 1; t >= 0; --t) {
        if (t >= T) continue;
        const int col = 32 * t + lane;
        const float inv = col < B ? 1.f / L[(int64_t)col * B + col] : 0.f;   // this lane's pivot
        stage(L, B, 32 * t, 32 * t, sm, lane);
        float s = y[t];
        for (int c = min(31, B - 1 - 32 * t); c >= 0; --c) {
            const float xc = __shfl_sync(0xffffffffu, s * inv, c);     // pivot lane c
            if (lane == c) s = xc;
            else if (lane < c) s = fmaf(-sm[c][lane], xc, s);
        }
        y[t] = s;
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kTiles; ++u) {
            if (u >= t) break;
            stage(L, B, 32 * t, 32 * u, sm, lane);
            float acc = 0.f;
#pragma unroll 8
            for (int c = 0; c < 32; ++c) acc = fmaf(sm[c][lane], __shfl_sync(0xffffffffu, s, c), acc);
            y[u] -= acc;
            __syncwarp();
        }
    }
}

}  // namespace ras
