// Tensor-core dense contraction used by the learned preconditioner (internal header).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

// C[m][n] = epilogue(sum_k A(m, k) B(n, k)), A(m, k) = A[m a_sr + k a_sk],
// B(n, k) = B[n b_sr + k b_sk]; one of each operand's strides must be 1.
// Epilogue: + bias[n] (if bias), ReLU (if relu), + skip[m ldskip + n] (if skip).
struct GemmArgs {
    int M = 0, N = 0, K = 0;
    int64_t a_sr = 0, a_sk = 1, b_sr = 0, b_sk = 1;
    float *C = nullptr;
    int64_t ldc = 0;
    const float *bias = nullptr;
    int relu = 0;
    const float *skip = nullptr;
    int64_t ldskip = 0;
    int kslice = 0;           // set by the launcher: K chunks per slice
    int64_t c_zstride = 0;    // set by the launcher: partial-tile stride of a K slice
};

// products: 3 = float32 operands (tf32 head x head + tail x head + head x tail),
// 2 = B exactly representable in tf32 (bf16 weights; head x B + tail x B).
// err: the context's device error word (raised when a bounded wait expires).
void gemm_tc(const GemmArgs &g, const float *A, const float *B, int products, unsigned *err, cudaStream_t s);
void gemm_tc(const GemmArgs &g, const float *A, const __nv_bfloat16 *B, int products, unsigned *err,
             cudaStream_t s);
