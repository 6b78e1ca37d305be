#pragma once
#include "common.cuh"

// Bounding box of n points spaced `stride` floats apart; host outputs.  Returns
// false when a coordinate is not finite.  Synchronises the stream.
bool bbox_host(const float *p, int64_t n, int stride, float lo[3], float hi[3], cudaStream_t s);

// Step 1 of Algorithm 1: writes 3N float4 centres and 3N targets; returns delta used.
float build_centers(const float *pts, const float *nrm, int64_t N, float delta, float target, float *centers,
                    float *targets, cudaStream_t s);
