// Shared host/device definitions of the library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/rbf.h"

struct rbf_ctx {
    int device = 0;
    int num_sms = 148;
    std::string last_error;
    // Device error word in pinned, mapped host memory: kernels with bounded waits
    // set it when a wait expires; the host reads it without a copy.
    unsigned *err_host = nullptr;
    unsigned *err_dev = nullptr;
    // Device address of the allocation-free product's file-scope scratch array,
    // resolved once when the context is created (noalloc.cu).
    float *noalloc_scratch = nullptr;
};

// noalloc.cu: with the context's device current, load the module that holds the
// allocation-free product (its scratch array is allocated by that load) and its
// kernels, and store the scratch array's device address in the context.
cudaError_t noalloc_prepare(rbf_ctx *ctx);

// The context's device error word (device pointer), and the host-side check that
// turns a raised word into a status (clearing it): kErrTimeout (a bounded wait
// expired) -> RBF_ERR_TIMEOUT, kErrRange (a value beyond a documented range) ->
// RBF_ERR_RANGE.  Kernels raise bits with atomicOr.
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrRange = 2u;
unsigned *ctx_error_word(rbf_ctx *ctx);
void ctx_check_device_error(rbf_ctx *ctx);
// probe.cu: one bounded wait that expires and raises *err (failure-detection check).
void launch_expiring_wait(unsigned *err, uint64_t limit_ns, cudaStream_t s);

// ------------------------------------------------------------------ errors
struct RbfError {
    rbf_status status;
    std::string msg;
};

[[noreturn]] inline void rbf_fail(rbf_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    throw RbfError{s, std::string(buf)};
}

#define RBF_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            (void)cudaGetLastError();                                                         \
            rbf_fail(e_ == cudaErrorMemoryAllocation ? RBF_ERR_OOM : RBF_ERR_CUDA, "%s: %s (%s:%d)", \
                     #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
        }                                                                                     \
    } while (0)

// Every kernel launch of the library is followed by RBF_LAUNCHED(): it checks the
// launch and counts it (rbf_launch_count).
void rbf_count_launch();
void rbf_count_launches(long long n);
#define RBF_LAUNCHED()             \
    do {                           \
        rbf_count_launch();        \
        RBF_CUDA(cudaGetLastError()); \
    } while (0)

#define RBF_CHECK(cond, st, ...)          \
    do {                                  \
        if (!(cond)) rbf_fail(st, __VA_ARGS__); \
    } while (0)

// ------------------------------------------------------------------ device buffers
// Device array.  Async = true: stream-ordered (cudaMallocAsync / cudaFreeAsync on
// the stream of the last allocation) for temporaries that live inside one call.
// Async = false: cudaMalloc / cudaFree, for buffers a plan keeps across calls
// (their release must not depend on a caller stream that may be gone).
template <typename T, bool Async = true>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            if (Async) cudaFreeAsync(p, s);
            else cudaFree(p);
        }
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count, cudaStream_t stream) {
        release();
        s = stream;
        n = count;
        if (count) {
            if (Async) RBF_CUDA(cudaMallocAsync((void **)&p, count * sizeof(T), stream));
            else RBF_CUDA(cudaMalloc((void **)&p, count * sizeof(T)));
        }
    }
    // grow-only reuse
    void ensure(size_t count, cudaStream_t stream) {
        if (count > n || !p) alloc(count, stream);
        s = stream;
    }
    void zero(cudaStream_t stream) {
        if (n) RBF_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), stream));
    }
};

template <typename T>
using PBuf = DevBuf<T, false>;

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t part1by2_u32(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t compact1by2_u32(uint32_t v) {
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x000003ffu;
    return v;
}

__host__ __device__ __forceinline__ uint32_t morton_host_dev(uint32_t x, uint32_t y, uint32_t z) {
    uint32_t r = 0;
    for (int b = 0; b < 10; ++b)
        r |= (((x >> b) & 1u) << (3 * b)) | (((y >> b) & 1u) << (3 * b + 1)) | (((z >> b) & 1u) << (3 * b + 2));
    return r;
}

// ------------------------------------------------------------------ primitives (scan.cu, sort.cu)
// out[i] = sum_{t<i} in[t] for i in [0, n]; out has n+1 entries (out[n] = total).
void scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of (key, val) pairs on the low `bits` bits of key.
// keys/vals are sorted in place (ping-pong buffers allocated internally).
void radix_sort_pairs(uint32_t *keys, int32_t *vals, int64_t n, int bits, cudaStream_t s);
