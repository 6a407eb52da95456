// Shared helpers of the BAE library: error reporting, complex arithmetic,
// launch checks. Device code targets sm_103a only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>

#include "../../include/bae.h"

namespace bae {

// Error carried from deep inside the library to the C ABI boundary, where
// it becomes a return code and the thread-local message.
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);

// Launch bookkeeping: every kernel launch of the library goes through
// BAE_LAUNCH, which counts it and, while profiling is on, brackets it with
// CUDA events on its stream (per-kernel device time, see bae_profile_*).
void count_launch();
void count_launches(long long k);   // k kernels launched at once (a graph)
void capture_begin();               // launches until capture_end() are counted, not timed
long long capture_end();            // returns the number counted
void prof_push(const char* name, cudaStream_t st);
void prof_pop(cudaStream_t st);

// Stream-ordered device allocation from the device's default memory pool
// (kept pooled: freed blocks are reused without returning to the driver).
void* dev_alloc(size_t bytes, cudaStream_t st);
// throws BAE_ERR_OOM when an injected allocation cap (bae_inject_fault)
// refuses an allocation of this size
void alloc_check(size_t bytes);
void dev_free(void* p, cudaStream_t st);
template <typename T>
T* dev_alloc_n(long long n, cudaStream_t st) {
    return static_cast<T*>(dev_alloc((size_t)(n > 0 ? n : 1) * sizeof(T), st));
}

#define BAE_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            int c_ = (e_ == cudaErrorMemoryAllocation) ? BAE_ERR_OOM : BAE_ERR_CUDA; \
            throw ::bae::Error(c_, std::string(#call) + ": " + cudaGetErrorString(e_) \
                                       + " (" __FILE__ ":" + std::to_string(__LINE__) + ")"); \
        }                                                                           \
    } while (0)

#define BAE_CHECK_LAUNCH() BAE_CUDA(cudaGetLastError())

// Restores the calling thread's current CUDA device on scope exit: every
// entry point switches to its context's device and leaves the caller's
// choice as it found it.
struct DeviceGuard {
    int saved = -1;
    DeviceGuard() {
        if (cudaGetDevice(&saved) != cudaSuccess) {
            cudaGetLastError();
            saved = -1;
        }
    }
    ~DeviceGuard() {
        if (saved >= 0) cudaSetDevice(saved);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Whether p is memory the kernels of the current device may read or write:
// true for device memory of the current device and for managed memory,
// false for host memory (pageable or pinned), which the callers stage.
// Device memory of another GPU is rejected (BAE_ERR_INVALID_ARG): the
// kernels of this device cannot be assumed to reach it.
bool is_device_ptr(const void* p);

#define BAE_LAUNCH(name, st, ...)            \
    do {                                     \
        ::bae::prof_push((name), (st));      \
        __VA_ARGS__;                         \
        ::bae::prof_pop(st);                 \
        ::bae::count_launch();               \
        BAE_CHECK_LAUNCH();                  \
    } while (0)

#define BAE_REQUIRE(cond, code, msg)                        \
    do {                                                    \
        if (!(cond)) throw ::bae::Error((code), (msg));     \
    } while (0)

// ----------------------------------------------------------- complex types
template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename Cplx<T>::type;

template <typename C> __device__ __forceinline__ C cmake(decltype(C::x) a, decltype(C::x) b) {
    C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    return cmake<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return cmake<C>(a.x * s, a.y * s); }

// read-only cached load of one complex value
template <typename C> __device__ __forceinline__ C ldg_c(const C* p) { return __ldg(p); }

// element type of the potential written by the last convolution pass, and
// the conversion to it (float32 -> float, float64 -> double)
template <typename T> struct OutOf { using type = T; };
__device__ __forceinline__ float to_out(float v) { return v; }
__device__ __forceinline__ double to_out(double v) { return v; }

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

inline bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

inline int ilog2(long long v) {
    int r = 0;
    while ((1LL << r) < v) ++r;
    return r;
}

// Linear index of node x = (i*N + j)*N + k of an N^3 grid after swapping
// grid axis 0 with axis sw (sw = 0: unchanged, 1: i <-> j, 2: i <-> k).
// The swap is its own inverse. The lattice Green's function of the
// 7-point operator is symmetric under permutations of the axes, so a
// convolution may run on the swapped grid and its output be read back at
// swapped indices.
__host__ __device__ __forceinline__ long long swap_axes(long long x, int sw, int N) {
    if (sw == 0) return x;
    const long long nn = (long long)N * N;
    const long long i = x / nn, j = (x / N) % N, k = x % N;
    return sw == 1 ? (j * N + i) * N + k : (k * N + j) * N + i;
}

}  // namespace bae
