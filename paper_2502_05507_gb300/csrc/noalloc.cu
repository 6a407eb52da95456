// bae_potential_apply_noalloc: the potential apply with its scratch in a
// fixed, file-scope device array instead of memory the library allocates.
//
// For callers that cannot allocate device memory while they run: code inside
// a memory budget enforced by someone else (a host application that hands
// the library a fixed arena, a real-time loop where a cudaMalloc/cudaFree
// would stall or synchronise the device, a plug-in whose host forbids
// allocations after start-up). Everything the apply needs besides its
// inputs and outputs is either part of the problem handle (built once, at
// set-up) or lives in g_noalloc_scratch below.
//
// The array is kNoAllocScratchBytes (8 MiB) in every process that loads the
// library, on every GPU it touches, for the life of the process.
#include <mutex>

#include "conv.cuh"
#include "internal.cuh"

namespace bae {

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;

// The scratch itself. Host code must not use this name as an address (it
// is a host-side stand-in); the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (with that device current).
void* scratch_on_current_device() {
    int dev = -1;
    BAE_CUDA(cudaGetDevice(&dev));
    BAE_REQUIRE(dev >= 0 && dev < kMaxDevices, BAE_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            throw Error(BAE_ERR_CUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = ptr;
    }
    return g_scratch_addr[dev];
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename T>
void apply_into(const ProblemView& pv, const double* q, double* v, unsigned char* scratch) {
    using C = cplx_t<T>;
    const long long N = pv.N, N1 = N + 1;
    const size_t bytes_A = align256((size_t)N * N * N1 * sizeof(C));
    const size_t bytes_B = align256((size_t)2 * N * N * N1 * sizeof(C));
    const size_t bytes_v = sizeof(T) == 8 ? 0 : align256((size_t)N * N * N * sizeof(T));
    const size_t need = bytes_A + bytes_B + bytes_v;
    if (need > kNoAllocScratchBytes)
        throw Error(BAE_ERR_INVALID_ARG,
                    "bae_potential_apply_noalloc: N=" + std::to_string(N) + " in " +
                        (sizeof(T) == 8 ? "float64" : "float32") + " needs " + std::to_string(need) +
                        " bytes of scratch; the static scratch holds " + std::to_string(kNoAllocScratchBytes) +
                        " (float32: N <= 64, float64: N <= 32)");
    ConvArgs<T> a;
    a.N = pv.N;
    a.nbatch = 1;
    a.mode = SRC_DENSITY;
    a.q = q;
    a.q_stride = pv.n_unk;
    a.no_tune = true;   // never times schedules inside this call
    a.rec = pv.rec;
    a.A = reinterpret_cast<C*>(scratch);
    a.B = reinterpret_cast<C*>(scratch + bytes_A);
    if constexpr (sizeof(T) == 8) {
        a.ghat = reinterpret_cast<const T*>(pv.ghat64);
        a.tw = reinterpret_cast<const C*>(pv.tw64);
        a.v = reinterpret_cast<T*>(v);                          // straight into the caller's output
    } else {
        a.ghat = reinterpret_cast<const T*>(pv.ghat32);
        a.tw = reinterpret_cast<const C*>(pv.tw32);
        a.v = reinterpret_cast<T*>(scratch + bytes_A + bytes_B);
    }
    // Every element of A, B and v that a pass reads is written earlier in the
    // same call, so nothing in the scratch has to be cleared first.
    conv_apply<T>(a, pv.stream);
    if constexpr (sizeof(T) == 4) widen<float>(a.v, (long long)N * N * N, v, pv.stream);
}

}  // namespace
}  // namespace bae

extern "C" int bae_potential_apply_noalloc(bae_problem* prob, int precision, const double* q, double* v) {
    using namespace bae;
    try {
        ProblemView pv;
        BAE_REQUIRE(prob && q && v, BAE_ERR_INVALID_ARG, "null argument");
        BAE_REQUIRE(problem_view(prob, pv), BAE_ERR_INVALID_ARG, "invalid problem handle");
        DeviceGuard dg;   // the caller's current device is restored on return
        BAE_CUDA(cudaSetDevice(pv.device));
        BAE_REQUIRE(precision == BAE_FP64 || precision == BAE_FP32, BAE_ERR_INVALID_ARG,
                    "precision must be BAE_FP64 or BAE_FP32");
        // device memory of another GPU is rejected inside is_device_ptr
        BAE_REQUIRE(is_device_ptr(q) && is_device_ptr(v), BAE_ERR_INVALID_ARG,
                    "bae_potential_apply_noalloc: q and v must be device memory (host arrays would need staging)");
        BAE_REQUIRE(pv.tw64 && pv.tw32, BAE_ERR_INVALID_ARG, "problem has no twiddle table");
        unsigned char* scratch = static_cast<unsigned char*>(scratch_on_current_device());
        if (precision == BAE_FP64) apply_into<double>(pv, q, v, scratch);
        else apply_into<float>(pv, q, v, scratch);
        BAE_CUDA(cudaStreamSynchronize(pv.stream));
        return BAE_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return BAE_ERR_CUDA;
    }
}
