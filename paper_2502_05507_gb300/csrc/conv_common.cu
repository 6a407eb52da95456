// Dispatch of the potential apply over the grid size, the schedule choice
// shared by all element types, and the gathers around the convolution.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>

#include "conv.cuh"
#include "conv_tune.cuh"

namespace bae {

namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = getenv("BAE_TUNE_FILE");
    if (!path) return;
    FILE* fp = fopen(path, "r");
    if (!fp) return;
    char key[128];
    int val;
    // one "key": value pair per line inside braces
    char line[256];
    while (fgets(line, sizeof line, fp))
        if (sscanf(line, " \"%127[^\"]\" : %d", key, &val) == 2) g_tune[key] = val;
    fclose(fp);
}

void tune_save_locked() {
    const char* path = getenv("BAE_TUNE_FILE");
    if (!path) return;
    FILE* fp = fopen(path, "w");
    if (!fp) return;
    fprintf(fp, "{\n");
    size_t k = 0;
    for (const auto& kv : g_tune)
        fprintf(fp, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++k < g_tune.size() ? "," : "");
    fprintf(fp, "}\n");
    fclose(fp);
}

}  // namespace

// -2: not set through the API, the environment decides
static std::atomic<int> g_forced{-2};

int forced_sched() {
    const int api = g_forced.load();
    if (api != -2) return api;
    static const int env = []() {
        // BAE_CONV_PLANE = 0 (passes), 1 (plane), 2 (passes, variant
        // geometry), 3 (persistent passes)
        const char* e = getenv("BAE_CONV_PLANE");
        if (!e || e[0] < '0' || e[0] > '3') return -1;
        return (int)(e[0] - '0');
    }();
    return env;
}

void set_forced_sched(int sched) { g_forced.store(sched); }


int tune_lookup(const std::string& key) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    return it == g_tune.end() ? -1 : it->second;
}

void tune_store(const std::string& key, int sched) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = sched;
    tune_save_locked();
}

namespace {

template <typename T>
const char* tname() {
    if constexpr (std::is_same<T, dsf>::value) return "df64";
    return sizeof(T) == 4 ? "f32" : "f64";
}

template <typename T>
const char* kname(const char* f32, const char* f64, const char* ds) {
    if constexpr (std::is_same<T, dsf>::value) return ds;
    return sizeof(T) == 4 ? f32 : f64;
}


// ------------------------------------------------------------------ gathers
template <typename T>
__global__ void k_closure_gather(const T* v, long long v_stride, const int* gm, const int* partner,
                                 const double* t, int n, double* out, long long out_stride, const int* active) {
    const int b = blockIdx.y;
    if (active && !active[b]) return;
    const T* vb = v + b * v_stride;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const double tr = t[r];
        out[b * out_stride + r] = tr * (double)vb[gm[r]] + (1.0 - tr) * (double)vb[partner[r]];
    }
}

// Rows of the direct formulation (eq. [direct_sys] with eq. [inhom]):
// y[r] = t x(m_r) + (1 - t) x(p(m_r)) on the n_gm gamma- rows (the closure),
// y[n_gm + k] = x(gp_k) - w(gp_k) on gamma+, for items with active[b] != 0;
// x is read like the convolution's density, w [nb][w_stride].
template <typename W, typename Y>
__global__ void k_direct_rows(const W* __restrict__ w, long long w_stride, const double* x, long long x_stride,
                              const int* x_row, long long x_row_stride, const int* __restrict__ gp,
                              const int* __restrict__ pu, const double* __restrict__ t, long long n_gm,
                              long long n_unk, const int* active, Y* y, long long y_stride) {
    const int b = blockIdx.y;
    if (active && !active[b]) return;
    const double* xb = x + b * x_stride + (x_row ? (long long)x_row[b] * x_row_stride : 0);
    const W* wb = w + b * w_stride;
    Y* yb = y + b * y_stride;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n_unk; r += (long long)gridDim.x * blockDim.x) {
        double v;
        if (r < n_gm) {
            const double tr = t[r];
            v = tr * xb[r] + (1.0 - tr) * xb[pu[r]];
        } else {
            v = xb[r] - (double)wb[gp[r - n_gm]];
        }
        yb[r] = (Y)v;
    }
}

// u[b][gm[r]] = q[b][r]: the gamma- values of the direct formulation's
// unknown into the reconstructed grid function
__global__ void k_scatter_gm(const double* q, long long q_stride, const int* __restrict__ gm, long long n,
                             double* u, long long n3) {
    const int b = blockIdx.y;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        u[b * n3 + gm[r]] = q[b * q_stride + r];
}

template <typename T>
__global__ void k_volume_combine(const T* v, const double* add, const uint8_t* flags, long long n3, double* u,
                                 int v_swap, int N) {
    const int b = blockIdx.y;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n3; x += (long long)gridDim.x * blockDim.x) {
        const bool np = (flags[x] & 3) != 0;   // M+ or gamma-
        double r = 0.0;
        if (np) {
            const long long xv = swap_axes(x, v_swap, N);
            r = (add ? add[b * n3 + xv] : 0.0) + (double)v[b * n3 + xv];
        }
        u[b * n3 + x] = r;
    }
}

__global__ void k_to_dsf(const double* in, long long n, dsf* out) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x)
        out[x] = dsf(in[x]);
}

template <typename T>
__global__ void k_widen(const T* v, long long n, double* out) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x)
        out[x] = (double)v[x];
}

}  // namespace

template <typename T>
void conv_apply(const ConvArgs<T>& a, cudaStream_t st) {
    switch (a.N) {
        case 8: run_conv<T, 16>(a, st); break;
        case 16: run_conv<T, 32>(a, st); break;
        case 32: run_conv<T, 64>(a, st); break;
        case 64: run_conv<T, 128>(a, st); break;
        case 128: run_conv<T, 256>(a, st); break;
        case 256: run_conv<T, 512>(a, st); break;
        default: throw Error(BAE_ERR_INVALID_ARG, "conv: N must be a power of two in [8, 256]");
    }
}

template <typename T>
bool conv_tuned(int N, int nbatch) {
    if (forced_sched() >= 0) return true;
    const std::string key = std::string(tname<T>()) + "/N" + std::to_string(N) + "/nb" + std::to_string(nbatch);
    return tune_lookup(key) >= 0;
}

template <typename T>
void conv_prepare(int N) {
    switch (N) {
        case 8: conv_configure<T, 16>(); break;
        case 16: conv_configure<T, 32>(); break;
        case 32: conv_configure<T, 64>(); break;
        case 64: conv_configure<T, 128>(); break;
        case 128: conv_configure<T, 256>(); break;
        case 256: conv_configure<T, 512>(); break;
        default: throw Error(BAE_ERR_INVALID_ARG, "conv: N must be a power of two in [8, 256]");
    }
}

template <typename T>
void closure_gather(const T* v, long long v_stride, const int* gm, const int* partner, const double* t,
                    int n, int nbatch, double* out, long long out_stride, cudaStream_t st, const int* active) {
    if (n == 0) return;
    dim3 grid(ceil_div(n, 256) < 1184 ? ceil_div(n, 256) : 1184, nbatch);
    BAE_LAUNCH(kname<T>("closure_gather.f32", "closure_gather.f64", "closure_gather.f64"), st, k_closure_gather<T><<<grid, 256, 0, st>>>(v, v_stride, gm, partner, t, n, out, out_stride, active));
}

__global__ void k_mask_bit(const uint8_t* __restrict__ flags, long long n, uint8_t bit, uint8_t* __restrict__ out) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x)
        out[x] = (flags[x] & bit) ? 1 : 0;
}

void mask_bit(const uint8_t* flags, long long n, uint8_t bit, uint8_t* out, cudaStream_t st) {
    const int grid = (int)(ceil_div(n, 256) < 2432 ? ceil_div(n, 256) : 2432);
    BAE_LAUNCH("k_mask_bit", st, k_mask_bit<<<grid, 256, 0, st>>>(flags, n, bit, out));
}

template <typename W, typename Y>
void direct_rows(const W* w, long long w_stride, const double* x, long long x_stride, const int* x_row,
                 long long x_row_stride, const int* gp, const int* pu, const double* t, long long n_gm, long long n_unk,
                 int nb, const int* active, Y* y, long long y_stride, cudaStream_t st) {
    dim3 grid(ceil_div(n_unk, 256) < 1184 ? ceil_div(n_unk, 256) : 1184, nb);
    BAE_LAUNCH("k_direct_rows", st, k_direct_rows<W, Y><<<grid, 256, 0, st>>>(w, w_stride, x, x_stride, x_row, x_row_stride,
                                                                              gp, pu, t, n_gm, n_unk, active, y, y_stride));
}

void scatter_gm(const double* q, long long q_stride, const int* gm, long long n, int nb, double* u, long long n3,
                cudaStream_t st) {
    dim3 grid(ceil_div(n, 256) < 1184 ? ceil_div(n, 256) : 1184, nb);
    BAE_LAUNCH("k_scatter_gm", st, k_scatter_gm<<<grid, 256, 0, st>>>(q, q_stride, gm, n, u, n3));
}

template <typename T>
void volume_combine(const T* v, const double* add, const uint8_t* flags, long long n3, int nbatch,
                    double* u, cudaStream_t st, int v_swap, int N) {
    BAE_REQUIRE(v_swap == 0 || (long long)N * N * N == n3, BAE_ERR_INVALID_ARG, "volume_combine: N must match n3");
    dim3 grid(ceil_div(n3, 256) < 2432 ? ceil_div(n3, 256) : 2432, nbatch);
    BAE_LAUNCH("k_volume_combine", st, k_volume_combine<T><<<grid, 256, 0, st>>>(v, add, flags, n3, u, v_swap, N));
}

template <typename T>
void widen(const T* v, long long n, double* out, cudaStream_t st) {
    BAE_LAUNCH("k_widen", st, k_widen<T><<<ceil_div(n, 256) < 2432 ? ceil_div(n, 256) : 2432, 256, 0, st>>>(v, n, out));
}

void to_dsf(const double* in, long long n, dsf* out, cudaStream_t st) {
    BAE_LAUNCH("k_to_dsf", st, k_to_dsf<<<ceil_div(n, 256) < 2432 ? ceil_div(n, 256) : 2432, 256, 0, st>>>(in, n, out));
}

template void conv_apply<float>(const ConvArgs<float>&, cudaStream_t);
template void conv_apply<double>(const ConvArgs<double>&, cudaStream_t);
template void conv_apply<dsf>(const ConvArgs<dsf>&, cudaStream_t);
template bool conv_tuned<float>(int, int);
template bool conv_tuned<double>(int, int);
template bool conv_tuned<dsf>(int, int);
template void conv_prepare<float>(int);
template void conv_prepare<double>(int);
template void conv_prepare<dsf>(int);
template void closure_gather<float>(const float*, long long, const int*, const int*, const double*, int, int, double*, long long, cudaStream_t, const int*);
template void closure_gather<double>(const double*, long long, const int*, const int*, const double*, int, int, double*, long long, cudaStream_t, const int*);
template void direct_rows<float, float>(const float*, long long, const double*, long long, const int*, long long, const int*, const int*, const double*, long long, long long, int, const int*, float*, long long, cudaStream_t);
template void direct_rows<float, double>(const float*, long long, const double*, long long, const int*, long long, const int*, const int*, const double*, long long, long long, int, const int*, double*, long long, cudaStream_t);
template void direct_rows<double, double>(const double*, long long, const double*, long long, const int*, long long, const int*, const int*, const double*, long long, long long, int, const int*, double*, long long, cudaStream_t);
template void volume_combine<float>(const float*, const double*, const uint8_t*, long long, int, double*, cudaStream_t,
                                     int, int);
template void volume_combine<double>(const double*, const double*, const uint8_t*, long long, int, double*,
                                      cudaStream_t, int, int);
template void widen<float>(const float*, long long, double*, cudaStream_t);
template void widen<double>(const double*, long long, double*, cudaStream_t);

}  // namespace bae
