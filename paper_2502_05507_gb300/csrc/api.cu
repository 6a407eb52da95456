// C ABI of the BAE library (include/bae.h): contexts, problems, the
// potential apply, and the GMRES solve of Algorithm 1 (FP64, or FP32
// convolution inside FP64 iterative refinement), single and batched.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <mutex>
#include <set>
#include <tuple>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "classify.cuh"
#include "common.cuh"
#include "conv.cuh"
#include "conv_tune.cuh"
#include "internal.cuh"
#include "krylov.cuh"
#include "lgf.cuh"
#include "precond.cuh"

namespace bae {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

// --------------------------------------------------- launches and profiling
static std::atomic<long long> g_launches{0};
static thread_local long long t_capture_kernels = -1;   // >= 0 while capturing a graph
void count_launch() {
    if (t_capture_kernels >= 0) ++t_capture_kernels;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void capture_begin() { t_capture_kernels = 0; }
long long capture_end() {
    const long long k = t_capture_kernels;
    t_capture_kernels = -1;
    return k;
}

namespace {
struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<ProfRec> recs;
    cudaEvent_t pending = nullptr;
    const char* pending_name = nullptr;
    bool overflow = false;
    cudaEvent_t next() {
        if (used >= pool.size()) { overflow = true; return nullptr; }
        return pool[used++];
    }
};
Profiler g_prof;
}  // namespace

void prof_push(const char* name, cudaStream_t st) {
    if (!g_prof.on || t_capture_kernels >= 0) return;
    g_prof.pending = g_prof.next();
    g_prof.pending_name = name;
    if (g_prof.pending) cudaEventRecord(g_prof.pending, st);
}

void prof_pop(cudaStream_t st) {
    if (!g_prof.on || !g_prof.pending || t_capture_kernels >= 0) return;
    cudaEvent_t e = g_prof.next();
    if (!e) return;
    cudaEventRecord(e, st);
    g_prof.recs.push_back({g_prof.pending_name, g_prof.pending, e});
    g_prof.pending = nullptr;
}

// host-side fault injection (bae_inject_fault): the cap on the size of one
// device allocation (0: none) and the number of fused Arnoldi launches whose
// barrier waits are made to run out
static std::atomic<long long> g_alloc_cap{0};
static std::atomic<long long> g_fault_barrier{0};

void alloc_check(size_t bytes) {
    const long long cap = g_alloc_cap.load();
    if (cap > 0 && (long long)bytes > cap)
        throw Error(BAE_ERR_OOM, "device allocation of " + std::to_string(bytes) +
                                     " bytes refused (injected allocation cap of " + std::to_string(cap) + " bytes)");
}

void* dev_alloc(size_t bytes, cudaStream_t st) {
    alloc_check(bytes);
    void* p = nullptr;
    BAE_CUDA(cudaMallocAsync(&p, bytes ? bytes : 16, st));
    return p;
}

void dev_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

namespace {

// Device buffer that grows on demand and frees itself (stream-ordered).
template <typename T>
struct Grow {
    T* p = nullptr;
    long long cap = 0;
    cudaStream_t st = nullptr;
    T* need(long long n) {
        if (n > cap) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            BAE_CUDA(cudaStreamIsCapturing(st, &cs));
            BAE_REQUIRE(cs == cudaStreamCaptureStatusNone, BAE_ERR_CUDA,
                        "internal: work-space growth during graph capture");
            dev_free(p, st);
            p = nullptr;
            cap = 0;
            p = dev_alloc_n<T>(n, st);
            cap = n;
        }
        return p;
    }
    void release() { dev_free(p, st); p = nullptr; cap = 0; }
    ~Grow() { release(); }
};

// One LGF spectrum, shared by every problem (and every context of a
// server) with the same (N, s); plain cudaMalloc so that it outlives the
// stream that built it.
struct Spectrum {
    int N = 0;
    double s = 0.0;
    double* g64 = nullptr;
    float* g32 = nullptr;
    dsf* gds = nullptr;
    double* near = nullptr;   // G_s on the offsets below NEAR_TN (preconditioner blocks)
    size_t bytes = 0;
    ~Spectrum() {
        if (g64) cudaFree(g64);
        if (g32) cudaFree(g32);
        if (gds) cudaFree(gds);
        if (near) cudaFree(near);
    }
};

// Work space shared by every problem of a context (calls on one context
// are serialised on its stream). Sized on demand for the largest call.
struct Workspace {
    Grow<double2> A, B;                       // convolution buffers (float64 sized)
    Grow<double> v64, up, vstage;             // [nb][N^3]
    Grow<float> v32;
    Grow<double> V, w, partial, h, hsave, x, r, bvec, tmp, qstage, n2;   // Krylov
    Grow<double> arnH, arnHu, arnCS, arnG, arnY, arnScal;
    Grow<int> active, arnI;
    Grow<unsigned int> arnCtr;
    Grow<unsigned long long> arnBar;
    Grow<double> in_f, in_g, out_q, out_u;    // staging of host arguments
    Grow<double> qpre, zpre;                  // M^{-1} y of the preconditioned inner solves
    Grow<float> arnV32, arnZ32;               // float32 copies of the newest basis vector and its M^{-1}
    Grow<double> ydir64, bprime;              // direct formulation: operator rows, [g; 0]
    Grow<float> ydir32;
    void set_stream(cudaStream_t st) {
        Grow<double>* ds[] = {&v64, &up, &vstage, &V, &w, &partial, &h, &hsave, &x, &r, &bvec, &tmp,
                              &qstage, &n2, &in_f, &in_g, &out_q, &out_u, &qpre, &zpre, &ydir64, &bprime};
        for (auto* d : ds) d->st = st;
        Grow<double>* ds2[] = {&arnH, &arnHu, &arnCS, &arnG, &arnY, &arnScal};
        for (auto* d : ds2) d->st = st;
        A.st = B.st = st;
        v32.st = st;
        arnV32.st = arnZ32.st = st;
        ydir32.st = st;
        active.st = arnI.st = st;
        arnCtr.st = st;
        arnBar.st = st;
    }
};

struct Twiddles {
    double2* tw64 = nullptr;
    float2* tw32 = nullptr;
    dsc* twds = nullptr;
};

}  // namespace

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type != cudaMemoryTypeDevice) return false;
    int cur = -1;
    BAE_CUDA(cudaGetDevice(&cur));
    BAE_REQUIRE(a.device == cur, BAE_ERR_INVALID_ARG,
                "array is device memory of GPU " + std::to_string(a.device) + ", the call runs on GPU " +
                    std::to_string(cur));
    return true;
}
}  // namespace bae

using namespace bae;

namespace bae {
// Spectra keyed by (N, bit pattern of s). Thread-safe: a context that needs
// a spectrum another one is building waits for it instead of building it
// twice. Entries live as long as the cache.
struct SpectrumCache {
    std::mutex mu;
    std::condition_variable cv;
    // key: (N, kind, bit pattern of s); kind 0 = the free-lattice G_s, 1 =
    // the finite-box Green's function of eq. [aux]
    std::map<std::tuple<int, int, uint64_t>, std::shared_ptr<Spectrum>> map;
    std::set<std::tuple<int, int, uint64_t>> building;

    std::shared_ptr<Spectrum> get(int N, double s, cudaStream_t st, int kind = 0) {
        uint64_t bits;
        std::memcpy(&bits, &s, sizeof(bits));
        const auto key = std::make_tuple(N, kind, bits);
        std::unique_lock<std::mutex> lock(mu);
        for (;;) {
            auto it = map.find(key);
            if (it != map.end()) return it->second;
            if (!building.count(key)) break;
            cv.wait(lock);
        }
        building.insert(key);
        lock.unlock();
        std::shared_ptr<Spectrum> sp;
        try {
            sp = std::make_shared<Spectrum>();
            sp->N = N;
            sp->s = s;
            const long long n3 = (long long)(N + 1) * (N + 1) * (N + 1);
            alloc_check(n3 * sizeof(double));
            BAE_CUDA(cudaMalloc(&sp->g64, n3 * sizeof(double)));
            alloc_check(n3 * sizeof(float));
            BAE_CUDA(cudaMalloc(&sp->g32, n3 * sizeof(float)));
            alloc_check(n3 * sizeof(dsf));
            BAE_CUDA(cudaMalloc(&sp->gds, n3 * sizeof(dsf)));
            sp->bytes = n3 * (sizeof(double) + sizeof(float) + sizeof(dsf));
            const double L = 2.0 * N;
            if (kind == 1) {
                box_spectrum(N, s, 1.0 / (L * L * L), sp->g64, sp->g32, st);
                to_dsf(sp->g64, n3, sp->gds, st);
            } else {
                lgf_spectrum(N, s, 1.0 / (L * L * L), sp->g64, sp->g32, st);
                to_dsf(sp->g64, n3, sp->gds, st);
                alloc_check(NEAR_TAB * sizeof(double));
                BAE_CUDA(cudaMalloc(&sp->near, NEAR_TAB * sizeof(double)));
                lgf_table(NEAR_TN, s, sp->near, st);
            }
            BAE_CUDA(cudaStreamSynchronize(st));
        } catch (...) {
            lock.lock();
            building.erase(key);
            cv.notify_all();
            throw;
        }
        lock.lock();
        building.erase(key);
        map[key] = sp;
        cv.notify_all();
        return sp;
    }

    size_t bytes() {
        std::lock_guard<std::mutex> lock(mu);
        size_t b = 0;
        for (auto& kv : map) b += kv.second->bytes;
        return b;
    }
};
}  // namespace bae

struct bae_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::shared_ptr<SpectrumCache> cache;
    std::map<int, Twiddles> tw;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t poll_ev[2] = {nullptr, nullptr};
    // second stream: set-up work that overlaps the main stream's (the
    // Schwarz rows), ordered by the fork and join events
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // a server slot: other slots' kernels run beside this context's on the
    // same GPU, so no kernel may assume that all of its CTAs are resident at
    // once (the Arnoldi step runs as two kernels, not the cooperative one)
    bool shared_gpu = false;
    int* pinned = nullptr;       // mapped host memory the kernels write the live flags into
    int* pinned_dev = nullptr;   // its device address
    int pinned_cap = 0;
    Workspace ws;

    // host-pinned, device-mapped polling buffer: [nb] live flags, then the
    // barrier error flag of the fused Arnoldi step
    int* pinned_flags(int nb) {
        if (nb + 1 > pinned_cap) {
            if (pinned) cudaFreeHost(pinned);
            pinned = nullptr;
            pinned_dev = nullptr;
            BAE_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&pinned), (size_t)(nb + 1) * sizeof(int),
                                   cudaHostAllocMapped));
            BAE_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&pinned_dev), pinned, 0));
            pinned_cap = nb + 1;
        }
        return pinned;
    }

    const Twiddles& twiddles(int L) {
        auto it = tw.find(L);
        if (it != tw.end()) return it->second;
        Twiddles t;
        t.tw64 = dev_alloc_n<double2>(L, stream);
        t.tw32 = dev_alloc_n<float2>(L, stream);
        t.twds = dev_alloc_n<dsc>(L, stream);
        make_twiddles(L, t.tw64, t.tw32, stream);
        to_dsf(reinterpret_cast<const double*>(t.tw64), 2LL * L, reinterpret_cast<dsf*>(t.twds), stream);
        return tw[L] = t;
    }

    std::shared_ptr<Spectrum> spectrum(int N, double s, int kind = 0) { return cache->get(N, s, stream, kind); }
};

struct bae_problem {
    bae_ctx* ctx = nullptr;
    Geometry geo;
    Precond pre;   // right preconditioner, built on the first mixed solve that asks for it
    std::shared_ptr<Spectrum> spec;
    std::shared_ptr<Spectrum> spec_box;   // finite-box spectrum, fetched by the first box apply
    double kappa2 = 0.0, s = 0.0;
    // direct formulation: the Arnoldi gather reads the operator rows as they
    // are (row r of the vector at index r, weight 1)
    int* iota = nullptr;
    double* ones = nullptr;
    bool direct() const { return geo.layer == BAE_LAYER_DIRECT; }
    Workspace& ws() { return ctx->ws; }
    long long n3() const { return (long long)geo.N * geo.N * geo.N; }
};

namespace bae {

void ctx_share_cache(bae_ctx* dst, const bae_ctx* src) { dst->cache = src->cache; }
void ctx_set_shared_gpu(bae_ctx* c) { c->shared_gpu = true; }

bool problem_view(const bae_problem* P, ProblemView& out) {
    if (!P || !P->spec) return false;
    out.device = P->ctx->device;
    out.N = P->geo.N;
    out.n_gm = P->geo.n_gm;
    out.n_unk = P->geo.n_unk;
    out.stream = P->ctx->stream;
    out.rec = P->geo.recipe();
    out.ghat64 = P->spec->g64;
    out.ghat32 = P->spec->g32;
    auto it = P->ctx->tw.find(2 * P->geo.N);
    if (it != P->ctx->tw.end()) {
        out.tw64 = it->second.tw64;
        out.tw32 = it->second.tw32;
    }
    return true;
}

namespace {

long long n_gm(const bae_problem* P) { return P->geo.n_gm; }
long long n_unk(const bae_problem* P) { return P->geo.n_unk; }

// Pruned applies (whose output is read at gamma-, the partners and M+
// only) transform only the planes that hold sources or read nodes, along
// the first axis of the grid they run on: the geometry's swapped view
// (Geometry::cv_swap), whose first axis is the one with the fewest such
// planes. Their recipe and flags are the view's, f is read through the
// swap, and their output is in the swapped layout: it is read back at
// gm_of / partner_of and through volume_combine's swap. Unpruned applies
// cover the whole grid in the plain layout.
bool use_view(const bae_problem* P, bool pruned) { return pruned && P->geo.cv_swap != 0; }
const int* gm_of(const bae_problem* P, bool pruned) { return use_view(P, pruned) ? P->geo.cv_gm : P->geo.gm; }
const int* partner_of(const bae_problem* P, bool pruned) {
    return use_view(P, pruned) ? P->geo.cv_partner : P->geo.partner;
}
int swap_of(const bae_problem* P, bool pruned) { return use_view(P, pruned) ? P->geo.cv_swap : 0; }

template <typename T>
ConvArgs<T> conv_args(bae_problem* P, int nb, bool pruned = false) {
    const int N = P->geo.N;
    const long long N1 = N + 1;
    ConvArgs<T> a;
    a.N = N;
    a.nbatch = nb;
    const bool view = use_view(P, pruned);
    if (pruned) {
        a.p0 = view ? P->geo.cv_lo : P->geo.plane_lo;
        a.p1 = view ? P->geo.cv_hi : P->geo.plane_hi;
        // the line range along the grid's second axis (y, or x when x and
        // y are swapped), rounded out to whole line pairs
        const int ax2 = (view && P->geo.cv_swap == 1) ? 0 : 1;
        a.q0 = P->geo.ext_lo[ax2] & ~1;
        a.q1 = std::min(N, (P->geo.ext_hi[ax2] + 1) & ~1);
    }
    a.rec = view ? P->geo.cv_recipe() : P->geo.recipe();
    a.flags = view ? P->geo.cv_flags : P->geo.flags;
    a.f_swap = swap_of(P, pruned);
    a.A = reinterpret_cast<cplx_t<T>*>(P->ws().A.need((long long)nb * N * N * N1));
    a.B = reinterpret_cast<cplx_t<T>*>(P->ws().B.need((long long)nb * N * 2 * N * N1));
    const Twiddles& tw = P->ctx->twiddles(2 * N);
    if constexpr (std::is_same<T, dsf>::value) {
        a.ghat = P->spec->gds;
        a.tw = tw.twds;
    } else if constexpr (sizeof(T) == 8) {
        a.ghat = reinterpret_cast<const T*>(P->spec->g64);
        a.tw = reinterpret_cast<const cplx_t<T>*>(tw.tw64);
    } else {
        a.ghat = reinterpret_cast<const T*>(P->spec->g32);
        a.tw = reinterpret_cast<const cplx_t<T>*>(tw.tw32);
    }
    return a;
}

template <typename T>
using out_t = typename OutOf<T>::type;

template <typename T>
out_t<T>* vbuf(bae_problem* P, int nb) {
    if constexpr (std::is_same<out_t<T>, double>::value) return P->ws().v64.need((long long)nb * P->n3());
    else return P->ws().v32.need((long long)nb * P->n3());
}

// v[b] = K q[b] on the N^3 grid (on the plane range only when pruned),
// q [nb][n_gm] on the device
template <typename T>
out_t<T>* apply_potential(bae_problem* P, int nb, const double* q, bool pruned = false) {
    ConvArgs<T> a = conv_args<T>(P, nb, pruned);
    a.mode = SRC_DENSITY;
    a.q = q;
    a.q_stride = n_unk(P);
    a.v = vbuf<T>(P, nb);
    conv_apply<T>(a, P->ctx->stream);
    return a.v;
}

// v[b] = sum_{x in M+} G(m - x) scale f[b](x)
template <typename T>
out_t<T>* apply_volume(bae_problem* P, int nb, const double* f, double scale, bool pruned = false) {
    ConvArgs<T> a = conv_args<T>(P, nb, pruned);
    a.mode = SRC_VOLUME;
    a.f = f;
    a.scale = scale;
    a.v = vbuf<T>(P, nb);
    conv_apply<T>(a, P->ctx->stream);
    return a.v;
}

// v[b] = G_box[chi_{M+} scale f[b]] (eq. [aux]): the finite-box particular
// solution, float64 or double-float
template <typename T>
out_t<T>* apply_box(bae_problem* P, int nb, const double* f, double scale, bool pruned) {
    static_assert(sizeof(T) == 8, "the finite-box apply is float64-accurate");
    if (!P->spec_box) P->spec_box = P->ctx->spectrum(P->geo.N, P->s, 1);
    ConvArgs<T> a = conv_args<T>(P, nb, pruned);
    if constexpr (std::is_same<T, dsf>::value) a.ghat = P->spec_box->gds;
    else a.ghat = reinterpret_cast<const T*>(P->spec_box->g64);
    a.mode = SRC_VOLUME;
    a.box = true;
    a.f = f;
    a.scale = scale;
    a.v = vbuf<T>(P, nb);
    conv_apply<T>(a, P->ctx->stream);
    return a.v;
}

double* apply_box64(bae_problem* P, int prec, int nb, const double* f, double scale, bool pruned = false) {
    return prec == BAE_DF64 ? apply_box<dsf>(P, nb, f, scale, pruned) : apply_box<double>(P, nb, f, scale, pruned);
}

// v[b] = K q[b] + sum_{x in M+} G(m - x) scale f[b](x): one convolution of
// the layer and volume sources (disjoint nodes)
template <typename T>
out_t<T>* apply_combined(bae_problem* P, int nb, const double* q, const double* f, double scale, bool pruned) {
    ConvArgs<T> a = conv_args<T>(P, nb, pruned);
    a.mode = SRC_DENSITY;
    a.q = q;
    a.q_stride = n_unk(P);
    a.f = f;
    a.scale = scale;
    a.v = vbuf<T>(P, nb);
    conv_apply<T>(a, P->ctx->stream);
    return a.v;
}

// Aq[b] = Phi K q[b], both [nb][n_gm] on the device
template <typename T>
void boundary_apply(bae_problem* P, int nb, const double* q, double* Aq) {
    out_t<T>* v = apply_potential<T>(P, nb, q, true);
    if (P->direct())
        direct_rows<out_t<T>, double>(v, P->n3(), q, n_unk(P), nullptr, 0, P->geo.gp, P->geo.partner_u, P->geo.t,
                                      n_gm(P), n_unk(P), nb, nullptr, Aq, n_unk(P), P->ctx->stream);
    else
        closure_gather<out_t<T>>(v, P->n3(), gm_of(P, true), partner_of(P, true), P->geo.t, (int)n_gm(P), nb, Aq, n_gm(P),
                                 P->ctx->stream);
}

void boundary_apply_prec(bae_problem* P, int prec, int nb, const double* q, double* Aq) {
    if (prec == BAE_FP32) boundary_apply<float>(P, nb, q, Aq);
    else if (prec == BAE_DF64) boundary_apply<dsf>(P, nb, q, Aq);
    else boundary_apply<double>(P, nb, q, Aq);
}

// K q[b] in float64 storage for the float64-accurate precisions
double* apply_potential64(bae_problem* P, int prec, int nb, const double* q, bool pruned = false) {
    return prec == BAE_DF64 ? apply_potential<dsf>(P, nb, q, pruned) : apply_potential<double>(P, nb, q, pruned);
}

double* apply_volume64(bae_problem* P, int prec, int nb, const double* f, double scale, bool pruned = false) {
    return prec == BAE_DF64 ? apply_volume<dsf>(P, nb, f, scale, pruned)
                            : apply_volume<double>(P, nb, f, scale, pruned);
}

double* apply_combined64(bae_problem* P, int prec, int nb, const double* q, const double* f, double scale,
                         bool pruned) {
    return prec == BAE_DF64 ? apply_combined<dsf>(P, nb, q, f, scale, pruned)
                            : apply_combined<double>(P, nb, q, f, scale, pruned);
}

// --------------------------------------------------------------- GMRES
struct RhsState {
    bool converged = false;
    int iterations = 0;
    double target = 0.0;     // absolute residual target
    double est = 0.0;        // last residual estimate
};

// v[b] = K q[b] on the grid with q read at q + b q_stride + (*q_row)
// q_row_stride, for items with active[b] != 0 (all device arrays;
// capturable in a graph); returns v [nb][N^3]
template <typename T>
out_t<T>* potential_rows(bae_problem* P, int nb, const double* q, long long q_stride, const int* q_row,
                         long long q_row_stride, const int* active, const float* q32 = nullptr) {
    ConvArgs<T> a = conv_args<T>(P, nb, true);
    a.mode = SRC_DENSITY;
    a.q = q;
    a.q_stride = q_stride;
    a.q_row = q_row;
    a.q_row_stride = q_row_stride;
    if (std::is_same<T, float>::value && q32) {
        a.q32 = q32;
        a.q32_stride = n_unk(P);
    }
    a.active = active;
    a.v = vbuf<T>(P, nb);
    conv_apply<T>(a, P->ctx->stream);
    return a.v;
}

// w[b] = A q[b] = Phi K q[b] (the potential, then the closure gather)
template <typename T>
void apply_rows(bae_problem* P, int nb, const double* q, long long q_stride, const int* q_row,
                long long q_row_stride, const int* active, double* out) {
    out_t<T>* v = potential_rows<T>(P, nb, q, q_stride, q_row, q_row_stride, active);
    if (P->direct())
        direct_rows<out_t<T>, double>(v, P->n3(), q, q_stride, q_row, q_row_stride, P->geo.gp, P->geo.partner_u,
                                      P->geo.t, n_gm(P), n_unk(P), nb, active, out, n_unk(P), P->ctx->stream);
    else
        closure_gather<out_t<T>>(v, P->n3(), gm_of(P, true), partner_of(P, true), P->geo.t, (int)n_gm(P), nb, out, n_gm(P),
                                 P->ctx->stream, active);
}

void apply_rows_prec(bae_problem* P, int prec, int nb, const double* q, long long q_stride, const int* q_row,
                     long long q_row_stride, const int* active, double* out) {
    if (prec == BAE_FP32) apply_rows<float>(P, nb, q, q_stride, q_row, q_row_stride, active, out);
    else if (prec == BAE_DF64) apply_rows<dsf>(P, nb, q, q_stride, q_row, q_row_stride, active, out);
    else apply_rows<double>(P, nb, q, q_stride, q_row, q_row_stride, active, out);
}

// A captured GMRES step and the values it was captured with: the next
// gmres call of the same solve (the inner solves of iterative refinement)
// replays it when every captured pointer and parameter is the same.
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
    std::vector<uintptr_t> key;
    StepGraph() = default;
    StepGraph(const StepGraph&) = delete;
    StepGraph& operator=(const StepGraph&) = delete;
    ~StepGraph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

// Restarted GMRES for the RHS b in `which` (rows of rhs/x [nb][n], device):
// every Arnoldi step (apply of precision `prec`, Gram-Schmidt, Givens) runs on the
// device; with use_graph it is captured once as a CUDA graph and replayed.
// The host only polls the convergence flags (double-buffered, one step
// behind) and closes each cycle. x_zero: x is known to be 0.
// pre: right-preconditioned (x is the preconditioned variable y of
// A M^{-1} y = rhs; the caller maps it back with M^{-1})
void gmres(bae_problem* P, int prec, int nb, const std::vector<int>& which, const double* rhs, double* x,
           bool x_zero, std::vector<RhsState>& S, int max_iter, int restart, std::vector<int>& applies,
           bool use_graph, bool pre = false, StepGraph* cache = nullptr) {
    cudaStream_t st = P->ctx->stream;
    Workspace& ws = P->ws();
    const int n = (int)n_unk(P);
    const int m = std::max(1, std::min(restart, max_iter));
    Arnoldi a;
    a.n = n;
    a.nb = nb;
    a.m = m;
    a.nchunk = arnoldi_chunks(n);
    a.V = ws.V.need((long long)nb * (m + 1) * n);
    a.w = ws.w.need((long long)nb * n);
    a.part = ws.partial.need((long long)nb * 2 * (m + 1) * a.nchunk);
    a.cf = ws.h.need((long long)nb * 2 * (m + 1));
    a.hs = ws.hsave.need((long long)nb * (m + 1));
    a.H = ws.arnH.need((long long)nb * m * (m + 1));
    a.Hu = ws.arnHu.need((long long)nb * m * (m + 1));
    a.cs = ws.arnCS.need((long long)nb * m * 2);
    a.sn = a.cs + (long long)nb * m;
    a.g = ws.arnG.need((long long)nb * (m + 1));
    a.y = ws.arnY.need((long long)nb * m);
    double* scal = ws.arnScal.need((long long)nb * 5);
    a.est = scal;
    a.target = scal + nb;
    a.inv = scal + 2 * nb;
    a.tco = scal + 3 * nb;
    int* ibuf = ws.arnI.need((long long)nb * 8 + 1);
    a.flag = ibuf;
    a.ncols = ibuf + nb;
    int* member = ibuf + 2 * nb;
    a.j = ibuf + 3 * nb;
    a.ctr = reinterpret_cast<unsigned int*>(ws.arnCtr.need((long long)nb * 3));
    // the fused cooperative step where the device can place it and has it
    // to itself
    arn_configure(m);
    a.coop_grid = P->ctx->shared_gpu ? 0 : arn_coop_grid(n, nb, m, &a.coop_resident, &a.coop_redundant);
    a.bar = ws.arnBar.need(2);
    a.bar2 = a.bar + 1;
    a.err = ibuf + 4 * nb;
    a.gflag = ibuf + 4 * nb + 1;
    a.live = ibuf + 5 * nb + 1;
    a.jstep = ibuf + 6 * nb + 1;
    a.ran = ibuf + 7 * nb + 1;
    a.v32 = ws.arnV32.need((long long)nb * n);
    double* r = ws.r.need((long long)nb * n);
    double* tmp = ws.tmp.need((long long)nb * n);
    double* npart = ws.n2.need((long long)nb * krylov_chunks(n) + nb);
    int* d_all = ws.active.need(nb);

    std::vector<int> all(nb), mem(nb, 0);
    std::vector<double> tgt(nb, 0.0);
    for (int b = 0; b < nb; ++b) {
        all[b] = b;
        tgt[b] = S[b].target;
    }
    for (int b : which)
        if (!S[b].converged) mem[b] = 1;
    BAE_CUDA(cudaMemcpyAsync(d_all, all.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st));
    BAE_CUDA(cudaMemcpyAsync(a.target, tgt.data(), nb * sizeof(double), cudaMemcpyHostToDevice, st));
    BAE_CUDA(cudaMemsetAsync(a.ctr, 0, (size_t)nb * 3 * sizeof(unsigned int), st));
    BAE_CUDA(cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned long long), st));
    BAE_CUDA(cudaMemsetAsync(a.err, 0, sizeof(int), st));

    // the kernels that decide the flags also write live[b] into mapped host
    // memory: no copy between the replayed steps
    volatile int* hlive = P->ctx->pinned_flags(nb);
    a.live_host = P->ctx->pinned_dev;
    a.err_host = P->ctx->pinned_dev + nb;
    hlive[nb] = 0;
    cudaEvent_t ev[2] = {P->ctx->poll_ev[0], P->ctx->poll_ev[1]};
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0;
    int iters_left = max_iter;
    std::vector<int> ncols(nb), flg(nb);
    int coop_err = 0;   // the fused step's barrier error flag, read with each cycle's results
    std::vector<double> est(nb);

    // one step: v = K V[j] for the iterating RHS, then the Arnoldi passes
    // (whose first pass gathers w = Phi v)
    a.v_f32 = prec == BAE_FP32;
    const bool direct = P->direct();
    a.v_stride = direct ? n : P->n3();
    a.gm = direct ? P->iota : gm_of(P, true);   // the step's applies are pruned
    a.partner = direct ? P->iota : partner_of(P, true);
    a.t = direct ? P->ones : P->geo.t;
    // direct formulation: the step's operator rows, in the apply's precision
    float* y32 = direct && prec == BAE_FP32 ? ws.ydir32.need((long long)nb * n) : nullptr;
    double* y64 = direct && prec != BAE_FP32 ? ws.ydir64.need((long long)nb * n) : nullptr;
    // right preconditioning: the step applies A to z = M^{-1} V[j]; the
    // fused step forms the next z itself (after arn_init: z of V[0] here)
    double* zpre = pre ? ws.zpre.need((long long)nb * n) : nullptr;
    a.z32 = pre ? ws.arnZ32.need((long long)nb * n) : nullptr;
    const bool fuse_pre = pre && a.coop_grid > 0;
    if (fuse_pre) {
        a.pre_col = P->pre.col;
        a.pre_val = P->pre.val;
        a.zpre = zpre;
    }
    auto one_step = [&]() {
        const double* q = a.V;
        long long qs = (long long)(m + 1) * n;
        const int* qrow = a.j;
        // the float32 apply reads the float32 copy of its density: z32, or
        // v32 (the newest basis vector, the row a.j selects)
        const float* q32 = a.v32;
        if (pre) {
            if (!fuse_pre) precond_apply(P->pre, a.V, qs, a.j, n, zpre, n, nb, a.flag, st, a.v32, a.z32);
            q = zpre;
            qs = n;
            qrow = nullptr;
            q32 = a.z32;
        }
        if (prec == BAE_FP32) a.v = potential_rows<float>(P, nb, q, qs, qrow, n, a.flag, q32);
        else if (prec == BAE_DF64) a.v = potential_rows<dsf>(P, nb, q, qs, qrow, n, a.flag);
        else a.v = potential_rows<double>(P, nb, q, qs, qrow, n, a.flag);
        if (direct) {
            if (y32) {
                direct_rows<float, float>(static_cast<const float*>(a.v), P->n3(), q, qs, qrow, n, P->geo.gp,
                                          P->geo.partner_u, P->geo.t, n_gm(P), n, nb, a.flag, y32, n, st);
                a.v = y32;
            } else {
                direct_rows<double, double>(static_cast<const double*>(a.v), P->n3(), q, qs, qrow, n, P->geo.gp,
                                            P->geo.partner_u, P->geo.t, n_gm(P), n, nb, a.flag, y64, n, st);
                a.v = y64;
            }
        }
        // fault injection (tests only): this launch's barrier waits run out
        // after ~8k polls (about a millisecond) instead of half a second
        const bool inject = a.coop_grid > 0 && !use_graph && g_fault_barrier.load() > 0;
        if (inject) {
            g_fault_barrier.fetch_sub(1);
            Arnoldi af = a;
            af.bar_extra = 1;
            af.spin_limit = 1 << 13;
            arn_step(af, st);
        } else {
            arn_step(a, st);
        }
    };
    // size every buffer and set every kernel attribute the step needs before
    // any capture (nothing may allocate or configure inside it)
    // and let the autotuner pick the convolution schedule for this batch size
    // on an uncaptured apply (its result is discarded)
    const bool tuned = prec == BAE_FP32 ? conv_tuned<float>(P->geo.N, nb)
                       : prec == BAE_DF64 ? conv_tuned<dsf>(P->geo.N, nb) : conv_tuned<double>(P->geo.N, nb);
    if (!tuned) apply_rows_prec(P, prec, nb, rhs, n, nullptr, 0, nullptr, ws.tmp.need((long long)nb * n));
    if (prec == BAE_FP32) {
        conv_args<float>(P, nb);
        vbuf<float>(P, nb);
        conv_prepare<float>(P->geo.N);
    } else if (prec == BAE_DF64) {
        conv_args<dsf>(P, nb);
        vbuf<dsf>(P, nb);
        conv_prepare<dsf>(P->geo.N);
    } else {
        conv_args<double>(P, nb);
        vbuf<double>(P, nb);
        conv_prepare<double>(P->geo.N);
    }

    // a graph captured by an earlier call with the same values is replayed
    std::vector<uintptr_t> key;
    if (use_graph && cache) {
        auto add = [&](const void* p) { key.push_back(reinterpret_cast<uintptr_t>(p)); };
        for (long long v : {(long long)prec, (long long)nb, (long long)m, (long long)n, (long long)pre,
                            (long long)fuse_pre, (long long)direct, (long long)a.coop_grid,
                            (long long)a.coop_resident, (long long)forced_sched()})
            key.push_back((uintptr_t)v);
        key.push_back((uintptr_t)a.coop_redundant);
        add(P); add(a.V); add(a.w); add(a.part); add(a.cf); add(a.hs); add(a.H); add(a.Hu); add(a.cs); add(a.g);
        add(a.y); add(scal); add(ibuf); add(a.ctr); add(a.bar); add(a.live_host); add(zpre); add(y32); add(y64);
        add(a.v32); add(a.z32);
        add(ws.A.p); add(ws.B.p); add(ws.v32.p); add(ws.v64.p); add(P->pre.col); add(P->pre.val);
        if (cache->exec && cache->key == key) {
            exec = cache->exec;
            graph_kernels = cache->kernels;
        }
    }
    // a graph made here goes to the cache (replacing its previous one) or is destroyed
    auto drop_exec = [&](bool keep) {
        if (!exec) return;
        if (cache && exec == cache->exec) return;
        if (keep && cache && !key.empty()) {
            if (cache->exec) cudaGraphExecDestroy(cache->exec);
            cache->exec = exec;
            cache->kernels = graph_kernels;
            cache->key = key;
        } else {
            cudaGraphExecDestroy(exec);
        }
        exec = nullptr;
    };
    try {
        while (iters_left > 0) {
            int any = 0;
            for (int b = 0; b < nb; ++b) any |= mem[b];
            if (!any) break;
            BAE_CUDA(cudaMemcpyAsync(member, mem.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st));
            // r = rhs - A x for the members
            if (x_zero) {
                BAE_CUDA(cudaMemcpyAsync(r, rhs, (size_t)nb * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
                x_zero = false;
            } else {
                if (pre) {
                    precond_apply(P->pre, x, n, nullptr, 0, zpre, n, nb, member, st);
                    apply_rows_prec(P, prec, nb, zpre, n, nullptr, 0, member, tmp);
                } else {
                    apply_rows_prec(P, prec, nb, x, n, nullptr, 0, member, tmp);
                }
                for (int b = 0; b < nb; ++b) applies[b] += mem[b];
                kr_sub(rhs, tmp, d_all, nb, n, r, st);
            }
            kr_norm2(r, d_all, nb, n, npart + nb, krylov_chunks(n), npart, st);
            arn_init(a, r, npart, member, st);
            if (fuse_pre)
                precond_apply(P->pre, a.V, (long long)(m + 1) * n, nullptr, 0, zpre, n, nb, member, st, a.v32, a.z32);
            // a column becomes final (and is rotated) one step later: one
            // more launch finishes the last column of the cycle
            const int steps = std::min(m, iters_left) + 1;
            int launched = 0;
            for (int it = 0; it < steps; ++it) {
                if (use_graph) {
                    if (!exec) {
                        cudaGraph_t graph;
                        capture_begin();
                        BAE_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                        try {
                            one_step();
                        } catch (...) {
                            cudaStreamEndCapture(st, &graph);
                            capture_end();
                            throw;
                        }
                        BAE_CUDA(cudaStreamEndCapture(st, &graph));
                        graph_kernels = capture_end();
                        const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
                        cudaGraphDestroy(graph);
                        BAE_CUDA(e);
                    }
                    BAE_CUDA(cudaGraphLaunch(exec, st));
                    count_launches(graph_kernels);
                } else {
                    one_step();
                }
                ++launched;
                BAE_CUDA(cudaEventRecord(ev[it & 1], st));
                if (it >= 1) {
                    // after step it - 1 completed the flags are those of that
                    // step or of a later one (they only drop to 0 in a cycle)
                    BAE_CUDA(cudaEventSynchronize(ev[(it - 1) & 1]));
                    int live = 0;
                    for (int b = 0; b < nb; ++b) live |= hlive[b];
                    if (!live || hlive[nb]) break;   // converged, or a barrier wait ran out
                }
            }
            // one host read per cycle: columns, estimates and the barrier
            // error flag, after the solution update
            arn_finish(a, x, st);
            BAE_CUDA(cudaMemcpyAsync(ncols.data(), a.ncols, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
            BAE_CUDA(cudaMemcpyAsync(est.data(), a.est, nb * sizeof(double), cudaMemcpyDeviceToHost, st));

            if (a.coop_grid > 0) BAE_CUDA(cudaMemcpyAsync(&coop_err, a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
            BAE_CUDA(cudaStreamSynchronize(st));
            BAE_REQUIRE(coop_err == 0, BAE_ERR_TIMEOUT,
                        "GMRES: a bounded grid-barrier wait of the fused Arnoldi step ran out");
            int maxc = 0;
            for (int b = 0; b < nb; ++b) maxc = std::max(maxc, ncols[b]);
            for (int b = 0; b < nb; ++b) {
                if (!mem[b]) continue;
                S[b].iterations += ncols[b];
                applies[b] += ncols[b];
                S[b].est = est[b];
                if (est[b] <= S[b].target) {
                    S[b].converged = true;
                    mem[b] = 0;
                }
            }
            iters_left -= std::max(maxc, 1);
            (void)launched;
        }
    } catch (...) {
        drop_exec(false);
        throw;
    }
    drop_exec(true);
}

// ------------------------------------------------------------ full solve
struct HostArg {
    const double* in = nullptr;
    double* out = nullptr;
};

// Zeros of a host output u (nb right-hand sides of N^3 values) outside the
// box [lo, hi) of every right-hand side, written by host threads while the
// device solves. The solution is 0 outside N+, which the box holds, so only
// the box is copied from the device. The destructor waits for the threads.
class HostZeroFill {
public:
    HostZeroFill(double* u, int nb, int N, const int lo[3], const int hi[3]) {
        // up to 8 threads (half the host's), one per ~4 MB of the array
        const unsigned hc = std::thread::hardware_concurrency();
        const long long work = (long long)nb * N * N * N / (512LL * 1024);
        const int nt = (int)std::max(1LL, std::min<long long>({8LL, (long long)(hc / 2), work}));
        for (int w = 0; w < nt; ++w)
            th_.emplace_back([=]() {
                const long long n3 = (long long)N * N * N, nn = (long long)N * N;
                for (long long it = w; it < (long long)nb * N; it += nt) {   // item: (b, i)
                    const long long b = it / N;
                    const int i = (int)(it % N);
                    double* plane = u + b * n3 + (long long)i * nn;
                    if (i < lo[0] || i >= hi[0]) {
                        std::memset(plane, 0, (size_t)nn * sizeof(double));
                        continue;
                    }
                    for (int j = 0; j < N; ++j) {
                        double* line = plane + (long long)j * N;
                        if (j < lo[1] || j >= hi[1]) {
                            std::memset(line, 0, (size_t)N * sizeof(double));
                        } else {
                            std::memset(line, 0, (size_t)lo[2] * sizeof(double));
                            std::memset(line + hi[2], 0, (size_t)(N - hi[2]) * sizeof(double));
                        }
                    }
                }
            });
    }
    ~HostZeroFill() { join(); }
    void join() {
        for (auto& t : th_)
            if (t.joinable()) t.join();
    }
    HostZeroFill(const HostZeroFill&) = delete;
    HostZeroFill& operator=(const HostZeroFill&) = delete;

private:
    std::vector<std::thread> th_;
};

int solve_impl(bae_problem* P, int nb, const double* f, const double* g, const bae_options* opts_in,
               double* density, double* u, bae_stats* stats) {
    bae_options o;
    bae_default_options(&o);
    if (opts_in) o = *opts_in;
    BAE_REQUIRE(nb >= 1, BAE_ERR_INVALID_ARG, "nrhs must be >= 1");
    BAE_REQUIRE(f && g, BAE_ERR_INVALID_ARG, "f and g must not be null");
    BAE_REQUIRE(o.tol > 0 && std::isfinite(o.tol), BAE_ERR_INVALID_ARG, "tol must be positive");
    BAE_REQUIRE(o.max_iter >= 1 && o.restart >= 1 && o.restart <= 1024, BAE_ERR_INVALID_ARG,
                "max_iter must be >= 1 and restart in [1, 1024]");
    BAE_REQUIRE(o.precision == BAE_FP64 || o.precision == BAE_MIXED || o.precision == BAE_DF64,
                BAE_ERR_INVALID_ARG, "precision must be BAE_FP64, BAE_MIXED or BAE_DF64");
    BAE_REQUIRE(o.residual_precision == BAE_FP64 || o.residual_precision == BAE_DF64, BAE_ERR_INVALID_ARG,
                "residual_precision must be BAE_FP64 or BAE_DF64");
    BAE_REQUIRE(o.precond >= 0 && o.precond <= 2, BAE_ERR_INVALID_ARG, "precond must be 0, 1 or 2");
    BAE_REQUIRE(o.particular == BAE_PARTICULAR_LATTICE || o.particular == BAE_PARTICULAR_BOX, BAE_ERR_INVALID_ARG,
                "particular must be BAE_PARTICULAR_LATTICE or BAE_PARTICULAR_BOX");
    BAE_REQUIRE(o.particular == BAE_PARTICULAR_LATTICE || P->geo.layer != BAE_LAYER_DIRECT, BAE_ERR_INVALID_ARG,
                "the finite-box particular solution is for the layer formulations (the direct formulation's "
                "difference potentials use the free-lattice G)");
    // arithmetic of every float64-accurate apply (particular solution,
    // refinement residuals, reconstruction)
    const int hp = o.precision == BAE_MIXED ? o.residual_precision : o.precision;
    cudaStream_t st = P->ctx->stream;
    BAE_CUDA(cudaEventRecord(P->ctx->ev0, st));
    const long long n3 = P->n3();
    const int ng = (int)n_gm(P);    // gamma- nodes: boundary points and g
    const int n = (int)n_unk(P);    // unknowns (ng, or ng + |gamma+| for the direct formulation)
    const bool direct = P->direct();
    const double h = P->geo.h;
    // the right preconditioner of the inner solves (restricted additive
    // Schwarz) is built on the side stream while this one checks the inputs
    // and forms the first right-hand side; the inner solves wait for it
    const bool any_pre = o.precision == BAE_MIXED && o.precond != 0;
    if (any_pre && !P->pre.built) {
        BAE_CUDA(cudaEventRecord(P->ctx->fork_ev, st));
        BAE_CUDA(cudaStreamWaitEvent(P->ctx->side, P->ctx->fork_ev, 0));
        build_precond(P->geo, P->s, P->spec->near, P->pre, P->ctx->side);
        BAE_CUDA(cudaEventRecord(P->ctx->join_ev, P->ctx->side));
        P->pre.pending = true;
    }

    // stage host inputs. The solve reads f only on M+ (the volume source
    // chi_{M+} f and the finiteness check), which lies inside the box of
    // planes [ext_lo, ext_hi) along each axis (gamma- encloses M+): one 3D
    // copy of that box per right-hand side; the rest of the device copy is
    // never read.
    const double* d_f = f;
    const double* d_g = g;
    long long h2d_rhs = 0;   // bytes copied per right-hand side
    if (!is_device_ptr(f)) {
        double* p = P->ws().in_f.need((long long)nb * n3);
        const Geometry& G = P->geo;
        const int NN = G.N;
        const cudaExtent ext = make_cudaExtent((size_t)(G.ext_hi[2] - G.ext_lo[2]) * sizeof(double),
                                               (size_t)(G.ext_hi[1] - G.ext_lo[1]), (size_t)(G.ext_hi[0] - G.ext_lo[0]));
        for (int b = 0; b < nb; ++b) {
            cudaMemcpy3DParms cp = {};
            cp.srcPtr = make_cudaPitchedPtr(const_cast<double*>(f) + (long long)b * n3, (size_t)NN * sizeof(double),
                                            (size_t)NN * sizeof(double), (size_t)NN);
            cp.dstPtr = make_cudaPitchedPtr(p + (long long)b * n3, (size_t)NN * sizeof(double),
                                            (size_t)NN * sizeof(double), (size_t)NN);
            cp.srcPos = make_cudaPos((size_t)G.ext_lo[2] * sizeof(double), (size_t)G.ext_lo[1], (size_t)G.ext_lo[0]);
            cp.dstPos = cp.srcPos;
            cp.extent = ext;
            cp.kind = cudaMemcpyHostToDevice;
            BAE_CUDA(cudaMemcpy3DAsync(&cp, st));
        }
        h2d_rhs += (long long)ext.width * ext.height * ext.depth;
        d_f = p;
    }
    if (!is_device_ptr(g)) {
        double* p = P->ws().in_g.need((long long)nb * ng);
        BAE_CUDA(cudaMemcpyAsync(p, g, (size_t)nb * ng * sizeof(double), cudaMemcpyHostToDevice, st));
        d_g = p;
        h2d_rhs += (long long)ng * sizeof(double);
    }
    // f on M+ and g must be finite: the flag is read with ||b|| below (one
    // host read; non-finite inputs only make the discarded b non-finite)
    int* d_bad = P->ws().arnI.need(4);
    BAE_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    kr_nonfinite(d_f, (long long)nb * n3, P->geo.flags, n3, d_bad, st);
    kr_nonfinite(d_g, (long long)nb * ng, nullptr, 1, d_bad, st);
    std::vector<bae_stats> st_local(nb);
    for (auto& s : st_local) {
        std::memset(&s, 0, sizeof(s));
        s.h2d_bytes = h2d_rhs;
    }
    // a host u: its zeros outside the box of N+ are written on the host
    // while the device works; only the box is copied back at the end
    const bool u_host = u && !is_device_ptr(u);
    std::unique_ptr<HostZeroFill> zero_fill;
    if (u_host) zero_fill.reset(new HostZeroFill(u, nb, P->geo.N, P->geo.ext_lo, P->geo.ext_hi));

    // particular solution u_p = G_h[chi_{M+} f] and b = g - Phi u_p. Mixed
    // precision needs u_p only for the first inner right-hand side, so there
    // it is a float32 apply: each float64-accurate residual below convolves
    // the layer and volume sources together, r = g - Phi (K q + u_p), and u
    // is that sum on N+. Otherwise u_p is float64 and kept for u.
    //
    // Direct formulation (eq. [direct_sys] with eq. [inhom]): the unknown
    // is u on gamma; with b' = [g; 0] and rows(w, x) = [closure of x; x -
    // w on gamma+], b = [g; u_p on gamma+] = b' - rows(u_p, 0), and every
    // residual is b - A x = b' - rows(P x + u_p, x) (one combined apply); u
    // is P x + u_p on M+ and x on gamma-.
    const bool mixed = o.precision == BAE_MIXED;
    // finite-box particular solution (eq. [aux]): kept in float64-accurate
    // arithmetic for b and for u, never folded into the residual applies
    // (the layer potential uses the free-lattice G, the box part does not)
    const bool box = o.particular == BAE_PARTICULAR_BOX;
    const bool comb = (mixed || direct) && !box;   // residuals convolve layer + volume sources together
    double* bvec = P->ws().x.need((long long)nb * n * 3);   // [b | q | r] blocks
    double* q = bvec + (long long)nb * n;
    double* res = q + (long long)nb * n;
    double* up = nullptr;
    BAE_CUDA(cudaMemsetAsync(q, 0, (size_t)nb * n * sizeof(double), st));
    double* bp = nullptr;
    if (direct) {
        bp = P->ws().bprime.need((long long)nb * n);
        BAE_CUDA(cudaMemsetAsync(bp, 0, (size_t)nb * n * sizeof(double), st));
        BAE_CUDA(cudaMemcpy2DAsync(bp, (size_t)n * sizeof(double), d_g, (size_t)ng * sizeof(double),
                                   (size_t)ng * sizeof(double), nb, cudaMemcpyDeviceToDevice, st));
    }
    if (mixed && !box) {
        const float* v = apply_volume<float>(P, nb, d_f, h * h, true);
        if (direct)
            direct_rows<float, double>(v, n3, q, n, nullptr, 0, P->geo.gp, P->geo.partner_u, P->geo.t, ng, n, nb,
                                       nullptr, res, n, st);
        else
            closure_gather<float>(v, n3, gm_of(P, true), partner_of(P, true), P->geo.t, n, nb, res, n, st);
        for (auto& s : st_local) s.applies_fp32 += 1;
    } else {
        up = P->ws().up.need((long long)nb * n3);
        double* v = box ? apply_box64(P, hp, nb, d_f, h * h, true) : apply_volume64(P, hp, nb, d_f, h * h, true);
        BAE_CUDA(cudaMemcpyAsync(up, v, (size_t)nb * n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        for (auto& s : st_local) s.applies_fp64 += 1;
        if (direct)
            direct_rows<double, double>(up, n3, q, n, nullptr, 0, P->geo.gp, P->geo.partner_u, P->geo.t, ng, n, nb,
                                        nullptr, res, n, st);
        else
            closure_gather<double>(up, n3, gm_of(P, true), partner_of(P, true), P->geo.t, n, nb, res, n, st);
    }
    {
        std::vector<int> all(nb);
        for (int b = 0; b < nb; ++b) all[b] = b;
        int* d_act = P->ws().active.need(nb);
        BAE_CUDA(cudaMemcpyAsync(d_act, all.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st));
        kr_sub(direct ? bp : d_g, res, d_act, nb, n, bvec, st);
    }

    // ||b||
    std::vector<double> bn2(nb), rn2(nb);
    double* n2 = P->ws().n2.need((long long)nb * krylov_chunks(n) + nb);
    std::vector<int> all(nb);
    for (int b = 0; b < nb; ++b) all[b] = b;
    int* d_act = P->ws().active.need(nb);
    BAE_CUDA(cudaMemcpyAsync(d_act, all.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st));
    kr_norm2(bvec, d_act, nb, n, n2 + nb, krylov_chunks(n), n2, st);
    BAE_CUDA(cudaMemcpyAsync(bn2.data(), n2, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    int bad = 0;
    BAE_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    BAE_CUDA(cudaStreamSynchronize(st));
    BAE_REQUIRE(!bad, BAE_ERR_INVALID_ARG, "f (on M+) or g contains non-finite values");

    std::vector<RhsState> S(nb);
    std::vector<int> iters_used(nb, 0);
    std::vector<bool> done(nb, false);
    std::vector<double> relres(nb, 0.0);
    double* v_last = nullptr;   // float64 K q of the final q, [nb][N^3]

    // residual r = b - A64 q = g - Phi (K q + u_p), with K q (+ u_p when
    // mixed) left in the float64 volume buffer
    auto true_residual = [&]() {
        int* d_all = P->ws().active.need(nb);
        BAE_CUDA(cudaMemcpyAsync(d_all, all.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st));
        double* tmp = P->ws().tmp.need((long long)nb * n);
        double* v = comb ? apply_combined64(P, hp, nb, q, d_f, h * h, true) : apply_potential64(P, hp, nb, q, true);
        if (direct)
            direct_rows<double, double>(v, n3, q, n, nullptr, 0, P->geo.gp, P->geo.partner_u, P->geo.t, ng, n, nb,
                                        nullptr, tmp, n, st);
        else
            closure_gather<double>(v, n3, gm_of(P, true), partner_of(P, true), P->geo.t, n, nb, tmp, n, st);
        for (auto& s : st_local) s.applies_fp64 += 1;
        kr_sub(direct ? bp : (comb ? d_g : bvec), tmp, d_all, nb, n, res, st);
        kr_norm2(res, d_all, nb, n, n2 + nb, krylov_chunks(n), n2, st);
        BAE_CUDA(cudaMemcpyAsync(rn2.data(), n2, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        BAE_CUDA(cudaStreamSynchronize(st));
        v_last = v;
        for (int b = 0; b < nb; ++b) relres[b] = bn2[b] > 0 ? std::sqrt(rn2[b] / bn2[b]) : 0.0;
    };

    if (o.precision != BAE_MIXED) {
        for (int b = 0; b < nb; ++b) S[b].target = o.tol * std::sqrt(bn2[b]);
        std::vector<int> applies(nb, 0);
        gmres(P, o.precision, nb, all, bvec, q, true, S, o.max_iter, o.restart, applies, o.use_graphs != 0);
        for (int b = 0; b < nb; ++b) {
            st_local[b].iterations = S[b].iterations;
            st_local[b].applies_fp64 += applies[b];
        }
        true_residual();
    } else {
        // iterative refinement: inner float32-apply GMRES on A d = r, q += d,
        // r = b - A64 q in float64
        double* d = P->ws().vstage.need((long long)nb * n);
        // right preconditioner of the inner solves (the inner unknown is y
        // with d = M^{-1} y), built on the side stream above
        if (P->pre.pending) {
            BAE_CUDA(cudaStreamWaitEvent(st, P->ctx->join_ev, 0));
            P->pre.pending = false;
        }
        double* dq = any_pre ? P->ws().qpre.need((long long)nb * n) : d;
        BAE_CUDA(cudaMemcpyAsync(res, bvec, (size_t)nb * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        rn2 = bn2;
        for (int b = 0; b < nb; ++b) relres[b] = bn2[b] > 0 ? 1.0 : 0.0;
        int iters_left = o.max_iter;
        StepGraph step_graph;   // the inner solves' captured step, shared by the refinement steps
        for (int step = 0; step < std::max(1, o.max_refine); ++step) {
            std::vector<int> act;
            for (int b = 0; b < nb; ++b)
                if (relres[b] > o.tol && bn2[b] > 0) act.push_back(b);
            if (act.empty() || iters_left <= 0) break;
            // every refinement step (precond 1) or the steps after the first
            // (precond 2)
            const bool use_pre = any_pre && (o.precond == 1 || (o.precond == 2 && step > 0));
            std::vector<RhsState> Si(nb);
            for (int b : act) {
                // reduce the residual by inner_tol; when that lands within ten
                // times the outer target, aim straight below the outer target
                // so that this is the last step (no further float64-accurate
                // residual and restart): at 0.3 tol ||b||, or 0.03 tol ||b|| in
                // a preconditioned step, whose float32 basis applies leave a
                // true residual up to ~10 times above the estimate
                const double floor_b = (use_pre ? 0.03 : 0.3) * o.tol * std::sqrt(bn2[b]);
                const double rn = std::sqrt(rn2[b]);
                double tgt = o.inner_tol * rn;
                if (tgt <= 10.0 * o.tol * std::sqrt(bn2[b])) tgt = floor_b;
                Si[b].target = std::max(tgt, floor_b);
            }
            for (int b = 0; b < nb; ++b)
                if (std::find(act.begin(), act.end(), b) == act.end()) Si[b].converged = true;
            BAE_CUDA(cudaMemsetAsync(d, 0, (size_t)nb * n * sizeof(double), st));
            std::vector<int> applies(nb, 0);
            gmres(P, BAE_FP32, nb, act, res, d, true, Si, iters_left, o.restart, applies, o.use_graphs != 0, use_pre,
                  &step_graph);
            if (use_pre) precond_apply(P->pre, d, n, nullptr, 0, dq, n, nb, nullptr, st);
            int used = 0;
            for (int b : act) {
                st_local[b].iterations += Si[b].iterations;
                st_local[b].refinements += 1;
                used = std::max(used, Si[b].iterations);
            }
            iters_left -= std::max(used, 1);
            int* d_a = P->ws().active.need(nb);
            BAE_CUDA(cudaMemcpyAsync(d_a, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            kr_add(use_pre ? dq : d, d_a, (int)act.size(), n, q, st);
            for (int b : act) st_local[b].applies_fp32 += applies[b];
            true_residual();
        }
        if (!v_last) true_residual();
    }

    // outputs: u = u_p + K q on N+ (v_last holds the sum when mixed), density q
    bool q_host = density && !is_device_ptr(density);
    long long d2h_u = 0;   // bytes of u copied per right-hand side
    if (u) {
        double* du = u_host ? P->ws().out_u.need((long long)nb * n3) : u;
        volume_combine<double>(v_last, direct ? nullptr : up, P->geo.flags, n3, nb, du, st, swap_of(P, true),
                               P->geo.N);
        if (direct) scatter_gm(q, n, P->geo.gm, ng, nb, du, n3, st);   // u on gamma- is the unknown there
        if (u_host) {   // the box that holds N+, one 3D copy per right-hand side
            const Geometry& G = P->geo;
            const size_t NN = (size_t)G.N;
            const cudaExtent ext = make_cudaExtent((size_t)(G.ext_hi[2] - G.ext_lo[2]) * sizeof(double),
                                                   (size_t)(G.ext_hi[1] - G.ext_lo[1]),
                                                   (size_t)(G.ext_hi[0] - G.ext_lo[0]));
            for (int b = 0; b < nb; ++b) {
                cudaMemcpy3DParms cp = {};
                cp.srcPtr = make_cudaPitchedPtr(du + (long long)b * n3, NN * sizeof(double), NN * sizeof(double), NN);
                cp.dstPtr = make_cudaPitchedPtr(u + (long long)b * n3, NN * sizeof(double), NN * sizeof(double), NN);
                cp.srcPos = make_cudaPos((size_t)G.ext_lo[2] * sizeof(double), (size_t)G.ext_lo[1],
                                         (size_t)G.ext_lo[0]);
                cp.dstPos = cp.srcPos;
                cp.extent = ext;
                cp.kind = cudaMemcpyDeviceToHost;
                BAE_CUDA(cudaMemcpy3DAsync(&cp, st));
            }
            d2h_u = (long long)ext.width * ext.height * ext.depth;
        }
    }
    if (density) {
        if (q_host) BAE_CUDA(cudaMemcpyAsync(density, q, (size_t)nb * n * sizeof(double), cudaMemcpyDeviceToHost, st));
        else BAE_CUDA(cudaMemcpyAsync(density, q, (size_t)nb * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    BAE_CUDA(cudaEventRecord(P->ctx->ev1, st));
    BAE_CUDA(cudaStreamSynchronize(st));
    if (zero_fill) zero_fill->join();   // the zeros outside the box are in place
    float ms = 0.f;
    BAE_CUDA(cudaEventElapsedTime(&ms, P->ctx->ev0, P->ctx->ev1));
    int rc = BAE_OK;
    for (int b = 0; b < nb; ++b) {
        st_local[b].rel_residual = relres[b];
        st_local[b].ms_total = ms;
        st_local[b].d2h_bytes = d2h_u + (q_host ? (long long)n * (long long)sizeof(double) : 0);
        if (!(relres[b] <= o.tol) && bn2[b] > 0) rc = BAE_ERR_NOT_CONVERGED;
    }
    if (stats)
        for (int b = 0; b < nb; ++b) stats[b] = st_local[b];
    if (rc != BAE_OK) set_last_error("GMRES did not reach the requested tolerance");
    return rc;
}

// Runs fn with device versions of (possibly host) in/out arrays.
struct Staged {
    bae_problem* P;
    double* dev = nullptr;
    const void* user = nullptr;
    size_t bytes = 0;
    bool host = false;
};

template <typename F>
int guarded(F&& fn) {
    DeviceGuard dg;   // the caller's current device is restored on return
    try {
        return fn();
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return BAE_ERR_OOM;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return BAE_ERR_CUDA;
    }
}

void check_device(bae_ctx* ctx) {
    BAE_REQUIRE(ctx, BAE_ERR_INVALID_ARG, "null context");
    BAE_CUDA(cudaSetDevice(ctx->device));
}

// copy a (host or device) input of `count` doubles into device memory
const double* device_in(Grow<double>& buf, const double* p, long long count, cudaStream_t st) {
    if (is_device_ptr(p)) return p;
    double* d = buf.need(count);
    BAE_CUDA(cudaMemcpyAsync(d, p, (size_t)count * sizeof(double), cudaMemcpyHostToDevice, st));
    return d;
}

template <typename T>
void copy_out(T* user, const T* dev, long long count, cudaStream_t st) {
    BAE_CUDA(cudaMemcpyAsync(user, dev, (size_t)count * sizeof(T), cudaMemcpyDefault, st));
}

}  // namespace
}  // namespace bae

// =================================================================== C ABI
extern "C" {

int bae_version(void) { return 1; }

long long bae_launch_count(void) { return bae::g_launches.load(); }

int bae_set_conv_schedule(int schedule) {
    return guarded([&]() -> int {
        BAE_REQUIRE(schedule >= BAE_SCHED_AUTO && schedule <= BAE_SCHED_PERSIST, BAE_ERR_INVALID_ARG,
                    "schedule must be BAE_SCHED_AUTO, BAE_SCHED_PASSES, BAE_SCHED_PLANE, BAE_SCHED_PASSES_ALT or "
                    "BAE_SCHED_PERSIST");
        bae::set_forced_sched(schedule);
        return BAE_OK;
    });
}

int bae_inject_fault(int kind, long long arg) {
    return guarded([&]() -> int {
        if (kind == BAE_FAULT_NONE) {
            g_alloc_cap.store(0);
            g_fault_barrier.store(0);
        } else if (kind == BAE_FAULT_BARRIER) {
            BAE_REQUIRE(arg >= 0, BAE_ERR_INVALID_ARG, "arg must be >= 0");
            g_fault_barrier.store(arg);
        } else if (kind == BAE_FAULT_ALLOC_CAP) {
            g_alloc_cap.store(arg > 0 ? arg : 0);
        } else {
            throw Error(BAE_ERR_INVALID_ARG, "unknown fault kind");
        }
        return BAE_OK;
    });
}

int bae_profile_start(int max_launches) {
    return guarded([&]() -> int {
        BAE_REQUIRE(max_launches > 0, BAE_ERR_INVALID_ARG, "max_launches must be positive");
        BAE_REQUIRE(!g_prof.on, BAE_ERR_INVALID_ARG, "profiling already started");
        const size_t need = 2 * (size_t)max_launches;
        while (g_prof.pool.size() < need) {
            cudaEvent_t e;
            BAE_CUDA(cudaEventCreate(&e));
            g_prof.pool.push_back(e);
        }
        g_prof.used = 0;
        g_prof.recs.clear();
        g_prof.overflow = false;
        g_prof.on = true;
        return BAE_OK;
    });
}

int bae_profile_stop(char* names, int names_len, double* total_ms, long long* launches, int max_kernels,
                     int* n_kernels) {
    return guarded([&]() -> int {
        BAE_REQUIRE(g_prof.on, BAE_ERR_INVALID_ARG, "profiling not started");
        g_prof.on = false;
        BAE_CUDA(cudaDeviceSynchronize());
        std::vector<std::string> order;
        std::map<std::string, std::pair<double, long long>> agg;
        for (const ProfRec& r : g_prof.recs) {
            float ms = 0.f;
            BAE_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
            auto it = agg.find(r.name);
            if (it == agg.end()) {
                order.push_back(r.name);
                agg[r.name] = {ms, 1};
            } else {
                it->second.first += ms;
                it->second.second += 1;
            }
        }
        std::string joined;
        int k = 0;
        for (const std::string& nm : order) {
            if (k >= max_kernels) break;
            if (total_ms) total_ms[k] = agg[nm].first;
            if (launches) launches[k] = agg[nm].second;
            joined += nm;
            joined += '\n';
            ++k;
        }
        if (n_kernels) *n_kernels = k;
        if (names && names_len > 0) {
            const size_t n = std::min((size_t)names_len - 1, joined.size());
            std::memcpy(names, joined.data(), n);
            names[n] = 0;
        }
        g_prof.recs.clear();
        if (g_prof.overflow) {
            set_last_error("profile event pool overflowed; some launches were not timed");
            return BAE_ERR_INVALID_ARG;
        }
        return BAE_OK;
    });
}

const char* bae_last_error(void) { return bae::g_last_error.c_str(); }

void bae_default_options(bae_options* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->max_iter = 500;
    o->restart = 200;
    o->precision = BAE_FP64;
    o->max_refine = 8;
    o->inner_tol = 1e-5;
    o->use_graphs = 0;
    o->residual_precision = BAE_DF64;
    o->precond = 1;
    o->particular = BAE_PARTICULAR_LATTICE;
}

int bae_ctx_create(int device, void* stream, bae_ctx** out) {
    return guarded([&]() -> int {
        BAE_REQUIRE(out, BAE_ERR_INVALID_ARG, "out is null");
        int count = 0;
        BAE_CUDA(cudaGetDeviceCount(&count));
        BAE_REQUIRE(device >= 0 && device < count, BAE_ERR_INVALID_ARG, "no such CUDA device");
        BAE_CUDA(cudaSetDevice(device));
        auto c = std::make_unique<bae_ctx>();
        c->device = device;
        if (stream) {
            c->stream = (cudaStream_t)stream;
        } else {
            BAE_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        BAE_CUDA(cudaEventCreate(&c->ev0));
        BAE_CUDA(cudaEventCreate(&c->ev1));
        BAE_CUDA(cudaEventCreateWithFlags(&c->poll_ev[0], cudaEventDisableTiming));
        BAE_CUDA(cudaEventCreateWithFlags(&c->poll_ev[1], cudaEventDisableTiming));
        BAE_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        BAE_CUDA(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
        BAE_CUDA(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
        // keep freed blocks of the default pool for reuse (problem set-up
        // and work space come from it)
        cudaMemPool_t pool;
        BAE_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
        uint64_t thr = UINT64_MAX;
        BAE_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        c->ws.set_stream(c->stream);
        c->cache = std::make_shared<SpectrumCache>();
        *out = c.release();
        return BAE_OK;
    });
}

void bae_ctx_destroy(bae_ctx* ctx) {
    if (!ctx) return;
    bae::DeviceGuard dg;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->cache.reset();
    for (auto& kv : ctx->tw) {
        dev_free(kv.second.tw64, ctx->stream);
        dev_free(kv.second.tw32, ctx->stream);
        dev_free(kv.second.twds, ctx->stream);
    }
    ctx->ws = Workspace();
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (cudaEvent_t e : ctx->poll_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
    }
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int bae_lgf_table(bae_ctx* ctx, int N, double s, double* values) {
    return guarded([&]() -> int {
        check_device(ctx);
        BAE_REQUIRE(values, BAE_ERR_INVALID_ARG, "values is null");
        BAE_REQUIRE(N >= 2 && N <= 256, BAE_ERR_INVALID_ARG, "N must be in [2, 256]");
        const long long ntri = (long long)N * (N + 1) * (N + 2) / 6;
        double* d = is_device_ptr(values) ? values : ctx->ws.out_u.need(ntri);
        lgf_table(N, s, d, ctx->stream);
        if (d != values) copy_out(values, d, ntri, ctx->stream);
        BAE_CUDA(cudaStreamSynchronize(ctx->stream));
        return BAE_OK;
    });
}

int bae_lgf_spectrum(bae_ctx* ctx, int N, double s, double* ghat) {
    return guarded([&]() -> int {
        check_device(ctx);
        BAE_REQUIRE(ghat, BAE_ERR_INVALID_ARG, "ghat is null");
        BAE_REQUIRE(is_pow2(N) && N >= 8 && N <= 256, BAE_ERR_INVALID_ARG, "N must be a power of two in [8, 256]");
        const long long n3 = (long long)(N + 1) * (N + 1) * (N + 1);
        double* d = is_device_ptr(ghat) ? ghat : ctx->ws.out_u.need(n3);
        lgf_spectrum(N, s, 1.0, d, nullptr, ctx->stream);
        if (d != ghat) copy_out(ghat, d, n3, ctx->stream);
        BAE_CUDA(cudaStreamSynchronize(ctx->stream));
        return BAE_OK;
    });
}

int bae_problem_create(bae_ctx* ctx, int N, double h, const double origin[3], const double* phi, double kappa2,
                       int layer, bae_problem** out) {
    return guarded([&]() -> int {
        check_device(ctx);
        BAE_REQUIRE(out && phi && origin, BAE_ERR_INVALID_ARG, "null argument");
        BAE_REQUIRE(is_pow2(N) && N >= 8 && N <= 256, BAE_ERR_INVALID_ARG, "N must be a power of two in [8, 256]");
        BAE_REQUIRE(std::isfinite(h) && h > 0, BAE_ERR_INVALID_ARG, "h must be positive and finite");
        BAE_REQUIRE(std::isfinite(kappa2) && kappa2 >= 0, BAE_ERR_INVALID_ARG, "kappa2 must be finite and >= 0");
        BAE_REQUIRE(std::isfinite(origin[0]) && std::isfinite(origin[1]) && std::isfinite(origin[2]),
                    BAE_ERR_INVALID_ARG, "origin must be finite");
        BAE_REQUIRE(layer == BAE_LAYER_DOUBLE || layer == BAE_LAYER_SINGLE || layer == BAE_LAYER_DIRECT,
                    BAE_ERR_INVALID_ARG, "unknown layer");
        auto P = std::make_unique<bae_problem>();
        P->ctx = ctx;
        P->kappa2 = kappa2;
        P->s = kappa2 * h * h;
        const long long n3 = (long long)N * N * N;
        const double* d_phi = device_in(ctx->ws.in_f, phi, n3, ctx->stream);
        try {
            build_geometry(d_phi, N, h, origin, layer, P->s, P->geo, ctx->stream);
        } catch (...) {
            P->geo.release();
            throw;
        }
        try {
            P->spec = ctx->spectrum(N, P->s);
            ctx->twiddles(2 * N);   // built here so that later applies allocate nothing
        // the Schwarz rows of the default (mixed, preconditioned) solve, built
        // on the side stream from here on; a solve waits for them only when it
        // uses them
        BAE_CUDA(cudaEventRecord(ctx->fork_ev, ctx->stream));
        BAE_CUDA(cudaStreamWaitEvent(ctx->side, ctx->fork_ev, 0));
        build_precond(P->geo, P->s, P->spec->near, P->pre, ctx->side);
        BAE_CUDA(cudaEventRecord(ctx->join_ev, ctx->side));
        P->pre.pending = true;
        if (P->direct()) {
            const long long nu = P->geo.n_unk;
            std::vector<int> io(nu);
            std::vector<double> on(nu, 1.0);
            for (long long r = 0; r < nu; ++r) io[r] = (int)r;
            P->iota = dev_alloc_n<int>(nu, ctx->stream);
            P->ones = dev_alloc_n<double>(nu, ctx->stream);
            BAE_CUDA(cudaMemcpyAsync(P->iota, io.data(), nu * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
            BAE_CUDA(cudaMemcpyAsync(P->ones, on.data(), nu * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
            BAE_CUDA(cudaStreamSynchronize(ctx->stream));
        }
        } catch (...) {
            // a failure after the geometry (no memory for the spectrum, the
            // Schwarz rows or the direct formulation's arrays) leaves the
            // context usable: everything made so far is freed
            cudaStreamSynchronize(ctx->side);
            cudaStreamSynchronize(ctx->stream);
            P->pre.release();
            if (P->iota) dev_free(P->iota, ctx->stream);
            if (P->ones) dev_free(P->ones, ctx->stream);
            P->geo.release();
            throw;
        }
        *out = P.release();
        return BAE_OK;
    });
}

void bae_problem_destroy(bae_problem* P) {
    if (!P) return;
    bae::DeviceGuard dg;
    cudaSetDevice(P->ctx->device);
    if (P->pre.pending) cudaStreamSynchronize(P->ctx->side);   // a build the main stream never waited for
    cudaStreamSynchronize(P->ctx->stream);
    P->pre.release();
    if (P->iota) dev_free(P->iota, P->ctx->stream);
    if (P->ones) dev_free(P->ones, P->ctx->stream);
    P->geo.release();
    delete P;
}

int bae_problem_sizes(const bae_problem* P, int64_t* n_gm, int64_t* n_gp, int64_t* n_mp) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P, BAE_ERR_INVALID_ARG, "null problem");
        if (n_gm) *n_gm = P->geo.n_gm;
        if (n_gp) *n_gp = P->geo.n_gp;
        if (n_mp) *n_mp = P->geo.n_mp;
        return BAE_OK;
    });
}

int bae_problem_plane_range(const bae_problem* P, int* lo, int* hi) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P && lo && hi, BAE_ERR_INVALID_ARG, "null argument");
        *lo = P->geo.plane_lo;
        *hi = P->geo.plane_hi;
        return BAE_OK;
    });
}

int bae_problem_conv_planes(const bae_problem* P, int* axis, int* lo, int* hi) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P && axis && lo && hi, BAE_ERR_INVALID_ARG, "null argument");
        const int sw = P->geo.cv_swap;
        *axis = sw;
        *lo = sw ? P->geo.cv_lo : P->geo.plane_lo;
        *hi = sw ? P->geo.cv_hi : P->geo.plane_hi;
        return BAE_OK;
    });
}

int bae_boundary_points(const bae_problem* P, double* xyz) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P && xyz, BAE_ERR_INVALID_ARG, "null argument");
        check_device(P->ctx);
        copy_out(xyz, P->geo.xstar, 3 * P->geo.n_gm, P->ctx->stream);
        BAE_CUDA(cudaStreamSynchronize(P->ctx->stream));
        return BAE_OK;
    });
}

int bae_classification(const bae_problem* P, uint8_t* flags, int32_t* gm_idx, int32_t* partner, double* t) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P, BAE_ERR_INVALID_ARG, "null problem");
        check_device(P->ctx);
        cudaStream_t st = P->ctx->stream;
        const long long n3 = (long long)P->geo.N * P->geo.N * P->geo.N;
        if (flags) copy_out(flags, P->geo.flags, n3, st);
        if (gm_idx) copy_out(gm_idx, P->geo.gm, P->geo.n_gm, st);
        if (partner) copy_out(partner, P->geo.partner, P->geo.n_gm, st);
        if (t) copy_out(t, P->geo.t, P->geo.n_gm, st);
        BAE_CUDA(cudaStreamSynchronize(st));
        return BAE_OK;
    });
}

int bae_interior_mask(const bae_problem* P, uint8_t* mask) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P && mask, BAE_ERR_INVALID_ARG, "null argument");
        check_device(P->ctx);
        cudaStream_t st = P->ctx->stream;
        const long long n3 = P->n3();
        if (is_device_ptr(mask)) {
            mask_bit(P->geo.flags, n3, 1, mask, st);
        } else {
            uint8_t* d = reinterpret_cast<uint8_t*>(P->ctx->ws.out_u.need((n3 + 7) / 8));
            mask_bit(P->geo.flags, n3, 1, d, st);
            BAE_CUDA(cudaMemcpyAsync(mask, d, (size_t)n3, cudaMemcpyDeviceToHost, st));
        }
        BAE_CUDA(cudaStreamSynchronize(st));
        return BAE_OK;
    });
}

int bae_problem_unknowns(const bae_problem* P, int64_t* n) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P && n, BAE_ERR_INVALID_ARG, "null argument");
        *n = P->geo.n_unk;
        return BAE_OK;
    });
}

int bae_gamma_plus(const bae_problem* P, int32_t* gp_idx) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P && gp_idx, BAE_ERR_INVALID_ARG, "null argument");
        check_device(P->ctx);
        cudaStream_t st = P->ctx->stream;
        copy_out(gp_idx, P->geo.gp, P->geo.n_gp, st);
        BAE_CUDA(cudaStreamSynchronize(st));
        return BAE_OK;
    });
}

int bae_potential_apply(bae_problem* P, int precision, const double* q, double* v) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P && q && v, BAE_ERR_INVALID_ARG, "null argument");
        BAE_REQUIRE(precision == BAE_FP64 || precision == BAE_FP32 || precision == BAE_DF64, BAE_ERR_INVALID_ARG,
                    "precision must be BAE_FP64, BAE_FP32 or BAE_DF64");
        check_device(P->ctx);
        cudaStream_t st = P->ctx->stream;
        const double* dq = device_in(P->ws().in_g, q, P->geo.n_unk, st);
        const long long n3 = P->n3();
        const bool vh = !is_device_ptr(v);
        double* dv = vh ? P->ws().out_u.need(n3) : v;
        if (precision != BAE_FP32) {
            double* r = apply_potential64(P, precision, 1, dq);
            BAE_CUDA(cudaMemcpyAsync(dv, r, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
            float* r = apply_potential<float>(P, 1, dq);
            widen<float>(r, n3, dv, st);
        }
        if (vh) copy_out(v, dv, n3, st);
        BAE_CUDA(cudaStreamSynchronize(st));
        return BAE_OK;
    });
}

int bae_boundary_apply(bae_problem* P, int precision, const double* q, double* Aq) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P && q && Aq, BAE_ERR_INVALID_ARG, "null argument");
        BAE_REQUIRE(precision == BAE_FP64 || precision == BAE_FP32 || precision == BAE_DF64, BAE_ERR_INVALID_ARG,
                    "precision must be BAE_FP64, BAE_FP32 or BAE_DF64");
        check_device(P->ctx);
        cudaStream_t st = P->ctx->stream;
        const long long n = P->geo.n_unk;
        const double* dq = device_in(P->ws().in_g, q, n, st);
        const bool oh = !is_device_ptr(Aq);
        double* dA = oh ? P->ws().out_q.need(n) : Aq;
        boundary_apply_prec(P, precision, 1, dq, dA);
        if (oh) copy_out(Aq, dA, n, st);
        BAE_CUDA(cudaStreamSynchronize(st));
        return BAE_OK;
    });
}

int bae_particular(bae_problem* P, int precision, const double* f, double* up) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P && f && up, BAE_ERR_INVALID_ARG, "null argument");
        BAE_REQUIRE(precision == BAE_FP64 || precision == BAE_FP32 || precision == BAE_DF64, BAE_ERR_INVALID_ARG,
                    "precision must be BAE_FP64, BAE_FP32 or BAE_DF64");
        check_device(P->ctx);
        cudaStream_t st = P->ctx->stream;
        const long long n3 = P->n3();
        const double* df = device_in(P->ws().in_f, f, n3, st);
        const bool oh = !is_device_ptr(up);
        double* du = oh ? P->ws().out_u.need(n3) : up;
        const double h2 = P->geo.h * P->geo.h;
        if (precision != BAE_FP32) {
            double* r = apply_volume64(P, precision, 1, df, h2);
            BAE_CUDA(cudaMemcpyAsync(du, r, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
            float* r = apply_volume<float>(P, 1, df, h2);
            widen<float>(r, n3, du, st);
        }
        if (oh) copy_out(up, du, n3, st);
        BAE_CUDA(cudaStreamSynchronize(st));
        return BAE_OK;
    });
}

int bae_box_particular(bae_problem* P, int precision, const double* f, double* up) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P && f && up, BAE_ERR_INVALID_ARG, "null argument");
        BAE_REQUIRE(precision == BAE_FP64 || precision == BAE_DF64, BAE_ERR_INVALID_ARG,
                    "precision must be BAE_FP64 or BAE_DF64");
        check_device(P->ctx);
        cudaStream_t st = P->ctx->stream;
        const long long n3 = P->n3();
        const double* df = device_in(P->ws().in_f, f, n3, st);
        const bool oh = !is_device_ptr(up);
        double* du = oh ? P->ws().out_u.need(n3) : up;
        double* r = apply_box64(P, precision, 1, df, P->geo.h * P->geo.h);
        BAE_CUDA(cudaMemcpyAsync(du, r, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (oh) copy_out(up, du, n3, st);
        BAE_CUDA(cudaStreamSynchronize(st));
        return BAE_OK;
    });
}

int bae_solve(bae_problem* P, const double* f, const double* g, const bae_options* opts, double* density,
              double* u, bae_stats* stats) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P, BAE_ERR_INVALID_ARG, "null problem");
        check_device(P->ctx);
        return solve_impl(P, 1, f, g, opts, density, u, stats);
    });
}

int bae_solve_batched(bae_problem* P, int nrhs, const double* f, const double* g, const bae_options* opts,
                      double* density, double* u, bae_stats* stats) {
    return guarded([&]() -> int {
        BAE_REQUIRE(P, BAE_ERR_INVALID_ARG, "null problem");
        BAE_REQUIRE(nrhs >= 1 && nrhs <= 65535, BAE_ERR_INVALID_ARG, "nrhs must be in [1, 65535]");
        check_device(P->ctx);
        return solve_impl(P, nrhs, f, g, opts, density, u, stats);
    });
}

}  // extern "C"
