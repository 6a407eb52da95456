// Lattice Green's function of (6+s) - (sum of the six neighbours), s = sigma h^2
// (Section 2.2, eq. [lgf] with h = 1), by Watson's Bessel integral
// (eq. [lgf_bessel], with exp(-(6+s)t) for sigma > 0):
//
//   G_s(n) = int_0^inf exp(-s t) Ie_a(2t) Ie_b(2t) Ie_c(2t) dt,  Ie_n(x) = e^{-x} I_n(x).
//
// The paper splits the integral at T* into a quadrature part and a tail
// evaluated from the large-argument expansion of I_n (mu = 4n^2). Here:
//  * [0, e^-Q] in t: 20-point Gauss-Legendre, Q = ceil(ln s) for s > 1 else 0;
//    [e^-Q, e^P] in u = ln t: unit panels of 16-point Gauss-Legendre (the
//    integrand is analytic in u), P chosen per offset from max(n).
//  * Ie_n(2 t_j), n < N, for every node t_j by Miller's backward recurrence
//    I_{k-1} = (2k/x) I_k + I_{k+1}, started at sqrt(N^2 + 80x) + 20 and
//    normalised by Ie_0 + 2 sum_k Ie_k = 1.
//  * Tail from T = e^P, T >= 100 max(n)^2: the product of the three
//    large-argument series (6 terms each) integrated term by term against
//    exp(-s t) t^{-3/2-k}: closed form for s = 0, erfc and upward recurrence
//    for 0 < s T <= 1. For s T* > 1 the panels are instead extended to
//    t = 45 / s, where exp(-s t) makes the rest negligible.
// The spectrum of the evenly embedded table is a separable cosine transform
// evaluated by three passes of a (N+1) x N cosine matrix.
#include <cmath>
#include <vector>

#include "lgf.cuh"

namespace bae {

namespace {

constexpr int NODES0 = 20;    // Gauss-Legendre points on [0, 1]
constexpr int NODESP = 16;    // points per unit panel in ln t
constexpr int TAIL_K = 7;     // tail series terms (k = 0..6)

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {   // final derivative at the converged node
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

struct Plan {
    int N = 0;
    double s = 0.0;
    int n_nodes = 0;
    int q0 = 0;                             // panels below t = 1
    std::vector<double> t, wexp;            // nodes and weights * exp(-s t)
    std::vector<int> panels;                // P per max index a
    std::vector<int> tail_mode;             // 0 none, 1 s = 0, 2 erfc recurrence
};

Plan make_plan(int N, double s) {
    Plan p;
    p.N = N;
    p.s = s;
    p.panels.resize(N);
    p.tail_mode.resize(N);
    int pmax = 1;
    for (int a = 0; a < N; ++a) {
        int P = 7;
        if (a > 0) P = std::max(7, (int)std::ceil(std::log(100.0 * a * a)));
        int mode = (s == 0.0) ? 1 : 2;
        if (s > 0.0 && s * std::exp((double)P) > 1.0) {
            P = std::max(1, (int)std::ceil(std::log(45.0 / s)));
            mode = 0;
        }
        p.panels[a] = P;
        p.tail_mode[a] = mode;
        pmax = std::max(pmax, P);
    }
    p.q0 = s > 1.0 ? (int)std::ceil(std::log(s)) : 0;
    const double t0 = std::exp(-(double)p.q0);
    std::vector<double> x20, w20, x16, w16;
    gauss_legendre(NODES0, x20, w20);
    gauss_legendre(NODESP, x16, w16);
    for (int i = 0; i < NODES0; ++i) {
        p.t.push_back(0.5 * t0 * (x20[i] + 1.0));
        p.wexp.push_back(0.5 * t0 * w20[i]);
    }
    for (int q = 1 - p.q0; q <= pmax; ++q)
        for (int i = 0; i < NODESP; ++i) {
            const double u = q - 0.5 + 0.5 * x16[i];
            const double tt = std::exp(u);
            p.t.push_back(tt);
            p.wexp.push_back(0.5 * w16[i] * tt);
        }
    p.n_nodes = (int)p.t.size();
    for (int j = 0; j < p.n_nodes; ++j) p.wexp[j] *= std::exp(-s * p.t[j]);
    return p;
}

// Ie_n(2 t_j), n < N, one CTA per node; thread 0 runs the recurrence.
__global__ void k_bessel_rows(const double* __restrict__ t, int N, double* __restrict__ rows) {
    extern __shared__ double s_row[];
    const int j = blockIdx.x;
    if (threadIdx.x == 0) {
        const double x = 2.0 * t[j];
        const long long M = (long long)ceil(sqrt((double)N * N + 80.0 * x)) + 20;
        const double twox = 2.0 / x;
        double y1 = 0.0, y0 = 1e-280, S = 0.0;
        for (int n = 0; n < N; ++n) s_row[n] = 0.0;
        for (long long k = M; k >= 1; --k) {
            if (k < N) s_row[k] = y0;
            S += 2.0 * y0;
            const double ym = (double)k * twox * y0 + y1;
            y1 = y0;
            y0 = ym;
            if (ym > 1e250) {
                y1 *= 1e-250;
                y0 *= 1e-250;
                S *= 1e-250;
                const int top = (int)(k < N ? k : N);
                for (int n = top; n < N; ++n) s_row[n] *= 1e-250;
            }
        }
        s_row[0] = y0;
        S += y0;
        const double inv = 1.0 / S;
        for (int n = 0; n < N; ++n) s_row[n] *= inv;
    }
    __syncthreads();
    for (int n = threadIdx.x; n < N; n += blockDim.x) rows[(long long)j * N + n] = s_row[n];
}

__device__ __forceinline__ long long tet(long long a) { return a * (a + 1) * (a + 2) / 6; }
__device__ __forceinline__ long long tri2(long long b) { return b * (b + 1) / 2; }

__device__ void decode_triple(long long idx, int& a, int& b, int& c) {
    long long A = (long long)cbrt(6.0 * (double)idx);
    while (A > 0 && tet(A) > idx) --A;
    while (tet(A + 1) <= idx) ++A;
    long long r = idx - tet(A);
    long long Bv = (long long)sqrt(2.0 * (double)r);
    while (Bv > 0 && tri2(Bv) > r) --Bv;
    while (tri2(Bv + 1) <= r) ++Bv;
    a = (int)A;
    b = (int)Bv;
    c = (int)(r - tri2(Bv));
}

// Coefficients alpha_j(n) of Ie_n(2t) ~ (4 pi t)^{-1/2} sum_j alpha_j t^{-j}:
// alpha_j = (-1)^j a_j(mu) / 2^j, a_j = prod_{i<=j} (mu - (2i-1)^2) / (j! 8^j).
__device__ void tail_alpha(int n, double* al) {
    const double mu = 4.0 * (double)n * (double)n;
    double c = 1.0;
    al[0] = 1.0;
    for (int j = 1; j < TAIL_K; ++j) {
        c *= (mu - (double)((2 * j - 1) * (2 * j - 1))) / (8.0 * j);
        al[j] = ((j & 1) ? -c : c) / (double)(1LL << j);
    }
}

__global__ void k_lgf_table(const double* __restrict__ rows, const double* __restrict__ wexp,
                            const int* __restrict__ panels, const int* __restrict__ tail_mode,
                            int N, double s, int q0, long long ntri, double* __restrict__ out) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ntri;
         idx += (long long)gridDim.x * blockDim.x) {
        int a, b, c;
        decode_triple(idx, a, b, c);
        const int P = panels[a];
        const int nn = NODES0 + NODESP * (P + q0);
        double acc = 0.0;
        for (int j = 0; j < nn; ++j) {
            const double* r = rows + (long long)j * N;
            acc += wexp[j] * (r[a] * r[b] * r[c]);
        }
        const int mode = tail_mode[a];
        if (mode != 0) {
            double al[TAIL_K], bl[TAIL_K], cl[TAIL_K], ab[TAIL_K];
            tail_alpha(a, al);
            tail_alpha(b, bl);
            tail_alpha(c, cl);
            for (int k = 0; k < TAIL_K; ++k) {
                double v = 0.0;
                for (int i = 0; i <= k; ++i) v += al[i] * bl[k - i];
                ab[k] = v;
            }
            const double T = exp((double)P);
            const double rT = 1.0 / sqrt(T);
            double E = 0.0, tail = 0.0, Tpow = rT;  // Tpow = T^{-1/2-k}
            const double eT = (mode == 2) ? exp(-s * T) : 1.0;
            for (int k = 0; k < TAIL_K; ++k) {
                if (mode == 1) {
                    E = Tpow / (k + 0.5);
                } else if (k == 0) {
                    E = 2.0 * rT * eT - 2.0 * sqrt(M_PI * s) * erfc(sqrt(s * T));
                } else {
                    E = (Tpow * eT - s * E) / (k + 0.5);
                }
                double beta = 0.0;
                for (int i = 0; i <= k; ++i) beta += ab[i] * cl[k - i];
                tail += beta * E;
                Tpow /= T;
            }
            acc += tail * (1.0 / (8.0 * M_PI * sqrt(M_PI)));  // (4 pi)^{-3/2}
        }
        out[idx] = acc;
    }
}

// cube[(i (N+1) + j)(N+1) + k] = G(sorted(i,j,k)) for i,j,k < N, 0 if any == N
__global__ void k_expand_cube(const double* __restrict__ table, int N, double* __restrict__ cube) {
    const long long N1 = N + 1;
    const long long n = N1 * N1 * N1;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n;
         x += (long long)gridDim.x * blockDim.x) {
        int i = (int)(x / (N1 * N1)), j = (int)((x / N1) % N1), k = (int)(x % N1);
        double v = 0.0;
        if (i < N && j < N && k < N) {
            int a = max(i, max(j, k)), c = min(i, min(j, k));
            int b = i + j + k - a - c;
            v = table[(long long)a * (a + 1) * (a + 2) / 6 + (long long)b * (b + 1) / 2 + c];
        }
        cube[x] = v;
    }
}

// cosine matrix Cm[k][n] = w(n) cos(pi k n / N), w(0) = 1, w(n) = 2, k <= N, n < N
__global__ void k_cos_matrix(int N, double* Cm) {
    const int N1 = N + 1;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N1 * N; x += gridDim.x * blockDim.x) {
        const int k = x / N, n = x % N;
        const int r = (int)(((long long)k * n) % (2 * N));
        Cm[x] = (n == 0 ? 1.0 : 2.0) * cospi((double)r / (double)N);
    }
}

// Lines of length N+1 (entry N ignored on input): out[line][k] = sum_n Cm[k][n] in[line][n].
// Line element e sits at base(line) + e * estride; 32 lines per CTA, one
// warp per output k group.
__global__ void k_cos_pass(const double* __restrict__ in, double* __restrict__ out, const double* __restrict__ Cm,
                           int N, long long nlines, long long estride, long long lstride_inner,
                           long long ninner, long long lstride_outer) {
    extern __shared__ double s_lines[];  // [32][N+1+1]
    const int N1 = N + 1;
    const int LS = N1 + 1;
    const long long line0 = (long long)blockIdx.x * 32;
    // load 32 lines
    for (int idx = threadIdx.x; idx < 32 * N; idx += blockDim.x) {
        const int ln = idx % 32, e = idx / 32;
        const long long line = line0 + ln;
        double v = 0.0;
        if (line < nlines) {
            const long long base = (line / ninner) * lstride_outer + (line % ninner) * lstride_inner;
            v = in[base + e * estride];
        }
        s_lines[ln * LS + e] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const long long line = line0 + lane;
    const long long base = (line / ninner) * lstride_outer + (line % ninner) * lstride_inner;
    for (int k = warp; k < N1; k += nwarp) {
        const double* crow = Cm + (long long)k * N;
        double acc = 0.0;
        for (int n = 0; n < N; ++n) acc += crow[n] * s_lines[lane * LS + n];
        if (line < nlines) out[base + k * estride] = acc;
    }
}

// The spectrum of the (2N)-periodic Green's function in closed form, i.e.
// the 2N-point trapezoid rule of the Fourier integral eq. [lgf] read in
// frequency space (Section 2.2, sigma > 0): scale / (6 + s - 2 sum_i
// cos(pi k_i / N)) on the octant 0 <= k_i <= N.
__global__ void k_periodic_spectrum(int N, double s, double scale, double* g64, float* g32) {
    const long long N1 = N + 1, n3 = N1 * N1 * N1;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n3; x += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(x / (N1 * N1)), j = (int)((x / N1) % N1), k = (int)(x % N1);
        const double c = cospi((double)i / N) + cospi((double)j / N) + cospi((double)k / N);
        const double v = scale / (6.0 + s - 2.0 * c);
        g64[x] = v;
        if (g32) g32[x] = (float)v;
    }
}

__global__ void k_scale_out(const double* in, long long n, double scale, double* g64, float* g32) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        const double v = in[x] * scale;
        g64[x] = v;
        if (g32) g32[x] = (float)v;
    }
}

__global__ void k_twiddles(int L, double2* tw64, float2* tw32) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)m / (double)L, &sn, &cs);
        if (tw64) tw64[m] = make_double2(cs, -sn);
        if (tw32) tw32[m] = make_float2((float)cs, (float)-sn);
    }
}

template <typename T>
struct DevBuf {
    T* p = nullptr;
    cudaStream_t st;
    DevBuf(size_t n, cudaStream_t s) : st(s) { p = dev_alloc_n<T>((long long)n, s); }
    ~DevBuf() { dev_free(p, st); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
};

void table_into(int N, double s, double* out, cudaStream_t st) {
    Plan plan = make_plan(N, s);
    DevBuf<double> d_t(plan.n_nodes, st), d_w(plan.n_nodes, st), d_rows((size_t)plan.n_nodes * N, st);
    DevBuf<int> d_p(N, st), d_m(N, st);
    BAE_CUDA(cudaMemcpyAsync(d_t.p, plan.t.data(), plan.n_nodes * sizeof(double), cudaMemcpyHostToDevice, st));
    BAE_CUDA(cudaMemcpyAsync(d_w.p, plan.wexp.data(), plan.n_nodes * sizeof(double), cudaMemcpyHostToDevice, st));
    BAE_CUDA(cudaMemcpyAsync(d_p.p, plan.panels.data(), N * sizeof(int), cudaMemcpyHostToDevice, st));
    BAE_CUDA(cudaMemcpyAsync(d_m.p, plan.tail_mode.data(), N * sizeof(int), cudaMemcpyHostToDevice, st));
    BAE_LAUNCH("k_bessel_rows", st, k_bessel_rows<<<plan.n_nodes, 128, N * sizeof(double), st>>>(d_t.p, N, d_rows.p));
    const long long ntri = (long long)N * (N + 1) * (N + 2) / 6;
    const int blocks = (int)std::min<long long>((ntri + 255) / 256, 152LL * 16);
    BAE_LAUNCH("k_lgf_table", st, k_lgf_table<<<blocks, 256, 0, st>>>(d_rows.p, d_w.p, d_p.p, d_m.p, N, s, plan.q0, ntri, out));
    BAE_CUDA(cudaStreamSynchronize(st));  // host vectors and scratch die here
}

}  // namespace

void lgf_table(int N, double s, double* out, cudaStream_t st) {
    BAE_REQUIRE(N >= 2 && N <= 256, BAE_ERR_INVALID_ARG, "lgf_table: N must be in [2, 256]");
    BAE_REQUIRE(std::isfinite(s) && s >= 0.0, BAE_ERR_INVALID_ARG, "lgf_table: s must be finite and >= 0");
    table_into(N, s, out, st);
}

// The spectrum of the finite-box Green's function of eq. [aux]: with the
// source extended oddly about the layers 0 and N in every axis, the box
// solve is the convolution with the (2N)-periodic Green's function, whose
// spectrum is scale / (6 + s - 2 sum cos(pi k_d / N)). Its only pole (s = 0,
// k = 0) multiplies a zero of the odd data and is set to 0.
__global__ void k_box_spectrum(int N, double s, double scale, double* g64, float* g32) {
    const long long N1 = N + 1, n3 = N1 * N1 * N1;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n3; x += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(x / (N1 * N1)), j = (int)((x / N1) % N1), k = (int)(x % N1);
        const double c = cospi((double)i / N) + cospi((double)j / N) + cospi((double)k / N);
        const double d = 6.0 + s - 2.0 * c;
        const double v = d != 0.0 ? scale / d : 0.0;
        g64[x] = v;
        if (g32) g32[x] = (float)v;
    }
}

void box_spectrum(int N, double s, double scale, double* g64, float* g32, cudaStream_t st) {
    BAE_REQUIRE(is_pow2(N) && N >= 8 && N <= 256, BAE_ERR_INVALID_ARG,
                "box_spectrum: N must be a power of two in [8, 256]");
    BAE_REQUIRE(std::isfinite(s) && s >= 0.0, BAE_ERR_INVALID_ARG, "box_spectrum: s must be finite and >= 0");
    const long long N1 = N + 1, n3 = N1 * N1 * N1;
    BAE_LAUNCH("k_box_spectrum", st,
               k_box_spectrum<<<(int)std::min<long long>((n3 + 255) / 256, 152LL * 16), 256, 0, st>>>(N, s, scale,
                                                                                                        g64, g32));
}

bool periodic_spectrum_applies(int N, double s) {
    if (!(s > 0.0)) return false;
    const double mu = std::acosh(1.0 + 0.5 * s);   // G_s ~ exp(-mu |n|) along an axis
    return std::pow(2.0 * N, 3) * std::exp(-mu * N) < 1e-14;
}

void lgf_spectrum(int N, double s, double scale, double* g64, float* g32, cudaStream_t st) {
    BAE_REQUIRE(is_pow2(N) && N >= 8 && N <= 256, BAE_ERR_INVALID_ARG,
                "lgf_spectrum: N must be a power of two in [8, 256]");
    BAE_REQUIRE(std::isfinite(s) && s >= 0.0, BAE_ERR_INVALID_ARG, "lgf_spectrum: s must be finite and >= 0");
    const long long N1 = N + 1;
    const long long n3 = N1 * N1 * N1;
    if (periodic_spectrum_applies(N, s)) {
        // the images of the (2N)-periodic Green's function are below
        // round-off: no table, no cosine transform
        BAE_LAUNCH("k_periodic_spectrum", st,
                   k_periodic_spectrum<<<(int)std::min<long long>((n3 + 255) / 256, 152LL * 16), 256, 0, st>>>(
                       N, s, scale, g64, g32));
        BAE_CUDA(cudaStreamSynchronize(st));
        return;
    }
    const long long ntri = (long long)N * (N + 1) * (N + 2) / 6;
    DevBuf<double> tab(ntri, st), c0(n3, st), c1(n3, st), Cm(N1 * N, st);
    table_into(N, s, tab.p, st);
    BAE_LAUNCH("k_expand_cube", st, k_expand_cube<<<(int)std::min<long long>((n3 + 255) / 256, 152LL * 16), 256, 0, st>>>(tab.p, N, c0.p));
    BAE_LAUNCH("k_cos_matrix", st, k_cos_matrix<<<ceil_div(N1 * N, 256), 256, 0, st>>>(N, Cm.p));
    const size_t smem = 32 * (N1 + 1) * sizeof(double);
    BAE_CUDA(cudaFuncSetAttribute(k_cos_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long nlines = N1 * N1;
    const int blocks = ceil_div(nlines, 32);
    // axis 3 (contiguous): line = (i, j), base = line * N1, element stride 1
    BAE_LAUNCH("k_cos_pass", st, k_cos_pass<<<blocks, 256, smem, st>>>(c0.p, c1.p, Cm.p, N, nlines, 1, N1, nlines, 0));
    // axis 2: line = (i, k), base = i * N1^2 + k, element stride N1
    BAE_LAUNCH("k_cos_pass", st, k_cos_pass<<<blocks, 256, smem, st>>>(c1.p, c0.p, Cm.p, N, nlines, N1, 1, N1, N1 * N1));
    // axis 1: line = (j, k), base = j * N1 + k, element stride N1^2
    BAE_LAUNCH("k_cos_pass", st, k_cos_pass<<<blocks, 256, smem, st>>>(c0.p, c1.p, Cm.p, N, nlines, N1 * N1, 1, nlines, 0));
    BAE_LAUNCH("k_scale_out", st, k_scale_out<<<(int)std::min<long long>((n3 + 255) / 256, 152LL * 16), 256, 0, st>>>(c1.p, n3, scale, g64, g32));
    BAE_CUDA(cudaStreamSynchronize(st));
}

void make_twiddles(int L, double2* tw64, float2* tw32, cudaStream_t st) {
    BAE_LAUNCH("k_twiddles", st, k_twiddles<<<ceil_div(L, 256), 256, 0, st>>>(L, tw64, tw32));
}

}  // namespace bae
