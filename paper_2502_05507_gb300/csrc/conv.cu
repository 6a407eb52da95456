// The matrix-free potential apply: source stencil, zero-padded (2N)^3 real
// FFT convolution with the lattice Green's function, and the gathers.
//
// v(m) = sum_x G_s(m - x) rho(x) for m, x in the N^3 grid (Section 3.2,
// eqs. [single_potential] and [double_potential]; Section 2.1, eq. [ps] for
// the volume source). Offsets m - x lie in (-N, N)^3, so the linear
// convolution equals the circular one on the (2N)^3 box with G embedded
// evenly (offset N unused). Its spectrum is real and even and is stored on
// the octant (N+1)^3 with the 1/(2N)^3 of the inverse transform folded in.
//
// Data layout (per right-hand side), i = x index (outermost), k = z (fastest):
//   A[i][j][kk]  i < N, j < N,  kk <= N   after the R2C pass along k
//   B[i][jj][kk] i < N, jj < 2N, kk <= N  after the pass along j
// Passes (forward, then inverse in reverse order):
//   kpass   : two real k-lines per complex FFT (x_a + i x_b), only the N
//             nonzero samples are loaded, spectra split by Hermitian symmetry
//   jpass   : FFT along j (N nonzero inputs, 2N outputs)      A -> B
//   ipass   : FFT along i (N nonzero), times ghat, inverse FFT, keep i < N,
//             in place in B
//   jpass^-1: inverse along j, keep j < N                     B -> A
//   kpass^-1: C2R of two lines per complex inverse FFT, keep k < N -> v
#include "conv.cuh"
#include "fft.cuh"

namespace bae {

namespace {

template <int L> struct Shape {
    static constexpr int TPL = L / 8;                       // threads per line
    static constexpr int PPC = (256 / TPL) > 0 ? 256 / TPL : 1;  // k-pass FFTs per CTA
    static constexpr int W = (256 / TPL) < 8 ? 8 : ((256 / TPL) > 32 ? 32 : 256 / TPL);  // columns per CTA
    static constexpr int STRIDE = L + 1;                    // padded line stride in smem
};

template <typename C>
__device__ __forceinline__ void load_twiddles(C* s_tw, const C* tw, int L) {
    for (int m = threadIdx.x; m < L; m += blockDim.x) s_tw[m] = tw[m];
}

// ------------------------------------------------------------- k pass (R2C)
template <typename T, int L>
__global__ void __launch_bounds__(256) k_kpass_fwd(ConvArgs<T> a) {
    using C = cplx_t<T>;
    using S = Shape<L>;
    constexpr int N = L / 2;
    constexpr int N1 = N + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s_tw = reinterpret_cast<C*>(smem_raw);
    C* s_lines = s_tw + L;

    const int b = blockIdx.z;
    const int p = threadIdx.x / S::TPL;          // FFT slot in this CTA
    const int t = threadIdx.x % S::TPL;
    const long long pair = (long long)blockIdx.x * S::PPC + p;
    const bool active = pair < (long long)N * N / 2;
    C* line = s_lines + p * S::STRIDE;

    load_twiddles(s_tw, a.tw, L);
    for (int k = t; k < L; k += S::TPL) line[k] = cmake<C>((T)0, (T)0);
    __syncthreads();

    if (active) {
        const long long la = 2 * pair, lb = la + 1;
        if (a.mode == SRC_DENSITY) {
            const double* q = a.q + (long long)b * a.q_stride;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const long long l = half ? lb : la;
                const int s0 = a.rec.line_off[l], s1 = a.rec.line_off[l + 1];
                for (int s = s0 + t; s < s1; s += S::TPL) {
                    const int k = a.rec.src_lin[s] - (int)(l * N);
                    double val = 0.0;
                    for (int e = a.rec.term_off[s]; e < a.rec.term_off[s + 1]; ++e)
                        val += (double)a.rec.term_coef[e] * q[a.rec.term_idx[e]];
                    if (half) line[k].y = (T)val; else line[k].x = (T)val;
                }
            }
        } else {
            const double* f = a.f + (long long)b * N * N * N;
            for (int k = t; k < N; k += S::TPL) {
                const long long xa = la * N + k, xb = lb * N + k;
                const double va = (a.flags[xa] & 1) ? a.scale * f[xa] : 0.0;
                const double vb = (a.flags[xb] & 1) ? a.scale * f[xb] : 0.0;
                line[k] = cmake<C>((T)va, (T)vb);
            }
        }
    }
    __syncthreads();
    fft_line<C, L, false>(line, s_tw, t);

    if (active) {
        C* A = a.A + (long long)b * N * N * N1;
        const long long la = 2 * pair, lb = la + 1;
        const T half = (T)0.5;
        for (int k = t; k <= N; k += S::TPL) {
            const C z = line[k];
            const C zr = line[(L - k) & (L - 1)];
            A[la * N1 + k] = cmake<C>((z.x + zr.x) * half, (z.y - zr.y) * half);
            A[lb * N1 + k] = cmake<C>((z.y + zr.y) * half, (zr.x - z.x) * half);
        }
    }
}

// ----------------------------------------------------- column passes (j, i)
enum ColMode { COL_FWD_J = 0, COL_CONV_I = 1, COL_INV_J = 2 };

template <typename T, int L, int MODE>
__global__ void __launch_bounds__(512) k_colpass(ConvArgs<T> a) {
    using C = cplx_t<T>;
    using S = Shape<L>;
    constexpr int N = L / 2;
    constexpr int N1 = N + 1;
    constexpr int W = S::W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s_tw = reinterpret_cast<C*>(smem_raw);
    C* s_lines = s_tw + L;

    const int b = blockIdx.z;
    const int o = blockIdx.y;               // i (j passes) or jj (i pass)
    const int col0 = blockIdx.x * W;        // first kk column
    const int nthr = blockDim.x;

    const C* in;
    C* out;
    long long stride;
    int n_in, n_out;
    C* Ab = a.A + (long long)b * N * N * N1;
    C* Bb = a.B + (long long)b * N * (2 * N) * N1;
    if (MODE == COL_FWD_J) {
        in = Ab + (long long)o * N * N1; out = Bb + (long long)o * (2 * N) * N1;
        stride = N1; n_in = N; n_out = 2 * N;
    } else if (MODE == COL_CONV_I) {
        in = Bb + (long long)o * N1; out = Bb + (long long)o * N1;
        stride = (long long)(2 * N) * N1; n_in = N; n_out = N;
    } else {
        in = Bb + (long long)o * (2 * N) * N1; out = Ab + (long long)o * N * N1;
        stride = N1; n_in = 2 * N; n_out = N;
    }

    load_twiddles(s_tw, a.tw, L);
    for (int idx = threadIdx.x; idx < W * L; idx += nthr) {
        const int w = idx % W, e = idx / W;
        const int col = col0 + w;
        C val = cmake<C>((T)0, (T)0);
        if (e < n_in && col < N1) val = in[e * stride + col];
        s_lines[w * S::STRIDE + e] = val;
    }
    __syncthreads();

    const int w = threadIdx.x / S::TPL;
    const int t = threadIdx.x % S::TPL;
    C* line = s_lines + w * S::STRIDE;
    fft_line<C, L, MODE == COL_INV_J>(line, s_tw, t);

    if (MODE == COL_CONV_I) {
        const int col = col0 + w;
        if (col < N1) {
            const int jj = o <= N ? o : L - o;
            const T* g = a.ghat + (long long)jj * N1 + col;
            for (int e = t; e < L; e += S::TPL) {
                const int ii = e <= N ? e : L - e;
                const T gv = g[(long long)ii * N1 * N1];
                line[e] = cscale(line[e], gv);
            }
        }
        __syncthreads();
        fft_line<C, L, true>(line, s_tw, t);
    }

    for (int idx = threadIdx.x; idx < W * n_out; idx += nthr) {
        const int ww = idx % W, e = idx / W;
        const int col = col0 + ww;
        if (col < N1) out[e * stride + col] = s_lines[ww * S::STRIDE + e];
    }
}

// ----------------------------------------------------------- k pass (C2R)
template <typename T, int L>
__global__ void __launch_bounds__(256) k_kpass_inv(ConvArgs<T> a) {
    using C = cplx_t<T>;
    using S = Shape<L>;
    constexpr int N = L / 2;
    constexpr int N1 = N + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s_tw = reinterpret_cast<C*>(smem_raw);
    C* s_lines = s_tw + L;

    const int b = blockIdx.z;
    const int p = threadIdx.x / S::TPL;
    const int t = threadIdx.x % S::TPL;
    const long long pair = (long long)blockIdx.x * S::PPC + p;
    const bool active = pair < (long long)N * N / 2;
    C* line = s_lines + p * S::STRIDE;
    const long long la = 2 * pair, lb = la + 1;
    const C* A = a.A + (long long)b * N * N * N1;

    load_twiddles(s_tw, a.tw, L);
    for (int k = t; k < L; k += S::TPL) {
        C z = cmake<C>((T)0, (T)0);
        if (active) {
            C xa, xb;
            if (k <= N) {
                xa = A[la * N1 + k];
                xb = A[lb * N1 + k];
                if (k == 0 || k == N) { xa.y = (T)0; xb.y = (T)0; }
            } else {
                xa = cconj(A[la * N1 + (L - k)]);
                xb = cconj(A[lb * N1 + (L - k)]);
            }
            z = cmake<C>(xa.x - xb.y, xa.y + xb.x);   // xa + i xb
        }
        line[k] = z;
    }
    __syncthreads();
    fft_line<C, L, true>(line, s_tw, t);
    if (active) {
        T* v = a.v + (long long)b * N * N * N;
        for (int k = t; k < N; k += S::TPL) {
            const C z = line[k];
            v[la * N + k] = z.x;
            v[lb * N + k] = z.y;
        }
    }
}

template <typename T>
const char* kname(const char* f32, const char* f64) { return sizeof(T) == 4 ? f32 : f64; }

template <typename T, int L>
void run_conv(const ConvArgs<T>& a, cudaStream_t st) {
    using C = cplx_t<T>;
    using S = Shape<L>;
    constexpr int N = L / 2;
    const size_t smem_k = (size_t)(L + S::PPC * S::STRIDE) * sizeof(C);
    const size_t smem_c = (size_t)(L + S::W * S::STRIDE) * sizeof(C);
    static bool configured = false;  // per instantiation
    if (!configured) {
        BAE_CUDA(cudaFuncSetAttribute(k_kpass_fwd<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k));
        BAE_CUDA(cudaFuncSetAttribute(k_kpass_inv<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k));
        BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_FWD_J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_CONV_I>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_INV_J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        configured = true;
    }
    const int nb = a.nbatch;
    const dim3 gk(ceil_div((long long)N * N / 2, S::PPC), 1, nb);
    const int tk = S::PPC * S::TPL;
    const int ncolblk = ceil_div(N + 1, S::W);
    const int tc = S::W * S::TPL;
    BAE_LAUNCH(kname<T>("conv_kfwd.f32", "conv_kfwd.f64"), st, k_kpass_fwd<T, L><<<gk, tk, smem_k, st>>>(a));
    BAE_LAUNCH(kname<T>("conv_jfwd.f32", "conv_jfwd.f64"), st, k_colpass<T, L, COL_FWD_J><<<dim3(ncolblk, N, nb), tc, smem_c, st>>>(a));
    BAE_LAUNCH(kname<T>("conv_i.f32", "conv_i.f64"), st, k_colpass<T, L, COL_CONV_I><<<dim3(ncolblk, 2 * N, nb), tc, smem_c, st>>>(a));
    BAE_LAUNCH(kname<T>("conv_jinv.f32", "conv_jinv.f64"), st, k_colpass<T, L, COL_INV_J><<<dim3(ncolblk, N, nb), tc, smem_c, st>>>(a));
    BAE_LAUNCH(kname<T>("conv_kinv.f32", "conv_kinv.f64"), st, k_kpass_inv<T, L><<<gk, tk, smem_k, st>>>(a));
}

// ------------------------------------------------------------------ gathers
template <typename T>
__global__ void k_closure_gather(const T* v, long long v_stride, const int* gm, const int* partner,
                                 const double* t, int n, double* out, long long out_stride) {
    const int b = blockIdx.y;
    const T* vb = v + b * v_stride;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const double tr = t[r];
        out[b * out_stride + r] = tr * (double)vb[gm[r]] + (1.0 - tr) * (double)vb[partner[r]];
    }
}

template <typename T>
__global__ void k_volume_combine(const T* v, const double* add, const uint8_t* flags, long long n3, double* u) {
    const int b = blockIdx.y;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n3; x += (long long)gridDim.x * blockDim.x) {
        const bool np = (flags[x] & 3) != 0;   // M+ or gamma-
        u[b * n3 + x] = np ? (add ? add[b * n3 + x] : 0.0) + (double)v[b * n3 + x] : 0.0;
    }
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
void closure_gather(const T* v, long long v_stride, const int* gm, const int* partner, const double* t,
                    int n, int nbatch, double* out, long long out_stride, cudaStream_t st) {
    if (n == 0) return;
    dim3 grid(ceil_div(n, 256) < 1184 ? ceil_div(n, 256) : 1184, nbatch);
    BAE_LAUNCH(kname<T>("closure_gather.f32", "closure_gather.f64"), st, k_closure_gather<T><<<grid, 256, 0, st>>>(v, v_stride, gm, partner, t, n, out, out_stride));
}

template <typename T>
void volume_combine(const T* v, const double* add, const uint8_t* flags, long long n3, int nbatch,
                    double* u, cudaStream_t st) {
    dim3 grid(ceil_div(n3, 256) < 2432 ? ceil_div(n3, 256) : 2432, nbatch);
    BAE_LAUNCH("k_volume_combine", st, k_volume_combine<T><<<grid, 256, 0, st>>>(v, add, flags, n3, u));
}

template <typename T>
void widen(const T* v, long long n, double* out, cudaStream_t st) {
    BAE_LAUNCH("k_widen", st, k_widen<T><<<ceil_div(n, 256) < 2432 ? ceil_div(n, 256) : 2432, 256, 0, st>>>(v, n, out));
}

template void conv_apply<float>(const ConvArgs<float>&, cudaStream_t);
template void conv_apply<double>(const ConvArgs<double>&, cudaStream_t);
template void closure_gather<float>(const float*, long long, const int*, const int*, const double*, int, int, double*, long long, cudaStream_t);
template void closure_gather<double>(const double*, long long, const int*, const int*, const double*, int, int, double*, long long, cudaStream_t);
template void volume_combine<float>(const float*, const double*, const uint8_t*, long long, int, double*, cudaStream_t);
template void volume_combine<double>(const double*, const double*, const uint8_t*, long long, int, double*, cudaStream_t);
template void widen<float>(const float*, long long, double*, cudaStream_t);
template void widen<double>(const double*, long long, double*, cudaStream_t);

}  // namespace bae
