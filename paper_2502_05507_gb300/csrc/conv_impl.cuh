#pragma once
// Kernels of the matrix-free potential apply: source stencil, zero-padded (2N)^3 real
// FFT convolution with the lattice Green's function, and the gathers.
//
// v(m) = sum_x G_s(m - x) rho(x) for m, x in the N^3 grid (Section 3.2,
// eqs. [single_potential] and [double_potential]; Section 2.1, eq. [ps] for
// the volume source). Offsets m - x lie in (-N, N)^3, so the linear
// convolution equals the circular one on the (2N)^3 box with G embedded
// evenly (offset N unused). Its spectrum is real and even and is stored on
// the octant (N+1)^3 with the 1/(2N)^3 of the inverse transform folded in.
//
// Data layout (per right-hand side), i = x index (outermost), k = z (fastest),
// rows of N + 1 elements of which columns kk < N are used (column 0 holds
// the real kk = 0 and kk = N spectra packed, see conv_geo.cuh):
//   A[i][j][kk]  i < N, j < N,  kk < N    after the R2C pass along k
//   B[i][jj][kk] i < N, jj < 2N, kk < N   after the pass along j
// Only the x-planes [p0, p1) of ConvArgs are transformed.
// Every pass transforms its lines in registers (four-step factorisation,
// one shared-memory exchange per transform, see fft2.cuh), reading and
// writing global memory directly. Passes (forward, then inverse in reverse
// order):
//   kpass   : two real k-lines per complex FFT (x_a + i x_b), only the N
//             nonzero samples are loaded, spectra split by Hermitian symmetry
//   jpass   : FFT along j (N nonzero inputs, 2N outputs)      A -> B
//   ipass   : FFT along i (N nonzero), times ghat, inverse FFT, keep i < N,
//             in place in B
//   jpass^-1: inverse along j, keep j < N                     B -> A
//   kpass^-1: C2R of two lines per complex inverse FFT, keep k < N -> v
//
// A thread holding sample n = t + R1 m of a line (0 <= t < R1, R1 R2 = 2N)
// holds a nonzero input / a kept output exactly when m < R2 / 2; the kernels
// test m, a compile-time index, so the compiler drops the arithmetic on the
// zero padding and on the discarded half.
#include <map>
#include <mutex>
#include <string>
#include <type_traits>

#include "conv_geo.cuh"
#include "conv_tune.cuh"

// Included once per element type by conv_<type>.cu, which instantiates
// run_conv and conv_configure for its transform lengths, so the kernels of
// the three element types compile in parallel.

namespace bae {

namespace {

// ------------------------------------------------------------- k pass (R2C)
// Two real k-lines (i, 2p) and (i, 2p+1) per complex transform z = x_a + i x_b.
// BOX: the finite auxiliary box of eq. [aux] (volume sources only): the
// upper half of each line holds the negated mirror of the lower half, x[2N -
// n] = -x[n], x[N] = 0 (odd about the layers 0 and N), instead of zeros.
template <typename T, int L, bool BOX, int V>
__device__ __forceinline__ void kpass_fwd_tile(const ConvArgs<T>& a, int bx, int bz) {
    using C = cplx_t<T>;
    using G = Geo<T, L, V>;
    using PL = typename G::PL;
    constexpr int N = L / 2, N1 = N + 1, TH = G::TH, S = G::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* xch = reinterpret_cast<C*>(smem_raw);                 // P * XS
    T* rho = reinterpret_cast<T*>(xch + G::P * G::XS);      // P * RS

    const int b = bz;
    if (a.active && !a.active[b]) return;   // whole CTA: no barrier is skipped
    const int t = threadIdx.x % TH;
    const int p = threadIdx.x / TH;
    const long long gp0 = (long long)bx * G::P;   // the CTA's first line pair
    const long long np = a.npairs();
    const bool active = gp0 + p < np;
    const long long la = a.pair_line(gp0 + p), lb = la + 1;
    T* r = rho + p * G::RS;

    C v[S];
    if (a.mode == SRC_DENSITY) {
        for (int k = t; k < 2 * N; k += TH)
            r[k] = active ? volume_or_zero(a, b, (k < N ? la : lb) * N + (k < N ? k : k - N)) : (T)0;
        __syncthreads();
        {
            // the sources of the CTA's lines are one contiguous range of the
            // recipe (from its first line to its last; across a plane
            // boundary the lines between are outside [q0, q1) and hold no
            // source): every thread of the CTA takes sources of the range,
            // so each chain of dependent loads (offsets, node, terms,
            // density) runs once, not once per line
            const long long gp1 = min(gp0 + (long long)G::P, np);
            if (gp0 < gp1) {
                const long long l0 = a.pair_line(gp0), l1 = a.pair_line(gp1 - 1) + 2;
                const double* q =
                    a.q + (long long)b * a.q_stride + (a.q_row ? (long long)a.q_row[b] * a.q_row_stride : 0);
                const float* q32 = a.q32 ? a.q32 + (long long)b * a.q32_stride : nullptr;
                const int s0 = a.rec.line_off[l0], s1 = a.rec.line_off[l1];
                const int npq = a.pairs_per_plane(), jlo = a.line_lo(), jhi = a.line_hi();
                for (int s = s0 + (int)threadIdx.x; s < s1; s += (int)blockDim.x) {
                    const int lin = a.rec.src_lin[s];
                    const int line = lin / N, ip = line / N, jl = line % N;
                    // pair within the CTA, half of the pair
                    const long long loc = (long long)(ip - a.plane_lo()) * npq + (jl - jlo) / 2 - gp0;
                    if (jl >= jlo && jl < jhi && loc >= 0 && loc < G::P)
                        rho[loc * G::RS + (jl & 1) * N + (lin % N)] = source_value<T>(a.rec, s, q, q32);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < S; ++m) {
            const int n = t + TH * m;
            v[m] = (m < S / 2) ? cmake<C>(r[n], r[N + n]) : cmake<C>((T)0, (T)0);
        }
    } else {
        const double* f = a.f + (long long)b * N * N * N;
#pragma unroll
        for (int m = 0; m < S; ++m) {
            const int n = t + TH * m;
            T va = (T)0.0, vb = (T)0.0;
            // the sample read: n in the lower half; 2N - n mirrored (BOX)
            const int nn = m < S / 2 ? n : ((BOX && n > N) ? 2 * N - n : -1);
            if (active && nn >= 0) {
                const long long xa = la * N + nn, xb = lb * N + nn;
                va = (a.flags[xa] & 1) ? (T)(a.scale * f[swap_axes(xa, a.f_swap, N)]) : (T)0;
                vb = (a.flags[xb] & 1) ? (T)(a.scale * f[swap_axes(xb, a.f_swap, N)]) : (T)0;
                if (m >= S / 2) {
                    va = -va;
                    vb = -vb;
                }
            }
            v[m] = cmake<C>(va, vb);
        }
    }
    const int base = p * G::XS;
    PL::template fwd<!BOX>(v, xch, base, 1, t, a.tw);
    // natural order into the exchange area, then split the two spectra
    // X_a = (Z[k] + conj Z[L-k]) / 2, X_b = (Z[k] - conj Z[L-k]) / 2i
    C* z = xch + base;
#pragma unroll
    for (int s = 0; s < S; ++s) z[PL::kidx(t, s)] = v[s];
    __syncthreads();
    if (active) {
        C* A = a.A + (long long)b * N * N * N1;
        for (int k = t; k < N; k += TH) {
            C xa, xb;
            split_lines(z, k, L, xa, xb);
            A[la * N1 + k] = xa;
            A[lb * N1 + k] = xb;
        }
    }
}

// PERSIST: a grid of at most the resident CTAs strides over the tiles (pair
// block, right-hand side); otherwise one tile per CTA of the grid (pair
// blocks, 1, right-hand sides). Separate instantiations: inside a tile loop
// the compiler keeps loop invariants (twiddles, offsets) in registers,
// which halves the occupancy of the one-tile form.
template <typename T, int L, bool BOX = false, int V = 0, bool PERSIST = false>
__global__ void __launch_bounds__(Geo<T, L, V>::KT, Geo<T, L, V>::MINB_KF) k_kpass_fwd(ConvArgs<T> a) {
    wait_prior_grid();   // results of the previous kernel on the stream
    if constexpr (PERSIST) {
        constexpr int N = L / 2;
        const long long gkx = (a.npairs() + Geo<T, L, V>::P - 1) / Geo<T, L, V>::P;
        const long long ntiles = gkx * a.nbatch;
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            kpass_fwd_tile<T, L, BOX, V>(a, (int)(tile % gkx), (int)(tile / gkx));
            __syncthreads();   // the next tile reuses the shared memory
        }
    } else {
        kpass_fwd_tile<T, L, BOX, V>(a, (int)blockIdx.x, (int)blockIdx.z);
    }
}

// ----------------------------------------------------- column passes (j, i)
enum ColMode { COL_FWD_J = 0, COL_CONV_I = 1, COL_INV_J = 2 };

// MP > 0 (the i pass of a narrow plane range, !BOX): the nonzero rows
// [p0, p1) lie in rows [lo0, lo0 + TH MP) with lo0 = p0 rounded down to a
// multiple of TH, so the pencil is transformed shifted down by lo0: slot m
// of thread t holds row lo0 + t + TH m, only slots m < MP are loaded (the
// first DFT drops the zero slots) and only they are stored back (the last
// DFT computes only those). A circular convolution commutes with the
// shift, so the rows written are the same as without it.
template <typename T, int L, int MODE, bool BOX, int V, int MP = 0>
__device__ __forceinline__ void colpass_tile(const ConvArgs<T>& a, int bx, int by, int bz) {
    using C = cplx_t<T>;
    using G = Geo<T, L, V>;
    using PL = typename G::PL;
    constexpr int N = L / 2, N1 = N + 1, TH = G::TH, S = G::S, W = G::W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* xch = reinterpret_cast<C*>(smem_raw);   // XL * W

    static_assert(MP == 0 || (MODE == COL_CONV_I && !BOX && MP <= S / 2), "narrow i pass only");
    const int b = bz;
    if (a.active && !a.active[b]) return;
    const int o = MODE == COL_CONV_I ? by : a.plane_lo() + by;   // jj, or i
    const int lo0 = MP > 0 ? (a.plane_lo() / TH) * TH : 0;       // row shift of a narrow i pass
    const int c = threadIdx.x % W;
    const int t = threadIdx.x / W;
    const int col = bx * W + c;             // kk (column 0 holds kk = 0 and N)
    const bool ok = col < N;
    const bool col0 = bx == 0;              // this CTA holds column 0 (c == 0)

    C* Ab = a.A + (long long)b * N * N * N1;
    C* Bb = a.B + (long long)b * N * (2 * N) * N1;
    const C* in;
    C* out;
    long long stride;
    if (MODE == COL_FWD_J) {
        in = Ab + (long long)o * N * N1 + col; out = Bb + (long long)o * (2 * N) * N1 + col; stride = N1;
    } else if (MODE == COL_CONV_I) {
        out = Bb + (long long)o * N1 + col; in = out; stride = (long long)(2 * N) * N1;
    } else {
        in = Bb + (long long)o * (2 * N) * N1 + col; out = Ab + (long long)o * N * N1 + col; stride = N1;
    }

    C v[S];
    const C zero = cmake<C>((T)0, (T)0);
    if (MODE == COL_INV_J) {
        // k-layout load of all L rows (column 0: merge slots k and L - k)
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int k = PL::kidx(t, s);
            C x = ok ? in[k * stride] : zero;
            if (col0 && c == 0) x = slot_merge(x, in[((L - k) & (L - 1)) * stride], k, N);
            v[s] = x;
        }
        PL::inv(v, xch, c, W, t, a.tw);
    } else if constexpr (MP > 0) {
        // n-layout load of the rows lo0 + t + TH m, m < MP
#pragma unroll
        for (int m = 0; m < S; ++m) {
            const int nn = lo0 + t + TH * m;
            const bool live = m < MP && nn >= a.plane_lo() && nn < a.plane_hi();
            v[m] = (ok && live) ? in[nn * stride] : zero;
        }
        PL::template fwd_nz<MP>(v, xch, c, W, t, a.tw);
    } else {
        // n-layout load of the N nonzero rows (BOX: and their negated
        // mirrors in the upper half)
#pragma unroll
        for (int m = 0; m < S; ++m) {
            const int n = t + TH * m;
            const int nn = m < S / 2 ? n : ((BOX && n > N) ? 2 * N - n : -1);
            // rows outside [p0, p1) (i pass) or [q0, q1) (j pass) are zero
            // (not even written)
            const bool live = nn >= 0 && (MODE != COL_CONV_I || (nn >= a.plane_lo() && nn < a.plane_hi())) &&
                              (MODE != COL_FWD_J || (nn >= a.line_lo() && nn < a.line_hi()));
            C x = (ok && live) ? in[nn * stride] : zero;
            if (BOX && m >= S / 2) x = cmake<C>(-x.x, -x.y);
            v[m] = x;
        }
        PL::template fwd<!BOX>(v, xch, c, W, t, a.tw);
    }

    if (MODE == COL_FWD_J) {
        if (col0) split_column0<PL, L>(v, xch, c, t);   // column 0: separate F0 and FN
        if (ok) {
#pragma unroll
            for (int s = 0; s < S; ++s) out[PL::kidx(t, s) * stride] = v[s];
        }
        return;
    }
    if (MODE == COL_CONV_I) {
        // times the real, even spectrum (octant fold), then back. Column 0
        // carries the kk = 0 spectrum in slots jj < N, the kk = N spectrum
        // in slots jj > N, and both (packed) at jj = 0 and N.
        const int jj = o <= N ? o : L - o;
        const int gc = (col0 && c == 0 && o > N) ? N : (ok ? col : 0);
        const T* g = a.ghat + (long long)jj * N1 + gc;
        if (col0 && (o == 0 || o == N)) {   // y = F0 + i FN, both Hermitian in p
            if (c == 0) {
#pragma unroll
                for (int s = 0; s < S; ++s) xch[PL::kidx(t, s)] = v[s];
            }
            __syncthreads();
            if (c == 0) {
                const T half = (T)0.5;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const int k = PL::kidx(t, s);
                    const int ii = k <= N ? k : L - k;
                    const T g0 = g[(long long)ii * N1 * N1], gn = g[(long long)ii * N1 * N1 + N];
                    // (g0 + gN) y(p) / 2 + (g0 - gN) conj y(-p) / 2
                    const C yr = cconj(xch[(L - k) & (L - 1)]);
                    const C y = v[s];
                    const T sp = (g0 + gn) * half, sm = (g0 - gn) * half;
                    v[s] = cmake<C>(y.x * sp + yr.x * sm, y.y * sp + yr.y * sm);
                }
            }
            __syncthreads();
            if (c != 0) {
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const int k = PL::kidx(t, s);
                    const int ii = k <= N ? k : L - k;
                    v[s] = cscale(v[s], g[(long long)ii * N1 * N1]);
                }
            }
        } else {
            // slot s holds frequency k = t + k0(s), k0(s) = kidx(0, s) a
            // compile-time multiple of TH, so the octant row min(k, L - k)
            // is t + k0 when k0 < N and (L - k0) - t otherwise (k0 + t <= N
            // in the first case, k0 >= N in the second): one per-thread
            // offset and compile-time terms instead of a select per slot
            constexpr int NN = N1 * N1;
            const int tn = t * NN;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int k0 = PL::kidx(0, s);
                const T gv = k0 < N ? g[tn + k0 * NN] : g[(L - k0) * NN - tn];
                v[s] = cscale(v[s], gv);
            }
        }
        PL::inv(v, xch, c, W, t, a.tw);
    }
    // n-layout store of the first N rows (narrow i pass: of the rows
    // lo0 + t + TH m, m < MP)
    if (ok) {
#pragma unroll
        for (int m = 0; m < S; ++m) {
            const int n = lo0 + t + TH * m;
            if (m < (MP > 0 ? MP : S / 2) && (MODE != COL_CONV_I || (n >= a.plane_lo() && n < a.plane_hi())) &&
                (MODE != COL_INV_J || (n >= a.line_lo() && n < a.line_hi())))
                out[n * stride] = v[m];
        }
    }
}

// tiles (column block, line, right-hand side), column blocks fastest:
// strided over a grid of resident CTAs (PERSIST) or one per CTA of the grid
// (column blocks, lines, right-hand sides)
template <typename T, int L, int MODE, bool BOX = false, int V = 0, bool PERSIST = false, int MP = 0>
__global__ void __launch_bounds__(Geo<T, L, V>::CT, Geo<T, L, V>::minb_col(MODE)) k_colpass(ConvArgs<T> a) {
    wait_prior_grid();   // results of the previous kernel on the stream
    if constexpr (PERSIST) {
        constexpr int N = L / 2;
        constexpr int ncb = (N + Geo<T, L, V>::W - 1) / Geo<T, L, V>::W;
        const int ny = MODE == COL_CONV_I ? 2 * N : a.plane_hi() - a.plane_lo();
        const long long per_b = (long long)ncb * ny;
        const long long ntiles = per_b * a.nbatch;
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const long long rem = tile % per_b;
            colpass_tile<T, L, MODE, BOX, V, MP>(a, (int)(rem % ncb), (int)(rem / ncb), (int)(tile / per_b));
            __syncthreads();   // the next tile reuses the shared memory
        }
    } else {
        colpass_tile<T, L, MODE, BOX, V, MP>(a, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z);
    }
}

// ----------------------------------------------------------- k pass (C2R)
template <typename T, int L, int V>
__device__ __forceinline__ void kpass_inv_tile(const ConvArgs<T>& a, int bx, int bz) {
    using C = cplx_t<T>;
    using G = Geo<T, L, V>;
    using PL = typename G::PL;
    constexpr int N = L / 2, N1 = N + 1, TH = G::TH, S = G::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* xch = reinterpret_cast<C*>(smem_raw);

    const int b = bz;
    if (a.active && !a.active[b]) return;
    const int t = threadIdx.x % TH;
    const int p = threadIdx.x / TH;
    const long long gp = (long long)bx * G::P + p;
    const bool active = gp < a.npairs();
    const long long la = a.pair_line(gp), lb = la + 1;
    const C* A = a.A + (long long)b * N * N * N1;

    C v[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int k = PL::kidx(t, s);
        C z = cmake<C>((T)0, (T)0);
        if (active) {
            const C xa = line_spectrum(A + la * N1, k, N);
            const C xb = line_spectrum(A + lb * N1, k, N);
            z = cmake<C>(xa.x - xb.y, xa.y + xb.x);   // xa + i xb
        }
        v[s] = z;
    }
    PL::inv(v, xch, p * G::XS, 1, t, a.tw);
    if (active) {
        typename OutOf<T>::type* out = a.v + (long long)b * N * N * N;
#pragma unroll
        for (int m = 0; m < S; ++m) {
            const int n = t + TH * m;
            if (m < S / 2) {
                out[la * N + n] = to_out(v[m].x);
                out[lb * N + n] = to_out(v[m].y);
            }
        }
    }
}

template <typename T, int L, int V = 0, bool PERSIST = false>
__global__ void __launch_bounds__(Geo<T, L, V>::KT, Geo<T, L, V>::MINB) k_kpass_inv(ConvArgs<T> a) {
    wait_prior_grid();   // results of the previous kernel on the stream
    if constexpr (PERSIST) {
        constexpr int N = L / 2;
        const long long gkx = (a.npairs() + Geo<T, L, V>::P - 1) / Geo<T, L, V>::P;
        const long long ntiles = gkx * a.nbatch;
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            kpass_inv_tile<T, L, V>(a, (int)(tile % gkx), (int)(tile / gkx));
            __syncthreads();   // the next tile reuses the shared memory
        }
    } else {
        kpass_inv_tile<T, L, V>(a, (int)blockIdx.x, (int)blockIdx.z);
    }
}

// ------------------------------------------ plane-fused passes (k with j)
// One CTA per (i plane, batch item) keeps the whole N x (N+1) plane of
// k-spectra in shared memory, so the forward k and j passes (and the
// inverse j and k passes) run in one kernel and A never goes to global
// memory: 16 N^3 fewer bytes per apply. Used where the plane fits next to
// the exchange buffers (float32 up to N = 128, 16-byte types up to N = 64).

template <typename T, int L>
__global__ void __launch_bounds__(512) k_plane_fwd(ConvArgs<T> a) {
    wait_prior_grid();   // results of the previous kernel on the stream
    using C = cplx_t<T>;
    using G = PlaneGeo<T, L>;
    constexpr int N = G::N, N1 = G::N1, R1 = G::R1, R2 = G::R2, Q = R2 / R1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* plane = reinterpret_cast<C*>(smem_raw);                 // [N][N1]
    C* xch = reinterpret_cast<C*>(smem_raw + G::PLANE);
    const int b = blockIdx.y;
    if (a.active && !a.active[b]) return;
    const int i = a.plane_lo() + (int)blockIdx.x;

    // ---- k lines of plane i, PP pairs per round
    {
        const int t = threadIdx.x % R1, p = threadIdx.x / R1;
        for (int round = 0; round < G::ROUNDS; ++round) {
            const int pr = round * G::PP + p;
            const bool act = pr < N / 2;      // the last round may be partial
            const int ja = 2 * pr, jb = ja + 1;
            const long long la = (long long)i * N + ja, lb = la + 1;   // global line indices
            C v[R2];
            if (a.mode == SRC_DENSITY) {
                // stage the two real lines in the plane rows they will own
                T* ra = reinterpret_cast<T*>(plane + (long long)(act ? ja : 0) * N1);
                T* rb = reinterpret_cast<T*>(plane + (long long)(act ? jb : 0) * N1);
                if (act)
                    for (int k = t; k < N; k += R1) {
                        ra[k] = volume_or_zero(a, b, la * N + k);
                        rb[k] = volume_or_zero(a, b, lb * N + k);
                    }
                __syncthreads();
                if (act) {
                    const double* q = a.q + (long long)b * a.q_stride + (a.q_row ? (long long)a.q_row[b] * a.q_row_stride : 0);
                    const float* q32 = a.q32 ? a.q32 + (long long)b * a.q32_stride : nullptr;
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const long long l = half ? lb : la;
                        T* r = half ? rb : ra;
                        const int s0 = a.rec.line_off[l], s1 = a.rec.line_off[l + 1];
                        for (int s = s0 + t; s < s1; s += R1) {
                            const int k = a.rec.src_lin[s] - (int)(l * N);
                            r[k] = source_value<T>(a.rec, s, q, q32);
                        }
                    }
                }
                __syncthreads();
#pragma unroll
                for (int m = 0; m < R2; ++m) {
                    const int n = t + R1 * m;
                    v[m] = (act && m < R2 / 2) ? cmake<C>(ra[n], rb[n]) : cmake<C>((T)0.0, (T)0.0);
                }
            } else {
                const double* f = a.f + (long long)b * N * N * N;
#pragma unroll
                for (int m = 0; m < R2; ++m) {
                    const int n = t + R1 * m;
                    T va = (T)0.0, vb = (T)0.0;
                    if (act && m < R2 / 2) {
                        const long long xa = la * N + n, xb = lb * N + n;
                        va = (a.flags[xa] & 1) ? (T)(a.scale * f[swap_axes(xa, a.f_swap, N)]) : (T)0.0;
                        vb = (a.flags[xb] & 1) ? (T)(a.scale * f[swap_axes(xb, a.f_swap, N)]) : (T)0.0;
                    }
                    v[m] = cmake<C>(va, vb);
                }
            }
            const int base = p * G::XS;
            fft_n2k<L, false, true>(v, xch, base, R1 + 1, 1, t, a.tw);
            C* z = xch + base;
#pragma unroll
            for (int q2 = 0; q2 < Q; ++q2)
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) z[t + q2 * R1 + R2 * k1] = v[q2 * R1 + k1];
            __syncthreads();
            if (act) {
                for (int k = t; k < N; k += R1) {
                    C xa, xb;
                    split_lines(z, k, L, xa, xb);
                    plane[(long long)ja * N1 + k] = xa;
                    plane[(long long)jb * N1 + k] = xb;
                }
            }
            __syncthreads();
        }
    }
    // ---- j columns of the plane, PW columns per round, straight to B
    {
        const int c = threadIdx.x % G::PW, t = threadIdx.x / G::PW;
        C* out = a.B + (long long)b * N * (2 * N) * N1 + (long long)i * (2 * N) * N1;
        for (int col0 = 0; col0 < N; col0 += G::PW) {
            const int col = col0 + c;
            const bool ok = col < N;
            C v[R2];
#pragma unroll
            for (int m = 0; m < R2; ++m) {
                const int n = t + R1 * m;
                v[m] = (ok && m < R2 / 2) ? plane[(long long)n * N1 + col] : cmake<C>((T)0.0, (T)0.0);
            }
            fft_n2k<L, false, true>(v, xch, c, R1 * G::PW, G::PW, t, a.tw);
            if (col0 == 0) split_column0<Plan2<L>, L>(v, xch, c, t);
            if (ok) {
#pragma unroll
                for (int q2 = 0; q2 < Q; ++q2)
#pragma unroll
                    for (int k1 = 0; k1 < R1; ++k1)
                        out[(long long)(t + q2 * R1 + R2 * k1) * N1 + col] = v[q2 * R1 + k1];
            }
        }
    }
}

template <typename T, int L>
__global__ void __launch_bounds__(512) k_plane_inv(ConvArgs<T> a) {
    wait_prior_grid();   // results of the previous kernel on the stream
    using C = cplx_t<T>;
    using G = PlaneGeo<T, L>;
    constexpr int N = G::N, N1 = G::N1, R1 = G::R1, R2 = G::R2, Q = R2 / R1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* plane = reinterpret_cast<C*>(smem_raw);
    C* xch = reinterpret_cast<C*>(smem_raw + G::PLANE);
    const int b = blockIdx.y;
    if (a.active && !a.active[b]) return;
    const int i = a.plane_lo() + (int)blockIdx.x;

    // ---- inverse j on every column, keep j < N in the plane
    {
        const int c = threadIdx.x % G::PW, t = threadIdx.x / G::PW;
        const C* in = a.B + (long long)b * N * (2 * N) * N1 + (long long)i * (2 * N) * N1;
        for (int col0 = 0; col0 < N; col0 += G::PW) {
            const int col = col0 + c;
            const bool ok = col < N;
            C v[R2];
#pragma unroll
            for (int q2 = 0; q2 < Q; ++q2)
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) {
                    const int k = t + q2 * R1 + R2 * k1;
                    C x = ok ? in[(long long)k * N1 + col] : cmake<C>((T)0.0, (T)0.0);
                    if (col == 0) x = slot_merge(x, in[(long long)((L - k) & (L - 1)) * N1], k, N);
                    v[q2 * R1 + k1] = x;
                }
            fft_k2n<L, true>(v, xch, c, R1 * G::PW, G::PW, t, a.tw);
            if (ok) {
#pragma unroll
                for (int m = 0; m < R2; ++m) {
                    const int n = t + R1 * m;
                    if (m < R2 / 2) plane[(long long)n * N1 + col] = v[m];
                }
            }
        }
        __syncthreads();
    }
    // ---- C2R of two k lines per transform, keep k < N
    {
        const int t = threadIdx.x % R1, p = threadIdx.x / R1;
        auto* out = a.v + (long long)b * N * N * N;
        for (int round = 0; round < G::ROUNDS; ++round) {
            const int pr = round * G::PP + p;
            const bool act = pr < N / 2;
            const int ja = act ? 2 * pr : 0, jb = ja + 1;
            const long long la = (long long)i * N + ja, lb = la + 1;
            C v[R2];
#pragma unroll
            for (int q2 = 0; q2 < Q; ++q2)
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) {
                    const int k = t + q2 * R1 + R2 * k1;
                    C xa = cmake<C>((T)0.0, (T)0.0), xb = xa;
                    if (act) {
                        xa = line_spectrum(plane + (long long)ja * N1, k, N);
                        xb = line_spectrum(plane + (long long)jb * N1, k, N);
                    }
                    v[q2 * R1 + k1] = cmake<C>(xa.x - xb.y, xa.y + xb.x);
                }
            fft_k2n<L, true>(v, xch, p * G::XS, R1 + 1, 1, t, a.tw);
            if (act) {
#pragma unroll
                for (int m = 0; m < R2; ++m) {
                    const int n = t + R1 * m;
                    if (m < R2 / 2) {
                        out[la * N + n] = to_out(v[m].x);
                        out[lb * N + n] = to_out(v[m].y);
                    }
                }
            }
        }
    }
}

template <typename T, int L>
void configure_conv() {
    using C = cplx_t<T>;
    using G = Geo<T, L>;
    constexpr int N = L / 2;
    const size_t smem_k = (size_t)G::P * G::XS * sizeof(C) + (size_t)G::P * G::RS * sizeof(T);
    const size_t smem_c = (size_t)G::XL * G::W * sizeof(C);
    // once per instantiation (thread-safe static initialisation)
    static const bool configured = [&]() {
        BAE_CUDA(cudaFuncSetAttribute(k_kpass_fwd<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k));
        BAE_CUDA(cudaFuncSetAttribute(k_kpass_inv<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k));
        BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_FWD_J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_CONV_I>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_INV_J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        // the persistent instantiations of the variant-0 passes
        BAE_CUDA(cudaFuncSetAttribute(k_kpass_fwd<T, L, false, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_k));
        BAE_CUDA(cudaFuncSetAttribute(k_kpass_inv<T, L, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_k));
        BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_FWD_J, false, 0, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_CONV_I, false, 0, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_INV_J, false, 0, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
        if constexpr (HasAlt<T, L>::value) {
            using GA = Geo<T, L, 1>;
            const size_t ak = (size_t)GA::P * GA::XS * sizeof(C) + (size_t)GA::P * GA::RS * sizeof(T);
            const size_t ac = (size_t)GA::XL * GA::W * sizeof(C);
            BAE_CUDA(cudaFuncSetAttribute(k_kpass_fwd<T, L, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ak));
            BAE_CUDA(cudaFuncSetAttribute(k_kpass_inv<T, L, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ak));
            BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_FWD_J, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ac));
            BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_CONV_I, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ac));
            BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_INV_J, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ac));
        }
        if constexpr (sizeof(C) == 16) {
            BAE_CUDA(cudaFuncSetAttribute(k_kpass_fwd<T, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k));
            BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_FWD_J, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_c));
            BAE_CUDA(cudaFuncSetAttribute(k_colpass<T, L, COL_CONV_I, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_c));
        }
        if constexpr (PlaneGeo<T, L>::FITS) {
            BAE_CUDA(cudaFuncSetAttribute(k_plane_fwd<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)PlaneGeo<T, L>::SMEM));
            BAE_CUDA(cudaFuncSetAttribute(k_plane_inv<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)PlaneGeo<T, L>::SMEM));
        }
        if constexpr (!PlaneGeo<T, L>::FITS && CPlaneGeo<T, L>::USE) cplane_ready<T, L>();
        return true;
    }();
    (void)configured;
}

// CTAs of `kernel` resident on one SM at `threads` threads and `smem`
// bytes (cached per kernel; every launch site uses one configuration)
template <typename K>
int resident_per_sm(K kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<const void*, int> cache;
    const void* key = reinterpret_cast<const void*>(kernel);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    BAE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem));
    cache[key] = n > 0 ? n : 1;
    return cache[key];
}

inline int sm_count() {
    static const int n = []() {
        int dev = 0, c = 0;
        BAE_CUDA(cudaGetDevice(&dev));
        BAE_CUDA(cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev));
        return c;
    }();
    return n;
}

// Grid of a persistent pass kernel: at most the CTAs resident at once
template <typename K>
dim3 persist_grid(long long ntiles, K kernel, int threads, size_t smem) {
    const long long cap = (long long)resident_per_sm(kernel, threads, smem) * sm_count();
    return dim3((unsigned)(ntiles < 1 ? 1 : (ntiles < cap ? ntiles : cap)));
}

// ------------------------------------------------------ narrow i pass
// The i pass where the planes [p0, p1) span few blocks of TH rows: the
// instantiation with MP slots (colpass_tile) for the smallest MP in {1, 2,
// 4} below S / 2 that covers them. float32 and double-float at L >= 128;
// the kernels are compiled in conv_inarrow_*.cu. Returns false (nothing
// launched) where no narrow instantiation covers the span.
template <typename T, int L> struct NarrowI {
    static constexpr bool value = (std::is_same<T, float>::value || std::is_same<T, dsf>::value) && L >= 128;
};

template <typename T, int L, int V, bool PERSIST, int MP>
void launch_narrow_mp(const ConvArgs<T>& a, dim3 grid, size_t smem, cudaStream_t st) {
    auto k = k_colpass<T, L, COL_CONV_I, false, V, PERSIST, MP>;
    static const bool configured = [&]() {
        BAE_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        return true;
    }();
    (void)configured;
    if constexpr (PERSIST) {   // a grid of this kernel's resident CTAs over every tile
        using G = Geo<T, L, V>;
        constexpr int N = L / 2;
        grid = persist_grid((long long)ceil_div(N, G::W) * 2 * N * a.nbatch, k, G::CT, smem);
    }
    BAE_LAUNCH(kname<T>("conv_i.f32", "conv_i.f64", "conv_i.df64"), st,
               launch_pdl(k, grid, Geo<T, L, V>::CT, smem, st, a));
}

}  // namespace

// external linkage: explicitly instantiated once, in conv_inarrow_*.cu.
// Every schedule's i pass takes the same transform (narrow or not) for the
// same plane range, so the schedules stay bit-identical to one another.
template <typename T, int L, int V, bool PERSIST>
bool launch_conv_i_narrow(const ConvArgs<T>& a, dim3 grid, size_t smem, cudaStream_t st) {
    constexpr int TH = Geo<T, L, V>::TH, S = Geo<T, L, V>::S;
    const int lo0 = (a.plane_lo() / TH) * TH;
    const int span = ceil_div(a.plane_hi() - lo0, TH);   // slots holding rows of [p0, p1)
    if (span <= 1 && 1 < S / 2) {
        launch_narrow_mp<T, L, V, PERSIST, 1>(a, grid, smem, st);
        return true;
    }
    if constexpr (2 < S / 2) {
        if (span <= 2) {
            launch_narrow_mp<T, L, V, PERSIST, 2>(a, grid, smem, st);
            return true;
        }
    }
    if constexpr (4 < S / 2) {
        if (span <= 4) {
            launch_narrow_mp<T, L, V, PERSIST, 4>(a, grid, smem, st);
            return true;
        }
    }
    return false;
}

// the narrow kernels are compiled once, in conv_inarrow_*.cu
#define BAE_NARROW_I(T, L, V, P) \
    extern template bool launch_conv_i_narrow<T, L, V, P>(const ConvArgs<T>&, dim3, size_t, cudaStream_t);
BAE_NARROW_I(float, 128, 0, false)
BAE_NARROW_I(float, 256, 0, false)
BAE_NARROW_I(float, 256, 1, false)
BAE_NARROW_I(float, 512, 0, false)
BAE_NARROW_I(float, 512, 1, false)
BAE_NARROW_I(float, 128, 0, true)
BAE_NARROW_I(float, 256, 0, true)
BAE_NARROW_I(float, 512, 0, true)
BAE_NARROW_I(dsf, 128, 0, false)
BAE_NARROW_I(dsf, 256, 0, false)
BAE_NARROW_I(dsf, 512, 0, false)
BAE_NARROW_I(dsf, 128, 0, true)
BAE_NARROW_I(dsf, 256, 0, true)
BAE_NARROW_I(dsf, 512, 0, true)
#undef BAE_NARROW_I

namespace {

// the i pass (not the finite box): narrow where it can be
template <typename T, int L, int V, bool PERSIST = false>
void launch_conv_i(const ConvArgs<T>& a, dim3 grid, size_t smem, cudaStream_t st) {
    if constexpr (NarrowI<T, L>::value && (V == 0 || (HasAlt<T, L>::value && !PERSIST))) {
        if (!a.box && launch_conv_i_narrow<T, L, V, PERSIST>(a, grid, smem, st)) return;
    }
    BAE_LAUNCH(kname<T>("conv_i.f32", "conv_i.f64", "conv_i.df64"), st,
               launch_pdl(k_colpass<T, L, COL_CONV_I, false, V, PERSIST>, grid, Geo<T, L, V>::CT, smem, st, a));
}

// The five pass kernels with the launch geometry of variant V: one tile per
// CTA, or (PERSIST) the persistent instantiations on grids of resident CTAs.
template <typename T, int L, int V, bool BOX = false, bool PERSIST = false>
void launch_passes(const ConvArgs<T>& a, cudaStream_t st) {
    using C = cplx_t<T>;
    using G = Geo<T, L, V>;
    constexpr int N = L / 2;
    const size_t smem_k = (size_t)G::P * G::XS * sizeof(C) + (size_t)G::P * G::RS * sizeof(T);
    const size_t smem_c = (size_t)G::XL * G::W * sizeof(C);
    const int nb = a.nbatch;
    const int np = a.plane_hi() - a.plane_lo();   // x-planes holding sources or read outputs
    const int gkx = ceil_div(a.npairs(), G::P);   // k-line pairs in [p0, p1) x [q0, q1)
    const int ncb = ceil_div(N, G::W);           // column 0 also holds kk = N
    auto kf = k_kpass_fwd<T, L, BOX, V, PERSIST>;
    auto jf = k_colpass<T, L, COL_FWD_J, BOX, V, PERSIST>;
    auto ci = k_colpass<T, L, COL_CONV_I, BOX, V, PERSIST>;
    auto ji = k_colpass<T, L, COL_INV_J, false, V, PERSIST>;
    auto ki = k_kpass_inv<T, L, V, PERSIST>;
    dim3 gk(gkx, 1, nb), gj(ncb, np, nb), gi(ncb, 2 * N, nb);
    if (PERSIST) {
        gk = persist_grid((long long)gkx * nb, kf, G::KT, smem_k);
        gj = persist_grid((long long)ncb * np * nb, jf, G::CT, smem_c);
        gi = persist_grid((long long)ncb * 2 * N * nb, ci, G::CT, smem_c);
    }
    const dim3 gji = PERSIST ? persist_grid((long long)ncb * np * nb, ji, G::CT, smem_c) : gj;
    const dim3 gki = PERSIST ? persist_grid((long long)gkx * nb, ki, G::KT, smem_k) : gk;
    BAE_LAUNCH(BOX ? kname<T>("conv_box_kfwd.f32", "conv_box_kfwd.f64", "conv_box_kfwd.df64")
                   : kname<T>("conv_kfwd.f32", "conv_kfwd.f64", "conv_kfwd.df64"), st,
               launch_pdl(kf, gk, G::KT, smem_k, st, a));
    BAE_LAUNCH(BOX ? kname<T>("conv_box_jfwd.f32", "conv_box_jfwd.f64", "conv_box_jfwd.df64")
                   : kname<T>("conv_jfwd.f32", "conv_jfwd.f64", "conv_jfwd.df64"), st,
               launch_pdl(jf, gj, G::CT, smem_c, st, a));
    if constexpr (!BOX)
        launch_conv_i<T, L, V, PERSIST>(a, gi, smem_c, st);
    else
        BAE_LAUNCH(BOX ? kname<T>("conv_box_i.f32", "conv_box_i.f64", "conv_box_i.df64")
                       : kname<T>("conv_i.f32", "conv_i.f64", "conv_i.df64"), st,
                   launch_pdl(ci, gi, G::CT, smem_c, st, a));
    BAE_LAUNCH(kname<T>("conv_jinv.f32", "conv_jinv.f64", "conv_jinv.df64"), st,
               launch_pdl(ji, gji, G::CT, smem_c, st, a));
    BAE_LAUNCH(kname<T>("conv_kinv.f32", "conv_kinv.f64", "conv_kinv.df64"), st,
               launch_pdl(ki, gki, G::KT, smem_k, st, a));
}

template <typename T, int L>
void launch_sched(const ConvArgs<T>& a, cudaStream_t st, int sched) {
    using C = cplx_t<T>;
    using G = Geo<T, L>;
    using PG = PlaneGeo<T, L>;
    constexpr int N = L / 2;
    const size_t smem_c = (size_t)G::XL * G::W * sizeof(C);
    const int nb = a.nbatch;
    const int np = a.plane_hi() - a.plane_lo();
    if (a.box) {
        // finite box: the forward passes with mirrored upper halves, the
        // ordinary inverse passes
        if constexpr (sizeof(C) == 16) {
            launch_passes<T, L, 0, true>(a, st);
            return;
        } else {
            throw Error(BAE_ERR_INVALID_ARG, "finite-box apply needs float64 or double-float");
        }
    }
    if (sched == SCHED_PASSES_ALT) {
        // the five passes with the variant-1 geometry (HasAlt), else variant 0
        if constexpr (HasAlt<T, L>::value) {
            launch_passes<T, L, 1>(a, st);
            return;
        }
        sched = SCHED_PASSES;
    }
    if (sched == SCHED_PERSIST) {
        launch_passes<T, L, 0, false, true>(a, st);
        return;
    }
    if (sched == SCHED_PASSES) {
        launch_passes<T, L, 0>(a, st);
        return;
    }
    // plane-fused k and j passes around the i pass
    if constexpr (PG::FITS)
        BAE_LAUNCH(kname<T>("conv_plane_fwd.f32", "conv_plane_fwd.f64", "conv_plane_fwd.df64"), st,
                   launch_pdl(k_plane_fwd<T, L>, dim3(np, nb), PG::PT, PG::SMEM, st, a));
    else if constexpr (CPlaneGeo<T, L>::USE)
        cplane_launch<T, L>(a, st, false);
    launch_conv_i<T, L, 0>(a, dim3(ceil_div(N, G::W), 2 * N, nb), smem_c, st);
    if constexpr (PG::FITS)
        BAE_LAUNCH(kname<T>("conv_plane_inv.f32", "conv_plane_inv.f64", "conv_plane_inv.df64"), st,
                   launch_pdl(k_plane_inv<T, L>, dim3(np, nb), PG::PT, PG::SMEM, st, a));
    else if constexpr (CPlaneGeo<T, L>::USE)
        cplane_launch<T, L>(a, st, true);
}

}  // namespace

template <typename T, int L>
void run_conv(const ConvArgs<T>& a, cudaStream_t st) {
    configure_conv<T, L>();
    if (a.box) {
        launch_sched<T, L>(a, st, SCHED_PASSES);
        return;
    }
    using PG = PlaneGeo<T, L>;
    // the schedules this (element type, L) can run: the five passes, their
    // variant geometry, the plane-fused passes (one CTA, or a cluster)
    bool plane = PG::FITS;
    if constexpr (!PG::FITS && CPlaneGeo<T, L>::USE) plane = cplane_ready<T, L>();
    const bool alt = HasAlt<T, L>::value;
    auto runnable = [&](int sc) {
        return sc == SCHED_PASSES || sc == SCHED_PERSIST || (sc == SCHED_PASSES_ALT && alt) ||
               (sc == SCHED_PLANE && plane);
    };
    if (forced_sched() >= 0) {
        launch_sched<T, L>(a, st, runnable(forced_sched()) ? forced_sched() : SCHED_PASSES);
        return;
    }
    const std::string key = std::string(tname<T>()) + "/N" + std::to_string(L / 2) + "/nb" + std::to_string(a.nbatch);
    int sched = tune_lookup(key);
    if (sched >= 0 && !runnable(sched)) sched = -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BAE_CUDA(cudaStreamIsCapturing(st, &cs));
    if (sched < 0 && (cs != cudaStreamCaptureStatusNone || a.no_tune))
        sched = (a.nbatch <= 4 && plane) ? SCHED_PLANE : SCHED_PASSES;
    if (sched >= 0) {
        launch_sched<T, L>(a, st, sched);
        return;
    }
    // time every runnable schedule on the real data: five rounds in rotating
    // order, three back-to-back applies per timing, keep each schedule's
    // best round (schedules are often within 10%, where a single launch
    // mostly measures launch jitter); every apply leaves a valid result
    int cand[4], nc = 0;
    for (int sc : {SCHED_PASSES, SCHED_PASSES_ALT, SCHED_PLANE, SCHED_PERSIST})
        if (runnable(sc)) cand[nc++] = sc;
    cudaEvent_t e[2];
    for (auto& x : e) BAE_CUDA(cudaEventCreate(&x));
    float best[4] = {1e30f, 1e30f, 1e30f, 1e30f};
    for (int rep = 0; rep < 5; ++rep)
        for (int k = 0; k < nc; ++k) {
            const int ci = (k + rep) % nc;
            BAE_CUDA(cudaEventRecord(e[0], st));
            for (int r = 0; r < 3; ++r) launch_sched<T, L>(a, st, cand[ci]);
            BAE_CUDA(cudaEventRecord(e[1], st));
            BAE_CUDA(cudaEventSynchronize(e[1]));
            float ms = 0.f;
            BAE_CUDA(cudaEventElapsedTime(&ms, e[0], e[1]));
            best[ci] = ms < best[ci] ? ms : best[ci];
        }
    for (auto& x : e) cudaEventDestroy(x);
    int bi = 0;
    for (int k = 1; k < nc; ++k)
        if (best[k] < best[bi]) bi = k;
    tune_store(key, cand[bi]);
}


template <typename T, int L>
void conv_configure() {
    configure_conv<T, L>();
}

}  // namespace bae
