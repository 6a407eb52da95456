// Launch geometry of the potential-apply kernels (shared by conv_impl.cuh
// and conv_cplane.cuh).
#pragma once

#include <type_traits>

#include "conv.cuh"
#include "fft2.cuh"

namespace bae {

// Transform plan of the pass kernels per element type and length: the
// three-level plans for 16-byte elements at L = 256 (8 x 8 x 4) and L = 512
// (8 x 8 x 8) (float64 and double-float, whose two-level 16 x 16 and
// 16 x 32 splits need ~170-255 registers per thread), the two-level plan
// elsewhere.
// V selects a geometry variant of the pass kernels for the autotuner:
// variant 1 exists for float32 at L = 256 (column blocks of half the width,
// 16 columns, three CTAs per SM) and L = 512 (the three-level plan), and
// for float64 at L = 256 (the three-level plan: more warps per SM, but a
// second twiddle stage on the narrow FP64 pipe, which costs more than the
// occupancy gains once a launch holds many right-hand sides); elsewhere it
// equals 0.
template <typename T, int L, int V = 0> struct PlanOf { using type = Plan2<L>; };
template <> struct PlanOf<double, 256, 1> { using type = Plan3_256; };
template <int V> struct PlanOf<dsf, 256, V> { using type = Plan3_256; };
template <int V> struct PlanOf<double, 512, V> { using type = Plan3_512; };
template <int V> struct PlanOf<dsf, 512, V> { using type = Plan3_512; };
template <> struct PlanOf<float, 512, 1> { using type = Plan3_512; };

template <typename T, int L> struct HasAlt {
    static constexpr bool value =
        (std::is_same<T, float>::value && (L == 256 || L == 512)) || (std::is_same<T, double>::value && L == 256);
};

// Launch geometry per transform length, precision and variant.
template <typename T, int L, int V = 0> struct Geo {
    using C = cplx_t<T>;
    using PL = typename PlanOf<T, L, V>::type;
    static constexpr bool THREE = PL::TH * PL::S == L && PL::TH > PL::S;
    static constexpr int TH = PL::TH, S = PL::S;   // threads per line, values per thread
    // column passes: W columns per CTA, TH threads per column (three-level:
    // 64-byte row segments at 64 threads per line, 128-byte ones at 32, so
    // that a CTA has 256 threads for the 16-byte types)
    static constexpr int WB = 65536 / (L * (int)sizeof(C));
    static constexpr int W0 = THREE ? (128 / (int)sizeof(C) / 2) * (64 / TH) : (WB > 32 ? 32 : (WB < 8 ? 8 : WB));
    static constexpr int W = (V == 1 && !THREE && HasAlt<T, L>::value) ? W0 / 2 : W0;
    static constexpr int CT = W * TH;
    static constexpr int XL = PL::XLEN;            // exchange positions per column
    // line passes (k): P line pairs per CTA, TH threads per pair
    static constexpr int PB = 65536 / (L * (int)sizeof(C));
    static constexpr int P = THREE ? 256 / TH : ((256 / TH) < PB ? (256 / TH) : (PB < 4 ? 4 : PB));
    static constexpr int KT = P * TH;
    static constexpr int XS = PL::XS;              // exchange stride per pair (odd)
    // stride of a pair's source lines (2N values) in the forward k pass:
    // for 4-byte values the lines of one warp (32 / TH of them) would start
    // on the same bank; TH values of padding shift each to its own banks
    static constexpr int RS = L + ((int)sizeof(T) == 4 && TH < 32 ? TH : 0);
    // resident CTAs per SM the compiler must allow (register cap): three per
    // SM for the three-level plan (at most 85 registers per thread, as its
    // kernels need) and for variant 1 of float32 at L = 256 (its i pass
    // otherwise takes 123 registers, two CTAs per SM), no constraint
    // otherwise
    static constexpr bool CAP3 = THREE || (V == 1 && std::is_same<T, float>::value && L == 256);
    static constexpr int MINB = CAP3 ? 3 : 1;
    // per pass, where it differs: the three-level i pass at L = 256
    // (spectral product and two transforms) fits 128 registers without
    // spilling at two CTAs per SM and runs ~3% faster so than with the
    // spills of the three-CTA cap; the float32 variant-1 forward passes at
    // L = 256 (forward k, forward j, i) fit 64 registers without spilling
    // at four CTAs per SM and run 4-11% faster so at 64 right-hand sides,
    // while the two inverse passes run 7% and 37% slower so and keep three;
    // the three-level forward k and both j passes of the 16-byte types fit
    // 64 registers too and run 4-12% faster at four CTAs per SM (L = 256
    // and 512; at L = 512 the i pass would spill and keeps three)
    static constexpr bool F4 = (V == 1 && std::is_same<T, float>::value && L == 256) ||
                               (THREE && (L == 256 || (L == 512 && sizeof(C) == 16)));
    static constexpr int minb_col(int mode) {
        if (THREE && L == 256 && mode == 1) return 2;
        if (THREE && L == 512 && mode == 1) return MINB;
        return (F4 && (mode != 2 || THREE)) ? 4 : MINB;
    }
    static constexpr int MINB_KF = F4 ? 4 : MINB;   // forward k pass
};

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


// ------------------------------------------ plane-fused passes (k with j)
// One CTA per (i plane, batch item) keeps the whole N x (N+1) plane of
// k-spectra in shared memory, so the forward k and j passes (and the
// inverse j and k passes) run in one kernel and A never goes to global
// memory: 16 N^3 fewer bytes per apply. Used where the plane fits next to
// the exchange buffers (float32 up to N = 128, 16-byte types up to N = 64).
template <typename T, int L> struct PlaneGeo {
    using C = cplx_t<T>;
    static constexpr int N = L / 2, N1 = N + 1;
    static constexpr int R1 = Factors<L>::R1, R2 = Factors<L>::R2;
    static constexpr int PT = 512;                  // threads per CTA
    static constexpr int PP = PT / R1;              // line pairs per round
    static constexpr int PW = PT / R1;              // columns per round
    static constexpr int XS = R2 * (R1 + 1) + 1;    // exchange stride per pair
    static constexpr size_t PLANE = (size_t)N * N1 * sizeof(C);
    static constexpr size_t XL = (size_t)PP * XS * sizeof(C);
    static constexpr size_t XC = (size_t)L * PW * sizeof(C);
    static constexpr size_t SMEM = PLANE + (XL > XC ? XL : XC);
    static constexpr int ROUNDS = (N / 2 + PP - 1) / PP;   // k-line rounds (last may be partial)
    static constexpr bool FITS = SMEM <= 227 * 1024;
};

// ---------------------------------------------------- source stencil value
// rho(x) = sum of coef * q over the terms of source node x (Section 3.2).
// For the float32 apply the sum is formed in float32: its value is rounded
// to float32 anyway, and on GB300 every float64 warp instruction occupies
// the FP64 pipe for ~64 cycles. The float64 and double-float applies sum in
// float64.
// Initial value of node x (linear index) of batch item b in a density
// apply: zero, or the volume source scale f on M+ when f is set (the
// combined apply K q + G_h[chi_{M+} f]; the layer sources sit on gamma- and
// D-nodes, outside M+, so the two never share a node)
template <typename T>
__device__ __forceinline__ T volume_or_zero(const ConvArgs<T>& a, int b, long long x) {
    if (a.f && (a.flags[x] & 1))
        return (T)(a.scale * a.f[(long long)b * a.N * a.N * a.N + swap_axes(x, a.f_swap, a.N)]);
    return (T)0.0;
}

template <typename T>
__device__ __forceinline__ T source_value(const SrcRecipe& rec, int s, const double* q, const float* q32) {
    if constexpr (std::is_same<T, float>::value) {
        if (!rec.wide) {   // small integer coefficients: a float32 sum
            float val = 0.f;
            for (int e = rec.term_off[s]; e < rec.term_off[s + 1]; ++e) {
                const int k = rec.term_idx[e];
                val = __fmaf_rn(rec.term_coef32[e], q32 ? q32[k] : (float)q[k], val);
            }
            return val;
        }
    }
    // float64 sum, one rounding to T
    double val = 0.0;
    for (int e = rec.term_off[s]; e < rec.term_off[s + 1]; ++e) val += rec.term_coef[e] * q[rec.term_idx[e]];
    return (T)val;
}

// ------------------------------------------ programmatic dependent launch
// The convolution kernels are launched with programmatic stream
// serialisation: the launch of a kernel is set up while the kernel before it
// on the stream is still running, and the kernel's first statement waits
// for that kernel's completion (and its memory) before reading anything. A
// launch without the attribute makes the wait a no-op.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename K, typename A>
void launch_pdl(K kernel, dim3 grid, int threads, size_t smem, cudaStream_t st, const A& a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BAE_CUDA(cudaLaunchKernelEx(&cfg, kernel, a));
}

// ------------------------------------------------ packed Nyquist column
// The k-spectrum of a real line is real at kk = 0 and at kk = N, so both
// live in column 0 as X0 + i XN and every pass after the k transform runs
// over N columns (not N + 1). X0 and XN are real along j, so after the j
// transform Z = F0 + i FN with F0, FN Hermitian in the j frequency q; the
// j pass separates them (two real transforms for the price of one complex
// one) and stores, per slot s of column 0,
//   s in (0, N): F0(s),  s in (N, 2N): FN(2N - s),  s = 0, N: Z(s) = F0 + i FN
// so that the i pass sees independent pencils (the kk = 0 spectrum for
// s < N, the kk = N spectrum for s > N) except at s = 0 and N, where it
// splits F0 and FN by the Hermitian symmetry in the i frequency. The
// inverse j pass merges the slots back into R0 + i RN.

// (X_a[k], X_b[k]) for k in [0, N) of two real lines transformed together
// as z = x_a + i x_b (natural order, length L), column 0 packed
template <typename C>
__device__ __forceinline__ void split_lines(const C* z, int k, int L, C& xa, C& xb) {
    using T = decltype(xa.x);
    if (k == 0) {
        const C z0 = z[0], zn = z[L / 2];
        xa = cmake<C>(z0.x, zn.x);
        xb = cmake<C>(z0.y, zn.y);
    } else {
        const T half = (T)0.5;
        const C zk = z[k], zr = z[L - k];
        xa = cmake<C>((zk.x + zr.x) * half, (zk.y - zr.y) * half);
        xb = cmake<C>((zk.y + zr.y) * half, (zr.x - zk.x) * half);
    }
}

// X[k], k in [0, 2N), of a real line from its packed row (columns 0..N-1)
template <typename C>
__device__ __forceinline__ C line_spectrum(const C* row, int k, int N) {
    using T = decltype(row[0].x);
    if (k == 0) return cmake<C>(row[0].x, (T)0.0);
    if (k == N) return cmake<C>(row[0].y, (T)0.0);
    if (k < N) return row[k];
    return cconj(row[2 * N - k]);
}

// slot k of column 0 after the forward j transform, from Z(k) and Z(2N - k)
template <typename C>
__device__ __forceinline__ C slot_split(C zk, C zr, int k, int N) {
    using T = decltype(zk.x);
    const T half = (T)0.5;
    if (k == 0 || k == N) return zk;
    if (k < N) return cmake<C>((zk.x + zr.x) * half, (zk.y - zr.y) * half);
    return cmake<C>((zr.y + zk.y) * half, (zk.x - zr.x) * half);
}

// After the forward j transform of a column group (column c held by the
// plan's TH threads t in k-layout, slot s holding k = PL::kidx(t, s); the
// exchange buffer free), replaces the outputs of column c == 0 by its
// slots. Every thread of the CTA calls it (two barriers).
template <typename PL, int L, typename C>
__device__ __forceinline__ void split_column0(C* v, C* xch, int c, int t) {
    if (c == 0) {
#pragma unroll
        for (int s = 0; s < PL::S; ++s) xch[PL::kidx(t, s)] = v[s];
    }
    __syncthreads();
    if (c == 0) {
#pragma unroll
        for (int s = 0; s < PL::S; ++s) {
            const int k = PL::kidx(t, s);
            v[s] = slot_split(v[s], xch[(L - k) & (L - 1)], k, L / 2);
        }
    }
    __syncthreads();
}

// R0(k) + i RN(k) for the inverse j transform, from slots k and 2N - k
template <typename C>
__device__ __forceinline__ C slot_merge(C sk, C sr, int k, int N) {
    if (k == 0 || k == N) return sk;
    if (k < N) return cmake<C>(sk.x - sr.y, sk.y + sr.x);
    return cmake<C>(sr.x + sk.y, sk.x - sr.y);
}

// ------------------------------ cluster plane passes (distributed shared memory)
// When a plane does not fit one SM (float32 at N = 256, 16-byte types at
// N >= 128), a cluster of CS CTAs holds it: CTA r keeps rows
// [r N/CS, (r+1) N/CS) of the k-spectra in its shared memory, transforms
// its own k-lines, and after a cluster barrier transforms its share of the
// j-columns reading the rows of the other CTAs through distributed shared
// memory. The inverse writes the inverse j-columns into the owners' rows,
// then each CTA runs the C2R of its own rows. As with the single-CTA
// plane, A never reaches global memory.
template <typename T, int L> struct CPlaneGeo {
    using C = cplx_t<T>;
    static constexpr int N = L / 2, N1 = N + 1;
    static constexpr int R1 = Factors<L>::R1, R2 = Factors<L>::R2;
    static constexpr int CS = (N * N1 * (int)sizeof(C) <= 140 * 1024) ? 1
                              : (N * N1 * (int)sizeof(C) <= 280 * 1024) ? 2
                              : (N * N1 * (int)sizeof(C) <= 560 * 1024) ? 4 : 8;
    static constexpr int NR = N / CS;                 // rows per CTA
    static constexpr int XS = R2 * (R1 + 1) + 1;
    static constexpr int PT0 = 256;
    static constexpr size_t ROWS = (size_t)NR * N1 * sizeof(C);
    static constexpr int PT = (ROWS + (size_t)(PT0 / R1) * XS * sizeof(C) <= 220 * 1024) ? PT0 : PT0 / 2;
    static constexpr int PP = PT / R1;                // line pairs per round
    static constexpr int PW = PT / R1;                // columns per round
    static constexpr int ROUNDS = (NR / 2 + PP - 1) / PP;
    static constexpr int CW = N / CS;                 // columns per CTA (column 0 packs kk = N)
    static constexpr size_t XL = (size_t)PP * XS * sizeof(C);
    static constexpr size_t XC = (size_t)L * PW * sizeof(C);
    static constexpr size_t SMEM = ROWS + (XL > XC ? XL : XC);
    static constexpr bool USE = CS > 1 && CS <= 8 && SMEM <= 227 * 1024 && NR % 2 == 0;
};

}  // namespace bae
