// Register-resident FFT building blocks for the convolution passes.
//
// A transform of length L = R1 * R2 (R2 = R1 or 2 R1) is done by R1 threads
// per line with the four-step factorisation n = n1 + R1 n2, k = k2 + R2 k1:
//   X[k2 + R2 k1] = sum_n1 W_R1^{n1 k1} W_L^{n1 k2} sum_n2 x[n1 + R1 n2] W_R2^{n2 k2}.
// "n-layout": thread t holds x[t + R1 m], m < R2 (global loads/stores of a
// strided line are coalesced across the columns a warp covers).
// "k-layout": thread t holds X[k2 + R2 k1] for k2 = t + q R1 (q < R2/R1),
// k1 < R1, in v[q R1 + k1].
// Forward: R2-point DFT in registers, twiddle, one exchange through shared
// memory, R1-point DFTs in registers. The inverse runs the same steps
// backwards from the k-layout to the n-layout. Every register DFT has
// compile-time indices and constant twiddles, so nothing is spilled to
// local memory; one shared-memory round trip per transform.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace bae {

// cos and sin of 2 pi m / 32 from the first-octant values by symmetry
struct Root32 {
    double c, s;
};
__host__ __device__ constexpr Root32 root32(int m) {
    // cos(pi j / 16), j = 0..8
    constexpr double C[9] = {1.0,
                             0.98078528040323044913,
                             0.92387953251128675613,
                             0.83146961230254523708,
                             0.70710678118654752440,
                             0.55557023301960222474,
                             0.38268343236508977173,
                             0.19509032201612826785,
                             0.0};
    m = ((m % 32) + 32) % 32;
    const int q = m / 8, r = m % 8;  // angle = q pi/2 + r pi/16
    const double cr = C[r], sr = C[8 - r];
    if (q == 0) return {cr, sr};
    if (q == 1) return {-sr, cr};
    if (q == 2) return {-cr, -sr};
    return {sr, -cr};
}

// x (c + i s)
template <typename C, typename T>
__device__ __forceinline__ C crot(C x, T c, T s) {
    return cmake<C>(x.x * c - x.y * s, x.x * s + x.y * c);
}

// x * exp(-/+ 2 pi i M / R) with compile-time M, R | 32
template <int R, int M, bool INV, typename C>
__device__ __forceinline__ C wmul(C x) {
    using T = decltype(x.x);
    constexpr int m = ((M * (32 / R)) % 32 + 32) % 32;
    if constexpr (m == 0) return x;
    if constexpr (m == 16) return cmake<C>(-x.x, -x.y);
    if constexpr (m == 8) {   // forward: -i, inverse: +i
        if constexpr (INV) return cmake<C>(-x.y, x.x);
        else return cmake<C>(x.y, -x.x);
    }
    if constexpr (m == 24) {  // forward: +i, inverse: -i
        if constexpr (INV) return cmake<C>(x.y, -x.x);
        else return cmake<C>(-x.y, x.x);
    }
    constexpr Root32 w = root32(m);
    const T c = (T)w.c;
    const T s = INV ? (T)w.s : (T)-w.s;
    return crot(x, c, s);
}

template <bool INV, typename C>
__device__ __forceinline__ void rdft2(C& a, C& b) {
    const C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <bool INV, typename C>
__device__ __forceinline__ void rdft4(C& x0, C& x1, C& x2, C& x3) {
    const C t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3);
    const C t3 = wmul<4, 1, INV>(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

// The radix-2 butterfly lo = e + W o, hi = e - W o with W = W_R^{+-K} a
// compile-time root. For float32 and float64 a general rotation is folded
// into the butterfly with fused multiply-adds (the factorisation of Linzer
// and Feig, "Implementation of efficient FFT algorithms on fused
// multiply-add architectures", IEEE Trans. Signal Process. 41, 1993):
// W o = f (o + i r o) with f the larger of |cos|, |sin| (so |r| <= 1), then
// e +- f u: six fused operations instead of a four-operation rotation and
// four additions. Rotations by multiples of pi/2 and the double-float type
// keep the plain form.
template <int R, int K, bool INV, typename C>
__device__ __forceinline__ void bfly(const C& e, const C& o, C& lo, C& hi) {
    using T = decltype(o.x);
    constexpr int m = ((K * (32 / R)) % 32 + 32) % 32;
    if constexpr (!(std::is_same<T, float>::value || std::is_same<T, double>::value) || m % 8 == 0) {
        const C w = wmul<R, K, INV>(o);
        lo = cadd(e, w);
        hi = csub(e, w);
    } else {
        constexpr Root32 w = root32(m);
        constexpr double c = w.c, sn = INV ? w.s : -w.s;   // W = c + i sn
        T ux, uy, f;
        if constexpr (c * c >= sn * sn) {   // W = c (1 + i sn/c)
            constexpr double r = sn / c;
            ux = fma_t((T)-r, o.y, o.x);
            uy = fma_t((T)r, o.x, o.y);
            f = (T)c;
        } else {                            // W = sn (c/sn + i)
            constexpr double r = c / sn;
            ux = fma_t((T)r, o.x, -o.y);
            uy = fma_t((T)r, o.y, o.x);
            f = (T)sn;
        }
        lo = cmake<C>(fma_t(f, ux, e.x), fma_t(f, uy, e.y));
        hi = cmake<C>(fma_t(-f, ux, e.x), fma_t(-f, uy, e.y));
    }
}

// the butterflies k = K .. R/2 - 1 of a radix-2 step: v[k], v[k + R/2]
template <int R, bool INV, typename C, int K>
struct Bflies {
    __device__ __forceinline__ static void run(const C* e, const C* o, C* v) {
        bfly<R, K, INV>(e[K], o[K], v[K], v[K + R / 2]);
        if constexpr (K + 1 < R / 2) Bflies<R, INV, C, K + 1>::run(e, o, v);
    }
};

// In-register DFT of v[0..R) in natural order, R in {2, 4, 8, 16, 32}.
template <int R, bool INV, typename C>
__device__ __forceinline__ void rdft(C* v);

template <int R, bool INV, typename C>
__device__ __forceinline__ void rdft(C* v) {
    if constexpr (R == 2) {
        rdft2<INV>(v[0], v[1]);
    } else if constexpr (R == 4) {
        rdft4<INV>(v[0], v[1], v[2], v[3]);
    } else {
        // radix-2 decimation in time: even and odd halves, then butterflies
        C e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        rdft<R / 2, INV>(e);
        rdft<R / 2, INV>(o);
        Bflies<R, INV, C, 0>::run(e, o, v);
    }
}

// rdft of v[0..R) whose upper half v[R/2..R) is zero (the zero-padded
// inputs of the forward transforms): the butterflies with a zero operand
// are dropped (same values as rdft up to the sign of zeros)
template <int R, bool INV, typename C>
__device__ __forceinline__ void rdft_zhi(C* v) {
    if constexpr (R == 2) {
        v[1] = v[0];
    } else if constexpr (R == 4) {
        const C x0 = v[0], x1 = v[1];
        const C t3 = wmul<4, 1, INV>(x1);
        v[0] = cadd(x0, x1);
        v[2] = csub(x0, x1);
        v[1] = cadd(x0, t3);
        v[3] = csub(x0, t3);
    } else {
        C e[R / 2], o[R / 2];   // both halves have a zero upper half again
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        rdft_zhi<R / 2, INV>(e);
        rdft_zhi<R / 2, INV>(o);
        Bflies<R, INV, C, 0>::run(e, o, v);
    }
}

// rdft of v[0..R) whose inputs v[M..R) are zero, 1 <= M (the shifted
// narrow inputs of the i pass): the butterflies with a zero operand are
// dropped (same values as rdft up to the sign of zeros)
template <int R, bool INV, int M, typename C>
__device__ __forceinline__ void rdft_zpre(C* v) {
    if constexpr (M >= R) {
        rdft<R, INV>(v);
    } else if constexpr (M == 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = v[0];
    } else if constexpr (R == 4) {   // M == 2 (M == 3: the full DFT)
        if constexpr (M == 2) rdft_zhi<4, INV>(v);
        else rdft<4, INV>(v);
    } else {
        C e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        rdft_zpre<R / 2, INV, (M + 1) / 2>(e);
        rdft_zpre<R / 2, INV, M / 2>(o);
        Bflies<R, INV, C, 0>::run(e, o, v);
    }
}

template <int L> struct Factors;
template <> struct Factors<16> { static constexpr int R1 = 4, R2 = 4; };
template <> struct Factors<32> { static constexpr int R1 = 4, R2 = 8; };
template <> struct Factors<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Factors<128> { static constexpr int R1 = 8, R2 = 16; };
template <> struct Factors<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct Factors<512> { static constexpr int R1 = 16, R2 = 32; };

// Exchange buffer for one transform: R2 x R1 complex at
// xch[base + k2 * sk + n1 * sn]; the caller picks the strides so that the
// lanes of a warp touch distinct banks (columns interleaved: sk = R1 W,
// sn = W, base = column; lines: sk = R1 + 1, sn = 1, base = line offset).

// n-layout -> k-layout (forward, or inverse when INV: then from the
// n-layout of X to the k-layout of the inverse transform, same steps with
// conjugate twiddles). tw: exp(-2 pi i m / L), m < L. ZHI: the input rows
// n >= L/2 are zero (v[m] = 0 for m >= R2 / 2); NZ > 0: only v[m < NZ] are
// nonzero (rows n < R1 NZ).
template <int L, bool INV, bool ZHI = false, int NZ = 0, typename C>
__device__ __forceinline__ void fft_n2k(C* v, C* xch, int base, int sk, int sn, int t, const C* __restrict__ tw) {
    constexpr int R1 = Factors<L>::R1, R2 = Factors<L>::R2, Q = R2 / R1;
    if constexpr (NZ > 0) rdft_zpre<R2, INV, NZ>(v);  // only v[m < NZ] nonzero
    else if constexpr (ZHI) rdft_zhi<R2, INV>(v);     // v[k2] = Y[t][k2]
    else rdft<R2, INV>(v);
#pragma unroll
    for (int k2 = 1; k2 < R2; ++k2) {
        const C w = ldg_c(tw + t * k2);
        v[k2] = INV ? cmulc(v[k2], w) : cmul(v[k2], w);
    }
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) xch[base + k2 * sk + t * sn] = v[k2];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[q * R1 + n1] = xch[base + (t + q * R1) * sk + n1 * sn];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) rdft<R1, INV>(v + q * R1);   // v[q R1 + k1] = X[k2 + R2 k1]
}

// k-layout -> n-layout (inverse when INV, the mirror of fft_n2k).
template <int L, bool INV, typename C>
__device__ __forceinline__ void fft_k2n(C* v, C* xch, int base, int sk, int sn, int t, const C* __restrict__ tw) {
    constexpr int R1 = Factors<L>::R1, R2 = Factors<L>::R2, Q = R2 / R1;
#pragma unroll
    for (int q = 0; q < Q; ++q) rdft<R1, INV>(v + q * R1);   // v[q R1 + n1] = Z[k2][n1]
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
            const int k2 = t + q * R1;
            if (n1 > 0 && k2 > 0) {
                const C w = ldg_c(tw + n1 * k2);
                v[q * R1 + n1] = INV ? cmulc(v[q * R1 + n1], w) : cmul(v[q * R1 + n1], w);
            }
            xch[base + k2 * sk + n1 * sn] = v[q * R1 + n1];
        }
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k2] = xch[base + k2 * sk + t * sn];
    __syncthreads();
    rdft<R2, INV>(v);                                   // v[n2] = x[t + R1 n2]
}


// ------------------------------------------------------------ transform plans
// A plan fixes how one line of length L is spread over the threads that
// transform it: TH threads per line, S values per thread. In both plans the
// n-layout is "thread t holds x[t + TH m] in slot m" (m < S), so a forward
// transform's zero upper half is exactly the slots m >= S / 2; the k-layout
// (after a forward transform, before an inverse one) is given by kidx(t, s).
// The exchange area of a line holds XLEN positions; position p of the line
// whose area starts at xch + base sits at xch[base + p * es], es = 1 for a
// private area per line (line passes; XS positions apart) or es = the number
// of lines interleaved element by element (column passes).

// Two levels (fft_n2k / fft_k2n above): TH = R1, S = R2.
template <int L>
struct Plan2 {
    static constexpr int R1 = Factors<L>::R1, R2 = Factors<L>::R2;
    static constexpr int TH = R1, S = R2;
    static constexpr int XS = R2 * (R1 + 1) + 1;   // private area stride (odd)
    static constexpr int XLEN = L;
    // slot s = q R1 + k1 holds X[t + q R1 + R2 k1]
    __host__ __device__ static constexpr int kidx(int t, int s) { return t + (s / R1) * R1 + R2 * (s % R1); }
    template <bool ZHI, typename C>
    __device__ __forceinline__ static void fwd(C* v, C* xch, int base, int es, int t, const C* __restrict__ tw) {
        fft_n2k<L, false, ZHI>(v, xch, base, es == 1 ? R1 + 1 : R1 * es, es, t, tw);
    }
    // forward transform whose slots m >= NZ are zero
    template <int NZ, typename C>
    __device__ __forceinline__ static void fwd_nz(C* v, C* xch, int base, int es, int t, const C* __restrict__ tw) {
        fft_n2k<L, false, false, NZ>(v, xch, base, es == 1 ? R1 + 1 : R1 * es, es, t, tw);
    }
    template <typename C>
    __device__ __forceinline__ static void inv(C* v, C* xch, int base, int es, int t, const C* __restrict__ tw) {
        fft_k2n<L, true>(v, xch, base, es == 1 ? R1 + 1 : R1 * es, es, t, tw);
    }
};

// Three levels for L = 512 = 8 x 8 x 8: 64 threads per line, 8 values each
// (the two-level 16 x 32 split holds 32 values per thread, which for
// 16-byte elements means ~200-255 registers and few warps per SM). With
// n = t + 64 m, t = t1 + 8 t2, and k = k3 + 8 k2 + 64 k1:
//   X[k] = sum_t1 W8^{t1 k1} W64^{t1 k2} sum_t2 W8^{t2 k2}
//          [ W512^{t k3} sum_m W8^{m k3} x[t + 64 m] ]
// stage A: thread t, DFT over m (slots k3), twiddle W512^{t k3};
// exchange; stage B: thread t1 + 8 k3, DFT over t2 (slots k2), twiddle
// W64^{t1 k2}; exchange; stage C: thread k3 + 8 k2, DFT over t1: slot k1
// holds X[t + 64 k1]. The inverse runs the stages backwards with conjugate
// twiddles. Positions are padded by one per 64 so that 16-byte accesses of
// the line passes do not collide in shared-memory banks.
struct Plan3_512 {
    static constexpr int TH = 64, S = 8;
    static constexpr int XLEN = 512 + 8;
    static constexpr int XS = XLEN + 1;
    __host__ __device__ static constexpr int kidx(int t, int s) { return t + 64 * s; }
    __device__ __forceinline__ static int pos(int p) { return p + (p >> 6); }

    template <bool ZHI, typename C>
    __device__ __forceinline__ static void fwd(C* v, C* xch, int base, int es, int t, const C* __restrict__ tw) {
        fwd_nz<ZHI ? 4 : 8>(v, xch, base, es, t, tw);
    }
    // forward transform whose slots m >= NZ are zero
    template <int NZ, typename C>
    __device__ __forceinline__ static void fwd_nz(C* v, C* xch, int base, int es, int t, const C* __restrict__ tw) {
        if constexpr (NZ == 4) rdft_zhi<8, false>(v);   // v[k3]
        else rdft_zpre<8, false, NZ>(v);
#pragma unroll
        for (int k3 = 1; k3 < 8; ++k3) v[k3] = cmul(v[k3], ldg_c(tw + t * k3));
#pragma unroll
        for (int k3 = 0; k3 < 8; ++k3) xch[base + pos(k3 * 64 + t) * es] = v[k3];
        __syncthreads();
        const int t1 = t & 7, k3 = t >> 3;
#pragma unroll
        for (int t2 = 0; t2 < 8; ++t2) v[t2] = xch[base + pos(k3 * 64 + t1 + 8 * t2) * es];
        __syncthreads();
        rdft<8, false>(v);                               // v[k2]
#pragma unroll
        for (int k2 = 1; k2 < 8; ++k2) v[k2] = cmul(v[k2], ldg_c(tw + 8 * t1 * k2));
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) xch[base + pos((k3 * 8 + k2) * 8 + t1) * es] = v[k2];
        __syncthreads();
        const int c3 = t & 7, c2 = t >> 3;
#pragma unroll
        for (int u1 = 0; u1 < 8; ++u1) v[u1] = xch[base + pos((c3 * 8 + c2) * 8 + u1) * es];
        __syncthreads();
        rdft<8, false>(v);                               // v[k1] = X[t + 64 k1]
    }

    template <typename C>
    __device__ __forceinline__ static void inv(C* v, C* xch, int base, int es, int t, const C* __restrict__ tw) {
        const int c3 = t & 7, c2 = t >> 3;               // this thread's (k3, k2)
        rdft<8, true>(v);                                // v[t1]
#pragma unroll
        for (int u1 = 0; u1 < 8; ++u1) xch[base + pos((c3 * 8 + c2) * 8 + u1) * es] = v[u1];
        __syncthreads();
        const int t1 = t & 7, k3 = t >> 3;
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) v[k2] = xch[base + pos((k3 * 8 + k2) * 8 + t1) * es];
        __syncthreads();
#pragma unroll
        for (int k2 = 1; k2 < 8; ++k2) v[k2] = cmulc(v[k2], ldg_c(tw + 8 * t1 * k2));
        rdft<8, true>(v);                                // v[t2]
#pragma unroll
        for (int t2 = 0; t2 < 8; ++t2) xch[base + pos(k3 * 64 + t1 + 8 * t2) * es] = v[t2];
        __syncthreads();
#pragma unroll
        for (int j3 = 0; j3 < 8; ++j3) v[j3] = xch[base + pos(j3 * 64 + t) * es];
        __syncthreads();
#pragma unroll
        for (int j3 = 1; j3 < 8; ++j3) v[j3] = cmulc(v[j3], ldg_c(tw + t * j3));
        rdft<8, true>(v);                                // v[m] = x[t + 64 m]
    }
};

// Three levels for L = 256 = 8 x 8 x 4: 32 threads per line (one warp), 8
// values each (the two-level 16 x 16 split holds 16 values per thread:
// 170-210 registers for 16-byte elements, one 256-thread CTA per SM). With
// n = t + 32 m, t = t1 + 4 t2 (t1 < 4, t2 < 8), k = k3 + 8 k2 + 64 k1:
//   X[k] = sum_t1 W4^{t1 k1} W32^{t1 k2} sum_t2 W8^{t2 k2}
//          [ W256^{t k3} sum_m W8^{m k3} x[t + 32 m] ]
// stage A: thread t, DFT over m (slots k3), twiddle W256^{t k3}; exchange;
// stage B: thread t1 + 4 k3, DFT over t2 (slots k2), twiddle W32^{t1 k2};
// exchange; stage C: thread u takes the two pairs (k3, k2) = (u % 8,
// u / 8 + 4 h), h < 2, each a 4-point DFT over t1. Slot s = h + 2 k1 then
// holds X[u + 32 s]. The inverse runs the stages backwards with conjugate
// twiddles. Positions are swizzled, p -> p ^ rev3((p >> 5) & 7) (rev3
// reverses three bits), so that the 16-byte accesses of a line (one warp)
// hit eight distinct bank groups in every stage: rows of 32 positions
// apart land on distinct groups, and the two 4-aligned blocks read in stage
// B land in different halves.
struct Plan3_256 {
    static constexpr int TH = 32, S = 8;
    static constexpr int XLEN = 256;
    static constexpr int XS = XLEN + 1;
    __host__ __device__ static constexpr int kidx(int t, int s) { return t + 32 * s; }
    __device__ __forceinline__ static int pos(int p) {
        const int r = (p >> 5) & 7;
        return p ^ (((r & 1) << 2) | (r & 2) | ((r >> 2) & 1));
    }

    template <bool ZHI, typename C>
    __device__ __forceinline__ static void fwd(C* v, C* xch, int base, int es, int t, const C* __restrict__ tw) {
        fwd_nz<ZHI ? 4 : 8>(v, xch, base, es, t, tw);
    }
    // forward transform whose slots m >= NZ are zero
    template <int NZ, typename C>
    __device__ __forceinline__ static void fwd_nz(C* v, C* xch, int base, int es, int t, const C* __restrict__ tw) {
        if constexpr (NZ == 4) rdft_zhi<8, false>(v);   // v[k3]
        else rdft_zpre<8, false, NZ>(v);
#pragma unroll
        for (int k3 = 1; k3 < 8; ++k3) v[k3] = cmul(v[k3], ldg_c(tw + t * k3));
#pragma unroll
        for (int k3 = 0; k3 < 8; ++k3) xch[base + pos(k3 * 32 + t) * es] = v[k3];
        __syncthreads();
        const int t1 = t & 3, k3 = t >> 2;
#pragma unroll
        for (int t2 = 0; t2 < 8; ++t2) v[t2] = xch[base + pos(k3 * 32 + t1 + 4 * t2) * es];
        __syncthreads();
        rdft<8, false>(v);                               // v[k2]
#pragma unroll
        for (int k2 = 1; k2 < 8; ++k2) v[k2] = cmul(v[k2], ldg_c(tw + 8 * t1 * k2));
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) xch[base + pos((k3 * 8 + k2) * 4 + t1) * es] = v[k2];
        __syncthreads();
        const int c3 = t & 7, c2 = t >> 3;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            C w[4];
#pragma unroll
            for (int u1 = 0; u1 < 4; ++u1) w[u1] = xch[base + pos((c3 * 8 + c2 + 4 * h) * 4 + u1) * es];
            rdft<4, false>(w);                           // w[k1]
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) v[h + 2 * k1] = w[k1];   // X[t + 32 (h + 2 k1)]
        }
        __syncthreads();
    }

    template <typename C>
    __device__ __forceinline__ static void inv(C* v, C* xch, int base, int es, int t, const C* __restrict__ tw) {
        const int c3 = t & 7, c2 = t >> 3;               // this thread's pairs (k3, k2 + 4 h)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            C w[4];
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) w[k1] = v[h + 2 * k1];
            rdft<4, true>(w);                            // w[t1]
#pragma unroll
            for (int u1 = 0; u1 < 4; ++u1) xch[base + pos((c3 * 8 + c2 + 4 * h) * 4 + u1) * es] = w[u1];
        }
        __syncthreads();
        const int t1 = t & 3, k3 = t >> 2;
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) v[k2] = xch[base + pos((k3 * 8 + k2) * 4 + t1) * es];
        __syncthreads();
#pragma unroll
        for (int k2 = 1; k2 < 8; ++k2) v[k2] = cmulc(v[k2], ldg_c(tw + 8 * t1 * k2));
        rdft<8, true>(v);                                // v[t2]
#pragma unroll
        for (int t2 = 0; t2 < 8; ++t2) xch[base + pos(k3 * 32 + t1 + 4 * t2) * es] = v[t2];
        __syncthreads();
#pragma unroll
        for (int j3 = 0; j3 < 8; ++j3) v[j3] = xch[base + pos(j3 * 32 + t) * es];
        __syncthreads();
#pragma unroll
        for (int j3 = 1; j3 < 8; ++j3) v[j3] = cmulc(v[j3], ldg_c(tw + t * j3));
        rdft<8, true>(v);                                // v[m] = x[t + 32 m]
    }
};

}  // namespace bae
