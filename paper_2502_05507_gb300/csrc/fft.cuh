// In-shared-memory radix-8/4/2 Stockham FFT used by the convolution passes.
//
// A CTA holds several lines of the same power-of-two length L in shared
// memory; L/8 threads cooperate on each line, every thread owning eight
// complex values per stage (one radix-8 butterfly, two radix-4 or four
// radix-2). Stages are separated by CTA-wide barriers, so every thread of
// the CTA must call fft_line with the same L and direction. Twiddles come
// from a table tw[m] = exp(-2 pi i m / L), m < L, staged in shared memory.
//
// Stockham autosort (no bit reversal): stage with span Ns and radix R reads
// x[j + r L/R], multiplies by W_{Ns R}^{r (j mod Ns)}, does an R-point DFT
// and writes to (j / Ns) Ns R + (j mod Ns) + r Ns.
#pragma once

#include "common.cuh"

namespace bae {

constexpr int const_log2(int v) { return v <= 1 ? 0 : 1 + const_log2(v >> 1); }

template <typename C, bool INV>
__device__ __forceinline__ void dft2(C& a, C& b) {
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
    C t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), d = csub(x1, x3);
    // forward multiplies d by -i, inverse by +i
    C t3 = INV ? cmake<C>(-d.y, d.x) : cmake<C>(d.y, -d.x);
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft8(C* v) {
    using T = decltype(v[0].x);
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<C, INV>(e0, e1, e2, e3);
    dft4<C, INV>(o0, o1, o2, o3);
    const T r = (T)0.70710678118654752440;
    if (!INV) {  // o_k *= exp(-i pi k / 4)
        o1 = cmake<C>((o1.x + o1.y) * r, (o1.y - o1.x) * r);
        o2 = cmake<C>(o2.y, -o2.x);
        o3 = cmake<C>((o3.y - o3.x) * r, -(o3.x + o3.y) * r);
    } else {     // o_k *= exp(+i pi k / 4)
        o1 = cmake<C>((o1.x - o1.y) * r, (o1.x + o1.y) * r);
        o2 = cmake<C>(-o2.y, o2.x);
        o3 = cmake<C>(-(o3.x + o3.y) * r, (o3.x - o3.y) * r);
    }
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <typename C, int R, bool INV>
__device__ __forceinline__ void dft_r(C* v) {
    if constexpr (R == 8) dft8<C, INV>(v);
    else if constexpr (R == 4) dft4<C, INV>(v[0], v[1], v[2], v[3]);
    else dft2<C, INV>(v[0], v[1]);
}

// One in-place Stockham stage; t in [0, L/8) is the thread's slot in its line.
template <typename C, int L, int R, bool INV>
__device__ __forceinline__ void stockham_stage(C* line, const C* tw, int t, int logNs) {
    constexpr int TPL = L / 8;
    constexpr int NB = 8 / R;            // butterflies per thread
    constexpr int LOGR = const_log2(R);
    constexpr int LOGL = const_log2(L);
    C v[8];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * TPL;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = line[j + r * (L / R)];
    }
    __syncthreads();
    const int Ns = 1 << logNs;
    const int shift = LOGL - logNs - LOGR;  // tw index = r k L / (Ns R)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * TPL;
        const int k = j & (Ns - 1);
        C* w = v + b * R;
        if (logNs > 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const C tv = tw[(r * k) << shift];
                w[r] = INV ? cmulc(w[r], tv) : cmul(w[r], tv);
            }
        }
        dft_r<C, R, INV>(w);
        const int idxD = ((j >> logNs) << (logNs + LOGR)) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) line[idxD + r * Ns] = w[r];
    }
    __syncthreads();
}

// Full length-L transform of one line held in shared memory (unnormalised;
// the inverse uses +i). All threads of the CTA must call it together.
template <typename C, int L, bool INV>
__device__ __forceinline__ void fft_line(C* line, const C* tw, int t) {
    constexpr int LOGL = const_log2(L);
    constexpr int N8 = LOGL / 3;
    constexpr int REM = LOGL % 3;
    int logNs = 0;
#pragma unroll
    for (int s = 0; s < N8; ++s) {
        stockham_stage<C, L, 8, INV>(line, tw, t, logNs);
        logNs += 3;
    }
    if constexpr (REM == 2) stockham_stage<C, L, 4, INV>(line, tw, t, logNs);
    if constexpr (REM == 1) stockham_stage<C, L, 2, INV>(line, tw, t, logNs);
}

}  // namespace bae
