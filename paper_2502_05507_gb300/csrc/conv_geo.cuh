// Launch geometry of the potential-apply kernels (shared by conv_impl.cuh
// and conv_cplane.cuh).
#pragma once

#include <type_traits>

#include "conv.cuh"
#include "fft2.cuh"

namespace bae {

// Launch geometry per transform length and precision.
template <typename T, int L> struct Geo {
    using C = cplx_t<T>;
    static constexpr int R1 = Factors<L>::R1, R2 = Factors<L>::R2;
    // column passes: W columns per CTA, R1 threads per column
    static constexpr int WB = 65536 / (L * (int)sizeof(C));
    static constexpr int W = WB > 32 ? 32 : (WB < 8 ? 8 : WB);
    static constexpr int CT = W * R1;
    // line passes (k): P line pairs per CTA, R1 threads per pair
    static constexpr int PB = 65536 / (L * (int)sizeof(C));
    static constexpr int P = (256 / R1) < PB ? (256 / R1) : (PB < 4 ? 4 : PB);
    static constexpr int KT = P * R1;
    static constexpr int XS = R2 * (R1 + 1) + 1;   // exchange stride per pair (odd)
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
    static constexpr int CW = (N1 + CS - 1) / CS;     // columns per CTA
    static constexpr size_t XL = (size_t)PP * XS * sizeof(C);
    static constexpr size_t XC = (size_t)L * PW * sizeof(C);
    static constexpr size_t SMEM = ROWS + (XL > XC ? XL : XC);
    static constexpr bool USE = CS > 1 && CS <= 8 && SMEM <= 227 * 1024 && NR % 2 == 0;
};

}  // namespace bae
