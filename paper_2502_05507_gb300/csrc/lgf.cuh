// Lattice Green's function table and spectrum (Section 2.2).
#pragma once

#include "common.cuh"

namespace bae {

// G_s(n) for all sorted offsets N > a >= b >= c >= 0, index
// a(a+1)(a+2)/6 + b(b+1)/2 + c, into `out` (device, N(N+1)(N+2)/6 doubles).
void lgf_table(int N, double s, double* out, cudaStream_t st);

// Octant spectrum of G_s evenly embedded in (2N)^3 (offset N set to 0):
// ghat[(k1 (N+1) + k2)(N+1) + k3] = sum_n Gemb(n) cos(pi k.n / N), times
// `scale`. Writes float64 into g64 and, if g32 is not null, float32 into g32.
// Whether the spectrum of the (2N)-periodic Green's function (closed form)
// equals the embedded G_s to round-off: (2N)^3 exp(-mu N) < 1e-14 with
// cosh(mu) = 1 + s/2; lgf_spectrum then skips the table.
bool periodic_spectrum_applies(int N, double s);

void lgf_spectrum(int N, double s, double scale, double* g64, float* g32, cudaStream_t st);

// Octant spectrum (same layout) of the finite-box Green's function of eq.
// [aux] (zero on the layers 0 and N of every axis), for sources extended
// oddly about those layers: scale / (6 + s - 2 sum cos(pi k_d / N)), 0 at
// the pole (s = 0, k = 0).
void box_spectrum(int N, double s, double scale, double* g64, float* g32, cudaStream_t st);

// Twiddle tables exp(-2 pi i m / L), m < L, on the device.
void make_twiddles(int L, double2* tw64, float2* tw32, cudaStream_t st);

}  // namespace bae
