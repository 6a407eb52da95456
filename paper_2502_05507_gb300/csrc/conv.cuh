// Host interface of the LGF convolution (the potential apply).
#pragma once

#include "common.cuh"
#include "dsf.cuh"

namespace bae {

// Compact description of the source stencil rho = B q (Section 3.2): the
// source nodes in lexicographic order, grouped by (i,j) grid line, each
// with its terms rho(x) = sum coef * q[idx].
struct SrcRecipe {
    const int* line_off = nullptr;   // N*N + 1 offsets into src_lin
    const int* src_lin = nullptr;    // linear grid index of each source node
    const int* term_off = nullptr;   // ns + 1 offsets into term_idx/term_coef
    const int* term_idx = nullptr;   // unknown number of each term
    const double* term_coef = nullptr;
    const float* term_coef32 = nullptr;   // the same coefficients rounded to float32
    // sum the terms in float64 before the float32 rounding (the direct
    // formulation's (6 + s) u(n) - sum u(y) cancels to O(h^2 u))
    bool wide = false;
};

enum SourceMode { SRC_DENSITY = 0, SRC_VOLUME = 1 };

template <typename T>
struct ConvArgs {
    int N = 0;
    int nbatch = 1;
    SourceMode mode = SRC_DENSITY;
    // SRC_DENSITY: q [nbatch][q_stride] float64 density on gamma-; when q_row
    // is set, batch item b reads q + b q_stride + q_row[b] q_row_stride (the
    // row indices live in device memory, so a captured graph can advance them)
    const double* q = nullptr;
    long long q_stride = 0;
    const int* q_row = nullptr;
    long long q_row_stride = 0;
    // optional float32 copy of the density the float32 apply reads (the
    // values of q rounded to float32; item b at q32 + b q32_stride, the row
    // q_row selects): saves the float64 -> float32 conversions, which run on
    // GB300's narrow float64 pipe
    const float* q32 = nullptr;
    long long q32_stride = 0;
    // optional per-item flags: items with active[b] == 0 are skipped
    const int* active = nullptr;
    SrcRecipe rec;
    // SRC_VOLUME: rho = scale * f on nodes with (flags & 1); in SRC_DENSITY
    // mode a non-null f adds these volume sources to the layer sources
    const double* f = nullptr;
    const uint8_t* flags = nullptr;
    double scale = 1.0;
    // the grid of this apply has axes 0 and f_swap swapped (swap_axes):
    // rec, flags and the output v are in the swapped layout, f in the
    // caller's, so f is read at swap_axes(x) (0: no swap)
    int f_swap = 0;
    // work buffers (per batch item): A = N*N*(N+1), B = N*2N*(N+1) complex
    cplx_t<T>* A = nullptr;
    cplx_t<T>* B = nullptr;
    const T* ghat = nullptr;      // (N+1)^3 octant, includes 1/(2N)^3
    const cplx_t<T>* tw = nullptr;  // exp(-2 pi i m / 2N), m < 2N
    typename OutOf<T>::type* v = nullptr;   // [nbatch][N^3] output potential
    // x-planes [p0, p1) hold every nonzero source and every output the
    // caller reads (p1 == 0: all N planes). Planes outside are skipped: their
    // sources are zero, and their part of v is left unwritten.
    int p0 = 0, p1 = 0;
    // finite auxiliary box (eq. [aux], SRC_VOLUME only, float64 and
    // double-float): the source is extended oddly about the layers 0 and N
    // of every axis (loads of the upper half return the negated mirror
    // instead of zero padding) and ghat is the box spectrum; runs the five
    // separate passes
    bool box = false;
    // never time schedules in this apply: use the choice made by an earlier
    // apply of the same (element type, N, batch size), else the default
    bool no_tune = false;
    __host__ __device__ int plane_lo() const { return p1 > 0 ? p0 : 0; }
    __host__ __device__ int plane_hi() const { return p1 > 0 ? p1 : N; }
    // lines [q0, q1) along the second axis (even bounds) hold every source
    // and every node read back (q1 == 0: all N). The k passes transform
    // only the line pairs of the planes [p0, p1) inside it; the forward j
    // pass reads the other rows as zeros and the inverse one does not write
    // them. The plane-fused kernels transform every line.
    int q0 = 0, q1 = 0;
    __host__ __device__ int line_lo() const { return q1 > 0 ? q0 : 0; }
    __host__ __device__ int line_hi() const { return q1 > 0 ? q1 : N; }
    __host__ __device__ int pairs_per_plane() const { return (line_hi() - line_lo()) / 2; }
    // line pairs of the k passes, and the first line of pair gp (pairs
    // numbered plane by plane)
    __host__ __device__ long long npairs() const { return (long long)(plane_hi() - plane_lo()) * pairs_per_plane(); }
    __host__ __device__ long long pair_line(long long gp) const {
        const int npq = pairs_per_plane();
        return (long long)(plane_lo() + gp / npq) * N + line_lo() + 2 * (gp % npq);
    }
};

template <typename T>
void conv_apply(const ConvArgs<T>& a, cudaStream_t st);

// The apply and the kernel set-up for one transform length L = 2N,
// instantiated per element type in conv_f32.cu, conv_f64.cu and
// conv_df64*.cu.
template <typename T, int L>
void run_conv(const ConvArgs<T>& a, cudaStream_t st);
template <typename T, int L>
void conv_configure();

// The cluster plane kernels (conv_cplane_*.cu) for L where one plane of
// k-spectra does not fit one CTA: cplane_ready sets their attributes and
// says whether the device can place a cluster; cplane_launch runs the
// forward (k, j) or the inverse (j, k) kernel.
template <typename T, int L>
bool cplane_ready();
template <typename T, int L>
void cplane_launch(const ConvArgs<T>& a, cudaStream_t st, bool inverse);

// Sets the kernel attributes conv_apply needs for grid size N (done on the
// first apply anyway; call it before capturing applies in a CUDA graph).
template <typename T>
void conv_prepare(int N);

// Whether the schedule for (element type, N, batch size) has been chosen
// already (an apply outside graph capture chooses it by timing both).
template <typename T>
bool conv_tuned(int N, int nbatch);

// out[b][r] = t[r] v[b][gm[r]] + (1 - t[r]) v[b][partner[r]]  (items with
// active[b] == 0 skipped when active is not null)
template <typename T>
void closure_gather(const T* v, long long v_stride, const int* gm, const int* partner, const double* t,
                    int n, int nbatch, double* out, long long out_stride, cudaStream_t st,
                    const int* active = nullptr);

// Rows of the direct formulation for items with active[b] != 0 (all
// device arrays, capturable): y[b][r] = t[r] x(r) + (1 - t[r]) x(pu[r]) for
// r < n_gm (the closure), y[b][n_gm + k] = x(n_gm + k) - w[b][gp[k]] (gamma+);
// x[b] at x + b x_stride (+ x_row[b] x_row_stride when x_row is set).
template <typename W, typename Y>
void direct_rows(const W* w, long long w_stride, const double* x, long long x_stride, const int* x_row,
                 long long x_row_stride, const int* gp, const int* pu, const double* t, long long n_gm, long long n_unk,
                 int nb, const int* active, Y* y, long long y_stride, cudaStream_t st);

// out[x] = (flags[x] & bit) != 0 for x < n
void mask_bit(const uint8_t* flags, long long n, uint8_t bit, uint8_t* out, cudaStream_t st);

// u[b][gm[r]] = q[b][r] for r < n
void scatter_gm(const double* q, long long q_stride, const int* gm, long long n, int nb, double* u, long long n3,
                cudaStream_t st);

// u[b][x] = (nplus(x) ? add[b][x] + v[b][x'] : 0) over the N^3 grid, with
// x' = swap_axes(x, v_swap, N): v and add in the swapped layout, u and
// flags in the grid's
template <typename T>
void volume_combine(const T* v, const double* add, const uint8_t* flags, long long n3, int nbatch,
                    double* u, cudaStream_t st, int v_swap = 0, int N = 0);

// out[i] = nearest double-float of in[i]
void to_dsf(const double* in, long long n, dsf* out, cudaStream_t st);

// v (T) -> out (double), plain copy
template <typename T>
void widen(const T* v, long long n, double* out, cudaStream_t st);

}  // namespace bae
