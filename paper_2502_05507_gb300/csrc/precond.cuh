// Restricted additive Schwarz right preconditioner of the boundary
// algebraic equation.
//
// The BAE matrix A (eq. [double_bae] or its single-layer form) is dense,
// but its near-field entries dominate. Section 4 remarks that right
// preconditioning by the dense D_- improves the spectrum but costs too much,
// and the numerical section asks for preconditioning; this is a local form:
// for every gamma- node r, S_r = the gamma- nodes of the 5 x 5 x 5
// neighbourhood of r (about 25 on a smooth surface; the MAXR nearest when
// there are more), and row r of M^{-1} is the row of r in inv(A[S_r, S_r]).
// GMRES solves A M^{-1} y = b, q = M^{-1} y.
//
// A M^{-1} v is computed as A z with z = M^{-1} v formed by a small sparse
// kernel in float64 (inside the captured GMRES step), so the convolution
// keeps the exact source recipe. Used by the float32 inner solves of the
// mixed precision (iterative refinement).
#pragma once

#include "classify.cuh"
#include "common.cuh"

namespace bae {

constexpr int MAXR = 32;   // members of a neighbourhood block, at most (one per lane of a warp)
constexpr int NB_R = 2;    // the neighbourhood: offsets up to NB_R per axis
static_assert(MAXR == 32, "a row's slots map onto the lanes of a warp (the fused Arnoldi step relies on it)");
constexpr int NEAR_TN = 8;  // the blocks use G_s at offsets [0, NEAR_TN)^3 (up to 2 NB_R + 2 per axis)
constexpr int NEAR_TAB = NEAR_TN * (NEAR_TN + 1) * (NEAR_TN + 2) / 6;   // sorted-table length

struct Precond {
    bool built = false;
    bool pending = false;          // built on another stream; the owner's stream has not waited yet
    cudaStream_t stream = nullptr; // owner's stream (frees)
    long long n = 0;
    // row r of M^{-1}: slot q at col[r * MAXR + q], val[r * MAXR + q] (unused
    // slots: column r, value 0)
    int* col = nullptr;
    float* val = nullptr;
    void release();
};

// Builds the preconditioner of the problem's BAE (layer and LGF parameter
// s = kappa^2 h^2 as in the geometry) on the geometry's stream: one warp
// per gamma- node (found through the geometry's node map) forms its
// neighbourhood block and solves for its row in float32 (a preconditioner
// only approximates the inverse; M^{-1} itself is applied exactly in
// float64, so the preconditioned system is unchanged).
// near: G_s on the sorted offsets below NEAR_TN (lgf_table(NEAR_TN, s)),
// device; computed here when null.
// Runs on stream `on` (which must already be ordered after the geometry's
// build); the arrays are freed on the geometry's stream.
void build_precond(const Geometry& g, double s, const double* near, Precond& out, cudaStream_t on);

// out[b] = M^{-1} in[b] with in[b] at in + b in_stride (+ row[b] row_stride
// when row is not null, device), out[b] at out + b out_stride, for items
// with active[b] != 0 when active is not null (a mask; all device arrays,
// capturable in a graph). in32 (optional): the selected input rows already
// rounded to float32, [nb][n] (read instead of converting in); out32
// (optional): out rounded to float32 as well, [nb][n].
void precond_apply(const Precond& p, const double* in, long long in_stride, const int* row, long long row_stride,
                   double* out, long long out_stride, int nb, const int* active, cudaStream_t st,
                   const float* in32 = nullptr, float* out32 = nullptr);

}  // namespace bae
