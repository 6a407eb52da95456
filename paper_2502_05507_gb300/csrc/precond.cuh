// Block-Jacobi right preconditioner of the boundary algebraic equation.
//
// The BAE matrix A (eq. [double_bae] or its single-layer form) is dense,
// but its near-field entries dominate. Section 4 remarks that right
// preconditioning by the dense D_- improves the spectrum but costs too much,
// and the numerical section asks for preconditioning; this is the local
// form: the gamma- nodes are grouped by 2 x 2 x 2 cells of the grid, the
// exact diagonal blocks A[B, B] of those groups are inverted, and GMRES
// solves A M^{-1} y = b with M = blockdiag(A[B, B]), q = M^{-1} y.
//
// A M^{-1} v is computed as A z with z = M^{-1} v formed by a small
// block-diagonal kernel in float64 (inside the captured GMRES step), so the
// convolution keeps the exact source recipe. Used by the float32 inner
// solves of the mixed precision (iterative refinement).
#pragma once

#include "classify.cuh"
#include "common.cuh"

namespace bae {

constexpr int MAXB = 8;   // gamma- nodes in a 2 x 2 x 2 cell, at most

struct Precond {
    bool built = false;
    cudaStream_t stream = nullptr;
    long long n = 0;
    // row r of M^{-1}: col[r * MAXB + q], val[r * MAXB + q], q < MAXB (unused
    // slots have value 0)
    int* col = nullptr;
    double* val = nullptr;
    void release();
};

// Builds the preconditioner of the problem's BAE (layer and LGF parameter
// s = kappa^2 h^2 as in the geometry) on the geometry's stream: a small LGF
// table, a cell table, and one thread per gamma- node that forms and inverts
// its cell's block.
void build_precond(const Geometry& g, double s, Precond& out);

// out[b] = M^{-1} in[b] with in[b] at in + b in_stride (+ row[b] row_stride
// when row is not null, device), out[b] at out + b out_stride, for items
// with active[b] != 0 when active is not null (a mask; all device arrays,
// capturable in a graph).
void precond_apply(const Precond& p, const double* in, long long in_stride, const int* row, long long row_stride,
                   double* out, long long out_stride, int nb, const int* active, cudaStream_t st);

}  // namespace bae
