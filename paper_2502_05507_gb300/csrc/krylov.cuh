// Deterministic batched vector kernels for GMRES (classical Gram-Schmidt
// with one reorthogonalisation). Every reduction uses a fixed partition of
// the vector and a fixed summation order, so results do not depend on
// timing or on which other right-hand sides share the launch.
#pragma once

#include "common.cuh"

namespace bae {

// Batch of nb vectors of length n with a Krylov basis each:
// V [nb][m+1][n], w [nb][n].
struct KrylovBatch {
    int n = 0;
    int nb = 0;
    int mp1 = 0;                  // m + 1 basis vectors per RHS
    double* V = nullptr;
    double* w = nullptr;
    double* partial = nullptr;    // [nb][mp1 + 1][nchunk]
    double* h = nullptr;          // [nb][mp1 + 1] reduced results
    int nchunk = 0;
};

int krylov_chunks(int n);

// h[b][i] = <V[b][i], w[b]> for i < cols (b in active list), deterministic.
void kr_dots(const KrylovBatch& k, const int* active, int na, int cols, cudaStream_t st);
// w[b] -= sum_{i < cols} V[b][i] h[b][i]; then h[b][mp1] = ||w[b]||^2.
void kr_update_norm(const KrylovBatch& k, const int* active, int na, int cols, cudaStream_t st);
// V[b][j] = w[b] / ||w[b]|| with the norm^2 left in h[b][mp1] by kr_update_norm
// (a zero vector if the norm is 0: breakdown)
void kr_scale_into(const KrylovBatch& k, const int* active, int na, int j, cudaStream_t st);
// x[b] += sum_{i < cols} V[b][i] y[b][i]   (x [nb][n], y [nb][ystride])
void kr_combine(const KrylovBatch& k, const int* active, int na, int cols, const double* y, int ystride,
                double* x, cudaStream_t st);
// y[b] = x[b] * alpha[b] for active b, vectors [nb][n]
void kr_scale(const double* x, const double* alpha, const int* active, int na, int n, double* y, cudaStream_t st);
// nrm2[b] = ||x[b]||^2 (deterministic), x [nb][n] with row stride n
void kr_norm2(const double* x, const int* active, int na, int n, double* partial, int nchunk, double* out,
              cudaStream_t st);
// y[b] = a[b] - c[b] for active b
void kr_sub(const double* a, const double* c, const int* active, int na, int n, double* y, cudaStream_t st);
// y[b] += x[b] for active b
void kr_add(const double* x, const int* active, int na, int n, double* y, cudaStream_t st);
// gather / scatter whole rows: dst[r] = src[active[r]] (rows of n doubles)
void kr_gather_rows(const double* src, const int* active, int na, long long n, double* dst, cudaStream_t st);
void kr_scatter_rows(const double* src, const int* active, int na, long long n, double* dst, cudaStream_t st);

}  // namespace bae
