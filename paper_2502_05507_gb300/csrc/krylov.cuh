// Deterministic batched vector kernels for GMRES (classical Gram-Schmidt
// with one reorthogonalisation). Every reduction uses a fixed partition of
// the vector and a fixed summation order (partial sums per chunk, then the
// last CTA to finish adds the partials in chunk order), so results do not
// depend on timing or on which other right-hand sides share the launch.
#pragma once

#include "common.cuh"

namespace bae {

int krylov_chunks(int n);

// *d_flag |= 1 if some x[i] is not finite, counting only i whose
// flags[i % period] has bit 0 (M+) when flags is not null
void kr_nonfinite(const double* x, long long n, const uint8_t* flags, long long period, int* d_flag,
                  cudaStream_t st);

// nrm2[b] = ||x[b]||^2 (deterministic), x [nb][n] with row stride n
void kr_norm2(const double* x, const int* active, int na, int n, double* partial, int nchunk, double* out,
              cudaStream_t st);
// y[b] = a[b] - c[b] for active b
void kr_sub(const double* a, const double* c, const int* active, int na, int n, double* y, cudaStream_t st);
// y[b] += x[b] for active b
void kr_add(const double* x, const int* active, int na, int n, double* y, cudaStream_t st);

}  // namespace bae

namespace bae {

// Device-resident state of a batch of restarted-GMRES cycles whose Arnoldi
// steps run without the host: the step index j, the Hessenberg columns, the
// Givens rotations and the per-RHS convergence flags live in device memory,
// so one Arnoldi step (apply + CGS2 + Givens) can be captured once as a
// CUDA graph and replayed.
struct Arnoldi {
    int n = 0, nb = 0, m = 0, nchunk = 0;
    double* V = nullptr;        // [nb][m+1][n]
    double* w = nullptr;        // [nb][n]
    double* part = nullptr;     // [nb][m+2][nchunk] partial sums
    double* h1 = nullptr;       // [nb][m+1] first projection, then the second
    double* hcol = nullptr;     // [nb][m+1] h1 + h2
    double* H = nullptr;        // [nb][m][m+1] rotated Hessenberg, column j at j (m+1)
    double* cs = nullptr;       // [nb][m]
    double* sn = nullptr;       // [nb][m]
    double* g = nullptr;        // [nb][m+1]
    double* y = nullptr;        // [nb][m] least-squares solution
    double* est = nullptr;      // [nb] residual estimate |g[j+1]|
    double* target = nullptr;   // [nb] absolute residual target
    double* inv = nullptr;      // [nb] 1 / ||w||
    int* flag = nullptr;        // [nb] 1 while the RHS is iterating in this cycle
    int* ncols = nullptr;       // [nb] basis vectors used this cycle
    unsigned int* ctr = nullptr;  // [nb][3] last-block counters (self-resetting)
    int* j = nullptr;           // [nb] current step of each RHS
    // w = A V[j] is formed inside the first projection pass from the
    // potential v [nb][v_stride] (float32 or float64) by the closure gather
    // w[r] = t[r] v[gm[r]] + (1 - t[r]) v[partner[r]] (eq. [double_bae])
    const void* v = nullptr;
    bool v_f32 = false;
    long long v_stride = 0;
    const int* gm = nullptr;
    const int* partner = nullptr;
    const double* t = nullptr;
    // fused step (one cooperative kernel with grid barriers), used when
    // coop_grid > 0: the barrier counter (reset to 0 before the first step,
    // a multiple of coop_grid between steps), an error flag set when a
    // barrier wait runs out, and [nb] squared norms
    int coop_grid = 0;
    bool coop_resident = false;   // one CTA per chunk, basis chunk in shared memory
    unsigned long long* bar = nullptr;
    int* err = nullptr;
    double* n2 = nullptr;
    // In the fused step the Givens rotations of column j run one step later,
    // on the last nb CTAs of the grid, while the other CTAs compute column
    // j + 1: the step stores column j (h1 + h2, and ||w - V h2|| after it)
    // in pcol[b][j % 2] and sets gflag[b]; the next step applies the
    // rotations, updates g and the residual estimate, and decides flag[b]
    // (the right-hand side that converged at column j has computed column
    // j + 1 for nothing). live[b] = flag[b] | gflag[b] tells the host that
    // another step is needed; bar2 counts the barriers of the chunk CTAs.
    int* gflag = nullptr;                  // [nb]
    int* live = nullptr;                   // [nb]
    int* live_host = nullptr;              // [nb] device address of mapped host memory, or null
    double* pcol = nullptr;                // [nb][2][m + 2]
    // right preconditioner rows (32 slots per row, column r and value 0 in
    // unused slots): when set, the fused step ends with z = M^{-1} V[j+1]
    // (the next step's apply reads z) after one more grid barrier
    const int* pre_col = nullptr;
    const float* pre_val = nullptr;
    double* zpre = nullptr;                // [nb][n]
    unsigned long long* bar2 = nullptr;
    // float32 copies, rounded where the float64 values are written: v32
    // [nb][n] of the newest basis vector V[j] and, with the preconditioner,
    // z32 [nb][n] of z = M^{-1} V[j]; the float32 applies and the
    // preconditioner read them instead of converting float64 values (GB300's
    // float64 pipe, which also converts, is narrow)
    float* v32 = nullptr;
    float* z32 = nullptr;
    // bounded barrier waits: polls before a wait gives up; err_host, when
    // set, is mapped host memory the failing CTA also flags (the host stops
    // the cycle after the step). bar_extra > 0 only under host fault
    // injection: the barriers then wait for that many CTAs more than the
    // grid has, so every wait runs out (see bae_inject_fault).
    long long spin_limit = 1LL << 22;
    int* err_host = nullptr;
    int bar_extra = 0;
};

// number of vector chunks (CTAs per RHS) of the Arnoldi passes
int arnoldi_chunks(int n);

// Start of a cycle: r [nb][n] residuals with squared norms nrm2[b]; RHS with
// member[b] != 0 and sqrt(nrm2) > target start iterating (V[b][0] = r/beta).
void arn_init(const Arnoldi& a, const double* r, const double* nrm2, const int* member, cudaStream_t st);
// One Arnoldi step after the potential v = K V[j] (gather into w = A V[j],
// CGS2 with the norm of the reorthogonalised vector from the Pythagorean
// identity, Givens, j++, next basis vector): three kernels.
void arn_step(const Arnoldi& a, cudaStream_t st);
// CTAs of the fused cooperative step for this batch (0 if the device cannot
// run it: no cooperative launch, or more than 64 right-hand sides); call
// before any graph capture.
// *resident: every (RHS, chunk) item gets its own resident CTA, which keeps
// its chunk of the basis in shared memory.
int arn_coop_grid(int n, int nb, int m, bool* resident);
// End of a cycle: y = R^{-1} g for every RHS with ncols > 0, x += V y
// (each RHS over its own ncols columns, read on the device).
void arn_finish(const Arnoldi& a, double* x, cudaStream_t st);

}  // namespace bae
