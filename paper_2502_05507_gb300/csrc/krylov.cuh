// Deterministic batched vector kernels for GMRES (classical Gram-Schmidt
// with one reorthogonalisation, delayed by one step). Every reduction uses
// a fixed partition of
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
// so one Arnoldi step can be captured once as a CUDA graph and replayed.
//
// Gram-Schmidt with delayed reorthogonalisation (DCGS2, one global
// reduction per step): row j of V holds u_j, the new direction after ONE
// classical projection, neither reorthogonalised nor normalised. Step j
// applies the operator to it (w = A M^{-1} u_j) and forms, in one reduction,
// c = Q^T u_j, u_j.u_j, b = Q^T w and u_j.w (Q = rows 0..j-1, orthonormal).
// Then r = sqrt(u.u - |c|^2), q_j = (u_j - Q c) / r (the second
// projection of u_j), t = (u.w - c.b) / r = q_j.w, and the next direction
// u_{j+1} = (w - Q b - q_j t) / r. Column j - 1 of the Hessenberg matrix
// becomes final in the same step (its pending part plus c, subdiagonal r);
// column j is h = ([b; t] - H c) / r with H the final columns 0..j-1
// (since w = A M^{-1} (r q_j + Q c)). The one-step delay matches the
// deferred Givens rotations: a cycle of k columns takes k + 1 steps.
struct Arnoldi {
    int n = 0, nb = 0, m = 0, nchunk = 0;
    double* V = nullptr;        // [nb][m+1][n]
    double* w = nullptr;        // [nb][n]
    double* part = nullptr;     // [nb][2 (m+1)][nchunk] partial sums: rows i <= j of Q^T u (i = j: u.u),
                                // then from row m + 1 those of Q^T w (m + 1 + j: u.w)
    double* cf = nullptr;       // [nb][2 (m+1)] the same sums reduced (read by the update pass)
    double* hs = nullptr;       // [nb][m+1] pending column j before its final terms
    double* Hu = nullptr;       // [nb][m][m+1] final columns, not rotated (for H c)
    double* H = nullptr;        // [nb][m][m+1] rotated Hessenberg, column j at j (m+1)
    double* cs = nullptr;       // [nb][m]
    double* sn = nullptr;       // [nb][m]
    double* g = nullptr;        // [nb][m+1]
    double* y = nullptr;        // [nb][m] least-squares solution
    double* est = nullptr;      // [nb] residual estimate |g[j]|
    double* target = nullptr;   // [nb] absolute residual target
    double* inv = nullptr;      // [nb] 1 / ||r|| at the start, then 1 / r of the step
    double* tco = nullptr;      // [nb] t = q_j.w of the step
    int* flag = nullptr;        // [nb] 1 while column j is to be computed in this cycle
    int* gflag = nullptr;       // [nb] 1 while column j - 1 waits to be finished
    int* live = nullptr;        // [nb] flag | gflag: the host runs another step
    int* live_host = nullptr;   // [nb] device address of mapped host memory, or null
    int* ncols = nullptr;       // [nb] basis vectors used this cycle
    int* jstep = nullptr;       // [nb] j and flag of the last step (two-kernel path:
    int* ran = nullptr;         //      the update kernel reads them)
    unsigned int* ctr = nullptr;  // [nb][3] last-block counters (self-resetting)
    int* j = nullptr;           // [nb] current step of each RHS
    // w = A u_j is formed inside the first pass from the potential v [nb][v_stride]
    // (float32 or float64) by the closure gather
    // w[r] = t[r] v[gm[r]] + (1 - t[r]) v[partner[r]] (eq. [double_bae])
    const void* v = nullptr;
    bool v_f32 = false;
    long long v_stride = 0;
    const int* gm = nullptr;
    const int* partner = nullptr;
    const double* t = nullptr;
    // fused step (one cooperative kernel with grid barriers), used when
    // coop_grid > 0: the chunk CTAs, then one CTA per right-hand side that
    // reduces its coefficients and finishes and rotates its column.
    // coop_resident: one CTA per chunk, basis chunk in shared memory.
    // coop_redundant: every chunk CTA holds one item and reduces its
    // right-hand side's coefficients itself (one grid barrier less).
    int coop_grid = 0;
    bool coop_resident = false;
    bool coop_redundant = false;
    unsigned long long* bar = nullptr;    // counter of the barriers of all CTAs
    unsigned long long* bar2 = nullptr;   // counter of the chunk CTAs' barrier
    int* err = nullptr;                   // set when a barrier wait runs out
    // right preconditioner rows (32 slots per row, column r and value 0 in
    // unused slots): when set, the fused step ends with z = M^{-1} u_{j+1}
    // (the next step's apply reads z) after one more grid barrier
    const int* pre_col = nullptr;
    const float* pre_val = nullptr;
    double* zpre = nullptr;                // [nb][n]
    // float32 copies, rounded where the float64 values are written: v32
    // [nb][n] of the newest direction u_{j+1} and, with the preconditioner,
    // z32 [nb][n] of z = M^{-1} u_{j+1}; the float32 applies and the
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
// One Arnoldi step after the potential v = K u_j (gather into w, the one
// reduction, q_j and u_{j+1}, the final column j - 1 and its rotations,
// j++): two kernels, or the fused cooperative kernel.
void arn_step(const Arnoldi& a, cudaStream_t st);
// Kernel attributes of the step kernels for restart length m; call before
// any graph capture.
void arn_configure(int m);
// CTAs of the fused cooperative step for this batch (0 if the device cannot
// run it: no cooperative launch, or more than 64 right-hand sides); call
// before any graph capture.
// *resident: every (RHS, chunk) item gets its own resident CTA, which keeps
// its chunk of the basis in shared memory. *redundant: every chunk CTA holds
// at most one item (the chunk CTAs reduce their coefficients themselves).
int arn_coop_grid(int n, int nb, int m, bool* resident, bool* redundant);
// End of a cycle: y = R^{-1} g for every RHS with ncols > 0, x += V y
// (each RHS over its own ncols columns, read on the device).
void arn_finish(const Arnoldi& a, double* x, cudaStream_t st);

}  // namespace bae
