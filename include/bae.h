/*
 * bae.h - C ABI of the GB300 (sm_103a) unfitted boundary algebraic equation
 * (BAE) solver with lattice Green's functions.
 *
 * Method: Xia, "Unfitted boundary algebraic equation method based on
 * difference potentials and lattice Green's function in 3D". Equations are
 * cited by their LaTeX labels in brackets, e.g. eq. [double_bae].
 *
 * Problem (Section 2, eq. [elliptic]):  -Lap u + kappa2 u = f in Omega,
 * u = g on dOmega, kappa2 >= 0, Omega = {phi < 0} given by level-set samples
 * on an N^3 Cartesian grid with spacing h. Node (i,j,k) sits at
 * origin + (i,j,k) h; every N^3 array is C-order (k fastest).
 *
 * Conventions for every entry point:
 *  - Return value: BAE_OK (0) or one of the BAE_ERR_* codes below; the
 *    thread-local message of the last failure is bae_last_error(). No C++
 *    exception crosses this boundary.
 *  - Array arguments are plain pointers that may point to device memory of
 *    the context's device or to host memory (pageable or pinned); the
 *    library detects which (cudaPointerGetAttributes) and stages host arrays
 *    through its own device buffers, copying on the context stream. Device
 *    memory of another GPU is rejected with BAE_ERR_INVALID_ARG. The
 *    caller owns every array it passes; the library never frees them.
 *  - Each call makes its context's device current while it runs and
 *    restores the calling thread's current device before it returns.
 *  - All work is issued on the context's stream. Entry points return after
 *    the stream has finished the call's work (results are ready to read).
 *  - Handles own their device memory; a problem must be destroyed before its
 *    context. Handles are not thread-safe: one call at a time per handle.
 *  - There is no CPU fallback: without a usable GPU every call that needs
 *    one returns BAE_ERR_CUDA.
 */
#ifndef BAE_H
#define BAE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define BAE_OK                 0
#define BAE_ERR_INVALID_ARG    1  /* bad size, null pointer, non-finite input  */
#define BAE_ERR_GEOMETRY       2  /* gamma- empty or touching the grid box faces */
#define BAE_ERR_OOM            3  /* device allocation failed                   */
#define BAE_ERR_NOT_CONVERGED  4  /* GMRES hit its limit; outputs still written */
#define BAE_ERR_TIMEOUT        5  /* a bounded device wait ran out             */
#define BAE_ERR_CUDA           6  /* any other CUDA failure                    */

/* layer type of the indirect formulation (Section 3.2) */
#define BAE_LAYER_DOUBLE 0     /* D(m,n), eq. [double_potential] (default)     */
#define BAE_LAYER_SINGLE 1     /* S(m,n) = G(m-n), eq. [single_potential]      */
#define BAE_LAYER_DIRECT 2     /* direct formulation: the unknown is u on
                                  gamma = gamma- then gamma+ (n_gm + n_gp values),
                                  difference potentials G_h[chi_{M-} L_h u]
                                  (eqs. [dp], [bep], [direct_sys])              */

/* arithmetic of the potential apply */
#define BAE_FP64  0            /* every step in float64                        */
#define BAE_MIXED 1            /* float32 convolution inside float64 iterative
                                  refinement (solve only)                      */
#define BAE_FP32  2            /* float32 convolution (apply entry points only)*/
#define BAE_DF64  3            /* double-float convolution: each value a pair of
                                  float32 (about 48 significant bits) on the
                                  float32 pipes; float64-accurate to ~1e-14
                                  (apply entry points, and the refinement
                                  residual of BAE_MIXED)                      */

typedef struct bae_ctx bae_ctx;
typedef struct bae_problem bae_problem;

typedef struct bae_options {
    double tol;          /* relative residual ||b - A q|| / ||b||, default 1e-10 */
    int    max_iter;     /* total GMRES iterations (all cycles), default 500    */
    int    restart;      /* GMRES restart length, 1..1024, default 200          */
    int    precision;    /* BAE_FP64 (every apply native float64), BAE_DF64
                            (every apply double-float) or BAE_MIXED (float32
                            applies inside iterative refinement), default
                            BAE_FP64                                         */
    int    max_refine;   /* outer refinement steps for BAE_MIXED, default 8     */
    double inner_tol;    /* inner float32 GMRES reduction per step, default 1e-5;
                            the step that can reach tol aims at 0.3 tol ||b|| */
    int    use_graphs;   /* 1: each Arnoldi step (apply, Gram-Schmidt, Givens) is captured
                            as a CUDA graph once per solve and replayed; 0:
                            launched kernel by kernel with programmatic
                            launch overlap (same kernels). Default 0: per
                            solve, the capture costs more than the launches
                            it saves (measured on the bench workloads). */
    int    residual_precision;  /* BAE_MIXED only: arithmetic of the particular
                            solution, the refinement residuals and the
                            reconstruction, BAE_DF64 (default) or BAE_FP64 */
    int    precond;      /* BAE_MIXED only: right-preconditions the inner
                            float32 GMRES with a restricted additive Schwarz
                            inverse of the BAE matrix (each gamma- node's row
                            of the inverse of its 5 x 5 x 5 neighbourhood
                            block, at most 32 nearest nodes; a local form of the right preconditioning
                            in Section 4's remark; built once per problem on
                            the device from a small LGF table): 1 (default)
                            in every refinement step, 2 in the steps after
                            the first, 0 never. The solution is the same to
                            tol.                                           */
    int    particular;   /* particular solution u_p = G_h[chi_{M+} f] (eq. [ps]):
                            BAE_PARTICULAR_LATTICE (default) convolves with the
                            free-lattice G_h; BAE_PARTICULAR_BOX solves the
                            auxiliary problem of eq. [aux] on the finite box
                            (zero on the layers 0 and N of every axis), as
                            Algorithm 1 prints it. u on N+ is the same discrete
                            solution either way; the density differs. The box
                            form costs one float64-accurate apply more per
                            solve (u_p is kept, not folded into the
                            residuals). Not for BAE_LAYER_DIRECT.           */
} bae_options;

#define BAE_PARTICULAR_LATTICE 0
#define BAE_PARTICULAR_BOX     1

typedef struct bae_stats {
    int    iterations;       /* GMRES iterations, all cycles and refinement steps */
    int    refinements;      /* outer refinement steps (BAE_MIXED), else 0        */
    int    applies_fp64;     /* float64-accurate applies (BAE_FP64 or BAE_DF64)   */
    int    applies_fp32;     /* float32 potential applies in this call            */
    double rel_residual;     /* final ||b - A q|| / ||b||, A applied in float64   */
    double ms_total;         /* wall time of the call on the context stream       */
    int64_t h2d_bytes;       /* bytes of this right-hand side's inputs (f, g) the
                                call copied from host memory (0: device inputs) */
    int64_t d2h_bytes;       /* bytes of its outputs (u, density) it copied to
                                host memory (0: device outputs)                 */
} bae_stats;

/* ------------------------------------------------------------- utilities */

/* ABI version, currently 1. */
int bae_version(void);

/* Message of the last failed call on this thread ("" if none). Owned by the
 * library; valid until the next call on this thread. */
const char* bae_last_error(void);

/* Fills *opts with the defaults listed in bae_options. */
void bae_default_options(bae_options* opts);

/* Number of CUDA kernels this library has launched in this process so far
 * (all contexts). */
long long bae_launch_count(void);

/* Schedule of the FFT convolution inside every potential apply of this
 * process (all contexts): BAE_SCHED_AUTO (-1, the default) times every
 * schedule the (precision, N) can run on the first apply of each
 * (precision, N, batch size) outside graph capture and keeps the fastest;
 * BAE_SCHED_PASSES (0) runs the k, j and i transforms as five separate
 * kernels; BAE_SCHED_PLANE (1) fuses the k and j transforms per x-plane (one
 * CTA per plane where the plane of k-spectra fits in shared memory, a
 * thread-block cluster sharing it through distributed shared memory where it
 * does not); BAE_SCHED_PASSES_ALT (2) runs the five passes with a second
 * launch geometry (float32: column blocks of half the width at N = 128, the
 * three-level 8 x 8 x 8 transform at N = 256; float64: the three-level
 * 8 x 8 x 4 transform at N = 128; elsewhere the same as BAE_SCHED_PASSES); BAE_SCHED_PERSIST (3) runs the five passes as
 * persistent kernels, each launched with at most the CTAs that are resident
 * at once, striding over the tiles of every right-hand side of the batch.
 * All compute the same convolution (Section 3.2, the
 * discrete potentials as lattice sums); they differ in rounding order only.
 * A schedule the size cannot run falls back to BAE_SCHED_PASSES. Overrides
 * the BAE_CONV_PLANE environment variable (0, 1, 2 or 3: the same values).
 * Returns BAE_ERR_INVALID_ARG for any other value. Not part of the method:
 * a performance control. */
#define BAE_SCHED_AUTO (-1)
#define BAE_SCHED_PASSES 0
#define BAE_SCHED_PLANE 1
#define BAE_SCHED_PASSES_ALT 2
#define BAE_SCHED_PERSIST 3
int bae_set_conv_schedule(int schedule);

/* Host-side fault injection for the library's own failure tests (the paper
 * has no counterpart). Nothing here faults or hangs a GPU: the failures are
 * made on the host or by bounded device waits. Process-wide.
 *  - BAE_FAULT_NONE: clears every injection (arg ignored).
 *  - BAE_FAULT_BARRIER: the next `arg` launches of the fused (cooperative)
 *    Arnoldi step wait at each grid barrier for one CTA more than the grid
 *    has, polling about a millisecond instead of half a second; the waits
 *    run out, the kernel records the error and returns, and the solve
 *    returns BAE_ERR_TIMEOUT. Steps replayed from a CUDA graph
 *    (use_graphs) are not affected. The context stays usable.
 *  - BAE_FAULT_ALLOC_CAP: every device allocation of the library (work
 *    space, problem data, spectra) larger than `arg` bytes fails as out of
 *    memory (BAE_ERR_OOM) until cleared; arg <= 0 clears it. A failed
 *    bae_problem_create frees what it had made; the context stays usable.
 * Returns BAE_ERR_INVALID_ARG for an unknown kind. */
#define BAE_FAULT_NONE 0
#define BAE_FAULT_BARRIER 1
#define BAE_FAULT_ALLOC_CAP 2
int bae_inject_fault(int kind, long long arg);

/* Process-wide kernel timing. bae_profile_start pre-creates CUDA events for
 * up to max_launches launches; from then on every kernel launch of the
 * library is bracketed by two events on its own stream. bae_profile_stop
 * synchronises the device, and for each distinct kernel (in order of first
 * launch, at most max_kernels) writes its name into `names` ('\n'-separated,
 * NUL-terminated, truncated to names_len bytes), its summed device time in
 * milliseconds into total_ms[k] and its launch count into launches[k];
 * *n_kernels gets the number written. Any output pointer may be NULL (host
 * memory). Returns BAE_ERR_INVALID_ARG if more than max_launches launches
 * happened (the excess is not timed). Not part of the method; a measurement
 * aid. */
int bae_profile_start(int max_launches);
int bae_profile_stop(char* names, int names_len, double* total_ms, long long* launches, int max_kernels,
                     int* n_kernels);

/* --------------------------------------------------------------- context */

/* Creates a context on CUDA device `device`. `stream` is a cudaStream_t
 * (for instance torch.cuda.current_stream().cuda_stream) or NULL for a new
 * non-blocking stream owned by the context. The context caches LGF spectra
 * per (N, s = kappa2 h^2) (numerical section: the table is precomputed once
 * and reused across problems). */
int bae_ctx_create(int device, void* stream, bae_ctx** out);

/* Frees the context, its cache and its stream (if it created one). */
void bae_ctx_destroy(bae_ctx* ctx);

/* ------------------------------------------------------ LGF (Section 2.2) */

/* G_s(n) of (6+s) - sum of the six neighbours (eq. [lgf] with h = 1, by
 * Watson's Bessel integral eq. [lgf_bessel] with exp(-(6+s)t)), for all
 * sorted offsets N > a >= b >= c >= 0 in lexicographic order of (a,b,c):
 * index(a,b,c) = a(a+1)(a+2)/6 + b(b+1)/2 + c; `values` holds
 * N(N+1)(N+2)/6 doubles. N in [2, 256], s >= 0 and finite. */
int bae_lgf_table(bae_ctx* ctx, int N, double s, double* values);

/* The real spectrum of G_s embedded evenly in the (2N)^3 periodic box
 * (offset N set to 0), on the octant 0 <= k_i <= N: ghat[(k1 (N+1) + k2)(N+1)
 * + k3] = sum_n Gemb(n) cos(pi k.n / N), unscaled. (N+1)^3 doubles. N must be
 * a power of two in [8, 256]. When (2N)^3 exp(-mu N) < 1e-14 (cosh mu =
 * 1 + s/2: G_s has decayed far below round-off within the box) it is the
 * closed-form spectrum of the (2N)-periodic Green's function,
 * 1 / (6 + s - 2 sum cos(pi k_i / N)) (the 2N-point trapezoid rule of
 * Section 2.2), equal to the embedded one to round-off. */
int bae_lgf_spectrum(bae_ctx* ctx, int N, double s, double* ghat);

/* -------------------------------------------------- problem (Algorithm 1) */

/* Classifies the grid from phi (N^3 doubles; phi < 0 is interior, phi == 0
 * exterior; Section 2.1 point sets M+-, N+-, gamma+-), builds the closure
 * (one row per gamma- node: among its M+ neighbours, in the order +x,-x,+y,
 * -y,+z,-z with x = array axis 0, the one with the largest
 * t = phi(p)/(phi(p)-phi(m)); x* = x_p + t (x_m - x_p); row
 * t v(m) + (1-t) v(p) = g(x*), the hat basis of eq. [bc]), and fetches or
 * builds the LGF spectrum for s = kappa2 h^2.
 * N: power of two in [8, 256]. h > 0. layer: BAE_LAYER_DOUBLE (a gamma- node
 * whose D_n is empty uses the single-layer column) or BAE_LAYER_SINGLE.
 * BAE_ERR_GEOMETRY if gamma- is empty or touches the box faces. */
int bae_problem_create(bae_ctx* ctx, int N, double h, const double origin[3],
                       const double* phi, double kappa2, int layer, bae_problem** out);

void bae_problem_destroy(bae_problem* prob);

/* |gamma-| (the boundary points, and the unknowns of the layer
 * formulations), |gamma+|, |M+|. Any pointer may be NULL. Host-side, no
 * device work. */
int bae_problem_sizes(const bae_problem* prob, int64_t* n_gm, int64_t* n_gp, int64_t* n_mp);

/* Unknowns of the boundary system: n_gm for the single and double layer,
 * n_gm + n_gp for BAE_LAYER_DIRECT (u on gamma-, then on gamma+). This is
 * the length of every density q below. Host-side, no device work. */
int bae_problem_unknowns(const bae_problem* prob, int64_t* n);

/* gp_idx[n_gp]: linear indices of gamma+ (lexicographic; the order of the
 * gamma+ unknowns of the direct formulation). Host or device pointer. */
int bae_gamma_plus(const bae_problem* prob, int32_t* gp_idx);

/* The x-planes [*lo, *hi) that hold every source (gamma-, the D-nodes, M+)
 * and every node a solve reads back (gamma-, the closure partners, M+): the
 * other planes are zero on input and unread on output. When
 * bae_problem_conv_planes reports axis 0, inside a solve and in
 * bae_boundary_apply the convolution transforms only these planes. Not a
 * quantity of the paper; a cost model aid. Host-side, no device work. */
int bae_problem_plane_range(const bae_problem* prob, int* lo, int* hi);

/* The planes that the applies inside a solve and bae_boundary_apply
 * transform: *axis is the grid axis (0 x, 1 y, 2 z) with the fewest planes
 * holding sources or read-back nodes (chosen only when it has at least a
 * tenth fewer than x; always 0 for BAE_LAYER_DIRECT or with the environment
 * variable BAE_CONV_AXIS=x at problem creation), [*lo, *hi) the range along
 * it. The convolution skips zero planes only along the first axis of the
 * grid it runs on, so those applies run on the grid with axes x and *axis
 * swapped; the lattice Green's function is symmetric under permutations of
 * the axes, so they compute the same potential (within rounding). Not a
 * quantity of the paper; a cost model aid. Host-side, no device work. */
int bae_problem_conv_planes(const bae_problem* prob, int* axis, int* lo, int* hi);

/* Boundary points x*(m) of the closure rows, gamma- in lexicographic order:
 * xyz[3r + c]. The caller evaluates g there. */
int bae_boundary_points(const bae_problem* prob, double* xyz);

/* Classification export, any pointer may be NULL:
 *  flags[N^3]: bit0 M+, bit1 gamma-, bit2 gamma+, bit3 D-node (outside N+,
 *              next to gamma-), bits 4..6 |D_n| on gamma- nodes;
 *  gm_idx[n_gm]: linear indices of gamma- (lexicographic);
 *  partner[n_gm]: linear index of the closure partner p(m);
 *  t[n_gm]: closure weight t(m). */
int bae_classification(const bae_problem* prob, uint8_t* flags, int32_t* gm_idx,
                       int32_t* partner, double* t);

/* mask[N^3] = 1 on M+ (phi < 0, the nodes where u is the solution of eq.
 * [discrete]), 0 elsewhere; host or device pointer. */
int bae_interior_mask(const bae_problem* prob, uint8_t* mask);

/* ---------------------------------------- the potential apply (hot path) */

/* v = K q on the whole N^3 grid, K the problem's layer potential
 * (Section 3.2: single eq. [single_potential], double eq. [double_potential]),
 * i.e. the source stencil rho = B q, the free-space convolution with G_s by
 * a zero-padded (2N)^3 FFT, v(m) = sum_x G_s(m-x) rho(x). For
 * BAE_LAYER_DIRECT, q is u on gamma and v the difference potential
 * P q = G_s * [chi_{M-} ((6 + s) q - sum of the six neighbours of q)]
 * (eq. [dp] with G_h = h^2 G_s, s = kappa2 h^2).
 * q: bae_problem_unknowns() doubles; v: N^3 doubles. precision BAE_FP64 or
 * BAE_FP32. */
int bae_potential_apply(bae_problem* prob, int precision, const double* q, double* v);

/* The boundary operator of eq. [double_bae] (or its single-layer analogue):
 * (A q)_m = t(m) (Kq)(m) + (1 - t(m)) (Kq)(p(m)) for every gamma- node m.
 * BAE_LAYER_DIRECT (eq. [direct_sys] with eq. [inhom]): the closure rows
 * t(m) q(m) + (1 - t(m)) q(p(m)) on gamma-, then q(p) - (P q)(p) on gamma+.
 * q, Aq: bae_problem_unknowns() doubles. precision BAE_FP64 or BAE_FP32. */
int bae_boundary_apply(bae_problem* prob, int precision, const double* q, double* Aq);

/* The same potential apply as bae_potential_apply, for callers that must not
 * allocate device memory while they run (a fixed memory budget owned by the
 * host application, a real-time loop in which cudaMalloc/cudaFree would
 * stall or synchronise the device, a plug-in host that forbids allocation
 * after start-up). This call allocates nothing: its work buffers are one
 * file-scope device array of 8 MiB that every GPU the library touches holds
 * until the process exits. The paper has no counterpart; this is a
 * deployment variant of the hot path.
 *  - q (bae_problem_unknowns() doubles) and v (N^3 doubles) must be device memory of the
 *    problem's device; host pointers are rejected (BAE_ERR_INVALID_ARG),
 *    since staging them would need allocations.
 *  - Size limit: float32 up to N = 64, float64 up to N = 32; larger problems
 *    are rejected with BAE_ERR_INVALID_ARG and a message giving the bytes
 *    needed. The problem handle, its spectrum and twiddles are built by
 *    bae_problem_create, which does allocate, at set-up.
 *  - The first call on a device looks up the device address of the array
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *  - The call never times convolution schedules: it uses the schedule an
 *    earlier apply of the same precision and N (one right-hand side) chose,
 *    or bae_set_conv_schedule's, else the plane-fused default.
 *  - Every call uses the same array and leaves its contents behind; nothing
 *    in it needs clearing, since each call writes every element it reads.
 *    Calls whose GPU work overlaps in time (several host threads, several
 *    contexts or streams on one device) race on the array: serialise them.
 * precision BAE_FP64 or BAE_FP32. Returns after the work has finished. */
int bae_potential_apply_noalloc(bae_problem* prob, int precision, const double* q, double* v);

/* Particular solution on the free lattice (eq. [ps] with G_h = h^2 G_s):
 * up(m) = sum_{x in M+} G_s(m-x) h^2 f(x) on the whole grid.
 * f, up: N^3 doubles (paper sign). precision BAE_FP64 or BAE_FP32. */
int bae_particular(bae_problem* prob, int precision, const double* f, double* up);

/* Particular solution on the finite auxiliary box (eq. [aux] with eq. [ps]):
 * up solves (6 + s) up(m) - sum of the six neighbours = h^2 f(m) [m in M+]
 * for every m with all indices in [1, N-1], with up = 0 on the layers of
 * index 0 and N (s = kappa2 h^2). It is the convolution of the source,
 * extended oddly about those layers, with the (2N)-periodic Green's
 * function, on the same zero-padded transform as the potential apply.
 * f, up: N^3 doubles (paper sign). precision BAE_FP64 or BAE_DF64. */
int bae_box_particular(bae_problem* prob, int precision, const double* f, double* up);

/* ---------------------------------------------------- solve (Algorithm 1) */

/* Solves the BAE of eq. [double_bae] (or single layer) by unrestarted-
 * per-cycle GMRES with zero initial guess and no preconditioner:
 *   b = g - Phi u_p,  A q = b,  u = u_p + K q.
 * BAE_LAYER_DIRECT solves eq. [direct_sys] with eq. [inhom] for q = u on
 * gamma: b = [g; u_p on gamma+], u = u_p + P q on M+ and q on gamma-
 * (eq. [discrete_green]); its Schwarz blocks (opts->precond) take the
 * gamma nodes of each neighbourhood (closure rows, and delta - P rows).
 * f: N^3 doubles (paper sign, -Lap u + kappa2 u = f); g: n_gm doubles, the
 * Dirichlet data at bae_boundary_points(). Outputs: density q
 * (bae_problem_unknowns() doubles)
 * and u (N^3 doubles: the discrete solution on N+ = M+ u gamma-, 0 elsewhere);
 * either may be NULL. opts may be NULL (defaults); stats may be NULL.
 * Only the values of f on M+ are read (eq. [ps] takes chi_{M+} f); from
 * host memory the call copies the box of planes that holds M+ (the planes
 * with a source, one plane of margin, along each axis) and reports the
 * bytes in stats->h2d_bytes. Likewise u, which is 0 outside N+: into host
 * memory the call copies that box and writes the zeros around it with
 * host threads while the device solves (stats->d2h_bytes). Inputs and
 * outputs may be host or device memory independently.
 * BAE_ERR_NOT_CONVERGED leaves valid outputs and stats. */
int bae_solve(bae_problem* prob, const double* f, const double* g, const bae_options* opts,
              double* density, double* u, bae_stats* stats);

/* nrhs independent right-hand sides on one problem: f [nrhs][N^3],
 * g [nrhs][n_gm], density [nrhs][n_gm], u [nrhs][N^3]. Every GMRES step
 * applies the potential to all unconverged right-hand sides in one batched
 * convolution. stats, if not NULL, points to nrhs entries. Returns the worst
 * per-RHS code. */
int bae_solve_batched(bae_problem* prob, int nrhs, const double* f, const double* g,
                      const bae_options* opts, double* density, double* u, bae_stats* stats);

/* ---------------------------------------------------------------- serving */

/* A solve server: a host scheduler admits submitted requests into one of
 * `slots` concurrent slots (each a context with its own CUDA stream and work
 * space) when a slot is free and the request's device-memory estimate fits
 * in hbm_budget_bytes next to the requests in flight; work of different
 * slots overlaps on the device. With two or more slots, the first half run
 * on streams of the device's highest priority and take small requests
 * (N <= 64) first, the others on the lowest priority and take large ones
 * first; a slot with none of its class queued takes the first request that
 * fits. Requests of any N, kappa2, geometry and
 * layer mix freely; LGF spectra are cached on the device per
 * (N, kappa2 h^2) and shared by all slots; Krylov state stays on the
 * device. A request's result does not depend on what else is in flight. */
typedef struct bae_server bae_server;

/* Called on a server thread once the request is classified: fill g[r] with
 * the Dirichlet data at xyz[3r..3r+2] (host arrays, n points). */
typedef void (*bae_boundary_fn)(const double* xyz, int64_t n, double* g, void* user);

typedef struct bae_request {
    int N;                       /* as bae_problem_create                        */
    double h;
    double origin[3];
    const double* phi;           /* N^3, host or device; valid until done        */
    double kappa2;
    int layer;
    const double* f;             /* N^3, host or device; valid until done        */
    bae_boundary_fn boundary;    /* Dirichlet data at the boundary points        */
    void* user;                  /* passed to boundary                           */
    double* u_out;               /* N^3 output, host or device (or NULL)         */
    bae_options opts;            /* solve options                                */
} bae_request;

typedef struct bae_result {
    int status;                  /* BAE_OK or the solve's error code            */
    int64_t n_gm;                /* length of the density (bae_problem_unknowns) */
    bae_stats stats;
    double t_submit, t_admit, t_done;  /* seconds on the server's steady clock   */
} bae_result;

#define BAE_PENDING 7            /* bae_server_poll: not finished yet          */

int bae_server_create(int device, int slots, int64_t hbm_budget_bytes, bae_server** out);
/* Queues a request (copied; the arrays it points to must stay valid until
 * the request is done). *ticket identifies it. */
int bae_server_submit(bae_server* srv, const bae_request* req, int64_t* ticket);
/* Waits up to timeout_ms (0: no wait, < 0: forever) for the request; returns
 * BAE_OK with *out filled when it is done, BAE_PENDING otherwise. */
int bae_server_poll(bae_server* srv, int64_t ticket, int timeout_ms, bae_result* out);
/* Copies the finished request's density (bae_problem_unknowns() doubles of
 * its problem) to out (host or device, capacity doubles). */
int bae_server_density(bae_server* srv, int64_t ticket, double* out, int64_t capacity);
/* Forgets a finished request. */
int bae_server_release(bae_server* srv, int64_t ticket);
/* Seconds on the server's steady clock (the time base of bae_result). */
double bae_server_clock(bae_server* srv);
/* Finishes the requests in flight, drops the queued ones, frees everything. */
void bae_server_destroy(bae_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* BAE_H */
