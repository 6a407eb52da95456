// Restricted additive Schwarz right preconditioner of the BAE (see
// precond.cuh): built on the device, one warp per gamma- node forms its
// neighbourhood block and solves for its own row of that block's inverse.
#include <algorithm>

#include "lgf.cuh"
#include "precond.cuh"

namespace bae {

namespace {


// G_s on the offset cube [-TE, TE]^3 in shared memory, filled from the
// sorted table (offsets below NEAR_TN per axis, sorted by absolute value)
constexpr int TE = NEAR_TN - 1, TW = 2 * TE + 1, TCUBE = TW * TW * TW;

__device__ __forceinline__ float lgf_sorted(const double* __restrict__ tab, int dx, int dy, int dz) {
    int a = dx < 0 ? -dx : dx, b = dy < 0 ? -dy : dy, c = dz < 0 ? -dz : dz;
    if (a < b) { const int x = a; a = b; b = x; }
    if (b < c) { const int x = b; b = c; c = x; }
    if (a < b) { const int x = a; a = b; b = x; }
    return (float)tab[a * (a + 1) * (a + 2) / 6 + b * (b + 1) / 2 + c];
}

__device__ __forceinline__ float lgf_at(const float* cube, int dx, int dy, int dz) {
    return cube[((dx + TE) * TW + (dy + TE)) * TW + (dz + TE)];
}

// potential at node x = (xi, xj, xk) of a unit density at gamma- node c:
// single layer G(x - c); double layer |D_c| G(x - c) - sum_{k in D_c}
// G(x - k), or the single-layer column when D_c is empty (eqs.
// [single_potential], [double_potential]); dmask bit d: neighbour d of c
// is a D-node (outside M+ and gamma-)
__device__ __forceinline__ float kval(const float* tab, int xi, int xj, int xk, int ci, int cj, int ck,
                                      unsigned dmask) {
    const int di = xi - ci, dj = xj - cj, dk = xk - ck;
    const float g0 = lgf_at(tab, di, dj, dk);
    if (dmask == 0) return g0;
    float acc = 0.f;
    int nd = 0;
    // neighbours +i, -i, +j, -j, +k, -k of c: x - k = (x - c) - e_d
    if (dmask & 1) { acc -= lgf_at(tab, di - 1, dj, dk); ++nd; }
    if (dmask & 2) { acc -= lgf_at(tab, di + 1, dj, dk); ++nd; }
    if (dmask & 4) { acc -= lgf_at(tab, di, dj - 1, dk); ++nd; }
    if (dmask & 8) { acc -= lgf_at(tab, di, dj + 1, dk); ++nd; }
    if (dmask & 16) { acc -= lgf_at(tab, di, dj, dk - 1); ++nd; }
    if (dmask & 32) { acc -= lgf_at(tab, di, dj, dk + 1); ++nd; }
    return acc + (float)nd * g0;
}

constexpr int RAS_WARPS = 6;    // nodes in flight per CTA, one warp each (static shared memory < 48 KB)
constexpr int NB_W = 2 * NB_R + 1, NB_N = NB_W * NB_W * NB_W;

// the offsets of the neighbourhood by increasing distance (ties in
// lexicographic order), so that a capped block keeps the nearest nodes
struct NbOffsets {
    signed char d[NB_N][3];
};
constexpr NbOffsets make_nb_offsets() {
    NbOffsets o{};
    int n = 0;
    for (int r2 = 0; r2 <= 3 * NB_R * NB_R; ++r2)
        for (int a = -NB_R; a <= NB_R; ++a)
            for (int b = -NB_R; b <= NB_R; ++b)
                for (int c = -NB_R; c <= NB_R; ++c)
                    if (a * a + b * b + c * c == r2) {
                        o.d[n][0] = (signed char)a;
                        o.d[n][1] = (signed char)b;
                        o.d[n][2] = (signed char)c;
                        ++n;
                    }
    return o;
}
__constant__ NbOffsets c_nb = make_nb_offsets();
static_assert(2 * NB_R + 2 < NEAR_TN, "the LGF table must reach the block's offsets");
constexpr int MS = MAXR + 1;    // odd row stride of a block in shared memory

struct RasNode {
    int g[3][MAXR], x[3][MAXR];   // coordinates of member p and of its partner
    float t[MAXR];
    unsigned dmask[MAXR];
    int S[MAXR];
    float M[MAXR * MS];
};

// One warp per gamma- node r. S = the gamma- nodes of the neighbourhood of
// r, nearest first (the lanes probe 32 offsets per round; a ballot keeps the
// order; at most MAXR, r itself first), A_S = A[S, S] from the LGF table
// (lanes over entries), and row r of M^{-1} = the row of r in inv(A_S), from
// Gaussian elimination with partial pivoting of A_S^T z = e_r: lane p owns
// row p of A_S^T, the pivot row of step c is the unused row with the
// largest |entry| in column c, and the back substitution runs over the
// columns with each row's right-hand side in its lane. A numerically
// singular block keeps the identity row.
// Per unknown s: its grid index, its closure partner (grid index; for the
// direct formulation the partner's unknown number, -1 on gamma+), t (float
// bits; 1 on gamma+) and a neighbour mask (bit d set for neighbour d
// outside N+ = M+ and gamma- in the double layer, outside M+ in the direct
// formulation; bit 6: a gamma+ unknown), 16 bytes read once per block member.
__global__ void k_member_info(const int* __restrict__ lin_of, const int* __restrict__ partner,
                              const int* __restrict__ partner_u, const double* __restrict__ t,
                              const uint8_t* __restrict__ flags, long long n, long long n_gm, int N, int layer,
                              int4* __restrict__ info) {
    const int off[6] = {N * N, -N * N, N, -N, 1, -1};
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int g = lin_of[s];
        unsigned dm = 0;
        if (layer == BAE_LAYER_DIRECT) {
            for (int d = 0; d < 6; ++d)
                if (!(flags[g + off[d]] & 1)) dm |= 1u << d;
            if (s < n_gm)
                info[s] = make_int4(g, partner_u[s], __float_as_int((float)t[s]), (int)dm);
            else
                info[s] = make_int4(g, -1, __float_as_int(1.f), (int)(dm | 64u));
            continue;
        }
        if (layer == BAE_LAYER_DOUBLE)
            for (int d = 0; d < 6; ++d)
                if (!(flags[g + off[d]] & 3)) dm |= 1u << d;
        info[s] = make_int4(g, partner[s], __float_as_int((float)t[s]), (int)dm);
    }
}

__global__ void __launch_bounds__(32 * RAS_WARPS) k_ras_rows(const int* __restrict__ lin_of, const int4* __restrict__ minfo,
                                                          const uint8_t* __restrict__ flags,
                                                          const double* __restrict__ tab64, const int* __restrict__ node_of,
                                                          long long n, int N, bool direct, float s6,
                                                          int* __restrict__ col, float* __restrict__ val) {
    __shared__ float tab[TCUBE];
    __shared__ signed char nbo[NB_N][3];
    __shared__ RasNode sh[RAS_WARPS];
    for (int e = threadIdx.x; e < TCUBE; e += blockDim.x)
        tab[e] = lgf_sorted(tab64, e / (TW * TW) - TE, (e / TW) % TW - TE, e % TW - TE);
    for (int e = threadIdx.x; e < NB_N; e += blockDim.x)
        for (int c = 0; c < 3; ++c) nbo[e][c] = c_nb.d[e][c];
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    RasNode& R = sh[w];
    const int NN = N * N;   // N^3 < 2^31
    constexpr int ROUNDS = (NB_N + 31) / 32;
    for (long long r = (long long)blockIdx.x * RAS_WARPS + w; r < n; r += (long long)gridDim.x * RAS_WARPS) {
        const int lin = lin_of[r];
        const int ri = lin / NN, rj = (lin / N) % N, rk = lin % N;
        const int member = direct ? 6 : 2;   // gamma nodes, or gamma- nodes
        // every probe's flags first (independent loads), then the node indices
        int y[ROUNDS], s[ROUNDS];
#pragma unroll
        for (int q = 0; q < ROUNDS; ++q) {
            const int e = q * 32 + lane;
            y[q] = -1;
            if (e < NB_N) {
                const int ii = ri + nbo[e][0], jj = rj + nbo[e][1], kk = rk + nbo[e][2];
                if ((unsigned)ii < (unsigned)N && (unsigned)jj < (unsigned)N && (unsigned)kk < (unsigned)N)
                    y[q] = (ii * N + jj) * N + kk;
            }
        }
#pragma unroll
        for (int q = 0; q < ROUNDS; ++q) s[q] = (y[q] >= 0 && (flags[y[q]] & member)) ? 0 : -1;
#pragma unroll
        for (int q = 0; q < ROUNDS; ++q)
            if (s[q] == 0) s[q] = node_of[y[q]];
        // members in probe order (nearest first), at most MAXR
        int k = 0, mine = -1;
#pragma unroll
        for (int q = 0; q < ROUNDS; ++q) {
            const unsigned ball = __ballot_sync(FULL, s[q] >= 0);
            const int p = k + __popc(ball & ((1u << lane) - 1));
            if (s[q] >= 0 && p < MAXR) R.S[p] = s[q];
            k = min(MAXR, k + __popc(ball));
        }
        __syncwarp();
        if (lane < k) mine = R.S[lane];
        if (mine >= 0) {
            const int4 f = minfo[mine];
            R.g[0][lane] = f.x / NN; R.g[1][lane] = (f.x / N) % N; R.g[2][lane] = f.x % N;
            if (direct) {
                R.x[0][lane] = f.y;   // the partner's unknown number (-1 on gamma+)
            } else {
                R.x[0][lane] = f.y / NN; R.x[1][lane] = (f.y / N) % N; R.x[2][lane] = f.y % N;
            }
            R.t[lane] = __int_as_float(f.z);
            R.dmask[lane] = (unsigned)f.w;
        }
        const int me = 0;   // offset 0 comes first: r itself
        __syncwarp();
        // M = A_S^T: M[q][p] = A_S[p][q] = t_p K(g_p, g_q) + (1 - t_p) K(x_p, g_q);
        // direct formulation: a gamma- row is the closure (t_p at itself,
        // 1 - t_p at its partner), a gamma+ row delta - P with
        // P(p, q) = (6 + s) G(p - q) [q in M-] - sum_{y ~ q, y in M-} G(p - y)
        float scale = 0.f;
        for (int e = lane; e < k * k; e += 32) {
            const int p = e / k, q = e - p * k;
            const int ci = R.g[0][q], cj = R.g[1][q], ck = R.g[2][q];
            const unsigned dm = R.dmask[q];
            const float tp = R.t[p];
            float v;
            if (!direct) {
                v = tp * kval(tab, R.g[0][p], R.g[1][p], R.g[2][p], ci, cj, ck, dm) +
                    (1.f - tp) * kval(tab, R.x[0][p], R.x[1][p], R.x[2][p], ci, cj, ck, dm);
            } else if (!(R.dmask[p] & 64u)) {
                v = (p == q ? tp : 0.f) + (R.S[q] == R.x[0][p] ? 1.f - tp : 0.f);
            } else {
                const int di = R.g[0][p] - ci, dj = R.g[1][p] - cj, dk = R.g[2][p] - ck;
                float pv = (dm & 64u) ? 0.f : s6 * lgf_at(tab, di, dj, dk);
                if (dm & 1) pv -= lgf_at(tab, di - 1, dj, dk);
                if (dm & 2) pv -= lgf_at(tab, di + 1, dj, dk);
                if (dm & 4) pv -= lgf_at(tab, di, dj - 1, dk);
                if (dm & 8) pv -= lgf_at(tab, di, dj + 1, dk);
                if (dm & 16) pv -= lgf_at(tab, di, dj, dk - 1);
                if (dm & 32) pv -= lgf_at(tab, di, dj, dk + 1);
                v = (p == q ? 1.f : 0.f) - pv;
            }
            R.M[q * MS + p] = v;
            scale = fmaxf(scale, fabsf(v));
        }
        for (int o = 16; o > 0; o >>= 1) scale = fmaxf(scale, __shfl_xor_sync(FULL, scale, o));
        __syncwarp();
        float zr = lane == me ? 1.f : 0.f;   // right-hand side of row `lane`
        bool used = lane >= k;
        int mystep = MAXR;                  // elimination step at which row `lane` was the pivot
        bool ok = true;
        for (int c = 0; c < k; ++c) {
            const float mc = lane < k ? R.M[lane * MS + c] : 0.f;
            // pivot: one integer max over the lanes of (|entry| bits with the
            // low 5 mantissa bits replaced by 31 - lane), so equal keys go to
            // the lower row; used rows take key 0
            const unsigned key = used ? 0u : ((__float_as_uint(fabsf(mc)) & ~31u) | (unsigned)(31 - lane));
            const unsigned top = __reduce_max_sync(FULL, key);
            const int bl = 31 - (int)(top & 31u);
            const float best = __uint_as_float(top & ~31u);
            if (top == 0u || !(best > 1e-6f * scale)) { ok = false; break; }   // warp-uniform
            const float pv = __shfl_sync(FULL, mc, bl);
            const float zp = __shfl_sync(FULL, zr, bl);
            if (lane == bl) { used = true; mystep = c; }
            if (!used) {
                const float f = __fdividef(mc, pv);
                if (f != 0.f) {
#pragma unroll 4
                    for (int q = c + 1; q < k; ++q) R.M[lane * MS + q] -= f * R.M[bl * MS + q];
                    zr -= f * zp;
                }
            }
            __syncwarp();
        }
        // back substitution: the pivot row of step c has entries only in
        // columns >= c; x_c from it, then the rows of earlier steps drop column c
        float xr = 0.f;   // x_lane
        if (ok)
            for (int c = k - 1; c >= 0; --c) {
                const int piv = __ffs(__ballot_sync(FULL, mystep == c)) - 1;
                const float xc = __fdividef(__shfl_sync(FULL, zr, piv), R.M[piv * MS + c]);
                if (lane == c) xr = xc;
                if (mystep < c) zr -= R.M[lane * MS + c] * xc;
            }
        else
            xr = lane == me ? 1.f : 0.f;
        // all MAXR slots: unused ones hold (r, 0)
        col[r * MAXR + lane] = lane < k ? R.S[lane] : (int)r;
        val[r * MAXR + lane] = lane < k ? xr : 0.f;
        __syncwarp();
    }
}

// y = M^{-1} x for one batch row per blockIdx.y: one warp per row, lane q
// takes slot q (row-major slots), a float32 product and a float32 shuffle
// tree (a float64 warp instruction holds a GB300 sub-partition's FP64 pipe
// for ~64 cycles; the inner float32 solves that apply M^{-1} round z to
// float32 anyway), the sum stored as float64
// in32 (optional): the same input already rounded to float32 ([nb][n], the
// row the row indices select); out32 (optional): y in float32 as well
__global__ void __launch_bounds__(256) k_precond_apply(const int* __restrict__ col,
                                                       const float* __restrict__ val, long long n, const double* in,
                                                       long long in_stride, const int* row, long long row_stride,
                                                       const float* in32, double* out, long long out_stride,
                                                       float* out32, const int* active) {
    const int b = blockIdx.y;
    if (active && !active[b]) return;
    const double* x = in + b * in_stride + (row ? (long long)row[b] * row_stride : 0);
    const float* x32 = in32 ? in32 + b * n : nullptr;
    double* y = out + b * out_stride;
    float* y32 = out32 ? out32 + b * n : nullptr;
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = w0; r < n; r += nw) {
        const int k = col[r * MAXR + lane];   // unused slots: 0 x[r]
        float v = val[r * MAXR + lane] * (x32 ? x32[k] : (float)x[k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            y[r] = (double)v;
            if (y32) y32[r] = v;
        }
    }
}

}  // namespace

void Precond::release() {
    if (col) dev_free(col, stream);
    if (val) dev_free(val, stream);
    col = nullptr;
    val = nullptr;
    built = false;
}

void build_precond(const Geometry& g, double s, const double* near, Precond& out, cudaStream_t st) {
    const int N = g.N;
    const bool direct = g.layer == BAE_LAYER_DIRECT;
    const long long n = direct ? g.n_unk : g.n_gm;
    // G_s at offsets [0, NEAR_TN)^3, the function the convolution's spectrum comes from
    double* own = nullptr;
    if (!near) {
        own = dev_alloc_n<double>(NEAR_TAB, st);
        lgf_table(NEAR_TN, s, own, st);
        near = own;
    }
    out.release();
    out.stream = g.stream;
    out.n = n;
    out.col = dev_alloc_n<int>(n * MAXR, st);
    out.val = dev_alloc_n<float>(n * MAXR, st);
    // grid index of every unknown: gamma-, then (direct) gamma+
    int* lin_of = g.gm;
    int* lin_own = nullptr;
    if (direct) {
        lin_own = dev_alloc_n<int>(n, st);
        BAE_CUDA(cudaMemcpyAsync(lin_own, g.gm, g.n_gm * sizeof(int), cudaMemcpyDeviceToDevice, st));
        BAE_CUDA(cudaMemcpyAsync(lin_own + g.n_gm, g.gp, g.n_gp * sizeof(int), cudaMemcpyDeviceToDevice, st));
        lin_of = lin_own;
    }
    int4* minfo = dev_alloc_n<int4>(n, st);
    BAE_LAUNCH("k_member_info", st,
               k_member_info<<<(int)std::min<long long>((n + 255) / 256, 152LL * 8), 256, 0, st>>>(
                   lin_of, g.partner, g.partner_u, g.t, g.flags, n, g.n_gm, N, g.layer, minfo));
    const int ctas = (int)std::min<long long>((n + RAS_WARPS - 1) / RAS_WARPS, 152LL * 4);
    BAE_LAUNCH("k_ras_rows", st,
               k_ras_rows<<<ctas, 32 * RAS_WARPS, 0, st>>>(lin_of, minfo, g.flags, near, g.node_of, n, N, direct,
                                                           (float)(6.0 + s), out.col, out.val));
    dev_free(minfo, st);
    if (lin_own) dev_free(lin_own, st);
    if (own) dev_free(own, st);
    out.built = true;
}

void precond_apply(const Precond& p, const double* in, long long in_stride, const int* row, long long row_stride,
                   double* out, long long out_stride, int nb, const int* active, cudaStream_t st, const float* in32,
                   float* out32) {
    BAE_REQUIRE(p.built, BAE_ERR_INVALID_ARG, "internal: preconditioner applied before it was built");
    if (p.n == 0 || nb == 0) return;
    const int ctas = (int)std::min<long long>((p.n + 7) / 8, 152LL * 16);   // 8 rows per 256-thread CTA
    BAE_LAUNCH("k_precond_apply", st,
               k_precond_apply<<<dim3(ctas, nb), 256, 0, st>>>(p.col, p.val, p.n, in, in_stride, row, row_stride,
                                                               in32, out, out_stride, out32, active));
}

}  // namespace bae
