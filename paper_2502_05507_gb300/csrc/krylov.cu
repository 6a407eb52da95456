// Batched GMRES vector kernels with fixed-order reductions (see krylov.cuh).
#include <algorithm>
#include <cstdlib>

#include "krylov.cuh"

namespace bae {

namespace {

constexpr int CH = 512;        // elements per chunk

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// x[b] += sum_{i < ncols[b]} V[b][i] y[b][i], V [nb][mp1][n], y [nb][ystride]
__global__ void k_combine(const double* __restrict__ V, int n, int mp1, const int* __restrict__ ncols,
                          const double* __restrict__ y, int ystride, double* __restrict__ x) {
    const int b = blockIdx.y;
    const int cols = ncols[b];
    if (cols <= 0) return;
    const double* yb = y + (long long)b * ystride;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < cols; ++i) acc += V[((long long)b * mp1 + i) * n + r] * yb[i];
        x[(long long)b * n + r] += acc;
    }
}

__global__ void k_norm2_partial(const double* __restrict__ x, const int* __restrict__ active, int n, double* partial,
                                int nchunk) {
    __shared__ double s_red[8];
    const int b = active[blockIdx.y];
    const int c = blockIdx.x;
    const long long r0 = (long long)c * CH;
    double acc = 0.0;
    for (int e = threadIdx.x; e < CH; e += blockDim.x) {
        const long long r = r0 + e;
        if (r < n) { const double v = x[(long long)b * n + r]; acc += v * v; }
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += s_red[q];
        partial[(long long)b * nchunk + c] = s;
    }
}

__global__ void k_norm2_final(const double* partial, const int* __restrict__ active, int na, int nchunk, double* out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < na; q += gridDim.x * blockDim.x) {
        const int b = active[q];
        double s = 0.0;
        for (int c = 0; c < nchunk; ++c) s += partial[(long long)b * nchunk + c];
        out[b] = s;
    }
}

__global__ void k_sub(const double* a, const double* c, const int* __restrict__ active, int n, double* y) {
    const int b = active[blockIdx.y];
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        y[(long long)b * n + r] = a[(long long)b * n + r] - c[(long long)b * n + r];
}

__global__ void k_add(const double* x, const int* __restrict__ active, int n, double* y) {
    const int b = active[blockIdx.y];
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        y[(long long)b * n + r] += x[(long long)b * n + r];
}

// *flag |= 1 if some x[i] with (flags == null or flags[i % period] & 1) is not finite
__global__ void k_nonfinite(const double* __restrict__ x, long long n, const uint8_t* __restrict__ flags,
                            long long period, int* flag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[i]) && (!flags || (flags[i % period] & 1))) atomicOr(flag, 1);
}

int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 1216); }

}  // namespace

int krylov_chunks(int n) { return ceil_div(n, CH); }

void kr_nonfinite(const double* x, long long n, const uint8_t* flags, long long period, int* d_flag,
                  cudaStream_t st) {
    if (n <= 0) return;
    BAE_LAUNCH("k_nonfinite", st, k_nonfinite<<<blocks_for(n), 256, 0, st>>>(x, n, flags, period, d_flag));
}

void kr_norm2(const double* x, const int* active, int na, int n, double* partial, int nchunk, double* out,
              cudaStream_t st) {
    if (na == 0) return;
    BAE_LAUNCH("k_norm2_partial", st, k_norm2_partial<<<dim3(nchunk, na), 256, 0, st>>>(x, active, n, partial, nchunk));
    BAE_LAUNCH("k_norm2_final", st, k_norm2_final<<<ceil_div(na, 128), 128, 0, st>>>(partial, active, na, nchunk, out));
}

void kr_sub(const double* a, const double* c, const int* active, int na, int n, double* y, cudaStream_t st) {
    if (na == 0) return;
    BAE_LAUNCH("k_sub", st, k_sub<<<dim3(blocks_for(n), na), 256, 0, st>>>(a, c, active, n, y));
}

void kr_add(const double* x, const int* active, int na, int n, double* y, cudaStream_t st) {
    if (na == 0) return;
    BAE_LAUNCH("k_add", st, k_add<<<dim3(blocks_for(n), na), 256, 0, st>>>(x, active, n, y));
}

}  // namespace bae

// ======================================================= device-side GMRES
namespace bae {

namespace {

__device__ __forceinline__ bool last_block(unsigned int* ctr, unsigned int nblocks, int* s_flag) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(ctr, 1u);
        *s_flag = (t == nblocks - 1) ? 1 : 0;
    }
    __syncthreads();
    return *s_flag != 0;
}

__global__ void k_arn_init(Arnoldi a, const double* __restrict__ nrm2, const int* __restrict__ member) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < a.nb; b += gridDim.x * blockDim.x) {
        const double beta = sqrt(nrm2[b]);
        const bool go = member[b] != 0 && beta > a.target[b];
        double* g = a.g + (long long)b * (a.m + 1);
        for (int i = 0; i <= a.m; ++i) g[i] = 0.0;
        g[0] = beta;
        a.est[b] = beta;
        a.flag[b] = go ? 1 : 0;
        a.live[b] = go ? 1 : 0;
        if (a.live_host) {
            a.live_host[b] = go ? 1 : 0;
            __threadfence_system();
        }
        if (a.gflag) a.gflag[b] = 0;
        a.inv[b] = beta > 0.0 ? 1.0 / beta : 0.0;
        a.ncols[b] = 0;
        a.j[b] = 0;
    }
}

__global__ void k_arn_row0(Arnoldi a, const double* __restrict__ r) {
    const int b = blockIdx.y;
    if (!a.flag[b]) return;
    const double s = a.inv[b];
    double* v = a.V + (long long)b * (a.m + 1) * a.n;
    float* v32 = a.v32 ? a.v32 + (long long)b * a.n : nullptr;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x) {
        const double x = r[(long long)b * a.n + i] * s;
        v[i] = x;
        if (v32) v32[i] = (float)x;
    }
}

constexpr int ACH = 64;   // vector elements per CTA in the Arnoldi passes

// sum over chunks of part[i][*] for rows i < cols, one warp per row, each
// lane a fixed stride of chunks, then a fixed shuffle tree
__device__ __forceinline__ void reduce_rows(const double* part, int nch, int cols, double* out, double* out2,
                                            const double* add) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < cols; i += nw) {
        double acc = 0.0;
        for (int c = lane; c < nch; c += 32) acc += __ldcg(part + (long long)i * nch + c);
        acc = warp_sum(acc);
        if (lane == 0) {
            if (add) out[i] = add[i] + acc; else out[i] = acc;
            if (out2) out2[i] = acc;
        }
    }
}

// The chunk [r0, r0 + 64) of the basis rows: element e of row i is
// base[i rs + off(e)], off(e) = min(r0 + e, n - 1) in global memory (indices
// clamped to the vector) or e in a shared-memory copy (row stride ACH + 1,
// so that lanes reading different rows hit different banks). oa, ob: the
// offsets of this lane's two elements (e = lane, lane + 32).
struct RowView {
    const double* base;
    long long rs, oa, ob;
    long long r0, nlast;   // global: r0 and n - 1; shared: nlast < 0
    __device__ __forceinline__ double at(int i, int e) const {
        const long long o = nlast < 0 ? (long long)e : min(r0 + e, nlast);
        return base[(long long)i * rs + o];
    }
};

constexpr int SV_STRIDE = ACH + 1;

__device__ __forceinline__ RowView global_rows(const double* Vb, long long n, long long r0) {
    const int lane = threadIdx.x & 31;
    return {Vb, n, min(r0 + lane, n - 1), min(r0 + lane + 32, n - 1), r0, n - 1};
}

__device__ __forceinline__ RowView shared_rows(const double* sV) {
    const int lane = threadIdx.x & 31;
    return {sV, SV_STRIDE, lane, lane + 32, 0, -1};
}

// The update of step j on the chunk [r0, r0 + ACH): with
// S_c = sum_{i<j} V[i] c[i] and S_b = sum_{i<j} V[i] b[i] (8 warps split the
// rows, warp q taking rows q, q + 8, ..., four rows per loop trip so that
// eight loads are in flight; partial sums added in warp order),
//   q_j = (u_j - S_c) inv,   u_{j+1} = (w - S_b - q_j t) inv,
// u_j read from row j of the view. q_j goes to row j of Vg and u_{j+1} to
// row j + 1 (and its float32 copy to v32). Indices past the end of the
// vector are clamped and their results not stored. s_acc: 2 x 8 x ACH.
__device__ __forceinline__ void chunk_next(const RowView& V, long long n, long long r0, int j, const double* s_c,
                                           const double* s_b, double t, double inv, const double* w, double* Vg,
                                           float* v32, double* s_acc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    int i = warp;
    for (; i + 24 < j; i += 32) {
        const double* v0 = V.base + (long long)i * V.rs;
        const double* v1 = v0 + 8 * V.rs;
        const double* v2 = v0 + 16 * V.rs;
        const double* v3 = v0 + 24 * V.rs;
        const double x0 = v0[V.oa], y0 = v0[V.ob], x1 = v1[V.oa], y1 = v1[V.ob];
        const double x2 = v2[V.oa], y2 = v2[V.ob], x3 = v3[V.oa], y3 = v3[V.ob];
        a0 += x0 * s_c[i] + x1 * s_c[i + 8] + x2 * s_c[i + 16] + x3 * s_c[i + 24];
        a1 += y0 * s_c[i] + y1 * s_c[i + 8] + y2 * s_c[i + 16] + y3 * s_c[i + 24];
        b0 += x0 * s_b[i] + x1 * s_b[i + 8] + x2 * s_b[i + 16] + x3 * s_b[i + 24];
        b1 += y0 * s_b[i] + y1 * s_b[i + 8] + y2 * s_b[i + 16] + y3 * s_b[i + 24];
    }
    for (; i < j; i += 8) {
        const double* v = V.base + (long long)i * V.rs;
        const double x = v[V.oa], y = v[V.ob];
        a0 += x * s_c[i];
        a1 += y * s_c[i];
        b0 += x * s_b[i];
        b1 += y * s_b[i];
    }
    s_acc[warp * ACH + lane] = a0;
    s_acc[warp * ACH + lane + 32] = a1;
    s_acc[(8 + warp) * ACH + lane] = b0;
    s_acc[(8 + warp) * ACH + lane + 32] = b1;
    __syncthreads();
    if (threadIdx.x < ACH) {
        const int e = threadIdx.x;
        const long long r = r0 + e;
        double sc = 0.0, sb = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            sc += s_acc[q * ACH + e];
            sb += s_acc[(8 + q) * ACH + e];
        }
        if (r < n) {
            const double qv = (V.at(j, e) - sc) * inv;
            const double un = (w[r] - sb - qv * t) * inv;
            Vg[(long long)j * n + r] = qv;
            Vg[(long long)(j + 1) * n + r] = un;
            if (v32) v32[r] = (float)un;
        }
    }
    __syncthreads();
}

// partial dots of the chunk against rows i < cols: part[i][c]. Warp q sums
// the elements [8q, 8q + 8) of 32 rows at a time (lane = row, two
// accumulators), then warp 0 adds the eight warp partials of its row in
// warp order: ~2 float64 warp instructions per row instead of a shuffle
// tree per row (each float64 warp instruction occupies GB300's FP64 pipe
// for ~64 cycles). s_red: 8 x 32 doubles of shared memory.
// The same sums when at most 32 / G rows are used (the first Arnoldi steps
// of a cycle): lane = (row r = lane % R, element group g = lane / R), each
// lane sums its row over the 8 / G elements g, g + G, ... of the warp's 8,
// and the G groups meet through the shuffle tree, so a float64 warp
// instruction has (nearly) all lanes busy instead of one per row.
template <int G>
__device__ __forceinline__ void chunk_dots_grouped(const RowView& V, int cols, const double* s_w, double* part,
                                                   int nch, int c, double* s_red) {
    constexpr int R = 32 / G, E = 8 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = lane % R, g = lane / R;
    double acc = 0.0;
    if (r < cols) {
        double p0 = 0.0, p1 = 0.0;
#pragma unroll
        for (int u = 0; u < E; ++u) {
            const int e = 8 * warp + g + G * u;
            if (u & 1) p1 = __fma_rn(V.at(r, e), s_w[e], p1);
            else p0 = __fma_rn(V.at(r, e), s_w[e], p0);
        }
        acc = E > 1 ? p0 + p1 : p0;
    }
#pragma unroll
    for (int o = R; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (g == 0) s_red[warp * 32 + r] = acc;
    __syncthreads();
    if (warp == 0 && lane < cols) {
        double t = s_red[lane];
#pragma unroll
        for (int q = 1; q < 8; ++q) t += s_red[q * 32 + lane];
        part[(long long)lane * nch + c] = t;
    }
    __syncthreads();
}

__device__ __forceinline__ void chunk_dots(const RowView& V, int cols, const double* s_w, double* part, int nch,
                                           int c, double* s_red) {
    if (cols <= 4) return chunk_dots_grouped<8>(V, cols, s_w, part, nch, c, s_red);
    if (cols <= 8) return chunk_dots_grouped<4>(V, cols, s_w, part, nch, c, s_red);
    if (cols <= 16) return chunk_dots_grouped<2>(V, cols, s_w, part, nch, c, s_red);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double wv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) wv[u] = s_w[8 * warp + u];
    for (int i0 = 0; i0 < cols; i0 += 32) {
        const int i = i0 + lane;
        double acc = 0.0;
        if (i < cols) {
            double x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = V.at(i, 8 * warp + u);
            double p0 = x[0] * wv[0], p1 = x[1] * wv[1];
#pragma unroll
            for (int u = 2; u < 8; u += 2) {
                p0 = __fma_rn(x[u], wv[u], p0);
                p1 = __fma_rn(x[u + 1], wv[u + 1], p1);
            }
            acc = p0 + p1;
        }
        s_red[warp * 32 + lane] = acc;
        __syncthreads();
        if (warp == 0 && i < cols) {
            double t = s_red[lane];
#pragma unroll
            for (int q = 1; q < 8; ++q) t += s_red[q * 32 + lane];
            part[(long long)i * nch + c] = t;
        }
        __syncthreads();
    }
}

// Applies the rotations (s_cs[i], s_sn[i]), i < j, to the Hessenberg column
// s_col[0..j+1] (s_col[j+1] = the new subdiagonal), forms the rotation that
// zeroes s_col[j+1] (stored in cs[j], sn[j]) and rotates g[j], g[j+1]. One
// thread; the two-kernel and the fused step share it.
__device__ __forceinline__ void givens_apply(double* s_col, const double* s_cs, const double* s_sn, int j, double* cs,
                                             double* sn, double* g) {
    for (int i = 0; i < j; ++i) {
        const double x0 = s_col[i], x1 = s_col[i + 1];
        s_col[i] = s_cs[i] * x0 + s_sn[i] * x1;
        s_col[i + 1] = -s_sn[i] * x0 + s_cs[i] * x1;
    }
    const double rr = hypot(s_col[j], s_col[j + 1]);
    const double cj = rr > 0.0 ? s_col[j] / rr : 1.0;
    const double sj = rr > 0.0 ? s_col[j + 1] / rr : 0.0;
    cs[j] = cj;
    sn[j] = sj;
    s_col[j] = rr;
    s_col[j + 1] = 0.0;
    g[j + 1] = -sj * g[j];
    g[j] = cj * g[j];
}

// ------------------------------------------------ the step's coefficients
// Rows [0, j] of the two sets of partial sums reduced into cf (Q^T u with
// u.u last, then from cf + m + 1 Q^T w with u.w last, when ran), one warp
// per row in the order of reduce_rows; then r and t by two warps with
// lane-strided sums and the fixed shuffle tree. Every CTA that needs them
// (the rotation CTA, a chunk CTA in the redundant mode, the last block of
// the two-kernel path) runs this same code, so all get the same bits.
__device__ __forceinline__ void step_coeffs(const Arnoldi& a, int b, int j, bool ran, double* cf, double* s_rt) {
    const int m = a.m, nch = a.nchunk;
    const double* part = a.part + (long long)b * 2 * (m + 1) * nch;
    reduce_rows(part, nch, j + 1, cf, nullptr, nullptr);
    if (ran) reduce_rows(part + (long long)(m + 1) * nch, nch, j + 1, cf + m + 1, nullptr, nullptr);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {   // r^2 = u.u - |c|^2 (Pythagoras: u_j is projected once, c = O(eps) |u_j|)
        double acc = 0.0;
        for (int i = lane; i < j; i += 32) acc += cf[i] * cf[i];
        acc = warp_sum(acc);
        if (lane == 0) s_rt[0] = sqrt(fmax(cf[j] - acc, 0.0));
    } else if (warp == 1 && ran) {   // t r = u.w - c.b
        double acc = 0.0;
        for (int i = lane; i < j; i += 32) acc += cf[i] * cf[m + 1 + i];
        acc = warp_sum(acc);
        if (lane == 0) s_rt[1] = cf[m + 1 + j] - acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double r = s_rt[0];
        s_rt[2] = r > 0.0 ? 1.0 / r : 0.0;                   // inv
        s_rt[3] = (ran && r > 0.0) ? s_rt[1] / r : 0.0;      // t
    }
    __syncthreads();
}

// The Hessenberg part of step j for right-hand side b (one CTA; cf and
// s_rt from step_coeffs): column j - 1 (pending) becomes final, hs + c with
// subdiagonal r, and is rotated (residual estimate, decision to go on);
// column j (when ran) is stored pending as h = ([b; t] - H c) / r. Then the
// flags and j advance. s_col: m + 2 doubles, s_cs / s_sn: m each.
__device__ __forceinline__ void step_hessenberg(const Arnoldi& a, int b, int j, bool ran, bool pend, const double* cf,
                                                const double* s_rt, double* s_col, double* s_cs, double* s_sn) {
    const int m = a.m;
    const double r = s_rt[0];
    double* hs = a.hs + (long long)b * (m + 1);
    double* Hu = a.Hu + (long long)b * m * (m + 1);
    if (pend) {   // column j - 1: rows 0 .. j
        for (int i = threadIdx.x; i <= j; i += blockDim.x) {
            const double x = i < j ? hs[i] + cf[i] : r;
            s_col[i] = x;
            Hu[(long long)(j - 1) * (m + 1) + i] = x;
        }
    }
    __syncthreads();   // Hu complete and hs read before hs is overwritten
    if (ran) {         // column j: rows 0 .. j, (H c)_i over the final columns k < j
        const double inv = s_rt[2], t = s_rt[3];
        for (int i = threadIdx.x; i <= j; i += blockDim.x) {
            double hc = 0.0;
            for (int k = (i > 0 ? i - 1 : 0); k < j; ++k) hc += Hu[(long long)k * (m + 1) + i] * cf[k];
            hs[i] = ((i < j ? cf[m + 1 + i] : t) - hc) * inv;
        }
    }
    double* cs = a.cs + (long long)b * m;
    double* sn = a.sn + (long long)b * m;
    if (pend) {
        for (int i = threadIdx.x; i < j - 1; i += blockDim.x) {
            s_cs[i] = cs[i];
            s_sn[i] = sn[i];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool converged = false;
        if (pend) {
            const int c = j - 1;
            givens_apply(s_col, s_cs, s_sn, c, cs, sn, a.g + (long long)b * (m + 1));
            const double e = fabs(a.g[(long long)b * (m + 1) + c + 1]);
            a.est[b] = e;
            a.ncols[b] = c + 1;
            converged = !(e > a.target[b] && r > 0.0);
        }
        const int gf = (ran && !converged) ? 1 : 0;
        const int fl = (gf && j + 1 < m) ? 1 : 0;
        a.gflag[b] = gf;
        a.flag[b] = fl;
        a.live[b] = gf | fl;
        if (a.live_host) {
            a.live_host[b] = gf | fl;
            __threadfence_system();
        }
        a.j[b] = ran ? j + 1 : j;
    }
    __syncthreads();
    if (pend) {
        double* col = a.H + ((long long)b * m + (j - 1)) * (m + 1);
        for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = s_col[i];
    }
}

// the coefficients the chunk update reads: c = cf[0..j), b = cf[m+1 ..
// m+1+j), inv, t
__device__ __forceinline__ void publish_coeffs(const Arnoldi& a, int b, int j, const double* cf, const double* s_rt) {
    const int m = a.m;
    double* out = a.cf + (long long)b * 2 * (m + 1);
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        out[i] = cf[i];
        out[m + 1 + i] = cf[m + 1 + i];
    }
    if (threadIdx.x == 0) {
        a.inv[b] = s_rt[2];
        a.tco[b] = s_rt[3];
    }
}

// w = the closure gather of the potential (eq. [double_bae]) on the chunk
// (into global w and s_w, zero past the end), and s_u = the chunk of u_j
template <typename VT>
__device__ __forceinline__ void gather_chunk(const Arnoldi& a, int b, long long r0, bool ran, const double* uj,
                                             double* s_w, double* s_u) {
    if (threadIdx.x < ACH) {
        const long long r = r0 + threadIdx.x;
        double val = 0.0, uv = 0.0;
        if (r < a.n) {
            uv = uj[r];
            if (ran) {
                const VT* vb = static_cast<const VT*>(a.v) + b * a.v_stride;
                const double tr = a.t[r];
                val = tr * (double)vb[a.gm[r]] + (1.0 - tr) * (double)vb[a.partner[r]];
                a.w[(long long)b * a.n + r] = val;
            }
        }
        s_w[threadIdx.x] = val;
        s_u[threadIdx.x] = uv;
    }
}

// ----------------------------------------------------- two-kernel step
// kernel 1: gather w (when the RHS computes a column), partial sums of
// Q^T u and u.u (and of Q^T w and u.w); the last CTA of each right-hand side
// reduces them and does the Hessenberg part; the update kernel reads the
// published coefficients and the step's j and flag.
template <typename VT>
__global__ void __launch_bounds__(256) k_arn_dots(Arnoldi a) {
    extern __shared__ double s_dyn[];
    const int m = a.m;
    double* s_cf = s_dyn;                     // 2 (m + 1)
    double* s_col = s_cf + 2 * (m + 1);       // m + 2
    double* s_cs = s_col + (m + 2);           // m
    double* s_sn = s_cs + m;                  // m
    __shared__ double s_w[ACH], s_u[ACH];
    __shared__ double s_red8[8 * 32];
    __shared__ double s_rt[4];
    __shared__ int s_last;
    const int b = blockIdx.y;
    const bool ran = a.flag[b] != 0, pend = a.gflag[b] != 0;
    if (!ran && !pend) {   // no update for this right-hand side in this step
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ran[b] = 0;
        return;
    }
    const int j = a.j[b];
    const int c = blockIdx.x;
    const long long r0 = (long long)c * ACH;
    const double* Vb = a.V + (long long)b * (m + 1) * a.n;
    gather_chunk<VT>(a, b, r0, ran, Vb + (long long)j * a.n, s_w, s_u);
    __syncthreads();
    double* part = a.part + (long long)b * 2 * (m + 1) * a.nchunk;
    const RowView V = global_rows(Vb, a.n, r0);
    chunk_dots(V, j + 1, s_u, part, a.nchunk, c, s_red8);
    if (ran) chunk_dots(V, j + 1, s_w, part + (long long)(m + 1) * a.nchunk, a.nchunk, c, s_red8);
    if (last_block(a.ctr + 3 * b + 0, gridDim.x, &s_last)) {
        step_coeffs(a, b, j, ran, s_cf, s_rt);
        if (ran) publish_coeffs(a, b, j, s_cf, s_rt);
        if (threadIdx.x == 0) {
            a.jstep[b] = j;
            a.ran[b] = ran ? 1 : 0;
            a.ctr[3 * b + 0] = 0;
        }
        step_hessenberg(a, b, j, ran, pend, s_cf, s_rt, s_col, s_cs, s_sn);
    }
}

// kernel 2: q_j into row j, u_{j+1} into row j + 1
__global__ void __launch_bounds__(256) k_arn_next(Arnoldi a) {
    extern __shared__ double s_dyn[];
    double* s_c = s_dyn;              // m + 1
    double* s_b = s_dyn + (a.m + 1);  // m + 1
    __shared__ double s_acc[2 * 8 * ACH];
    const int b = blockIdx.y;
    if (!a.ran[b]) return;
    const int j = a.jstep[b];
    const int m = a.m;
    const double* cf = a.cf + (long long)b * 2 * (m + 1);
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        s_c[i] = cf[i];
        s_b[i] = cf[m + 1 + i];
    }
    __syncthreads();
    const long long r0 = (long long)blockIdx.x * ACH;
    double* Vb = a.V + (long long)b * (m + 1) * a.n;
    chunk_next(global_rows(Vb, a.n, r0), a.n, r0, j, s_c, s_b, a.tco[b], a.inv[b], a.w + (long long)b * a.n, Vb,
               a.v32 ? a.v32 + (long long)b * a.n : nullptr, s_acc);
}

// ------------------------------------------------ fused cooperative step
// The two kernels above as one cooperative launch: the chunk CTAs (all
// resident at once) form the partial sums, meet the rotation CTAs (one per
// right-hand side) at a grid barrier, and, once the coefficients are
// known, write q_j and u_{j+1}; the rotation CTAs reduce the coefficients,
// publish them (a second grid barrier the chunk CTAs wait at) and then
// finish and rotate the Hessenberg column while the chunk CTAs update. In
// the redundant mode (one item per chunk CTA) every chunk CTA reduces its
// right-hand side's coefficients itself and the second barrier goes. With
// the preconditioner, z = M^{-1} u_{j+1} follows one more barrier. The
// sums use the same partition and order as the two-kernel step, so both
// give bit-identical results.
constexpr int COOP_MAX_NB = 64;

// All CTAs of the grid wait here until every CTA has arrived. The counter
// only grows (by G per barrier), so the k-th barrier of a CTA completes when
// it reaches the next multiple of G. A wait that runs out (after `limit`
// polls) sets *err, and the mapped host copy *err_host when given, and the
// barrier returns false in every thread of the CTA: the caller then returns
// without touching the step state (the host reports BAE_ERR_TIMEOUT).
__device__ __forceinline__ bool grid_barrier(unsigned long long* ctr, unsigned long long G, int* err,
                                             int* err_host, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long old = atomicAdd(ctr, 1ull);
        const unsigned long long target = (old / G + 1) * G;
        long long spins = 0;
        int ok = 1;
        while (*reinterpret_cast<volatile unsigned long long*>(ctr) < target) {
            if (++spins > limit) {
                atomicOr(err, 1);
                if (err_host) {
                    *reinterpret_cast<volatile int*>(err_host) = 1;
                    __threadfence_system();
                }
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// arrival without waiting (the CTA's writes made visible first)
__device__ __forceinline__ void grid_arrive(unsigned long long* ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1ull);
    }
}

// SV: every CTA holds exactly one (RHS, chunk) item and keeps its chunk of
// the rows V[0..j] in shared memory (copied asynchronously while the
// gather runs), so both passes read it from there; the sums are the same
// expressions in the same order as with global rows.
// Compiled for four resident CTAs per SM (64 registers, a few spilled
// values): more CTAs take more of the (RHS, chunk) items at once, and the
// 64-right-hand-side step is 12% faster than at three CTAs per SM (80
// registers, no spill); left free, the compiler takes ~90 registers and
// only two CTAs fit.
template <typename VT, bool SV>
__global__ void __launch_bounds__(256, 4) k_arn_step_coop(Arnoldi a) {
    // launched with programmatic stream serialisation: the launch is set up
    // while the apply's last kernel runs; nothing is read before that kernel
    // has completed
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    extern __shared__ double s_dyn[];
    const int m = a.m;
    double* s_cf = s_dyn;                     // 2 (m + 1)
    double* s_col = s_cf + 2 * (m + 1);       // m + 2
    double* s_cs = s_col + (m + 2);           // m
    double* s_sn = s_cs + m;                  // m
    double* s_V = s_sn + m;                   // SV: (m + 1) x SV_STRIDE
    __shared__ double s_acc[2 * 8 * ACH];
    __shared__ double s_w[ACH], s_u[ACH];
    __shared__ double s_rt[4];
    __shared__ int s_j[COOP_MAX_NB], s_flag[COOP_MAX_NB], s_pend[COOP_MAX_NB];
    const unsigned long long G = gridDim.x;
    const int NI = (int)gridDim.x - a.nb;   // chunk CTAs; the last nb CTAs reduce and rotate
    const int items = a.nb * a.nchunk;
    // step index and flags as they were at the start of the step (the
    // rotation CTAs advance them)
    for (int b = threadIdx.x; b < a.nb; b += blockDim.x) {
        s_j[b] = a.j[b];
        s_flag[b] = a.flag[b];
        s_pend[b] = a.gflag[b];
    }
    __syncthreads();

    if ((int)blockIdx.x >= NI) {
        // ---- the coefficients and the Hessenberg column of one right-hand side
        const int b = (int)blockIdx.x - NI;
        const int j = s_j[b];
        const bool ran = s_flag[b] != 0, pend = s_pend[b] != 0;
        if (!grid_barrier(a.bar, G + a.bar_extra, a.err, a.err_host, a.spin_limit)) return;   // partial sums complete
        if (ran || pend) {
            step_coeffs(a, b, j, ran, s_cf, s_rt);
            if (ran && !a.coop_redundant) publish_coeffs(a, b, j, s_cf, s_rt);
        }
        if (!a.coop_redundant) grid_arrive(a.bar);   // the chunk CTAs may update
        if (ran || pend) step_hessenberg(a, b, j, ran, pend, s_cf, s_rt, s_col, s_cs, s_sn);
        return;
    }

    if (SV && blockIdx.x < items && (s_flag[blockIdx.x / a.nchunk] || s_pend[blockIdx.x / a.nchunk])) {
        // the chunk of V[0..j] into shared memory, clamped at the vector end
        const int b = blockIdx.x / a.nchunk;
        const long long r0 = (long long)(blockIdx.x % a.nchunk) * ACH;
        const double* Vb = a.V + (long long)b * (m + 1) * a.n;
        const int cnt = (s_j[b] + 1) * ACH;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int i = e / ACH, l = e % ACH;
            const double* src = Vb + (long long)i * a.n + min(r0 + l, (long long)a.n - 1);
            const unsigned dst = (unsigned)__cvta_generic_to_shared(s_V + i * SV_STRIDE + l);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    // phase 1: w = gather of v, partial sums against V[0..j] of u_j and w
    for (int item = blockIdx.x; item < items; item += NI) {
        const int b = item / a.nchunk, c = item % a.nchunk;
        const bool ran = s_flag[b] != 0;
        if (!ran && !s_pend[b]) continue;
        const int j = s_j[b];
        const long long r0 = (long long)c * ACH;
        const double* Vb = a.V + (long long)b * (m + 1) * a.n;
        gather_chunk<VT>(a, b, r0, ran, Vb + (long long)j * a.n, s_w, s_u);
        if (SV) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        const RowView V = SV ? shared_rows(s_V) : global_rows(Vb, a.n, r0);
        double* part = a.part + (long long)b * 2 * (m + 1) * a.nchunk;
        chunk_dots(V, j + 1, s_u, part, a.nchunk, c, s_acc);
        if (ran) chunk_dots(V, j + 1, s_w, part + (long long)(m + 1) * a.nchunk, a.nchunk, c, s_acc);
        __syncthreads();
    }
    if (!grid_barrier(a.bar, G + a.bar_extra, a.err, a.err_host, a.spin_limit)) return;   // all G CTAs
    if (!a.coop_redundant && !grid_barrier(a.bar, G + a.bar_extra, a.err, a.err_host, a.spin_limit))
        return;   // the rotation CTAs have published the coefficients
    // phase 2: q_j into row j, u_{j+1} into row j + 1
    for (int item = blockIdx.x; item < items; item += NI) {
        const int b = item / a.nchunk, c = item % a.nchunk;
        if (!s_flag[b]) continue;
        const int j = s_j[b];
        double* s_c = s_cf;
        double* s_b = s_cf + m + 1;
        double t, inv;
        if (a.coop_redundant) {   // the same reduction as the rotation CTA
            step_coeffs(a, b, j, true, s_cf, s_rt);
            t = s_rt[3];
            inv = s_rt[2];
        } else {
            const double* cf = a.cf + (long long)b * 2 * (m + 1);
            for (int i = threadIdx.x; i < j; i += blockDim.x) {
                s_c[i] = __ldcg(cf + i);
                s_b[i] = __ldcg(cf + m + 1 + i);
            }
            t = __ldcg(a.tco + b);
            inv = __ldcg(a.inv + b);
            __syncthreads();
        }
        double* Vb = a.V + (long long)b * (m + 1) * a.n;
        const long long r0 = (long long)c * ACH;
        const RowView V = SV ? shared_rows(s_V) : global_rows(Vb, a.n, r0);
        chunk_next(V, a.n, r0, j, s_c, s_b, t, inv, a.w + (long long)b * a.n, Vb,
                   a.v32 ? a.v32 + (long long)b * a.n : nullptr, s_acc);
    }
    if (!a.pre_col) return;
    // phase 3: z = M^{-1} u_{j+1} on the chunk's rows: warp w takes rows
    // 8 w .. 8 w + 7 of each item, lane q slot q, the same float32 products
    // and shuffle tree as the separate preconditioner kernel. The slots of the
    // CTA's first item are loaded before the barrier (they do not depend on
    // u_{j+1}); u_{j+1} is read through L2 (other CTAs wrote it).
    constexpr int RW = ACH / 8;   // rows per warp (8 warps)
    static_assert(ACH % 8 == 0, "rows per warp");
    const int lane = threadIdx.x & 31, wr = (threadIdx.x >> 5) * RW;
    int pc[RW];
    float pv[RW];
    auto load_slots = [&](int item) {
        const long long r0 = (long long)(item % a.nchunk) * ACH + wr;
#pragma unroll
        for (int u = 0; u < RW; ++u) {
            const long long r = r0 + u;
            pc[u] = r < a.n ? __ldg(a.pre_col + r * 32 + lane) : 0;
            pv[u] = r < a.n ? __ldg(a.pre_val + r * 32 + lane) : 0.f;
        }
    };
    if ((int)blockIdx.x < items) load_slots(blockIdx.x);
    if (!grid_barrier(a.bar2, (unsigned long long)NI + a.bar_extra, a.err, a.err_host, a.spin_limit))
        return;   // u_{j+1} complete
    for (int item = blockIdx.x; item < items; item += NI) {
        const int b = item / a.nchunk, c = item % a.nchunk;
        if (item != (int)blockIdx.x) load_slots(item);
        if (!s_flag[b]) continue;
        // u_{j+1} in float32 (v32, written in phase 2 with the same rounding
        // the conversion here would make)
        const float* x = a.v32 + (long long)b * a.n;
        double* z = a.zpre + (long long)b * a.n;
        float* z32 = a.z32 ? a.z32 + (long long)b * a.n : nullptr;
        const long long r0 = (long long)c * ACH + wr;
        float xv[RW];
#pragma unroll
        for (int u = 0; u < RW; ++u) xv[u] = r0 + u < a.n ? __ldcg(x + pc[u]) : 0.f;
#pragma unroll
        for (int u = 0; u < RW; ++u) {
            float v = pv[u] * xv[u];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && r0 + u < a.n) {
                z[r0 + u] = (double)v;
                if (z32) z32[r0 + u] = v;
            }
        }
    }
}

// y = R^{-1} g, one warp per RHS (column-oriented back substitution)
__global__ void k_arn_backsub(Arnoldi a) {
    extern __shared__ double s_rhs[];
    const int b = blockIdx.x;
    const int c = a.ncols[b];
    const int m = a.m;
    double* y = a.y + (long long)b * m;
    const double* g = a.g + (long long)b * (m + 1);
    const double* H = a.H + (long long)b * m * (m + 1);
    for (int l = threadIdx.x; l < m; l += blockDim.x) {
        s_rhs[l] = l < c ? g[l] : 0.0;
        y[l] = 0.0;
    }
    __syncwarp();
    for (int i = c - 1; i >= 0; --i) {
        const double d = H[(long long)i * (m + 1) + i];
        const double yi = d != 0.0 ? s_rhs[i] / d : 0.0;
        __syncwarp();
        for (int l = threadIdx.x; l < i; l += blockDim.x) s_rhs[l] -= H[(long long)i * (m + 1) + l] * yi;
        if (threadIdx.x == 0) y[i] = yi;
        __syncwarp();
    }
}

}  // namespace

void arn_init(const Arnoldi& a, const double* r, const double* nrm2, const int* member, cudaStream_t st) {
    BAE_LAUNCH("k_arn_init", st, k_arn_init<<<ceil_div(a.nb, 128), 128, 0, st>>>(a, nrm2, member));
    BAE_LAUNCH("k_arn_row0", st, k_arn_row0<<<dim3(blocks_for(a.n), a.nb), 256, 0, st>>>(a, r));
}

int arnoldi_chunks(int n) { return ceil_div(n, ACH); }

// dynamic shared memory of the step kernels: cf, the column, cs and sn
static size_t step_smem(int m) { return (size_t)(5 * m + 4) * sizeof(double); }

void arn_configure(int m) {
    const int sh = (int)step_smem(m);
    BAE_CUDA(cudaFuncSetAttribute(k_arn_dots<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh));
    BAE_CUDA(cudaFuncSetAttribute(k_arn_dots<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh));
    BAE_CUDA(cudaFuncSetAttribute(k_arn_step_coop<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh));
    BAE_CUDA(cudaFuncSetAttribute(k_arn_step_coop<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh));
}

int arn_coop_grid(int n, int nb, int m, bool* resident, bool* redundant) {
    static const bool off = []() {
        const char* e = getenv("BAE_ARNOLDI_COOP");
        return e && e[0] == '0';
    }();
    *resident = false;
    *redundant = false;
    if (off || nb > COOP_MAX_NB || n <= 0) return 0;
    int dev = 0, coop = 0, sms = 0;
    BAE_CUDA(cudaGetDevice(&dev));
    BAE_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    BAE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (!coop) return 0;
    arn_configure(m);
    const size_t sh = step_smem(m);
    const long long items = (long long)nb * ceil_div(n, ACH);
    // resident basis chunks: one item per CTA, all CTAs on the device at once
    const size_t sh_sv = sh + (size_t)(m + 1) * SV_STRIDE * sizeof(double);
    if (sh_sv <= 200 * 1024) {
        BAE_CUDA(cudaFuncSetAttribute(k_arn_step_coop<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sh_sv));
        BAE_CUDA(cudaFuncSetAttribute(k_arn_step_coop<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sh_sv));
        int s32 = 0, s64 = 0;
        BAE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s32, k_arn_step_coop<float, true>, 256, sh_sv));
        BAE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s64, k_arn_step_coop<double, true>, 256, sh_sv));
        if (items + nb <= (long long)std::min(s32, s64) * sms) {   // one CTA per chunk plus one rotation CTA per right-hand side
            *resident = true;
            *redundant = true;
            return (int)(items + nb);
        }
    }
    int k32 = 0, k64 = 0;
    BAE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k32, k_arn_step_coop<float, false>, 256, sh));
    BAE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k64, k_arn_step_coop<double, false>, 256, sh));
    const long long cap = (long long)std::min(k32, k64) * sms;
    // persistent chunk CTAs plus one rotation CTA per right-hand side
    if (cap <= nb) return 0;
    const long long grid = std::min(cap, items + nb);
    *redundant = items <= grid - nb;   // one item per chunk CTA
    return (int)grid;
}

void arn_step(const Arnoldi& a, cudaStream_t st) {
    BAE_REQUIRE(a.v && a.gm && a.partner && a.t, BAE_ERR_INVALID_ARG, "arn_step: gather inputs not set");
    BAE_REQUIRE(a.cf && a.hs && a.Hu && a.tco && a.gflag && a.live, BAE_ERR_INVALID_ARG,
                "arn_step: step state not set");
    const size_t sh = step_smem(a.m);
    if (a.coop_grid > 0) {
        BAE_REQUIRE(a.bar && a.bar2 && a.err && a.nb <= COOP_MAX_NB && a.coop_grid > a.nb &&
                        (!a.coop_redundant || (long long)a.nb * a.nchunk <= a.coop_grid - a.nb),
                    BAE_ERR_INVALID_ARG, "arn_step: cooperative step state not set");
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(a.coop_grid);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = sh + (a.coop_resident ? (size_t)(a.m + 1) * SV_STRIDE * sizeof(double) : 0);
        cfg.stream = st;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        if (a.coop_resident) {
            BAE_REQUIRE(a.coop_grid == a.nb * a.nchunk + a.nb, BAE_ERR_INVALID_ARG,
                        "arn_step: resident step needs one CTA per chunk and per right-hand side");
            if (a.v_f32)
                BAE_LAUNCH("k_arn_step_coop.f32", st, BAE_CUDA(cudaLaunchKernelEx(&cfg, k_arn_step_coop<float, true>, a)));
            else
                BAE_LAUNCH("k_arn_step_coop.f64", st, BAE_CUDA(cudaLaunchKernelEx(&cfg, k_arn_step_coop<double, true>, a)));
        } else if (a.v_f32) {
            BAE_LAUNCH("k_arn_step_coop.f32", st, BAE_CUDA(cudaLaunchKernelEx(&cfg, k_arn_step_coop<float, false>, a)));
        } else {
            BAE_LAUNCH("k_arn_step_coop.f64", st, BAE_CUDA(cudaLaunchKernelEx(&cfg, k_arn_step_coop<double, false>, a)));
        }
        return;
    }
    BAE_REQUIRE(a.jstep && a.ran, BAE_ERR_INVALID_ARG, "arn_step: step state not set");
    const dim3 grid(a.nchunk, a.nb);
    if (a.v_f32)
        BAE_LAUNCH("k_arn_dots.f32", st, k_arn_dots<float><<<grid, 256, sh, st>>>(a));
    else
        BAE_LAUNCH("k_arn_dots.f64", st, k_arn_dots<double><<<grid, 256, sh, st>>>(a));
    BAE_LAUNCH("k_arn_next", st, k_arn_next<<<grid, 256, (size_t)2 * (a.m + 1) * sizeof(double), st>>>(a));
}

void arn_finish(const Arnoldi& a, double* x, cudaStream_t st) {
    BAE_LAUNCH("k_arn_backsub", st, k_arn_backsub<<<a.nb, 32, a.m * sizeof(double), st>>>(a));
    BAE_LAUNCH("k_combine", st, k_combine<<<dim3(blocks_for(a.n), a.nb), 256, 0, st>>>(a.V, a.n, a.m + 1, a.ncols, a.y, a.m, x));
}

}  // namespace bae
