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

// w[r0 .. r0+ACH) -= V[0..cols) h over the chunk; 8 warps split the rows
// (warp q takes rows q, q+8, ...; four rows per loop trip so that eight
// loads are in flight), partial sums combined in warp order. Indices past
// the end of the vector are clamped (their results are never stored).
// Leaves the new chunk in s_w (zero past the end) and stores it into w, or,
// when dst is set, stores scale times it into dst instead.
__device__ __forceinline__ void chunk_update(const RowView& V, long long n, long long r0, int cols, const double* s_h,
                                             double* w, double* s_acc, double* s_w, double* dst = nullptr,
                                             double scale = 1.0, float* dst32 = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double a0 = 0.0, a1 = 0.0;
    int i = warp;
    for (; i + 24 < cols; i += 32) {
        const double* v0 = V.base + (long long)i * V.rs;
        const double* v1 = v0 + 8 * V.rs;
        const double* v2 = v0 + 16 * V.rs;
        const double* v3 = v0 + 24 * V.rs;
        const double x0 = v0[V.oa], y0 = v0[V.ob], x1 = v1[V.oa], y1 = v1[V.ob];
        const double x2 = v2[V.oa], y2 = v2[V.ob], x3 = v3[V.oa], y3 = v3[V.ob];
        a0 += x0 * s_h[i] + x1 * s_h[i + 8] + x2 * s_h[i + 16] + x3 * s_h[i + 24];
        a1 += y0 * s_h[i] + y1 * s_h[i + 8] + y2 * s_h[i + 16] + y3 * s_h[i + 24];
    }
    for (; i < cols; i += 8) {
        const double* v = V.base + (long long)i * V.rs;
        a0 += v[V.oa] * s_h[i];
        a1 += v[V.ob] * s_h[i];
    }
    s_acc[warp * ACH + lane] = a0;
    s_acc[warp * ACH + lane + 32] = a1;
    __syncthreads();
    if (threadIdx.x < ACH) {
        const long long r = r0 + threadIdx.x;
        double sub = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) sub += s_acc[q * ACH + threadIdx.x];
        double val = 0.0;
        if (r < n) {
            val = w[r] - sub;
            if (dst) {
                const double y = val * scale;
                dst[r] = y;
                if (dst32) dst32[r] = (float)y;
            } else {
                w[r] = val;
            }
        }
        s_w[threadIdx.x] = val;
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
// thread; the three-kernel and the fused step share it.
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

// pass 1: w = A V[j] by the closure gather of the potential v (the same
// expression as closure_gather), then h1 = V^T w over rows i <= j
template <typename VT>
__global__ void __launch_bounds__(256) k_arn_gather_dots(Arnoldi a) {
    __shared__ double s_w[ACH];
    __shared__ double s_red8[8 * 32];
    __shared__ int s_last;
    const int b = blockIdx.y;
    if (!a.flag[b]) return;
    const int cols = a.j[b] + 1;
    const int c = blockIdx.x;
    const long long r0 = (long long)c * ACH;
    double* w = a.w + (long long)b * a.n;
    if (threadIdx.x < ACH) {
        const long long r = r0 + threadIdx.x;
        double val = 0.0;
        if (r < a.n) {
            const VT* vb = static_cast<const VT*>(a.v) + b * a.v_stride;
            const double tr = a.t[r];
            val = tr * (double)vb[a.gm[r]] + (1.0 - tr) * (double)vb[a.partner[r]];
            w[r] = val;
        }
        s_w[threadIdx.x] = val;
    }
    __syncthreads();
    double* part = a.part + (long long)b * (a.m + 2) * a.nchunk;
    const double* Vb = a.V + (long long)b * (a.m + 1) * a.n;
    chunk_dots(global_rows(Vb, a.n, r0), cols, s_w, part, a.nchunk, c, s_red8);
    if (last_block(a.ctr + 3 * b + 0, gridDim.x, &s_last)) {
        reduce_rows(part, a.nchunk, cols, a.h1 + (long long)b * (a.m + 1), nullptr, nullptr);
        if (threadIdx.x == 0) a.ctr[3 * b + 0] = 0;
    }
}

// pass 2: w -= V h1, then h2 = V^T w and ||w||^2. The last block forms
// hcol = h1 + h2 and the new subdiagonal entry ||w - V h2|| by the
// Pythagorean identity ||w||^2 - ||h2||^2 (V orthonormal), applies the
// Givens rotations (staged in shared memory), updates the residual
// estimate and the flag, sets inv = 1 / ||w - V h2|| and advances j.
__global__ void __launch_bounds__(256) k_arn_update_dots(Arnoldi a) {
    extern __shared__ double s_dyn[];
    const int m = a.m;
    double* s_h = s_dyn;                 // m + 1: h1
    double* s_col = s_dyn + (m + 1);     // m + 2: the new Hessenberg column
    double* s_cs = s_col + (m + 2);      // m
    double* s_sn = s_cs + m;             // m
    __shared__ double s_acc[8 * ACH];
    __shared__ double s_w[ACH];
    __shared__ double s_n2;
    __shared__ int s_last;
    const int b = blockIdx.y;
    if (!a.flag[b]) return;
    const int j = a.j[b];
    const int cols = j + 1;
    const int c = blockIdx.x;
    const long long r0 = (long long)c * ACH;
    double* h1 = a.h1 + (long long)b * (m + 1);
    for (int i = threadIdx.x; i < cols; i += blockDim.x) s_h[i] = h1[i];
    __syncthreads();
    const double* Vb = a.V + (long long)b * (m + 1) * a.n;
    chunk_update(global_rows(Vb, a.n, r0), a.n, r0, cols, s_h, a.w + (long long)b * a.n, s_acc, s_w);
    double* part = a.part + (long long)b * (m + 2) * a.nchunk;
    chunk_dots(global_rows(Vb, a.n, r0), cols, s_w, part, a.nchunk, c, s_acc);
    if (threadIdx.x >= 224) {   // the last warp: ||w||^2 over the chunk
        const int l = threadIdx.x - 224;
        double acc = s_w[l] * s_w[l] + s_w[l + 32] * s_w[l + 32];
        acc = warp_sum(acc);
        if (l == 0) part[(long long)(m + 1) * a.nchunk + c] = acc;
    }
    if (last_block(a.ctr + 3 * b + 1, gridDim.x, &s_last)) {
        double* hc = a.hcol + (long long)b * (m + 1);
        // hcol = h1 + h2 (h1 still in s_h), then h1 <- h2
        reduce_rows(part, a.nchunk, cols, hc, h1, s_h);
        if (threadIdx.x < 32) {
            double acc = 0.0;
            for (int q = threadIdx.x; q < a.nchunk; q += 32) acc += __ldcg(part + (long long)(m + 1) * a.nchunk + q);
            acc = warp_sum(acc);
            if (threadIdx.x == 0) s_n2 = acc;
        }
        __syncthreads();
        double* cs = a.cs + (long long)b * m;
        double* sn = a.sn + (long long)b * m;
        for (int i = threadIdx.x; i <= j; i += blockDim.x) s_col[i] = __ldcg(hc + i);
        for (int i = threadIdx.x; i < j; i += blockDim.x) {
            s_cs[i] = cs[i];
            s_sn[i] = sn[i];
        }
        if (threadIdx.x < 32) {   // ||h2||^2 in a fixed order
            double acc = 0.0;
            for (int i = threadIdx.x; i <= j; i += 32) {
                const double x = __ldcg(h1 + i);
                acc += x * x;
            }
            acc = warp_sum(acc);
            if (threadIdx.x == 0) s_n2 = fmax(s_n2 - acc, 0.0);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double hn = sqrt(s_n2);
            double* g = a.g + (long long)b * (m + 1);
            s_col[j + 1] = hn;
            givens_apply(s_col, s_cs, s_sn, j, cs, sn, g);
            const double e = fabs(g[j + 1]);
            a.est[b] = e;
            a.ncols[b] = j + 1;
            a.inv[b] = hn > 0.0 ? 1.0 / hn : 0.0;
            a.flag[b] = (e > a.target[b] && hn > 0.0 && j + 1 < m) ? 1 : 0;
            a.live[b] = a.flag[b];
            if (a.live_host) {
                a.live_host[b] = a.flag[b];
                __threadfence_system();
            }
            a.j[b] = j + 1;   // every block of this RHS has read j already
            a.ctr[3 * b + 1] = 0;
        }
        __syncthreads();
        double* col = a.H + ((long long)b * m + j) * (m + 1);
        for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) col[i] = s_col[i];
    }
}

// pass 3: V[j] = (w - V h2) / ||w - V h2|| with j already advanced (w itself
// is not written back: the next step's gather replaces it)
__global__ void __launch_bounds__(256) k_arn_update_next(Arnoldi a) {
    extern __shared__ double s_dyn[];
    double* s_h = s_dyn;
    __shared__ double s_acc[8 * ACH];
    __shared__ double s_w[ACH];
    const int b = blockIdx.y;
    if (!a.flag[b]) return;
    const int j = a.j[b];
    const int cols = j;   // rows 0 .. j-1: the basis before this step's vector
    const int c = blockIdx.x;
    const long long r0 = (long long)c * ACH;
    const double* h2 = a.h1 + (long long)b * (a.m + 1);
    for (int i = threadIdx.x; i < cols; i += blockDim.x) s_h[i] = h2[i];
    __syncthreads();
    double* Vb = a.V + (long long)b * (a.m + 1) * a.n;
    chunk_update(global_rows(Vb, a.n, r0), a.n, r0, cols, s_h, a.w + (long long)b * a.n, s_acc, s_w,
                 Vb + (long long)j * a.n, a.inv[b], a.v32 ? a.v32 + (long long)b * a.n : nullptr);
}

// ------------------------------------------------ fused cooperative step
// The three passes above and their last-CTA reductions as one cooperative
// launch: the CTAs (all resident at once) meet at four grid barriers, and
// the reductions are spread over all warps instead of one CTA. The sums use
// the same partition and order as the three-kernel step, so both give
// bit-identical results.
constexpr int COOP_MAX_NB = 64;
constexpr long long BAR_SPIN_LIMIT = 1LL << 22;   // about half a second of waiting

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

// out[b][i] = sum over chunks of part[b][i][*] for rows i <= j_b of the
// iterating right-hand sides, one warp per row, in the order of reduce_rows;
// with add, also out2 = out and out = add + out. Row m + 1 (the squared
// norm partials) goes to n2[b] when n2 is set.
__device__ __forceinline__ void coop_reduce(const Arnoldi& a, int nctas, const int* s_j, const int* s_flag,
                                            double* out, double* out2, const double* add, double* n2) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = nctas * (blockDim.x >> 5);
    const int rows = a.m + 2;
    for (int item = gw; item < a.nb * rows; item += nw) {
        const int b = item / rows, i = item % rows;
        if (!s_flag[b]) continue;
        const bool norm = i == a.m + 1;
        if (norm ? !n2 : i > s_j[b]) continue;
        const double* p = a.part + ((long long)b * (a.m + 2) + i) * a.nchunk;
        double acc = 0.0;
        for (int c = lane; c < a.nchunk; c += 32) acc += __ldcg(p + c);
        acc = warp_sum(acc);
        if (lane == 0) {
            if (norm) {
                n2[b] = acc;
            } else {
                const long long o = (long long)b * (a.m + 1) + i;
                if (add) out[o] = __ldcg(add + o) + acc; else out[o] = acc;
                if (out2) out2[o] = acc;
            }
        }
    }
}

// SV: every CTA holds exactly one (RHS, chunk) item and keeps its chunk of
// the basis rows V[0..j] in shared memory (copied asynchronously while the
// gather runs), so the three projections read it from there; the sums are
// the same expressions in the same order as with global rows.
// Compiled for three resident CTAs per SM (at most 85 registers; it needs
// 80 without spilling): left free, the compiler takes 91 and only two CTAs
// fit, which made the 64-right-hand-side step ~40% slower.
template <typename VT, bool SV>
__global__ void __launch_bounds__(256, 3) k_arn_step_coop(Arnoldi a) {
    extern __shared__ double s_dyn[];
    const int m = a.m;
    double* s_h = s_dyn;                 // m + 1
    double* s_col = s_dyn + (m + 1);     // m + 2
    double* s_cs = s_col + (m + 2);      // m
    double* s_sn = s_cs + m;             // m
    double* s_V = s_sn + m;              // SV: (m + 1) x SV_STRIDE
    __shared__ double s_acc[8 * ACH];
    __shared__ double s_w[ACH];
    __shared__ double s_red[2];
    __shared__ int s_j[COOP_MAX_NB], s_flag[COOP_MAX_NB];
    const unsigned long long G = gridDim.x;
    const int NI = (int)gridDim.x - a.nb;   // chunk CTAs; the last nb CTAs do the rotations
    const int items = a.nb * a.nchunk;
    // step index and flags as they were at the start of the step (the
    // rotation CTAs advance them at the end)
    for (int b = threadIdx.x; b < a.nb; b += blockDim.x) {
        s_j[b] = a.j[b];
        s_flag[b] = a.flag[b];
    }
    __syncthreads();

    if ((int)blockIdx.x >= NI) {
        // ---- rotations of the column stored by the previous step
        const int b = (int)blockIdx.x - NI;
        const int j = s_j[b];
        const bool pending = a.gflag[b] != 0;   // column j - 1 waits in pcol[b][(j - 1) % 2]
        const int c = j - 1;
        double* cs = a.cs + (long long)b * m;
        double* sn = a.sn + (long long)b * m;
        if (pending) {
            const double* pc = a.pcol + ((long long)b * 2 + (c & 1)) * (m + 2);
            for (int i = threadIdx.x; i <= c + 1; i += blockDim.x) s_col[i] = pc[i];
            for (int i = threadIdx.x; i < c; i += blockDim.x) {
                s_cs[i] = cs[i];
                s_sn[i] = sn[i];
            }
        }
        // every chunk CTA has read j and the flags once all CTAs are here
        if (!grid_barrier(a.bar, G + a.bar_extra, a.err, a.err_host, a.spin_limit)) return;
        if (threadIdx.x == 0) {
            bool converged = false;
            if (pending) {
                const double hn = s_col[c + 1];
                givens_apply(s_col, s_cs, s_sn, c, cs, sn, a.g + (long long)b * (m + 1));
                const double e = fabs(a.g[(long long)b * (m + 1) + c + 1]);
                a.est[b] = e;
                a.ncols[b] = c + 1;
                converged = !(e > a.target[b] && hn > 0.0);
            }
            const bool ran = s_flag[b] != 0;   // the chunk CTAs computed column j in this step
            const int gf = (ran && !converged) ? 1 : 0;
            const int fl = (ran && !converged && j + 1 < m) ? 1 : 0;
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
        if (pending) {
            double* col = a.H + ((long long)b * m + c) * (m + 1);
            for (int i = threadIdx.x; i <= c + 1; i += blockDim.x) col[i] = s_col[i];
        }
        return;   // takes part in the first barrier only
    }

    if (SV && blockIdx.x < items && s_flag[blockIdx.x / a.nchunk]) {
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
    // phase 1: w = gather of v, partial dots against V[0..j]
    for (int item = blockIdx.x; item < items; item += NI) {
        const int b = item / a.nchunk, c = item % a.nchunk;
        if (!s_flag[b]) continue;
        const long long r0 = (long long)c * ACH;
        double* w = a.w + (long long)b * a.n;
        if (threadIdx.x < ACH) {
            const long long r = r0 + threadIdx.x;
            double val = 0.0;
            if (r < a.n) {
                const VT* vb = static_cast<const VT*>(a.v) + b * a.v_stride;
                const double tr = a.t[r];
                val = tr * (double)vb[a.gm[r]] + (1.0 - tr) * (double)vb[a.partner[r]];
                w[r] = val;
            }
            s_w[threadIdx.x] = val;
        }
        if (SV) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        const RowView V = SV ? shared_rows(s_V) : global_rows(a.V + (long long)b * (m + 1) * a.n, a.n, r0);
        chunk_dots(V, s_j[b] + 1, s_w, a.part + (long long)b * (m + 2) * a.nchunk, a.nchunk, c, s_acc);
        __syncthreads();
    }
    if (!grid_barrier(a.bar, G + a.bar_extra, a.err, a.err_host, a.spin_limit)) return;   // all G CTAs
    const unsigned long long GI = (unsigned long long)NI;
    // phase 2: h1
    coop_reduce(a, NI, s_j, s_flag, a.h1, nullptr, nullptr, nullptr);
    if (!grid_barrier(a.bar2, GI + a.bar_extra, a.err, a.err_host, a.spin_limit)) return;   // chunk CTAs only
    // phase 3: w -= V h1, partial dots for h2 and ||w||^2
    for (int item = blockIdx.x; item < items; item += NI) {
        const int b = item / a.nchunk, c = item % a.nchunk;
        if (!s_flag[b]) continue;
        const int cols = s_j[b] + 1;
        const long long r0 = (long long)c * ACH;
        const double* h1 = a.h1 + (long long)b * (m + 1);
        for (int i = threadIdx.x; i < cols; i += blockDim.x) s_h[i] = __ldcg(h1 + i);
        __syncthreads();
        const double* Vb = a.V + (long long)b * (m + 1) * a.n;
        double* part = a.part + (long long)b * (m + 2) * a.nchunk;
        const RowView V = SV ? shared_rows(s_V) : global_rows(Vb, a.n, r0);
        chunk_update(V, a.n, r0, cols, s_h, a.w + (long long)b * a.n, s_acc, s_w);
        chunk_dots(V, cols, s_w, part, a.nchunk, c, s_acc);
        if (threadIdx.x >= 224) {
            const int l = threadIdx.x - 224;
            double acc = s_w[l] * s_w[l] + s_w[l + 32] * s_w[l + 32];
            acc = warp_sum(acc);
            if (l == 0) part[(long long)(m + 1) * a.nchunk + c] = acc;
        }
        __syncthreads();
    }
    if (!grid_barrier(a.bar2, GI + a.bar_extra, a.err, a.err_host, a.spin_limit)) return;
    // phase 4: h2 (into h1), hcol = h1 + h2, ||w||^2
    coop_reduce(a, NI, s_j, s_flag, a.hcol, a.h1, a.h1, a.n2);
    if (!grid_barrier(a.bar2, GI + a.bar_extra, a.err, a.err_host, a.spin_limit)) return;

    // phase 5: hn = sqrt(||w||^2 - ||h2||^2) (every CTA, same order), then
    // V[j+1] = (w - V h2) / hn; the CTA of chunk 0 stores the column
    // (hcol, then hn) for the rotations of the next step
    for (int item = blockIdx.x; item < items; item += NI) {
        const int b = item / a.nchunk, c = item % a.nchunk;
        if (!s_flag[b]) continue;
        const int j = s_j[b], cols = j + 1;
        const double* h2 = a.h1 + (long long)b * (m + 1);
        for (int i = threadIdx.x; i < cols; i += blockDim.x) s_h[i] = __ldcg(h2 + i);
        if (threadIdx.x < 32) {
            double acc = 0.0;
            for (int i = threadIdx.x; i <= j; i += 32) {
                const double x = __ldcg(h2 + i);
                acc += x * x;
            }
            acc = warp_sum(acc);
            if (threadIdx.x == 0) {
                const double hn = sqrt(fmax(__ldcg(a.n2 + b) - acc, 0.0));
                s_red[0] = hn;
                s_red[1] = hn > 0.0 ? 1.0 / hn : 0.0;
            }
        }
        __syncthreads();
        if (c == 0) {
            double* pc = a.pcol + ((long long)b * 2 + (j & 1)) * (m + 2);
            const double* hc = a.hcol + (long long)b * (m + 1);
            for (int i = threadIdx.x; i <= j; i += blockDim.x) pc[i] = __ldcg(hc + i);
            if (threadIdx.x == 0) pc[j + 1] = s_red[0];
        }
        double* Vb = a.V + (long long)b * (m + 1) * a.n;
        const long long r0 = (long long)c * ACH;
        const RowView V = SV ? shared_rows(s_V) : global_rows(Vb, a.n, r0);
        chunk_update(V, a.n, r0, cols, s_h, a.w + (long long)b * a.n, s_acc, s_w, Vb + (long long)(j + 1) * a.n,
                     s_red[1], a.v32 ? a.v32 + (long long)b * a.n : nullptr);
        __syncthreads();
    }
    if (!a.pre_col) return;
    // phase 6: z = M^{-1} V[j+1] on the chunk's rows: warp w takes rows
    // 8 w .. 8 w + 7 of each item, lane q slot q, the same float32 products
    // and shuffle tree as the separate preconditioner kernel. The slots of the
    // CTA's first item are loaded before the barrier (they do not depend on
    // V[j+1]); V[j+1] is read through L2 (other CTAs wrote it).
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
    if (!grid_barrier(a.bar2, GI + a.bar_extra, a.err, a.err_host, a.spin_limit)) return;   // V[j+1] complete
    for (int item = blockIdx.x; item < items; item += NI) {
        const int b = item / a.nchunk, c = item % a.nchunk;
        if (item != (int)blockIdx.x) load_slots(item);
        if (!s_flag[b]) continue;
        // V[j+1] in float32 (v32, written in phase 5 with the same rounding
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

int arn_coop_grid(int n, int nb, int m, bool* resident) {
    static const bool off = []() {
        const char* e = getenv("BAE_ARNOLDI_COOP");
        return e && e[0] == '0';
    }();
    if (off || nb > COOP_MAX_NB || n <= 0) return 0;
    int dev = 0, coop = 0, sms = 0;
    BAE_CUDA(cudaGetDevice(&dev));
    BAE_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    BAE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (!coop) return 0;
    const size_t sh = (size_t)(4 * m + 3) * sizeof(double);
    const long long items = (long long)nb * ceil_div(n, ACH);
    // resident basis chunks: one item per CTA, all CTAs on the device at once
    const size_t sh_sv = sh + (size_t)(m + 1) * SV_STRIDE * sizeof(double);
    *resident = false;
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
            return (int)(items + nb);
        }
    }
    int k32 = 0, k64 = 0;
    BAE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k32, k_arn_step_coop<float, false>, 256, sh));
    BAE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k64, k_arn_step_coop<double, false>, 256, sh));
    const long long cap = (long long)std::min(k32, k64) * sms;
    // persistent chunk CTAs plus one rotation CTA per right-hand side
    if (cap <= nb) return 0;
    return (int)std::min(cap, items + nb);
}

void arn_step(const Arnoldi& a, cudaStream_t st) {
    BAE_REQUIRE(a.v && a.gm && a.partner && a.t, BAE_ERR_INVALID_ARG, "arn_step: gather inputs not set");
    const size_t sh_h = (size_t)(a.m + 1) * sizeof(double);
    const size_t sh_g = (size_t)(4 * a.m + 3) * sizeof(double);
    if (a.coop_grid > 0) {
        BAE_REQUIRE(a.bar && a.bar2 && a.err && a.n2 && a.gflag && a.live && a.pcol && a.nb <= COOP_MAX_NB &&
                        a.coop_grid > a.nb,
                    BAE_ERR_INVALID_ARG, "arn_step: cooperative step state not set");
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(a.coop_grid);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = sh_g + (a.coop_resident ? (size_t)(a.m + 1) * SV_STRIDE * sizeof(double) : 0);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
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
    const dim3 grid(a.nchunk, a.nb);
    if (a.v_f32)
        BAE_LAUNCH("k_arn_gather_dots.f32", st, k_arn_gather_dots<float><<<grid, 256, 0, st>>>(a));
    else
        BAE_LAUNCH("k_arn_gather_dots.f64", st, k_arn_gather_dots<double><<<grid, 256, 0, st>>>(a));
    BAE_LAUNCH("k_arn_update_dots", st, k_arn_update_dots<<<grid, 256, sh_g, st>>>(a));
    BAE_LAUNCH("k_arn_update_next", st, k_arn_update_next<<<grid, 256, sh_h, st>>>(a));
}

void arn_finish(const Arnoldi& a, double* x, cudaStream_t st) {
    BAE_LAUNCH("k_arn_backsub", st, k_arn_backsub<<<a.nb, 32, a.m * sizeof(double), st>>>(a));
    BAE_LAUNCH("k_combine", st, k_combine<<<dim3(blocks_for(a.n), a.nb), 256, 0, st>>>(a.V, a.n, a.m + 1, a.ncols, a.y, a.m, x));
}

}  // namespace bae
