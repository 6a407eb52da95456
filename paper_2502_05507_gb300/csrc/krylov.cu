// Batched GMRES vector kernels with fixed-order reductions (see krylov.cuh).
#include "krylov.cuh"

namespace bae {

namespace {

constexpr int CH = 512;        // elements per chunk
constexpr int ICH = 16;        // basis vectors per CTA in the dot kernel

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// partial[b][i][c] = sum over chunk c of V[b][i][r] w[b][r], i in [i0, i0+ICH) n [0, cols)
__global__ void __launch_bounds__(256) k_dots(KrylovBatch k, const int* __restrict__ active, int cols) {
    __shared__ double s_w[CH];
    const int b = active[blockIdx.y];
    const int c = blockIdx.x;
    const long long r0 = (long long)c * CH;
    const double* w = k.w + (long long)b * k.n;
    for (int e = threadIdx.x; e < CH; e += blockDim.x) s_w[e] = (r0 + e < k.n) ? w[r0 + e] : 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i0 = blockIdx.z * ICH;
    for (int i = i0 + warp; i < i0 + ICH && i < cols; i += 8) {
        const double* v = k.V + ((long long)b * k.mp1 + i) * k.n;
        double acc = 0.0;
        for (int e = lane; e < CH; e += 32)
            if (r0 + e < k.n) acc += v[r0 + e] * s_w[e];
        acc = warp_sum(acc);
        if (lane == 0) k.partial[((long long)b * (k.mp1 + 1) + i) * k.nchunk + c] = acc;
    }
}

// h[b][i] = sum_c partial[b][i][c] for i in rows [i_lo, i_hi)
__global__ void k_reduce(KrylovBatch k, const int* __restrict__ active, int i_lo, int i_hi) {
    const int b = active[blockIdx.y];
    for (int i = i_lo + blockIdx.x * blockDim.x + threadIdx.x; i < i_hi; i += gridDim.x * blockDim.x) {
        const double* p = k.partial + ((long long)b * (k.mp1 + 1) + i) * k.nchunk;
        double acc = 0.0;
        for (int c = 0; c < k.nchunk; ++c) acc += p[c];
        k.h[(long long)b * (k.mp1 + 1) + i] = acc;
    }
}

// w[b] -= sum_i V[b][i] h[b][i]; partial of ||w||^2 into row mp1
__global__ void __launch_bounds__(256) k_update_norm(KrylovBatch k, const int* __restrict__ active, int cols) {
    __shared__ double s_h[256];
    __shared__ double s_red[8];
    const int b = active[blockIdx.y];
    const int c = blockIdx.x;
    const long long r0 = (long long)c * CH;
    double* w = k.w + (long long)b * k.n;
    const double* hb = k.h + (long long)b * (k.mp1 + 1);
    double nrm = 0.0;
    for (int e = threadIdx.x; e < CH; e += blockDim.x) {
        const long long r = r0 + e;
        double acc = (r < k.n) ? w[r] : 0.0;
        for (int i0 = 0; i0 < cols; i0 += 256) {
            // stage h in shared memory, 256 at a time (same for every e)
            __syncthreads();
            if (i0 + (int)threadIdx.x < cols) s_h[threadIdx.x] = hb[i0 + threadIdx.x];
            __syncthreads();
            const int iend = min(cols - i0, 256);
            if (r < k.n)
                for (int i = 0; i < iend; ++i)
                    acc -= k.V[((long long)b * k.mp1 + i0 + i) * k.n + r] * s_h[i];
        }
        if (r < k.n) {
            w[r] = acc;
            nrm += acc * acc;
        }
    }
    nrm = warp_sum(nrm);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += s_red[q];
        k.partial[((long long)b * (k.mp1 + 1) + k.mp1) * k.nchunk + c] = s;
    }
}

__global__ void k_scale_into(KrylovBatch k, const int* __restrict__ active, int j) {
    const int b = active[blockIdx.y];
    const double n2 = k.h[(long long)b * (k.mp1 + 1) + k.mp1];
    const double s = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
    const double* w = k.w + (long long)b * k.n;
    double* v = k.V + ((long long)b * k.mp1 + j) * k.n;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < k.n; r += (long long)gridDim.x * blockDim.x)
        v[r] = w[r] * s;
}

__global__ void k_combine(KrylovBatch k, const int* __restrict__ active, int cols, const double* __restrict__ y,
                          int ystride, double* __restrict__ x) {
    const int b = active[blockIdx.y];
    const double* yb = y + (long long)b * ystride;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < k.n; r += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < cols; ++i) acc += k.V[((long long)b * k.mp1 + i) * k.n + r] * yb[i];
        x[(long long)b * k.n + r] += acc;
    }
}

__global__ void k_scale(const double* __restrict__ x, const double* __restrict__ alpha, const int* __restrict__ active,
                        int n, double* __restrict__ y) {
    const int b = active[blockIdx.y];
    const double a = alpha[b];
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        y[(long long)b * n + r] = x[(long long)b * n + r] * a;
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

__global__ void k_gather_rows(const double* src, const int* __restrict__ active, long long n, double* dst) {
    const int q = blockIdx.y;
    const int b = active[q];
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        dst[(long long)q * n + r] = src[(long long)b * n + r];
}

__global__ void k_scatter_rows(const double* src, const int* __restrict__ active, long long n, double* dst) {
    const int q = blockIdx.y;
    const int b = active[q];
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        dst[(long long)b * n + r] = src[(long long)q * n + r];
}

int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 1216); }

}  // namespace

int krylov_chunks(int n) { return ceil_div(n, CH); }

void kr_dots(const KrylovBatch& k, const int* active, int na, int cols, cudaStream_t st) {
    if (na == 0 || cols == 0) return;
    BAE_LAUNCH("k_dots", st, k_dots<<<dim3(k.nchunk, na, ceil_div(cols, ICH)), 256, 0, st>>>(k, active, cols));
    BAE_LAUNCH("k_reduce", st, k_reduce<<<dim3(ceil_div(cols, 128), na), 128, 0, st>>>(k, active, 0, cols));
}

void kr_update_norm(const KrylovBatch& k, const int* active, int na, int cols, cudaStream_t st) {
    if (na == 0) return;
    BAE_LAUNCH("k_update_norm", st, k_update_norm<<<dim3(k.nchunk, na), 256, 0, st>>>(k, active, cols));
    BAE_LAUNCH("k_reduce", st, k_reduce<<<dim3(1, na), 32, 0, st>>>(k, active, k.mp1, k.mp1 + 1));
}

void kr_scale_into(const KrylovBatch& k, const int* active, int na, int j, cudaStream_t st) {
    if (na == 0) return;
    BAE_LAUNCH("k_scale_into", st, k_scale_into<<<dim3(blocks_for(k.n), na), 256, 0, st>>>(k, active, j));
}

void kr_combine(const KrylovBatch& k, const int* active, int na, int cols, const double* y, int ystride, double* x,
                cudaStream_t st) {
    if (na == 0 || cols == 0) return;
    BAE_LAUNCH("k_combine", st, k_combine<<<dim3(blocks_for(k.n), na), 256, 0, st>>>(k, active, cols, y, ystride, x));
}

void kr_scale(const double* x, const double* alpha, const int* active, int na, int n, double* y, cudaStream_t st) {
    if (na == 0) return;
    BAE_LAUNCH("k_scale", st, k_scale<<<dim3(blocks_for(n), na), 256, 0, st>>>(x, alpha, active, n, y));
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

void kr_gather_rows(const double* src, const int* active, int na, long long n, double* dst, cudaStream_t st) {
    if (na == 0) return;
    BAE_LAUNCH("k_gather_rows", st, k_gather_rows<<<dim3(blocks_for(n), na), 256, 0, st>>>(src, active, n, dst));
}

void kr_scatter_rows(const double* src, const int* active, int na, long long n, double* dst, cudaStream_t st) {
    if (na == 0) return;
    BAE_LAUNCH("k_scatter_rows", st, k_scatter_rows<<<dim3(blocks_for(n), na), 256, 0, st>>>(src, active, n, dst));
}

}  // namespace bae
