// Restricted additive Schwarz right preconditioner of the BAE (see
// precond.cuh): built on the device (a node map, then one thread per
// gamma- node forms its neighbourhood block and solves for its own row of
// that block's inverse).
#include <algorithm>

#include "lgf.cuh"
#include "precond.cuh"

namespace bae {

namespace {


// node_of[lin] = gamma- index of grid node lin, -1 elsewhere
__global__ void k_node_map(const int* __restrict__ gm, long long n, int* node_of) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        node_of[gm[r]] = (int)r;
}

// G_s at a lattice offset from the sorted table (offsets below NEAR_TN per axis)
__device__ __forceinline__ float lgf_at(const float* tab, int dx, int dy, int dz) {
    int a = dx < 0 ? -dx : dx, b = dy < 0 ? -dy : dy, c = dz < 0 ? -dz : dz;
    if (a < b) { const int x = a; a = b; b = x; }
    if (b < c) { const int x = b; b = c; c = x; }
    if (a < b) { const int x = a; a = b; b = x; }
    return tab[a * (a + 1) * (a + 2) / 6 + b * (b + 1) / 2 + c];
}

// potential at node x of a unit density at gamma- node c: single layer
// G(x - c); double layer |D_c| G(x - c) - sum_{k in D_c} G(x - k), or the
// single-layer column when D_c is empty (eqs. [single_potential],
// [double_potential])
__device__ float kval(const float* tab, const uint8_t* flags, int N, int layer, long long x, long long c) {
    const long long NN = (long long)N * N;
    const int xi = (int)(x / NN), xj = (int)((x / N) % N), xk = (int)(x % N);
    const int ci = (int)(c / NN), cj = (int)((c / N) % N), ck = (int)(c % N);
    const float g0 = lgf_at(tab, xi - ci, xj - cj, xk - ck);
    if (layer != BAE_LAYER_DOUBLE) return g0;
    float acc = 0.f;
    int nd = 0;
    const int d[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    for (int q = 0; q < 6; ++q) {
        const int ki = ci + d[q][0], kj = cj + d[q][1], kk = ck + d[q][2];
        if (flags[((long long)ki * N + kj) * N + kk] & 3) continue;   // in N+ = M+ and gamma-
        acc -= lgf_at(tab, xi - ki, xj - kj, xk - kk);
        ++nd;
    }
    return nd == 0 ? g0 : acc + (float)nd * g0;
}

// One thread per gamma- node r: S = the gamma- nodes of the 3 x 3 x 3
// neighbourhood of r (in node order), A_S = A[S, S] from the LGF table, and
// row r of M^{-1} = the row of r in inv(A_S), from the LU solve (partial
// pivoting) of A_S^T z = e_r; a numerically singular block keeps the identity
// row. Written into the MAXR slots of r.
__global__ void __launch_bounds__(64) k_ras_rows(const int* __restrict__ gm, const int* __restrict__ partner,
                                                 const double* __restrict__ t, const uint8_t* __restrict__ flags,
                                                 const double* __restrict__ tab64, const int* __restrict__ node_of,
                                                 long long n, int N, int layer, int* col, double* val) {
    __shared__ float tab[NEAR_TAB];
    for (int e = threadIdx.x; e < NEAR_TAB; e += blockDim.x) tab[e] = (float)tab64[e];
    __syncthreads();
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const long long lin = gm[r], NN = (long long)N * N;
        int S[MAXR];
        int k = 0, me = 0;
        for (int di = -1; di <= 1; ++di)
            for (int dj = -1; dj <= 1; ++dj)
                for (int dk = -1; dk <= 1; ++dk) {
                    const int s = node_of[lin + di * NN + dj * N + dk];   // gamma- is not on a box face
                    if (s < 0) continue;
                    if (s == (int)r) me = k;
                    S[k++] = s;
                }
        // M = A_S^T, row-major: M[q][p] = A_S[p][q] (float32)
        float M[MAXR][MAXR], z[MAXR];
        float scale = 0.f;
        for (int p = 0; p < k; ++p) {
            const int rp = S[p];
            const float tp = (float)t[rp];
            for (int q = 0; q < k; ++q) {
                const long long cq = gm[S[q]];
                const float v = tp * kval(tab, flags, N, layer, gm[rp], cq) + (1.f - tp) * kval(tab, flags, N, layer, partner[rp], cq);
                M[q][p] = v;
                scale = fmaxf(scale, fabsf(v));
            }
            z[p] = p == me ? 1.f : 0.f;
        }
        bool ok = true;
        for (int c = 0; c < k; ++c) {   // forward elimination with partial pivoting
            int piv = c;
            for (int q = c + 1; q < k; ++q)
                if (fabsf(M[q][c]) > fabsf(M[piv][c])) piv = q;
            if (!(fabsf(M[piv][c]) > 1e-6f * scale)) {
                ok = false;
                break;
            }
            if (piv != c) {
                for (int q = c; q < k; ++q) {
                    const float x = M[piv][q];
                    M[piv][q] = M[c][q];
                    M[c][q] = x;
                }
                const float x = z[piv];
                z[piv] = z[c];
                z[c] = x;
            }
            const float dinv = 1.f / M[c][c];
            for (int p = c + 1; p < k; ++p) {
                const float f = M[p][c] * dinv;
                if (f == 0.f) continue;
                for (int q = c + 1; q < k; ++q) M[p][q] -= f * M[c][q];
                z[p] -= f * z[c];
            }
        }
        if (ok)
            for (int c = k - 1; c >= 0; --c) {   // back substitution
                float x = z[c];
                for (int q = c + 1; q < k; ++q) x -= M[c][q] * z[q];
                z[c] = x / M[c][c];
            }
        for (int q = 0; q < MAXR; ++q) {
            const bool use = q < k;
            col[r * MAXR + q] = use ? S[q] : (int)r;
            val[r * MAXR + q] = use ? (ok ? (double)z[q] : (q == me ? 1.0 : 0.0)) : 0.0;
        }
    }
}

__global__ void k_precond_apply(const int* __restrict__ col, const double* __restrict__ val, long long n,
                                const double* in, long long in_stride, const int* row, long long row_stride, double* out,
                                long long out_stride, const int* active) {
    const int b = blockIdx.y;
    if (active && !active[b]) return;
    const double* x = in + b * in_stride + (row ? (long long)row[b] * row_stride : 0);
    double* y = out + b * out_stride;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int q = 0; q < MAXR; ++q) {
            const double v = val[r * MAXR + q];
            if (v != 0.0) acc += v * x[col[r * MAXR + q]];
        }
        y[r] = acc;
    }
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 4864); }

}  // namespace

void Precond::release() {
    if (col) dev_free(col, stream);
    if (val) dev_free(val, stream);
    col = nullptr;
    val = nullptr;
    built = false;
}

void build_precond(const Geometry& g, double s, const double* near, Precond& out) {
    cudaStream_t st = g.stream;
    const int N = g.N;
    const long long n = g.n_gm, n3 = (long long)N * N * N;
    // G_s at offsets [0, NEAR_TN)^3, the function the convolution's spectrum comes from
    double* own = nullptr;
    if (!near) {
        own = dev_alloc_n<double>(NEAR_TAB, st);
        lgf_table(NEAR_TN, s, own, st);
        near = own;
    }
    int* node_of = dev_alloc_n<int>(n3, st);
    BAE_CUDA(cudaMemsetAsync(node_of, 0xff, (size_t)n3 * sizeof(int), st));
    out.release();
    out.stream = st;
    out.n = n;
    out.col = dev_alloc_n<int>(n * MAXR, st);
    out.val = dev_alloc_n<double>(n * MAXR, st);
    BAE_LAUNCH("k_node_map", st, k_node_map<<<grid_for(n), 256, 0, st>>>(g.gm, n, node_of));
    BAE_LAUNCH("k_ras_rows", st,
               k_ras_rows<<<grid_for(n), 64, 0, st>>>(g.gm, g.partner, g.t, g.flags, near, node_of, n, N, g.layer,
                                                       out.col, out.val));
    dev_free(node_of, st);
    if (own) dev_free(own, st);
    out.built = true;
}

void precond_apply(const Precond& p, const double* in, long long in_stride, const int* row, long long row_stride,
                   double* out, long long out_stride, int nb, const int* active, cudaStream_t st) {
    if (p.n == 0 || nb == 0) return;
    BAE_LAUNCH("k_precond_apply", st,
               k_precond_apply<<<dim3(std::min(grid_for(p.n), 1216), nb), 256, 0, st>>>(
                   p.col, p.val, p.n, in, in_stride, row, row_stride, out, out_stride, active));
}

}  // namespace bae
