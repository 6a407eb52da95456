// Block-Jacobi right preconditioner of the BAE (see precond.cuh): built on
// the device in two kernels (cell table, then one thread per gamma- node
// forms and inverts its cell's block and keeps its own row of the inverse).
#include <algorithm>

#include "lgf.cuh"
#include "precond.cuh"

namespace bae {

namespace {

constexpr int TN = 8;   // LGF table extent: the block entries need offsets up to 3 per axis
constexpr int TAB = TN * (TN + 1) * (TN + 2) / 6;

__device__ __forceinline__ long long cell_of(long long lin, int N) {
    const long long i = lin / ((long long)N * N), j = (lin / N) % N, k = lin % N;
    const long long C = N / 2 + 1;
    return ((i / 2) * C + j / 2) * C + k / 2;
}

// every gamma- node enters its 2 x 2 x 2 cell (at most 8 per cell)
__global__ void k_cell_fill(const int* __restrict__ gm, long long n, int N, int* count, int* members) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const long long c = cell_of(gm[r], N);
        const int slot = atomicAdd(count + c, 1);
        if (slot < MAXB) members[c * MAXB + slot] = (int)r;
    }
}

// G_s at a lattice offset from the sorted table (offsets below TN per axis)
__device__ __forceinline__ double lgf_at(const double* tab, long long dx, long long dy, long long dz) {
    long long a = dx < 0 ? -dx : dx, b = dy < 0 ? -dy : dy, c = dz < 0 ? -dz : dz;
    if (a < b) { const long long x = a; a = b; b = x; }
    if (b < c) { const long long x = b; b = c; c = x; }
    if (a < b) { const long long x = a; a = b; b = x; }
    return tab[a * (a + 1) * (a + 2) / 6 + b * (b + 1) / 2 + c];
}

// potential at node x of a unit density at gamma- node c: single layer
// G(x - c); double layer |D_c| G(x - c) - sum_{k in D_c} G(x - k), or the
// single-layer column when D_c is empty (eqs. [single_potential],
// [double_potential])
__device__ double kval(const double* tab, const uint8_t* flags, int N, int layer, long long x, long long c) {
    const long long NN = (long long)N * N;
    const long long xi = x / NN, xj = (x / N) % N, xk = x % N;
    const long long ci = c / NN, cj = (c / N) % N, ck = c % N;
    const double g0 = lgf_at(tab, xi - ci, xj - cj, xk - ck);
    if (layer != BAE_LAYER_DOUBLE) return g0;
    double acc = 0.0;
    int nd = 0;
    const int d[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    for (int q = 0; q < 6; ++q) {
        const long long ki = ci + d[q][0], kj = cj + d[q][1], kk = ck + d[q][2];
        if (flags[(ki * N + kj) * N + kk] & 3) continue;   // in N+ = M+ and gamma-
        acc -= lgf_at(tab, xi - ki, xj - kj, xk - kk);
        ++nd;
    }
    return nd == 0 ? g0 : acc + nd * g0;
}

// one thread per gamma- node r: its cell's block A[B, B] (members in node
// order), inverted by Gauss-Jordan with partial pivoting (the identity if a
// pivot is negligible), row r of the inverse into the 8 slots of r
__global__ void k_block_rows(const int* __restrict__ gm, const int* __restrict__ partner, const double* __restrict__ t,
                             const uint8_t* __restrict__ flags, const double* __restrict__ tab, long long n, int N,
                             int layer, const int* __restrict__ count, const int* __restrict__ members, int* col,
                             double* val) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const long long cell = cell_of(gm[r], N);
        const int k = min(count[cell], MAXB);
        int mem[MAXB];
        for (int p = 0; p < k; ++p) mem[p] = members[cell * MAXB + p];
        for (int p = 1; p < k; ++p)   // node order, the same in every member's thread
            for (int q = p; q > 0 && mem[q - 1] > mem[q]; --q) {
                const int x = mem[q - 1];
                mem[q - 1] = mem[q];
                mem[q] = x;
            }
        double a[MAXB][MAXB], inv[MAXB][MAXB];
        double scale = 0.0;
        for (int p = 0; p < k; ++p) {
            const int rp = mem[p];
            const double tp = t[rp];
            for (int q = 0; q < k; ++q) {
                const long long cq = gm[mem[q]];
                a[p][q] = tp * kval(tab, flags, N, layer, gm[rp], cq) + (1.0 - tp) * kval(tab, flags, N, layer, partner[rp], cq);
                inv[p][q] = p == q ? 1.0 : 0.0;
                scale = fmax(scale, fabs(a[p][q]));
            }
        }
        bool ok = true;
        for (int c = 0; c < k && ok; ++c) {
            int piv = c;
            for (int q = c + 1; q < k; ++q)
                if (fabs(a[q][c]) > fabs(a[piv][c])) piv = q;
            if (!(fabs(a[piv][c]) > 1e-12 * scale)) {
                ok = false;
                break;
            }
            if (piv != c)
                for (int q = 0; q < k; ++q) {
                    double x = a[piv][q]; a[piv][q] = a[c][q]; a[c][q] = x;
                    x = inv[piv][q]; inv[piv][q] = inv[c][q]; inv[c][q] = x;
                }
            const double dinv = 1.0 / a[c][c];
            for (int q = 0; q < k; ++q) {
                a[c][q] *= dinv;
                inv[c][q] *= dinv;
            }
            for (int p = 0; p < k; ++p) {
                if (p == c) continue;
                const double f = a[p][c];
                if (f == 0.0) continue;
                for (int q = 0; q < k; ++q) {
                    a[p][q] -= f * a[c][q];
                    inv[p][q] -= f * inv[c][q];
                }
            }
        }
        int me = 0;
        for (int p = 0; p < k; ++p)
            if (mem[p] == (int)r) me = p;
        for (int q = 0; q < MAXB; ++q) {
            const bool use = q < k;
            col[r * MAXB + q] = use ? mem[q] : (int)r;
            val[r * MAXB + q] = use ? (ok ? inv[me][q] : (q == me ? 1.0 : 0.0)) : 0.0;
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
#pragma unroll
        for (int q = 0; q < MAXB; ++q) acc += val[r * MAXB + q] * x[col[r * MAXB + q]];
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

void build_precond(const Geometry& g, double s, Precond& out) {
    cudaStream_t st = g.stream;
    const int N = g.N;
    const long long n = g.n_gm;
    const long long C = N / 2 + 1, cells = C * C * C;
    // G_s at offsets [0, TN)^3, the function the convolution's spectrum comes from
    double* tab = dev_alloc_n<double>(TAB, st);
    lgf_table(TN, s, tab, st);
    int* count = dev_alloc_n<int>(cells, st);
    int* members = dev_alloc_n<int>(cells * MAXB, st);
    BAE_CUDA(cudaMemsetAsync(count, 0, (size_t)cells * sizeof(int), st));
    out.release();
    out.stream = st;
    out.n = n;
    out.col = dev_alloc_n<int>(n * MAXB, st);
    out.val = dev_alloc_n<double>(n * MAXB, st);
    BAE_LAUNCH("k_cell_fill", st, k_cell_fill<<<grid_for(n), 256, 0, st>>>(g.gm, n, N, count, members));
    BAE_LAUNCH("k_block_rows", st,
               k_block_rows<<<grid_for(n), 128, 0, st>>>(g.gm, g.partner, g.t, g.flags, tab, n, N, g.layer, count,
                                                          members, out.col, out.val));
    dev_free(members, st);
    dev_free(count, st);
    dev_free(tab, st);
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
