// Classification of the grid from level-set samples (Section 2.1), the
// Dirichlet closure (eq. [bc], hat functions on the grid edge to the M+
// neighbour whose phi-linear zero crossing is nearest), and the source
// stencil of the layer potentials (Section 3.2) in a form the convolution's
// first pass reads line by line.
//
// Every list is produced in lexicographic (i,j,k) order by a deterministic
// exclusive scan, so the results are bit-identical from run to run.
#include <algorithm>
#include <vector>

#include "classify.cuh"

namespace bae {

namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_E = 8;
constexpr int SCAN_CHUNK = SCAN_T * SCAN_E;

__constant__ int c_dir[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

// ---------------------------------------------------------------- scans
// Block-local exclusive scan of SCAN_CHUNK ints; block totals to sums[].
__device__ int block_exclusive_scan(int v, int* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    const int before = warp > 0 ? s_warp[warp - 1] : 0;
    const int total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    s_warp[32] = total;
    return before + x - v;  // exclusive
}

__global__ void k_scan_local(const int* __restrict__ in, int* __restrict__ out, long long n, int* __restrict__ sums) {
    __shared__ int s_warp[33];
    const long long base = (long long)blockIdx.x * SCAN_CHUNK + threadIdx.x * SCAN_E;
    int v[SCAN_E], tot = 0;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e) {
        v[e] = (base + e < n) ? in[base + e] : 0;
        tot += v[e];
    }
    const int ex = block_exclusive_scan(tot, s_warp);
    int run = ex;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e) {
        if (base + e < n) out[base + e] = run;
        run += v[e];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = s_warp[32];
}

// single CTA: exclusive scan of nb block sums in place; grand total to *total
__global__ void k_scan_sums(int* sums, int nb, int* total) {
    __shared__ int s_warp[33];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x * SCAN_E) {
        int v[SCAN_E], tot = 0;
        const int b0 = base + threadIdx.x * SCAN_E;
#pragma unroll
        for (int e = 0; e < SCAN_E; ++e) {
            v[e] = (b0 + e < nb) ? sums[b0 + e] : 0;
            tot += v[e];
        }
        const int ex = block_exclusive_scan(tot, s_warp);
        int run = ex + s_carry;
#pragma unroll
        for (int e = 0; e < SCAN_E; ++e) {
            if (b0 + e < nb) sums[b0 + e] = run;
            run += v[e];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s_carry;
}

__global__ void k_scan_add(int* out, long long n, const int* sums) {
    const int add = sums[blockIdx.x];
    const long long base = (long long)blockIdx.x * SCAN_CHUNK + threadIdx.x * SCAN_E;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e)
        if (base + e < n) out[base + e] += add;
}

// exclusive scan of n ints on the device; returns the total (synchronises)
int exclusive_scan(const int* in, int* out, long long n, int* scratch_sums, int* d_total, cudaStream_t st) {
    const int nb = ceil_div(n, SCAN_CHUNK);
    BAE_LAUNCH("k_scan_local", st, k_scan_local<<<nb, SCAN_T, 0, st>>>(in, out, n, scratch_sums));
    BAE_LAUNCH("k_scan_sums", st, k_scan_sums<<<1, 1024, 0, st>>>(scratch_sums, nb, d_total));
    BAE_LAUNCH("k_scan_add", st, k_scan_add<<<nb, SCAN_T, 0, st>>>(out, n, scratch_sums));
    int total = 0;
    BAE_CUDA(cudaMemcpyAsync(&total, d_total, sizeof(int), cudaMemcpyDeviceToHost, st));
    BAE_CUDA(cudaStreamSynchronize(st));
    return total;
}

// ------------------------------------------------------------ point sets
__global__ void k_inside(const double* __restrict__ phi, long long n3, uint8_t* __restrict__ inside, int* err) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n3; x += (long long)gridDim.x * blockDim.x) {
        const double p = phi[x];
        if (!isfinite(p)) atomicOr(err, 1);
        inside[x] = p < 0.0 ? 1 : 0;
    }
}

__device__ __forceinline__ bool in_grid(int i, int j, int k, int N) {
    return (unsigned)i < (unsigned)N && (unsigned)j < (unsigned)N && (unsigned)k < (unsigned)N;
}

__device__ __forceinline__ int IN(const uint8_t* inside, int i, int j, int k, int N) {
    return in_grid(i, j, k, N) ? inside[((long long)i * N + j) * N + k] : 0;
}

// node has an M+ neighbour (grid-outside counts as exterior)
__device__ __forceinline__ bool has_in_nb(const uint8_t* inside, int i, int j, int k, int N) {
    for (int d = 0; d < 6; ++d)
        if (IN(inside, i + c_dir[d][0], j + c_dir[d][1], k + c_dir[d][2], N)) return true;
    return false;
}

__device__ __forceinline__ bool is_gm(const uint8_t* inside, int i, int j, int k, int N) {
    return in_grid(i, j, k, N) && !IN(inside, i, j, k, N) && has_in_nb(inside, i, j, k, N);
}

__device__ __forceinline__ bool is_nplus(const uint8_t* inside, int i, int j, int k, int N) {
    return in_grid(i, j, k, N) && (IN(inside, i, j, k, N) || has_in_nb(inside, i, j, k, N));
}

__global__ void k_flags(const uint8_t* __restrict__ inside, int N, uint8_t* __restrict__ flags, int* err) {
    const long long n3 = (long long)N * N * N;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n3; x += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(x / ((long long)N * N)), j = (int)((x / N) % N), k = (int)(x % N);
        const bool in = inside[x] != 0;
        const bool face = (i == 0 || j == 0 || k == 0 || i == N - 1 || j == N - 1 || k == N - 1);
        bool out_nb = false;
        for (int d = 0; d < 6; ++d)
            if (!IN(inside, i + c_dir[d][0], j + c_dir[d][1], k + c_dir[d][2], N)) out_nb = true;
        const bool gm = !in && has_in_nb(inside, i, j, k, N);
        const bool gp = in && out_nb;
        int cnt = 0;
        bool dnode = false;
        if (gm) {
            for (int d = 0; d < 6; ++d)
                if (!is_nplus(inside, i + c_dir[d][0], j + c_dir[d][1], k + c_dir[d][2], N)) ++cnt;
        } else if (!in) {  // outside N+ (not gm, not M+): next to a gamma- node?
            for (int d = 0; d < 6; ++d)
                if (is_gm(inside, i + c_dir[d][0], j + c_dir[d][1], k + c_dir[d][2], N)) dnode = true;
        }
        if ((gm || in) && face) atomicOr(err, 2);
        flags[x] = (uint8_t)((in ? 1 : 0) | (gm ? 2 : 0) | (gp ? 4 : 0) | (dnode ? 8 : 0) | (cnt << 4));
    }
}

__global__ void k_pred(const uint8_t* __restrict__ flags, long long n3, int mask, int* __restrict__ out) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n3; x += (long long)gridDim.x * blockDim.x)
        out[x] = (flags[x] & mask) ? 1 : 0;
}

__global__ void k_scatter_list(const uint8_t* __restrict__ flags, long long n3, int mask, const int* __restrict__ pos,
                               int* __restrict__ list) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n3; x += (long long)gridDim.x * blockDim.x)
        if (flags[x] & mask) list[pos[x]] = (int)x;
}

__global__ void k_index_map(const int* __restrict__ list, int n, int* __restrict__ map) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) map[list[r]] = r;
}

// Closure per gamma- node: partner p with the largest t = phi(p)/(phi(p)-phi(m)),
// first in the order +x,-x,+y,-y,+z,-z on ties; x* = x_p + t (x_m - x_p).
// Separate round-to-nearest operations (no contraction) so that the values
// are reproducible by any IEEE float64 implementation of the same formula.
__global__ void k_closure(const double* __restrict__ phi, const uint8_t* __restrict__ flags, const int* __restrict__ gm,
                          int n, int N, double h, double o0, double o1, double o2,
                          int* __restrict__ partner, double* __restrict__ tw, double* __restrict__ xstar) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int m = gm[r];
        const int i = m / (N * N), j = (m / N) % N, k = m % N;
        const double pm = phi[m];
        double best = -1.0;
        int bp = m, bd = 0;
        for (int d = 0; d < 6; ++d) {
            const int ii = i + c_dir[d][0], jj = j + c_dir[d][1], kk = k + c_dir[d][2];
            const int p = (ii * N + jj) * N + kk;   // in the grid: gamma- is off the faces
            if (flags[p] & 1) {
                const double pp = phi[p];
                const double t = __ddiv_rn(pp, __dsub_rn(pp, pm));
                if (t > best) { best = t; bp = p; bd = d; }
            }
        }
        partner[r] = bp;
        tw[r] = best;
        const int ip[3] = {i + c_dir[bd][0], j + c_dir[bd][1], k + c_dir[bd][2]};
        const int im[3] = {i, j, k};
        const double org[3] = {o0, o1, o2};
        for (int c = 0; c < 3; ++c) {
            const double xp = __dadd_rn(org[c], __dmul_rn((double)ip[c], h));
            const double xm = __dadd_rn(org[c], __dmul_rn((double)im[c], h));
            xstar[3 * (long long)r + c] = __dadd_rn(xp, __dmul_rn(best, __dsub_rn(xm, xp)));
        }
    }
}

// ------------------------------------------------------------ source recipe
// number of terms of each source node: 1 for gamma- nodes, the number of
// gamma- neighbours for D-nodes
__global__ void k_term_count(const int* __restrict__ src, int ns, const uint8_t* __restrict__ flags, int N,
                             int* __restrict__ cnt) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        const int x = src[s];
        if (flags[x] & 2) { cnt[s] = 1; continue; }
        const int i = x / (N * N), j = (x / N) % N, k = x % N;
        int c = 0;
        for (int d = 0; d < 6; ++d) {
            const int ii = i + c_dir[d][0], jj = j + c_dir[d][1], kk = k + c_dir[d][2];
            if (in_grid(ii, jj, kk, N) && (flags[(ii * N + jj) * N + kk] & 2)) ++c;
        }
        cnt[s] = c;
    }
}

// rho(x) = coef(x) q(x) on gamma- (coef = |D_x| for the double layer, or 1
// when D_x is empty or for the single layer); rho(k) = -sum q(n) over the
// gamma- neighbours n of a D-node k (k is in D_n for each of them).
__global__ void k_term_fill(const int* __restrict__ src, int ns, const uint8_t* __restrict__ flags, int N,
                            const int* __restrict__ gidx, const int* __restrict__ off, int layer,
                            int* __restrict__ tidx, float* __restrict__ tcoef) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        const int x = src[s];
        int e = off[s];
        const uint8_t f = flags[x];
        if (f & 2) {
            const int c = f >> 4;
            tidx[e] = gidx[x];
            tcoef[e] = (layer == BAE_LAYER_DOUBLE && c > 0) ? (float)c : 1.0f;
            continue;
        }
        const int i = x / (N * N), j = (x / N) % N, k = x % N;
        for (int d = 0; d < 6; ++d) {
            const int ii = i + c_dir[d][0], jj = j + c_dir[d][1], kk = k + c_dir[d][2];
            if (!in_grid(ii, jj, kk, N)) continue;
            const int y = (ii * N + jj) * N + kk;
            if (flags[y] & 2) {
                tidx[e] = gidx[y];
                tcoef[e] = -1.0f;
                ++e;
            }
        }
    }
}

// line_off[l] = first source with src_lin >= l * N  (lower bound)
__global__ void k_line_offsets(const int* __restrict__ src, int ns, int N, int* __restrict__ line_off) {
    const int nl = N * N;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l <= nl; l += gridDim.x * blockDim.x) {
        const long long key = (long long)l * N;
        int lo = 0, hi = ns;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((long long)src[mid] < key) lo = mid + 1; else hi = mid;
        }
        line_off[l] = lo;
    }
}

struct Scratch {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch() { for (void* p : ptrs) dev_free(p, st); }
    template <typename T> T* get(long long n) { T* p = dev_alloc_n<T>(n, st); ptrs.push_back(p); return p; }
};

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }

}  // namespace

void Geometry::release() {
    void* ps[] = {flags, gm, partner, t, xstar, line_off, src_lin, term_off, term_idx, term_coef};
    for (void* p : ps) if (p) dev_free(p, stream);
    flags = nullptr; gm = partner = nullptr; t = xstar = nullptr;
    line_off = src_lin = term_off = term_idx = nullptr; term_coef = nullptr;
}

void build_geometry(const double* phi, int N, double h, const double origin[3], int layer, Geometry& g,
                    cudaStream_t st) {
    const long long n3 = (long long)N * N * N;
    Scratch sc(st);
    g.stream = st;
    g.N = N;
    g.h = h;
    for (int c = 0; c < 3; ++c) g.origin[c] = origin[c];
    g.layer = layer;

    int* d_err = sc.get<int>(2);
    BAE_CUDA(cudaMemsetAsync(d_err, 0, 2 * sizeof(int), st));
    uint8_t* inside = sc.get<uint8_t>(n3);
    BAE_LAUNCH("k_inside", st, k_inside<<<grid_for(n3), 256, 0, st>>>(phi, n3, inside, d_err));
    g.flags = dev_alloc_n<uint8_t>(n3, st);
    BAE_LAUNCH("k_flags", st, k_flags<<<grid_for(n3), 256, 0, st>>>(inside, N, g.flags, d_err));
    int err = 0;
    BAE_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    BAE_CUDA(cudaStreamSynchronize(st));
    if (err & 1) throw Error(BAE_ERR_INVALID_ARG, "phi contains non-finite values");
    if (err & 2) throw Error(BAE_ERR_GEOMETRY, "M+ or gamma- reaches the faces of the grid box");

    int* pred = sc.get<int>(n3);
    int* pos = sc.get<int>(n3);
    int* sums = sc.get<int>(ceil_div(n3, SCAN_CHUNK) + 1);
    int* d_total = d_err + 1;
    auto make_list = [&](int mask, long long& count) -> int* {
        BAE_LAUNCH("k_pred", st, k_pred<<<grid_for(n3), 256, 0, st>>>(g.flags, n3, mask, pred));
        count = exclusive_scan(pred, pos, n3, sums, d_total, st);
        int* list = dev_alloc_n<int>(count, st);
        BAE_LAUNCH("k_scatter_list", st, k_scatter_list<<<grid_for(n3), 256, 0, st>>>(g.flags, n3, mask, pos, list));
        return list;
    };
    g.gm = make_list(2, g.n_gm);
    if (g.n_gm == 0) throw Error(BAE_ERR_GEOMETRY, "gamma- is empty (no interior node)");
    {
        long long dummy;
        int* l = make_list(4, g.n_gp);
        dev_free(l, st);
        l = make_list(1, g.n_mp);
        dev_free(l, st);
        (void)dummy;
    }
    // closure
    g.partner = dev_alloc_n<int>(g.n_gm, st);
    g.t = dev_alloc_n<double>(g.n_gm, st);
    g.xstar = dev_alloc_n<double>(3 * g.n_gm, st);
    BAE_LAUNCH("k_closure", st, k_closure<<<grid_for(g.n_gm), 256, 0, st>>>(phi, g.flags, g.gm, (int)g.n_gm, N, h, origin[0], origin[1], origin[2],
                                                g.partner, g.t, g.xstar));

    // source recipe
    int* gidx = sc.get<int>(n3);
    BAE_CUDA(cudaMemsetAsync(gidx, 0xff, n3 * sizeof(int), st));
    BAE_LAUNCH("k_index_map", st, k_index_map<<<grid_for(g.n_gm), 256, 0, st>>>(g.gm, (int)g.n_gm, gidx));
    g.src_lin = make_list(layer == BAE_LAYER_DOUBLE ? (2 | 8) : 2, g.n_src);
    int* cnt = sc.get<int>(g.n_src + 1);
    BAE_LAUNCH("k_term_count", st, k_term_count<<<grid_for(g.n_src), 256, 0, st>>>(g.src_lin, (int)g.n_src, g.flags, N, cnt));
    g.term_off = dev_alloc_n<int>(g.n_src + 1, st);
    BAE_CUDA(cudaMemsetAsync(cnt + g.n_src, 0, sizeof(int), st));
    g.n_terms = exclusive_scan(cnt, g.term_off, g.n_src + 1, sums, d_total, st);
    g.term_idx = dev_alloc_n<int>(g.n_terms, st);
    g.term_coef = dev_alloc_n<float>(g.n_terms, st);
    BAE_LAUNCH("k_term_fill", st, k_term_fill<<<grid_for(g.n_src), 256, 0, st>>>(g.src_lin, (int)g.n_src, g.flags, N, gidx, g.term_off, layer,
                                                   g.term_idx, g.term_coef));
    g.line_off = dev_alloc_n<int>((long long)N * N + 1, st);
    BAE_LAUNCH("k_line_offsets", st, k_line_offsets<<<grid_for((long long)N * N + 1), 256, 0, st>>>(g.src_lin, (int)g.n_src, N, g.line_off));
    // x-planes holding every source (gamma- and D-nodes, or M+ for the
    // volume term) and every gathered node (gamma- and the partners, one
    // step from gamma-): the lists are in lexicographic order, so the first
    // and last entries bound them
    int ends[4] = {0, 0, 0, 0};
    BAE_CUDA(cudaMemcpyAsync(ends + 0, g.gm, sizeof(int), cudaMemcpyDeviceToHost, st));
    BAE_CUDA(cudaMemcpyAsync(ends + 1, g.gm + (g.n_gm - 1), sizeof(int), cudaMemcpyDeviceToHost, st));
    BAE_CUDA(cudaMemcpyAsync(ends + 2, g.src_lin, sizeof(int), cudaMemcpyDeviceToHost, st));
    BAE_CUDA(cudaMemcpyAsync(ends + 3, g.src_lin + (g.n_src - 1), sizeof(int), cudaMemcpyDeviceToHost, st));
    BAE_CUDA(cudaStreamSynchronize(st));
    const long long nn = (long long)N * N;
    const long long first = std::min(ends[0], ends[2]) / nn, last = std::max(ends[1], ends[3]) / nn;
    g.plane_lo = (int)std::max(0LL, first - 1);
    g.plane_hi = (int)std::min((long long)N, last + 2);
}

}  // namespace bae
