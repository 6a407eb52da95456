// Classification of the grid from level-set samples (Section 2.1), the
// Dirichlet closure (eq. [bc], hat functions on the grid edge to the M+
// neighbour whose phi-linear zero crossing is nearest), and the source
// stencil of the layer potentials (Section 3.2) in a form the convolution's
// first pass reads line by line.
//
// Every list is produced in lexicographic (i,j,k) order by a deterministic
// exclusive scan, so the results are bit-identical from run to run.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "classify.cuh"

namespace bae {

namespace {

constexpr int SCAN_E = 8;   // entries per thread of the line-count scans

__constant__ int c_dir[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

// ---------------------------------------------------------------- scans
// exclusive scan over the CTA (blockDim.x a multiple of 32, at most 1024);
// the CTA total is left in s_warp[32]
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

// ------------------------------------------------------------ point sets
// One CTA per grid line (i, j), its threads over k.
constexpr int LINE_T = 128;

// slots of the small device record the host reads once
enum { I_ERR = 0, I_GP, I_MP, I_FIRST, I_LAST, I_NGM, I_NSRC, I_NTERM, I_NGPL, I_FIRSTY, I_LASTY, I_FIRSTZ, I_LASTZ,
       I_COUNT };

__device__ __forceinline__ bool in_grid(int i, int j, int k, int N) {
    return (unsigned)i < (unsigned)N && (unsigned)j < (unsigned)N && (unsigned)k < (unsigned)N;
}

// bits per node from phi: bit0 in M+ (phi < 0), bit1 an M+ neighbour, bit2
// a neighbour outside M+ (nodes outside the box count as exterior)
__global__ void __launch_bounds__(LINE_T) k_nbits(const double* __restrict__ phi, int N, uint8_t* __restrict__ nb,
                                                 int* __restrict__ info) {
    const int line = blockIdx.x, i = line / N, j = line - i * N;
    const long long base = (long long)line * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double p = phi[base + k];
        if (!isfinite(p)) atomicOr(info + I_ERR, 1);
        bool h = false, e = false;
        for (int d = 0; d < 6; ++d) {
            const int ii = i + c_dir[d][0], jj = j + c_dir[d][1], kk = k + c_dir[d][2];
            if (in_grid(ii, jj, kk, N) && phi[((long long)ii * N + jj) * N + kk] < 0.0) h = true;
            else e = true;
        }
        nb[base + k] = (uint8_t)((p < 0.0 ? 1 : 0) | (h ? 2 : 0) | (e ? 4 : 0));
    }
}

// Node flags from the bits of the node and its six neighbours: M+ (bit0),
// gamma- = outside M+ with an M+ neighbour (bit1), gamma+ = M+ with an
// exterior neighbour (bit2), D-node = outside N+ = M+ and gamma-, next to a
// gamma- node (bit3), and for gamma- nodes |D_n| = the neighbours outside
// N+ (bits 4-6). Per line: the gamma- nodes, the sources (flags & src_mask)
// and their stencil terms (a D-node: one per gamma- neighbour; a gamma- node:
// 1, or with `direct` 1 + its neighbours in gamma = gamma- u gamma+), the
// gamma+ nodes; M+ and gamma+ totals and the range of source planes go to
// info.
__global__ void __launch_bounds__(LINE_T) k_flags_lines(const uint8_t* __restrict__ nb, int N, int src_mask,
                                                       bool direct, uint8_t* __restrict__ flags,
                                                       int* __restrict__ cnt_gm, int* __restrict__ cnt_src,
                                                       int* __restrict__ cnt_term, int* __restrict__ cnt_gp,
                                                       int* __restrict__ info) {
    __shared__ int s_red[5][LINE_T / 32];
    const int line = blockIdx.x, i = line / N, j = line - i * N;
    const long long base = (long long)line * N;
    int c[5] = {0, 0, 0, 0, 0};   // gamma-, sources, terms, gamma+, M+
    int klo = N, khi = -1;        // k range of this thread's sources
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int me = nb[base + k];
        bool out_nb = false;
        int n_out = 0, n_gm = 0, n_gam = 0;
        for (int d = 0; d < 6; ++d) {
            const int ii = i + c_dir[d][0], jj = j + c_dir[d][1], kk = k + c_dir[d][2];
            const int q = in_grid(ii, jj, kk, N) ? nb[((long long)ii * N + jj) * N + kk] : 0;
            if (!(q & 1)) out_nb = true;
            if (!(q & 3)) ++n_out;               // not in N+
            if (!(q & 1) && (q & 2)) ++n_gm;     // a gamma- node
            if ((q & 1) ? (q & 4) : (q & 2)) ++n_gam;   // gamma+ or gamma-
        }
        const bool in = me & 1, gm = !in && (me & 2);
        const bool gp = in && out_nb;
        const bool dnode = !in && !gm && n_gm > 0;
        const bool face = (i == 0 || j == 0 || k == 0 || i == N - 1 || j == N - 1 || k == N - 1);
        if ((gm || in) && face) atomicOr(info + I_ERR, 2);
        const int f = (in ? 1 : 0) | (gm ? 2 : 0) | (gp ? 4 : 0) | (dnode ? 8 : 0) | ((gm ? n_out : 0) << 4);
        flags[base + k] = (uint8_t)f;
        const bool src = (f & src_mask) != 0;
        if (src) {
            klo = min(klo, k);
            khi = max(khi, k);
        }
        c[0] += gm;
        c[1] += src;
        c[2] += src ? (gm ? (direct ? 1 + n_gam : 1) : n_gm) : 0;
        c[3] += gp;
        c[4] += in;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < 5; ++e) {
        const int v = __reduce_add_sync(0xffffffffu, c[e]);
        if (lane == 0) s_red[e][w] = v;
    }
    klo = __reduce_min_sync(0xffffffffu, klo);
    khi = __reduce_max_sync(0xffffffffu, khi);
    if (lane == 0 && khi >= 0) {
        atomicMax(info + I_FIRSTZ, N - klo);
        atomicMax(info + I_LASTZ, khi + 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int t[5] = {0, 0, 0, 0, 0};
        for (int e = 0; e < 5; ++e)
            for (int x = 0; x < (int)(blockDim.x >> 5); ++x) t[e] += s_red[e][x];
        cnt_gm[line] = t[0];
        cnt_src[line] = t[1];
        cnt_term[line] = t[2];
        cnt_gp[line] = t[3];
        if (t[3]) atomicAdd(info + I_GP, t[3]);
        if (t[4]) atomicAdd(info + I_MP, t[4]);
        if (t[1]) {
            atomicMax(info + I_FIRST, N - i);
            atomicMax(info + I_LAST, i + 1);
            atomicMax(info + I_FIRSTY, N - j);
            atomicMax(info + I_LASTY, j + 1);
        }
    }
}

// In-place exclusive scans of the four per-line counts (nl + 1 entries,
// the last one becomes the total), one CTA each; totals to info.
__global__ void __launch_bounds__(1024) k_scan_lines(int* c0, int* c1, int* c2, int* c3, int nl, int* info) {
    __shared__ int s_warp[33];
    __shared__ int s_carry;
    int* arr = blockIdx.x == 0 ? c0 : (blockIdx.x == 1 ? c1 : (blockIdx.x == 2 ? c2 : c3));
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base <= nl; base += blockDim.x * SCAN_E) {
        int v[SCAN_E], tot = 0;
        const int b0 = base + threadIdx.x * SCAN_E;
#pragma unroll
        for (int e = 0; e < SCAN_E; ++e) {
            v[e] = (b0 + e < nl) ? arr[b0 + e] : 0;
            tot += v[e];
        }
        const int ex = block_exclusive_scan(tot, s_warp);
        int run = ex + s_carry;
#pragma unroll
        for (int e = 0; e < SCAN_E; ++e) {
            if (b0 + e <= nl) arr[b0 + e] = run;
            run += v[e];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) info[I_NGM + blockIdx.x] = s_carry;
}

// The lists in lexicographic order: per line, the CTA scans its nodes
// (gamma-, source and term counts packed in one int: at most 256, 256 and
// 1792 per line; gamma+ in a second scan) from the line's offsets.
// node_of[x] = index of gamma- node x, n_gm + index of gamma+ node x (set
// only there: the unknown numbers of the direct formulation); term_off[s] =
// first term of source s.
__global__ void __launch_bounds__(LINE_T) k_scatter_lines(const uint8_t* __restrict__ flags, int N, int src_mask,
                                                         bool direct, const int* __restrict__ off_gm,
                                                         const int* __restrict__ off_src,
                                                         const int* __restrict__ off_term,
                                                         const int* __restrict__ off_gp, const int* __restrict__ info,
                                                         int* __restrict__ gm, int* __restrict__ gp,
                                                         int* __restrict__ node_of, int* __restrict__ src_lin,
                                                         int* __restrict__ term_off) {
    __shared__ int s_warp[33];
    const int line = blockIdx.x, i = line / N, j = line - i * N;
    if (line == (int)gridDim.x - 1 && threadIdx.x == 0) term_off[info[I_NSRC]] = info[I_NTERM];
    int pg = off_gm[line], ps = off_src[line], pt = off_term[line], pp = off_gp[line];
    const int ngm = info[I_NGM];
    if (ps == off_src[line + 1] && pp == off_gp[line + 1]) return;   // nothing on this line: the whole CTA
    const int base = line * N;
    for (int k0 = 0; k0 < N; k0 += blockDim.x) {
        const int k = k0 + (int)threadIdx.x;
        int g = 0, s = 0, nt = 0, p = 0;
        if (k < N) {
            const int f = flags[base + k];
            g = (f >> 1) & 1;
            p = (f >> 2) & 1;
            s = (f & src_mask) != 0;
            if (s) {
                const int want = g ? 6 : 2;   // gamma- and gamma+ neighbours, or gamma- neighbours
                nt = g ? 1 : 0;
                if (!g || direct)
                    for (int d = 0; d < 6; ++d) {
                        const int ii = i + c_dir[d][0], jj = j + c_dir[d][1], kk = k + c_dir[d][2];
                        if (in_grid(ii, jj, kk, N) && (flags[(ii * N + jj) * N + kk] & want)) ++nt;
                    }
            }
        }
        const int ex = block_exclusive_scan(g | (s << 10) | (nt << 20), s_warp);
        const int tot = s_warp[32];
        const int exp_ = block_exclusive_scan(p, s_warp);
        const int totp = s_warp[32];
        if (p) {
            gp[pp + exp_] = base + k;
            node_of[base + k] = ngm + pp + exp_;
        }
        pp += totp;
        if (g) {
            gm[pg + (ex & 1023)] = base + k;
            node_of[base + k] = pg + (ex & 1023);
        }
        if (s) {
            src_lin[ps + ((ex >> 10) & 1023)] = base + k;
            term_off[ps + ((ex >> 10) & 1023)] = pt + (ex >> 20);
        }
        pg += tot & 1023;
        ps += (tot >> 10) & 1023;
        pt += tot >> 20;
    }
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

// unknown number of each gamma- node's closure partner (a gamma+ node)
__global__ void k_partner_unknown(const int* __restrict__ partner, int n, const int* __restrict__ node_of,
                                  int* __restrict__ pu) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) pu[r] = node_of[partner[r]];
}

// ------------------------------------------------------------ source recipe
// rho(x) = coef(x) q(x) on gamma- (coef = |D_x| for the double layer, or 1
// when D_x is empty or for the single layer); rho(k) = -sum q(n) over the
// gamma- neighbours n of a D-node k (k is in D_n for each of them).
//
// Direct formulation (eq. [dp]): rho = chi_{M-} (6 + s - neighbour sum) u
// on gamma: at a gamma- node n, (6 + s) u(n) minus u at its neighbours in
// gamma (gamma- and gamma+); at a D-node, minus u at its gamma- neighbours
// (a node outside N+ has no gamma+ neighbour). gidx holds the unknown
// number of every gamma node.
__global__ void k_term_fill(const int* __restrict__ src, int ns, const uint8_t* __restrict__ flags, int N,
                            const int* __restrict__ gidx, const int* __restrict__ off, int layer, double s6,
                            int* __restrict__ tidx, double* __restrict__ tcoef) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        const int x = src[s];
        int e = off[s];
        const uint8_t f = flags[x];
        if ((f & 2) && layer == BAE_LAYER_DIRECT) {
            tidx[e] = gidx[x];
            tcoef[e] = s6;
            ++e;
            const int i = x / (N * N), j = (x / N) % N, k = x % N;
            for (int d = 0; d < 6; ++d) {
                const int y = ((i + c_dir[d][0]) * N + j + c_dir[d][1]) * N + k + c_dir[d][2];   // in the grid
                if (flags[y] & 6) {
                    tidx[e] = gidx[y];
                    tcoef[e] = -1.0;
                    ++e;
                }
            }
            continue;
        }
        if (f & 2) {
            const int c = f >> 4;
            tidx[e] = gidx[x];
            tcoef[e] = (layer == BAE_LAYER_DOUBLE && c > 0) ? (double)c : 1.0;
            continue;
        }
        const int i = x / (N * N), j = (x / N) % N, k = x % N;
        for (int d = 0; d < 6; ++d) {
            const int ii = i + c_dir[d][0], jj = j + c_dir[d][1], kk = k + c_dir[d][2];
            if (!in_grid(ii, jj, kk, N)) continue;
            const int y = (ii * N + jj) * N + kk;
            if (flags[y] & 2) {
                tidx[e] = gidx[y];
                tcoef[e] = -1.0;
                ++e;
            }
        }
    }
}

struct Scratch {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch() { for (void* p : ptrs) dev_free(p, st); }
    template <typename T> T* get(long long n) { T* p = dev_alloc_n<T>(n, st); ptrs.push_back(p); return p; }
};

// out[i] = nearest float32 of in[i]
__global__ void k_to_float(const double* __restrict__ in, long long n, float* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 32); }

// ------------------------------------------------- swapped convolution view
// out[swap_axes(x)] = in[x] over the N^3 grid. sw = 1 maps k-lines onto
// k-lines (a copy, grid-stride); sw = 2 transposes the (i, k) plane of
// every j through a 32 x 32 shared-memory tile (grid: k tiles, i tiles, j;
// 256 threads), so that reads and writes are both coalesced.
template <typename T>
__global__ void k_swap_grid(const T* __restrict__ in, T* __restrict__ out, int N, int sw) {
    if (sw == 1) {
        const long long n3 = (long long)N * N * N;
        for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n3; x += (long long)gridDim.x * blockDim.x)
            out[swap_axes(x, 1, N)] = in[x];
        return;
    }
    __shared__ T tile[32][33];
    const int j = blockIdx.z, i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, k = k0 + tx;
        if (i < N && k < N) tile[r][tx] = in[((long long)i * N + j) * N + k];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int k = k0 + r, i = i0 + tx;
        if (i < N && k < N) out[((long long)k * N + j) * N + i] = tile[tx][r];
    }
}

// smap[src_lin[s]] = s (smap preset to -1)
__global__ void k_src_map(const int* __restrict__ src_lin, int ns, int* __restrict__ smap) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) smap[src_lin[s]] = s;
}

// Per line of the swapped grid: the number of its sources (swapped flags &
// src_mask: the nodes the plain recipe lists) and of their terms.
__global__ void __launch_bounds__(LINE_T) k_view_count(const uint8_t* __restrict__ vflags, int N, int sw,
                                                      int src_mask, const int* __restrict__ smap,
                                                      const int* __restrict__ term_off, int* __restrict__ cnt_src,
                                                      int* __restrict__ cnt_term) {
    __shared__ int s_red[2][LINE_T / 32];
    const long long base = (long long)blockIdx.x * N;
    int c0 = 0, c1 = 0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int s = (vflags[base + k] & src_mask) ? smap[swap_axes(base + k, sw, N)] : -1;
        if (s >= 0) {   // every source node of the swapped flags is in the plain recipe
            c0 += 1;
            c1 += term_off[s + 1] - term_off[s];
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    c0 = __reduce_add_sync(0xffffffffu, c0);
    c1 = __reduce_add_sync(0xffffffffu, c1);
    if (lane == 0) {
        s_red[0][w] = c0;
        s_red[1][w] = c1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int t0 = 0, t1 = 0;
        for (int x = 0; x < (int)(blockDim.x >> 5); ++x) {
            t0 += s_red[0][x];
            t1 += s_red[1][x];
        }
        cnt_src[blockIdx.x] = t0;
        cnt_term[blockIdx.x] = t1;
    }
}

// The swapped recipe in lexicographic order of the swapped grid: per line,
// the CTA scans its sources (count in bits 0-10, terms from bit 11) from
// the line's offsets; vorig[pos] = the source's number in the plain recipe.
__global__ void __launch_bounds__(LINE_T) k_view_scatter(const uint8_t* __restrict__ vflags, int N, int sw,
                                                        int src_mask, const int* __restrict__ smap,
                                                        const int* __restrict__ term_off,
                                                        const int* __restrict__ off_src,
                                                        const int* __restrict__ off_term, int n_src, int n_terms,
                                                        int* __restrict__ vsrc_lin, int* __restrict__ vterm_off,
                                                        int* __restrict__ vorig) {
    __shared__ int s_warp[33];
    const int line = blockIdx.x;
    if (line == (int)gridDim.x - 1 && threadIdx.x == 0) vterm_off[n_src] = n_terms;
    int ps = off_src[line], pt = off_term[line];
    if (ps == off_src[line + 1]) return;   // no source on this line: the whole CTA
    const long long base = (long long)line * N;
    for (int k0 = 0; k0 < N; k0 += blockDim.x) {
        const int k = k0 + (int)threadIdx.x;
        int sf = 0, nt = 0, s = -1;
        if (k < N && (vflags[base + k] & src_mask)) s = smap[swap_axes(base + k, sw, N)];
        if (s >= 0) {   // the same nodes as k_view_count counts
            sf = 1;
            nt = term_off[s + 1] - term_off[s];
        }
        const int ex = block_exclusive_scan(sf | (nt << 11), s_warp);
        const int tot = s_warp[32];
        if (sf) {
            const int pos = ps + (ex & 2047);
            vsrc_lin[pos] = (int)(base + k);
            vterm_off[pos] = pt + (ex >> 11);
            vorig[pos] = s;
        }
        ps += tot & 2047;
        pt += tot >> 11;
    }
}

// the terms of swapped source pos: those of plain source vorig[pos]
__global__ void k_view_terms(const int* __restrict__ vorig, const int* __restrict__ vterm_off, int ns,
                             const int* __restrict__ term_off, const int* __restrict__ term_idx,
                             const double* __restrict__ term_coef, const float* __restrict__ term_coef32,
                             int* __restrict__ vidx, double* __restrict__ vcoef, float* __restrict__ vcoef32) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < ns; p += gridDim.x * blockDim.x) {
        const int s = vorig[p];
        if (s < 0 || s >= ns) continue;   // preset -1: a position no scatter wrote
        const int o = term_off[s], n = term_off[s + 1] - o, d = vterm_off[p];
        for (int e = 0; e < n; ++e) {
            vidx[d + e] = term_idx[o + e];
            vcoef[d + e] = term_coef[o + e];
            vcoef32[d + e] = term_coef32[o + e];
        }
    }
}

// out[r] = swap_axes(in[r])
__global__ void k_swap_index(const int* __restrict__ in, long long n, int N, int sw, int* __restrict__ out) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        out[r] = (int)swap_axes(in[r], sw, N);
}

// Builds the swapped view (Geometry::cv_*) of a built geometry.
void build_view(Geometry& g, int sw, int src_mask, Scratch& sc, cudaStream_t st) {
    const int N = g.N;
    const long long n3 = (long long)N * N * N, nl = (long long)N * N;
    g.cv_swap = sw;
    g.cv_lo = g.ext_lo[sw];
    g.cv_hi = g.ext_hi[sw];
    g.cv_flags = dev_alloc_n<uint8_t>(n3, st);
    if (sw == 1)
        BAE_LAUNCH("k_swap_grid", st, k_swap_grid<uint8_t><<<grid_for(n3), 256, 0, st>>>(g.flags, g.cv_flags, N, sw));
    else
        BAE_LAUNCH("k_swap_grid", st,
                   k_swap_grid<uint8_t><<<dim3(ceil_div(N, 32), ceil_div(N, 32), N), 256, 0, st>>>(g.flags, g.cv_flags,
                                                                                                   N, sw));
    int* smap = sc.get<int>(n3);
    BAE_CUDA(cudaMemsetAsync(smap, 0xff, n3 * sizeof(int), st));
    BAE_LAUNCH("k_src_map", st, k_src_map<<<grid_for(g.n_src), 256, 0, st>>>(g.src_lin, (int)g.n_src, smap));
    g.cv_line_off = dev_alloc_n<int>(nl + 1, st);   // per-line source counts, then their scan
    int* off_src = g.cv_line_off;
    int* off_term = sc.get<int>(nl + 1);
    int* info = sc.get<int>(I_COUNT);
    BAE_LAUNCH("k_view_count", st,
               k_view_count<<<(unsigned)nl, LINE_T, 0, st>>>(g.cv_flags, N, sw, src_mask, smap, g.term_off, off_src,
                                                             off_term));
    // blocks 0 and 1 scan the two counts (the other two arrays are not read)
    BAE_LAUNCH("k_scan_lines", st, k_scan_lines<<<2, 1024, 0, st>>>(off_src, off_term, off_src, off_term, (int)nl, info));
    g.cv_src_lin = dev_alloc_n<int>(g.n_src, st);
    g.cv_term_off = dev_alloc_n<int>(g.n_src + 1, st);
    int* vorig = sc.get<int>(std::max(1LL, g.n_src));
    BAE_CUDA(cudaMemsetAsync(vorig, 0xff, std::max(1LL, g.n_src) * sizeof(int), st));
    BAE_LAUNCH("k_view_scatter", st,
               k_view_scatter<<<(unsigned)nl, LINE_T, 0, st>>>(g.cv_flags, N, sw, src_mask, smap, g.term_off, off_src,
                                                               off_term, (int)g.n_src, (int)g.n_terms, g.cv_src_lin,
                                                               g.cv_term_off, vorig));
    g.cv_term_idx = dev_alloc_n<int>(g.n_terms, st);
    g.cv_term_coef = dev_alloc_n<double>(g.n_terms, st);
    g.cv_term_coef32 = dev_alloc_n<float>(g.n_terms, st);
    BAE_LAUNCH("k_view_terms", st,
               k_view_terms<<<grid_for(g.n_src), 256, 0, st>>>(vorig, g.cv_term_off, (int)g.n_src, g.term_off,
                                                               g.term_idx, g.term_coef, g.term_coef32, g.cv_term_idx,
                                                               g.cv_term_coef, g.cv_term_coef32));
    g.cv_gm = dev_alloc_n<int>(g.n_gm, st);
    g.cv_partner = dev_alloc_n<int>(g.n_gm, st);
    BAE_LAUNCH("k_swap_index", st, k_swap_index<<<grid_for(g.n_gm), 256, 0, st>>>(g.gm, g.n_gm, N, sw, g.cv_gm));
    BAE_LAUNCH("k_swap_index", st,
               k_swap_index<<<grid_for(g.n_gm), 256, 0, st>>>(g.partner, g.n_gm, N, sw, g.cv_partner));
}

}  // namespace

void Geometry::release() {
    void* ps[] = {flags,    gm,          gp,         node_of,     partner,      partner_u,   t,
                  xstar,    line_off,    src_lin,    term_off,    term_idx,     term_coef,   term_coef32,
                  cv_flags, cv_gm,       cv_partner, cv_line_off, cv_src_lin,   cv_term_off, cv_term_idx,
                  cv_term_coef, cv_term_coef32};
    for (void* p : ps) if (p) dev_free(p, stream);
    flags = nullptr; gm = gp = node_of = partner = partner_u = nullptr; t = xstar = nullptr;
    line_off = src_lin = term_off = term_idx = nullptr; term_coef = nullptr; term_coef32 = nullptr;
    cv_flags = nullptr; cv_gm = cv_partner = cv_line_off = cv_src_lin = cv_term_off = cv_term_idx = nullptr;
    cv_term_coef = nullptr; cv_term_coef32 = nullptr;
    cv_swap = 0;
}

void build_geometry(const double* phi, int N, double h, const double origin[3], int layer, double s, Geometry& g,
                    cudaStream_t st) {
    const long long n3 = (long long)N * N * N;
    Scratch sc(st);
    g.stream = st;
    g.N = N;
    g.h = h;
    for (int c = 0; c < 3; ++c) g.origin[c] = origin[c];
    g.layer = layer;

    const long long nl = (long long)N * N;
    int* info = sc.get<int>(I_COUNT);
    BAE_CUDA(cudaMemsetAsync(info, 0, I_COUNT * sizeof(int), st));
    uint8_t* nbits = sc.get<uint8_t>(n3);
    BAE_LAUNCH("k_nbits", st, k_nbits<<<(unsigned)nl, LINE_T, 0, st>>>(phi, N, nbits, info));
    const bool direct = layer == BAE_LAYER_DIRECT;
    // gamma- and D-nodes (double layer, direct formulation), or gamma- only
    const int src_mask = layer == BAE_LAYER_SINGLE ? 2 : (2 | 8);
    g.flags = dev_alloc_n<uint8_t>(n3, st);
    g.line_off = dev_alloc_n<int>(nl + 1, st);   // per-line source counts, then their scan
    int* off_gm = sc.get<int>(nl + 1);
    int* off_term = sc.get<int>(nl + 1);
    int* off_gp = sc.get<int>(nl + 1);
    BAE_LAUNCH("k_flags_lines", st,
               k_flags_lines<<<(unsigned)nl, LINE_T, 0, st>>>(nbits, N, src_mask, direct, g.flags, off_gm, g.line_off,
                                                              off_term, off_gp, info));
    BAE_LAUNCH("k_scan_lines", st, k_scan_lines<<<4, 1024, 0, st>>>(off_gm, g.line_off, off_term, off_gp, (int)nl, info));
    int rec[I_COUNT];
    BAE_CUDA(cudaMemcpyAsync(rec, info, sizeof(rec), cudaMemcpyDeviceToHost, st));
    BAE_CUDA(cudaStreamSynchronize(st));
    if (rec[I_ERR] & 1) throw Error(BAE_ERR_INVALID_ARG, "phi contains non-finite values");
    if (rec[I_ERR] & 2) throw Error(BAE_ERR_GEOMETRY, "M+ or gamma- reaches the faces of the grid box");
    g.n_gm = rec[I_NGM];
    g.n_src = rec[I_NSRC];
    g.n_terms = rec[I_NTERM];
    g.n_gp = rec[I_GP];
    g.n_mp = rec[I_MP];
    if (g.n_gm == 0) throw Error(BAE_ERR_GEOMETRY, "gamma- is empty (no interior node)");

    g.n_unk = direct ? g.n_gm + g.n_gp : g.n_gm;
    g.gm = dev_alloc_n<int>(g.n_gm, st);
    g.gp = dev_alloc_n<int>(std::max(1LL, g.n_gp), st);
    g.node_of = dev_alloc_n<int>(n3, st);
    g.src_lin = dev_alloc_n<int>(g.n_src, st);
    g.term_off = dev_alloc_n<int>(g.n_src + 1, st);
    BAE_LAUNCH("k_scatter_lines", st,
               k_scatter_lines<<<(unsigned)nl, LINE_T, 0, st>>>(g.flags, N, src_mask, direct, off_gm, g.line_off,
                                                                off_term, off_gp, info, g.gm, g.gp, g.node_of,
                                                                g.src_lin, g.term_off));
    // closure
    g.partner = dev_alloc_n<int>(g.n_gm, st);
    g.t = dev_alloc_n<double>(g.n_gm, st);
    g.xstar = dev_alloc_n<double>(3 * g.n_gm, st);
    BAE_LAUNCH("k_closure", st, k_closure<<<grid_for(g.n_gm), 256, 0, st>>>(phi, g.flags, g.gm, (int)g.n_gm, N, h, origin[0], origin[1], origin[2],
                                                g.partner, g.t, g.xstar));
    if (direct) {
        g.partner_u = dev_alloc_n<int>(g.n_gm, st);
        BAE_LAUNCH("k_partner_unknown", st,
                   k_partner_unknown<<<grid_for(g.n_gm), 256, 0, st>>>(g.partner, (int)g.n_gm, g.node_of, g.partner_u));
    }
    // source recipe
    g.term_idx = dev_alloc_n<int>(g.n_terms, st);
    g.term_coef = dev_alloc_n<double>(g.n_terms, st);
    BAE_LAUNCH("k_term_fill", st, k_term_fill<<<grid_for(g.n_src), 256, 0, st>>>(g.src_lin, (int)g.n_src, g.flags, N, g.node_of, g.term_off, layer,
                                                   6.0 + s, g.term_idx, g.term_coef));
    g.term_coef32 = dev_alloc_n<float>(g.n_terms, st);
    BAE_LAUNCH("k_to_float", st, k_to_float<<<grid_for(g.n_terms), 256, 0, st>>>(g.term_coef, g.n_terms, g.term_coef32));
    // planes holding every source (gamma- and D-nodes, or M+ for the
    // volume term, whose planes lie between) and every gathered node
    // (gamma- and the partners, one step from gamma-), along each axis
    const int slot[3][2] = {{I_FIRST, I_LAST}, {I_FIRSTY, I_LASTY}, {I_FIRSTZ, I_LASTZ}};
    for (int ax = 0; ax < 3; ++ax) {
        const long long first = N - rec[slot[ax][0]], last = rec[slot[ax][1]] - 1;
        g.ext_lo[ax] = (int)std::max(0LL, first - 1);
        g.ext_hi[ax] = (int)std::min((long long)N, last + 2);
    }
    g.plane_lo = g.ext_lo[0];
    g.plane_hi = g.ext_hi[0];
    // the axis of fewest planes (by more than a tenth) for the pruned
    // applies, which transform only the planes of their first axis
    const char* env = std::getenv("BAE_CONV_AXIS");
    const bool keep_x = env && (env[0] == 'x' || env[0] == 'X');
    int sw = 0;
    if (!direct && !keep_x)
        for (int ax = 1; ax < 3; ++ax)
            if (10 * (g.ext_hi[ax] - g.ext_lo[ax]) < 9 * (g.ext_hi[sw] - g.ext_lo[sw])) sw = ax;
    if (sw) build_view(g, sw, src_mask, sc, st);
}

}  // namespace bae
