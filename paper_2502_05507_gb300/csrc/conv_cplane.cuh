// Cluster plane kernels of the potential apply (see CPlaneGeo in
// conv_geo.cuh): instantiated per element type in conv_cplane_*.cu so they
// compile in parallel with the other passes.
#pragma once

#include <cooperative_groups.h>

#include "conv_geo.cuh"

namespace cg = cooperative_groups;

namespace bae {

namespace {


template <typename T, int L>
__global__ void __launch_bounds__(CPlaneGeo<T, L>::PT) k_cplane_fwd(ConvArgs<T> a) {
    wait_prior_grid();   // no-op: launched without programmatic serialisation
    using C = cplx_t<T>;
    using G = CPlaneGeo<T, L>;
    constexpr int N = G::N, N1 = G::N1, R1 = G::R1, R2 = G::R2, Q = R2 / R1, NR = G::NR;
    static_assert(NR % R1 == 0, "a CTA's rows must hold whole R1 groups");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* rows = reinterpret_cast<C*>(smem_raw);                 // [NR][N1]
    C* xch = reinterpret_cast<C*>(smem_raw + G::ROWS);
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int i = a.plane_lo() + (int)(blockIdx.x / G::CS);
    const int b = blockIdx.y;
    const bool skip = a.active && !a.active[b];               // uniform over the cluster

    if (!skip) {   // ---- own k lines: rows j = r NR + jl
        const int t = threadIdx.x % R1, p = threadIdx.x / R1;
        for (int round = 0; round < G::ROUNDS; ++round) {
            const int pr = round * G::PP + p;
            const bool act = pr < NR / 2;
            const int jla = 2 * pr, jlb = jla + 1;
            const long long la = (long long)i * N + r * NR + jla, lb = la + 1;
            C v[R2];
            if (a.mode == SRC_DENSITY) {
                T* ra = reinterpret_cast<T*>(rows + (long long)(act ? jla : 0) * N1);
                T* rb = reinterpret_cast<T*>(rows + (long long)(act ? jlb : 0) * N1);
                if (act)
                    for (int k = t; k < N; k += R1) {
                        ra[k] = volume_or_zero(a, b, la * N + k);
                        rb[k] = volume_or_zero(a, b, lb * N + k);
                    }
                __syncthreads();
                if (act) {
                    const double* q = a.q + (long long)b * a.q_stride + (a.q_row ? (long long)a.q_row[b] * a.q_row_stride : 0);
                    const float* q32 = a.q32 ? a.q32 + (long long)b * a.q32_stride : nullptr;
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const long long l = half ? lb : la;
                        T* rr = half ? rb : ra;
                        const int s0 = a.rec.line_off[l], s1 = a.rec.line_off[l + 1];
                        for (int s = s0 + t; s < s1; s += R1) {
                            const int k = a.rec.src_lin[s] - (int)(l * N);
                            rr[k] = source_value<T>(a.rec, s, q, q32);
                        }
                    }
                }
                __syncthreads();
#pragma unroll
                for (int m = 0; m < R2; ++m) {
                    const int n = t + R1 * m;
                    v[m] = (act && m < R2 / 2) ? cmake<C>(ra[n], rb[n]) : cmake<C>((T)0.0, (T)0.0);
                }
            } else {
                const double* f = a.f + (long long)b * N * N * N;
#pragma unroll
                for (int m = 0; m < R2; ++m) {
                    const int n = t + R1 * m;
                    T va = (T)0.0, vb = (T)0.0;
                    if (act && m < R2 / 2) {
                        const long long xa = la * N + n, xb = lb * N + n;
                        va = (a.flags[xa] & 1) ? (T)(a.scale * f[swap_axes(xa, a.f_swap, N)]) : (T)0.0;
                        vb = (a.flags[xb] & 1) ? (T)(a.scale * f[swap_axes(xb, a.f_swap, N)]) : (T)0.0;
                    }
                    v[m] = cmake<C>(va, vb);
                }
            }
            const int base = p * G::XS;
            fft_n2k<L, false, true>(v, xch, base, R1 + 1, 1, t, a.tw);
            C* z = xch + base;
#pragma unroll
            for (int q2 = 0; q2 < Q; ++q2)
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) z[t + q2 * R1 + R2 * k1] = v[q2 * R1 + k1];
            __syncthreads();
            if (act) {
                for (int k = t; k < N; k += R1) {
                    C xa, xb;
                    split_lines(z, k, L, xa, xb);
                    rows[(long long)jla * N1 + k] = xa;
                    rows[(long long)jlb * N1 + k] = xb;
                }
            }
            __syncthreads();
        }
    }
    cluster.sync();
    if (!skip) {   // ---- own share of the j columns, rows from the whole cluster
        const int c = threadIdx.x % G::PW, t = threadIdx.x / G::PW;
        C* out = a.B + (long long)b * N * (2 * N) * N1 + (long long)i * (2 * N) * N1;
        const C* part[G::CS];
#pragma unroll
        for (int q = 0; q < G::CS; ++q) part[q] = cluster.map_shared_rank(rows, q);
        const int cbeg = r * G::CW, cend = cbeg + G::CW;
        for (int col0 = cbeg; col0 < cend; col0 += G::PW) {
            const int col = col0 + c;
            const bool ok = col < cend;
            C v[R2];
#pragma unroll
            for (int m = 0; m < R2; ++m) {
                // n = t + R1 m < N exactly when m < R2 / 2 (t < R1, R1 R2 = 2N); row n
                // lives in CTA (R1 m) / NR (R1 divides NR)
                constexpr int HALF = R2 / 2;
                const int n = t + R1 * m;
                const int owner = m < HALF ? (R1 * m) / NR : 0;
                v[m] = (ok && m < HALF) ? part[owner][(long long)(n - owner * NR) * N1 + col] : cmake<C>((T)0.0, (T)0.0);
            }
            fft_n2k<L, false, true>(v, xch, c, R1 * G::PW, G::PW, t, a.tw);
            if (col0 == 0) split_column0<Plan2<L>, L>(v, xch, c, t);
            if (ok) {
#pragma unroll
                for (int q2 = 0; q2 < Q; ++q2)
#pragma unroll
                    for (int k1 = 0; k1 < R1; ++k1)
                        out[(long long)(t + q2 * R1 + R2 * k1) * N1 + col] = v[q2 * R1 + k1];
            }
        }
    }
    cluster.sync();   // no CTA leaves while others may still read its rows
}

template <typename T, int L>
__global__ void __launch_bounds__(CPlaneGeo<T, L>::PT) k_cplane_inv(ConvArgs<T> a) {
    wait_prior_grid();   // no-op: launched without programmatic serialisation
    using C = cplx_t<T>;
    using G = CPlaneGeo<T, L>;
    constexpr int N = G::N, N1 = G::N1, R1 = G::R1, R2 = G::R2, Q = R2 / R1, NR = G::NR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* rows = reinterpret_cast<C*>(smem_raw);
    C* xch = reinterpret_cast<C*>(smem_raw + G::ROWS);
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int i = a.plane_lo() + (int)(blockIdx.x / G::CS);
    const int b = blockIdx.y;
    const bool skip = a.active && !a.active[b];
    static_assert(NR % R1 == 0, "a CTA's rows must hold whole R1 groups");
    cluster.sync();   // every CTA of the cluster runs before any remote write

    if (!skip) {   // ---- inverse j on own columns, rows j < N into their owners
        const int c = threadIdx.x % G::PW, t = threadIdx.x / G::PW;
        const C* in = a.B + (long long)b * N * (2 * N) * N1 + (long long)i * (2 * N) * N1;
        C* part[G::CS];
#pragma unroll
        for (int q = 0; q < G::CS; ++q) part[q] = cluster.map_shared_rank(rows, q);
        const int cbeg = r * G::CW, cend = cbeg + G::CW;
        for (int col0 = cbeg; col0 < cend; col0 += G::PW) {
            const int col = col0 + c;
            const bool ok = col < cend;
            C v[R2];
#pragma unroll
            for (int q2 = 0; q2 < Q; ++q2)
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) {
                    const int k = t + q2 * R1 + R2 * k1;
                    C x = ok ? in[(long long)k * N1 + col] : cmake<C>((T)0.0, (T)0.0);
                    if (col == 0) x = slot_merge(x, in[(long long)((L - k) & (L - 1)) * N1], k, N);
                    v[q2 * R1 + k1] = x;
                }
            fft_k2n<L, true>(v, xch, c, R1 * G::PW, G::PW, t, a.tw);
            if (ok) {
#pragma unroll
                for (int m = 0; m < R2; ++m) {
                    const int n = t + R1 * m;   // < N exactly when m < R2 / 2
                    const int owner = m < R2 / 2 ? (R1 * m) / NR : 0;
                    if (m < R2 / 2) part[owner][(long long)(n - owner * NR) * N1 + col] = v[m];
                }
            }
        }
    }
    cluster.sync();   // every row of this CTA is written
    if (!skip) {   // ---- C2R of own rows
        const int t = threadIdx.x % R1, p = threadIdx.x / R1;
        auto* out = a.v + (long long)b * N * N * N;
        for (int round = 0; round < G::ROUNDS; ++round) {
            const int pr = round * G::PP + p;
            const bool act = pr < NR / 2;
            const int jla = act ? 2 * pr : 0, jlb = jla + 1;
            const long long la = (long long)i * N + r * NR + jla, lb = la + 1;
            C v[R2];
#pragma unroll
            for (int q2 = 0; q2 < Q; ++q2)
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) {
                    const int k = t + q2 * R1 + R2 * k1;
                    C xa = cmake<C>((T)0.0, (T)0.0), xb = xa;
                    if (act) {
                        xa = line_spectrum(rows + (long long)jla * N1, k, N);
                        xb = line_spectrum(rows + (long long)jlb * N1, k, N);
                    }
                    v[q2 * R1 + k1] = cmake<C>(xa.x - xb.y, xa.y + xb.x);
                }
            fft_k2n<L, true>(v, xch, p * G::XS, R1 + 1, 1, t, a.tw);
            if (act) {
#pragma unroll
                for (int m = 0; m < R2; ++m) {
                    const int n = t + R1 * m;
                    if (m < R2 / 2) {
                        out[la * N + n] = to_out(v[m].x);
                        out[lb * N + n] = to_out(v[m].y);
                    }
                }
            }
        }
    }
}

// launch with a (cs, 1, 1) thread-block cluster
template <typename K, typename A>
void launch_cluster(K kernel, int cs, dim3 grid, int threads, size_t smem, cudaStream_t st, const A& a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BAE_CUDA(cudaLaunchKernelEx(&cfg, kernel, a));
}

// whether the device can place one cluster of the cluster-plane kernels
// (CS CTAs of ~200 KB shared memory each within one GPC)
template <typename T, int L>
bool cplane_ok() {
    static const bool ok = []() {
        using G = CPlaneGeo<T, L>;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(G::CS * (L / 2), 1);
        cfg.blockDim = dim3(G::PT);
        cfg.dynamicSmemBytes = G::SMEM;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = G::CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_cplane_fwd<T, L>, &cfg) != cudaSuccess) n = 0;
        int m = 0;
        if (n > 0 && cudaOccupancyMaxActiveClusters(&m, k_cplane_inv<T, L>, &cfg) != cudaSuccess) m = 0;
        cudaGetLastError();
        return n > 0 && m > 0;
    }();
    return ok;
}

}  // namespace

template <typename T, int L>
bool cplane_ready() {
    using G = CPlaneGeo<T, L>;
    static const bool ok = []() {
        BAE_CUDA(cudaFuncSetAttribute(k_cplane_fwd<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM));
        BAE_CUDA(cudaFuncSetAttribute(k_cplane_inv<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM));
        return cplane_ok<T, L>();
    }();
    return ok;
}

template <typename T, int L>
void cplane_launch(const ConvArgs<T>& a, cudaStream_t st, bool inverse) {
    using G = CPlaneGeo<T, L>;
    const dim3 grid(G::CS * (a.plane_hi() - a.plane_lo()), a.nbatch);
    if (!inverse)
        BAE_LAUNCH(kname<T>("conv_cplane_fwd.f32", "conv_cplane_fwd.f64", "conv_cplane_fwd.df64"), st,
                   launch_cluster(k_cplane_fwd<T, L>, G::CS, grid, G::PT, G::SMEM, st, a));
    else
        BAE_LAUNCH(kname<T>("conv_cplane_inv.f32", "conv_cplane_inv.f64", "conv_cplane_inv.df64"), st,
                   launch_cluster(k_cplane_inv<T, L>, G::CS, grid, G::PT, G::SMEM, st, a));
}

}  // namespace bae
