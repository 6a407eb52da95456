"""The schedules of the FFT convolution inside the potential apply
(Section 3.2: the discrete potentials as lattice sums with the LGF): five
separate transform passes, the same with the second launch geometry
(float32: half-width column blocks at N = 128, the three-level transform at
N = 256), the five passes as persistent kernels over all right-hand sides,
or the k and j transforms fused per x-plane (one CTA per plane
where the plane fits in shared memory, a thread-block cluster sharing it
through distributed shared memory where it does not: float32 at N = 256,
float64 and double-float at N >= 128). Every schedule the autotuner can
pick is here.

Each schedule is forced in turn and compared with the oracle: its FFT
convolution at N = 64, and at N = 256 plain sums over the nonzero sources at
sampled targets, with LGF values from the oracle's quadrature. The N = 128
case is in test_gpu_fullsize.py. A batched solve at N = 256 runs the cluster
kernels with several right-hand sides inside the captured GMRES graph."""
import numpy as np
import pytest

import workloads as W
from oracle import grid as OG
from oracle import lgf as OL
from oracle import potentials as OP

pytestmark = pytest.mark.gpu

TOL = {"fp32": 2e-6, "fp64": 1e-12, "df64": 1e-12}


@pytest.fixture
def schedule():
    from paper_2502_05507_gb300 import set_conv_schedule
    yield set_conv_schedule
    set_conv_schedule("auto")


def _gpu(P, layer="double"):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_05507_gb300 import Context, Problem
    ctx = Context(0)
    prob = Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, layer)
    return ctx, prob


def _apply(prob, q, precision):
    import torch
    return prob.potential_apply(torch.from_numpy(q).cuda(), precision).cpu().numpy().reshape(-1)


@pytest.mark.parametrize("precision", ["fp32", "fp64", "df64"])
def test_schedules_n64_vs_oracle_fft(schedule, precision):
    P = W.torus_helmholtz(64, kappa2=10.0)
    s = P.kappa2 * P.grid.h ** 2
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    q = W.random_density(cls.gm_idx.size, seed=41)
    spec = OP.lgf_spectrum(OL.LGFTable(64, s))
    ref = OP.fft_convolve(OP.source_density(cls, q, "double"), spectrum=spec, workers=-1).reshape(-1)
    scale = np.max(np.abs(ref))
    ctx, prob = _gpu(P)
    try:
        out = {}
        for name in ("passes", "passes_alt", "persist", "plane"):
            schedule(name)
            out[name] = _apply(prob, q, precision)
            assert np.max(np.abs(out[name] - ref)) <= TOL[precision] * scale, name
        # same convolution, different rounding order only
        assert np.max(np.abs(out["passes"] - out["plane"])) <= TOL[precision] * scale
    finally:
        prob.close()
        ctx.close()


def _sampled_direct(cls, q, targets, s, layer="double"):
    """v at the targets as the plain sum over the nonzero source nodes, with
    G_s from the oracle's quadrature at exactly the offsets needed."""
    N = cls.N
    shape = (N, N, N)
    rho = OP.source_density(cls, q, layer).reshape(-1)
    nz = np.flatnonzero(rho)
    src = np.stack(np.unravel_index(nz, shape), axis=1)
    tg = np.stack(np.unravel_index(np.asarray(targets), shape), axis=1)
    off = (tg[:, None, :] - src[None, :, :]).reshape(-1, 3)
    canon, inv = np.unique(np.sort(np.abs(off), axis=1), axis=0, return_inverse=True)
    G = OL.lgf_triples(canon, s)[inv.reshape(-1)].reshape(len(tg), len(nz))
    return G @ rho[nz], nz


@pytest.mark.parametrize("kappa2", [0.0, 1.0])
def test_schedules_n256_vs_sampled_direct_sums(schedule, kappa2):
    P = W.star(256, kappa2=kappa2)
    s = P.kappa2 * P.grid.h ** 2
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    rng = np.random.default_rng(43)
    q = np.zeros(cls.gm_idx.size)
    q[rng.choice(q.size, 10, replace=False)] = rng.standard_normal(10)
    rho = OP.source_density(cls, q, "double").reshape(-1)
    nz = np.flatnonzero(rho)
    # the source nodes (where |v| peaks), random N+ nodes, gamma- nodes
    targets = np.concatenate([nz, rng.choice(np.flatnonzero(cls.nplus), 60, replace=False),
                              rng.choice(cls.gm_idx, 20, replace=False)])
    ref, _ = _sampled_direct(cls, q, targets, s)
    scale = np.max(np.abs(ref))
    ctx, prob = _gpu(P)
    try:
        full = {}
        for precision in ("fp32", "fp64", "df64"):
            for name in ("passes", "passes_alt", "persist", "plane"):
                schedule(name)
                v = _apply(prob, q, precision)
                err = np.max(np.abs(v[targets] - ref))
                assert err <= TOL[precision] * scale, (precision, name, err / scale)
                full[precision, name] = v
            for other in ("passes_alt", "persist", "plane"):
                d = np.max(np.abs(full[precision, "passes"] - full[precision, other]))
                assert d <= TOL[precision] * scale, (precision, other, d / scale)
    finally:
        prob.close()
        ctx.close()


def test_batched_solve_n256_cluster_schedule(schedule):
    """Two right-hand sides at N = 256 in mixed precision: the inner float32
    GMRES applies run the cluster kernels with two batch items inside the
    captured graph; both schedules converge to the same solution."""
    import torch
    P = W.star(256, kappa2=1.0)
    ctx, prob = _gpu(P)
    try:
        xyz = np.asarray(prob.boundary_points())
        g1 = P.g_at(xyz)
        g2 = np.sin(xyz[:, 0]) * np.exp(0.5 * xyz[:, 1]) + xyz[:, 2] ** 2
        f = np.stack([P.f(), np.zeros_like(P.f())])
        g = np.stack([g1, g2])
        res = {}
        for name in ("passes", "passes_alt", "persist", "plane"):
            schedule(name)
            q, u, st = prob.solve_batched(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), tol=1e-10,
                                          precision="mixed")
            for s_ in st:
                assert s_["rel_residual"] <= 1e-10, s_
            res[name] = u.cpu().numpy()
        mp = OG.classify(P.phi, P.grid.h, P.grid.origin).inside.reshape(-1)
        for b in range(2):
            a = res["passes"][b].reshape(-1)[mp]
            c = res["plane"][b].reshape(-1)[mp]
            assert np.max(np.abs(a - c)) <= 1e-8 * np.max(np.abs(a)), b
    finally:
        prob.close()
        ctx.close()
