"""Pins of the oracle's potentials (Section 3.2) and particular solution."""
import numpy as np
import pytest

import workloads as W
from oracle import fd, grid, lgf
from oracle import potentials as pot


def lattice_op(v, s):
    """(6+s) v - sum of the 6 neighbours, on interior nodes (zero on faces)."""
    out = np.zeros_like(v)
    c = (slice(1, -1),) * 3
    acc = (6.0 + s) * v[c]
    for ax in range(3):
        for st in (1, -1):
            acc = acc - np.roll(v, st, axis=ax)[c]
    out[c] = acc
    return out


@pytest.fixture(scope="module")
def sphere16():
    P = W.sphere_exp(16, radius=0.55, kappa2=10.0)
    cls = grid.classify(P.phi, P.grid.h, P.grid.origin)
    s = P.kappa2 * P.grid.h ** 2
    return P, cls, lgf.LGFTable(16, s), s


@pytest.mark.parametrize("layer", ["double", "single"])
def test_potential_lattice_harmonic_on_Mplus(sphere16, layer):
    # Propositions of Section 3.2: L_h v = 0 on M+ for both layers
    P, cls, T, s = sphere16
    q = W.random_density(cls.gm_idx.size, seed=1)
    all_idx = np.arange(16 ** 3)
    v = pot.direct_potential(T, cls, q, all_idx, layer).reshape((16,) * 3)
    r = lattice_op(v, s)
    assert np.max(np.abs(r[cls.inside])) < 1e-13 * np.max(np.abs(v))
    # and L_h v reproduces the source density rho = B q off M+
    rho = pot.source_density(cls, q, layer)
    inner = np.zeros_like(cls.inside)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.max(np.abs(r[inner] - rho[inner])) < 1e-12


def test_double_layer_from_definition(sphere16):
    # layer_matrix builds D(m,n) = sum_{k in D_n} [G(m-n) - G(m-k)] column by
    # column; D_n from the brute-force set definition
    P, cls, T, s = sphere16
    bf = grid.classify_bruteforce(P.phi)
    shape = (16,) * 3
    rng = np.random.default_rng(3)
    cols = rng.choice(cls.gm_idx.size, 8, replace=False)
    tg = rng.choice(16 ** 3, 50, replace=False)
    K = pot.layer_matrix(T, cls, tg, "double")
    for col in cols:
        n = tuple(int(v) for v in np.unravel_index(cls.gm_idx[col], shape))
        Dn = bf["D"][n]
        for r, t in enumerate(tg):
            m = np.array(np.unravel_index(t, shape))
            ref = sum(T(m - np.array(n)) - T(m - np.array(k)) for k in Dn) if Dn else T(m - np.array(n))
            assert K[r, col] == pytest.approx(ref, abs=1e-15)


def test_double_layer_diagonal_closed_form():
    # s = 0: D(n, n) = |D_n| (G(0) - G(e1)) = |D_n| / 6 by (6)G(0) - 6G(e1) = 1
    P = W.sphere_exp(12, radius=0.6)
    cls = grid.classify(P.phi, P.grid.h, P.grid.origin)
    T = lgf.LGFTable(12, 0.0)
    K = pot.layer_matrix(T, cls, cls.gm_idx, "double")
    c = cls.count.reshape(-1)[cls.gm_idx]
    d = np.diag(K)
    sel = c > 0
    assert np.max(np.abs(d[sel] - c[sel] / 6.0)) < 1e-14


@pytest.mark.parametrize("layer", ["double", "single"])
def test_direct_equals_fft(sphere16, layer):
    P, cls, T, s = sphere16
    q = W.random_density(cls.gm_idx.size, seed=2)
    all_idx = np.arange(16 ** 3)
    v_dir = pot.direct_potential(T, cls, q, all_idx, layer)
    v_fft = pot.fft_convolve(pot.source_density(cls, q, layer), table=T).reshape(-1)
    assert np.max(np.abs(v_dir - v_fft)) < 1e-12 * np.max(np.abs(v_dir))
    # layer_matrix (column by column) agrees with the source-density sum
    K = pot.layer_matrix(T, cls, cls.gm_idx, layer)
    assert np.max(np.abs(K @ q - v_dir[cls.gm_idx])) < 1e-12 * np.max(np.abs(v_dir))


def test_particular_solution_lattice_equation(sphere16):
    # eq. [ps] on the free lattice: (6+s) u_p - sum u_p(nbr) = h^2 f chi_{M+}
    P, cls, T, s = sphere16
    h = P.grid.h
    f = P.f()
    rho = (h * h) * np.where(cls.inside, f, 0.0)
    up = pot.fft_convolve(rho, table=T)
    r = lattice_op(up, s)
    inner = np.zeros_like(cls.inside)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.max(np.abs(r[inner] - rho[inner])) < 1e-13 * np.max(np.abs(rho))
    up_dir = pot.direct_particular(T, cls, f, h, cls.gm_idx)
    assert np.max(np.abs(up_dir - up.reshape(-1)[cls.gm_idx])) < 1e-12 * np.max(np.abs(up))


def test_dense_equivalence_of_boundary_maps():
    # Section 3.2: S+ S-^{-1} = D+ D-^{-1}, and both equal the gamma- -> gamma+
    # map of the lattice Dirichlet problem on M+ (solved here by sparse FD)
    P = W.sphere_exp(12, radius=0.6, kappa2=1.0)
    cls = grid.classify(P.phi, P.grid.h, P.grid.origin)
    s = P.kappa2 * P.grid.h ** 2
    T = lgf.LGFTable(12, s)
    Sp = pot.layer_matrix(T, cls, cls.gp_idx, "single")
    Sm = pot.layer_matrix(T, cls, cls.gm_idx, "single")
    Dp = pot.layer_matrix(T, cls, cls.gp_idx, "double")
    Dm = pot.layer_matrix(T, cls, cls.gm_idx, "double")
    MS = Sp @ np.linalg.inv(Sm)
    MD = Dp @ np.linalg.inv(Dm)
    assert np.max(np.abs(MS - MD)) < 1e-10
    rng = np.random.default_rng(4)
    vals = rng.standard_normal(cls.gm_idx.size)
    u = fd.harmonic_extension(cls, s, vals)
    assert np.max(np.abs(MS @ vals - u[cls.gp_idx])) < 1e-10


def test_single_layer_smallest_singular_value():
    # Theorem of Section 3.3: every singular value of S- is >= 1/12
    for N, rad in ((12, 0.6), (16, 0.5)):
        P = W.sphere_exp(N, radius=rad)
        cls = grid.classify(P.phi, P.grid.h, P.grid.origin)
        T = lgf.LGFTable(N, 0.0)
        Sm = pot.layer_matrix(T, cls, cls.gm_idx, "single")
        assert np.allclose(Sm, Sm.T, atol=0)
        assert np.linalg.svd(Sm, compute_uv=False).min() >= 1.0 / 12.0


# ------------------------------------------ finite-box particular solution
def _box_sparse(f, h, s, inside):
    """eq. [aux] with q = chi_{M+} f assembled as a sparse system over the box
    nodes M0 = [1, N-1]^3 (u = 0 on the layers 0 and N) and solved directly."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    N = f.shape[0]
    n = N - 1
    idx = np.arange(n ** 3).reshape(n, n, n)
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                r = idx[i, j, k]
                rows.append(r), cols.append(r), vals.append(6.0 + s)
                for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    a, b, c = i + d[0], j + d[1], k + d[2]
                    if 0 <= a < n and 0 <= b < n and 0 <= c < n:
                        rows.append(r), cols.append(idx[a, b, c]), vals.append(-1.0)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n ** 3, n ** 3))
    rhs = (h * h) * np.where(inside, f, 0.0)[1:, 1:, 1:].reshape(-1)
    u = np.zeros((N, N, N))
    u[1:, 1:, 1:] = spl.spsolve(A.tocsc(), rhs).reshape(n, n, n)
    return u


@pytest.mark.parametrize("kappa2", [0.0, 10.0])
def test_box_particular_solves_aux_problem(kappa2):
    # eq. [aux]: the difference equation on M0 and zero on the box layer, and
    # the same values as a sparse direct solve of that system
    P = W.sphere_exp(8, radius=0.55, kappa2=kappa2)
    h, s = P.grid.h, kappa2 * P.grid.h ** 2
    inside = P.phi < 0
    f = P.f()
    u = pot.box_particular(f, h, s, inside)
    assert np.all(u[0, :, :] == 0) and np.all(u[:, 0, :] == 0) and np.all(u[:, :, 0] == 0)
    ext = np.zeros((9, 9, 9))                  # append the zero layer N
    ext[:8, :8, :8] = u
    r = lattice_op(ext, s)[1:8, 1:8, 1:8]
    rhs = (h * h) * np.where(inside, f, 0.0)[1:, 1:, 1:]
    assert np.max(np.abs(r - rhs)) <= 1e-13 * np.max(np.abs(rhs))
    ref = _box_sparse(f, h, s, inside)
    assert np.max(np.abs(u - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_box_particular_route_equals_fd():
    # Algorithm 1 with the finite-box particular solution: a different
    # density, the same discrete solution on N+ as the sparse FD system
    from oracle import solve as S
    P = W.torus_helmholtz(16, kappa2=10.0)
    r = S.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2, tol=1e-13, potential="fft",
                particular="box")
    u_fd, cls = S.solve_fd(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2)
    m = cls.nplus
    assert np.max(np.abs(r.u[m] - u_fd[m])) <= 1e-11 * np.max(np.abs(u_fd[m]))
    r0 = S.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2, tol=1e-13, potential="fft")
    assert np.max(np.abs(r.q - r0.q)) > 1e-6 * np.max(np.abs(r0.q))   # the densities differ


@pytest.mark.parametrize("s", [0.0, 0.5])
@pytest.mark.parametrize("perm", [(1, 0, 2), (2, 1, 0)])
def test_lattice_convolution_commutes_with_axis_swaps(s, perm):
    # The GPU convolution may run on the grid with two axes swapped and be
    # read back through the swap: that rests on G_s being symmetric under
    # permutations of the axes, so that G * (rho o P) = (G * rho) o P. The
    # plain lattice sum on the original grid, with G by quadrature of eq.
    # [lgf_bessel] at each signed, unsorted offset (no symmetry assumed), is
    # compared with the FFT route on the swapped grid read back at the
    # swapped node.
    N = 12
    rng = np.random.default_rng(7)
    rho = np.zeros((N, N, N))
    idx = rng.integers(2, N - 2, size=(24, 3))
    rho[idx[:, 0], idx[:, 1], idx[:, 2]] = rng.standard_normal(24)
    T = lgf.LGFTable(N, s)
    v_swapped = pot.fft_convolve(np.ascontiguousarray(np.transpose(rho, perm)), table=T)
    src = np.argwhere(rho != 0)
    for m in rng.integers(0, N, size=(5, 3)):
        direct = sum(rho[tuple(x)] * lgf.lgf_entry(tuple(int(v) for v in m - x), s) for x in src)
        mp = tuple(int(m[a]) for a in perm)   # node m seen on the swapped grid
        assert v_swapped[mp] == pytest.approx(direct, rel=1e-11, abs=1e-13)
