"""Point sets and the Dirichlet closure (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 2.1: M+ are the grid nodes inside Omega, M- the rest of the grid;
N+- are the 7-point stencils of M+-; gamma = N+ n N-, gamma+ = gamma n M+,
gamma- = gamma n M-. Section 3.2: D_n is the set of neighbours of a source
node n in gamma- that lie outside N+. Section 4.2 states that phi < 0 is the
interior; a node with phi == 0 is exterior.

Closure (eq. [bc], second-order hat functions; the paper does not say which
boundary point x* each row uses). Reading taken here: every node m in gamma-
has a row; among its six neighbours p in M+ (tested in the order +x, -x, +y,
-y, +z, -z, x being array axis 0) take the one whose linear zero crossing of
phi along the edge m-p lies closest to m, i.e. the largest
    t = phi(p) / (phi(p) - phi(m))  in (0, 1],
the first one on ties. x* = x_p + t (x_m - x_p) and the hat basis on that
edge gives the row  t v(m) + (1 - t) v(p) = g(x*).

Geometry check: no M+ or gamma- node may lie on a face of the grid box, so
that N+ and every D_n stay inside the N^3 grid.

Parity: classify() is pinned against classify_bruteforce(), which builds the
same sets from the paper's set definitions with Python sets on tiny grids.
The closure choice itself is a reading ("parity unpinned" beyond agreement
with the paper's error tables, see tests/test_oracle_solve.py).
"""
from __future__ import annotations

import dataclasses

import numpy as np

# neighbour order used everywhere: +x, -x, +y, -y, +z, -z (x = axis 0 = i)
DIRS = ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))


class GeometryError(ValueError):
    pass


def _shifted(mask: np.ndarray, d, outside_value: bool) -> np.ndarray:
    """out[x] = mask[x + d], with outside_value where x + d leaves the grid."""
    N = mask.shape[0]
    out = np.full(mask.shape, outside_value, dtype=bool)
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    for ax in range(3):
        if d[ax] == 1:
            src[ax], dst[ax] = slice(1, N), slice(0, N - 1)
        elif d[ax] == -1:
            src[ax], dst[ax] = slice(0, N - 1), slice(1, N)
    out[tuple(dst)] = mask[tuple(src)]
    return out


@dataclasses.dataclass
class Classification:
    N: int
    inside: np.ndarray     # M+ mask, N^3 bool
    gm: np.ndarray         # gamma- mask
    gp: np.ndarray         # gamma+ mask
    nplus: np.ndarray      # N+ mask = M+ u gamma-
    dnode: np.ndarray      # nodes outside N+ adjacent to some gamma- node
    count: np.ndarray      # |D_n| on every node (0 off gamma-), int
    gm_idx: np.ndarray     # linear indices of gamma-, lexicographic
    gp_idx: np.ndarray
    mp_idx: np.ndarray     # linear indices of M+
    partner: np.ndarray    # closure partner p(m) (linear index), per gamma- node
    t: np.ndarray          # closure weight t(m) on v(m), per gamma- node
    xstar: np.ndarray      # (n_gm, 3) boundary points x*


def classify(phi: np.ndarray, h: float, origin: float, check_geometry: bool = True) -> Classification:
    phi = np.asarray(phi, dtype=np.float64)
    N = phi.shape[0]
    inside = phi < 0.0
    has_in_nb = np.zeros_like(inside)
    has_out_nb = np.zeros_like(inside)
    for d in DIRS:
        has_in_nb |= _shifted(inside, d, False)
        has_out_nb |= _shifted(~inside, d, True)
    gm = ~inside & has_in_nb
    gp = inside & has_out_nb
    nplus = inside | gm
    count = np.zeros(phi.shape, dtype=np.int64)
    dnode = np.zeros_like(inside)
    for d in DIRS:
        count += (gm & ~_shifted(nplus, d, False)).astype(np.int64)
        dnode |= _shifted(gm, d, False)
    dnode &= ~nplus

    gm_idx = np.flatnonzero(gm)
    if check_geometry:
        if gm_idx.size == 0:
            raise GeometryError("empty gamma-: no interior node")
        ijk = np.stack(np.unravel_index(np.concatenate([gm_idx, np.flatnonzero(inside)]), phi.shape), axis=1)
        if (ijk.min() < 1) or (ijk.max() > N - 2):
            raise GeometryError("M+ or gamma- touches the grid box faces")

    # closure partner and weight
    ijk = np.stack(np.unravel_index(gm_idx, phi.shape), axis=1)
    pm = phi.reshape(-1)[gm_idx]
    tcand = np.full((6, gm_idx.size), -np.inf)
    pcand = np.zeros((6, gm_idx.size), dtype=np.int64)
    for di, d in enumerate(DIRS):
        q = ijk + np.array(d)
        ok = np.all((q >= 0) & (q < N), axis=1)
        qc = np.clip(q, 0, N - 1)
        lin = np.ravel_multi_index(qc.T, phi.shape)
        pp = phi.reshape(-1)[lin]
        isin = ok & (pp < 0.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            tt = pp / (pp - pm)
        tcand[di] = np.where(isin, tt, -np.inf)
        pcand[di] = lin
    best = np.argmax(tcand, axis=0)  # first maximum = tie-break in DIRS order
    cols = np.arange(gm_idx.size)
    t = tcand[best, cols]
    partner = pcand[best, cols]

    # boundary points x* = x_p + t (x_m - x_p), evaluated componentwise
    ip = np.stack(np.unravel_index(partner, phi.shape), axis=1).astype(np.float64)
    im = ijk.astype(np.float64)
    xp = origin + ip * h
    xm = origin + im * h
    xstar = xp + t[:, None] * (xm - xp)

    return Classification(N=N, inside=inside, gm=gm, gp=gp, nplus=nplus, dnode=dnode, count=count,
                          gm_idx=gm_idx, gp_idx=np.flatnonzero(gp), mp_idx=np.flatnonzero(inside),
                          partner=partner, t=t, xstar=xstar)


def classify_bruteforce(phi: np.ndarray):
    """The point sets of Section 2.1 straight from their definitions, with
    Python sets of index triples. For tiny grids only. Returns a dict of
    sorted lists plus |D_n| per gamma- node."""
    phi = np.asarray(phi)
    N = phi.shape[0]
    nodes = [(i, j, k) for i in range(N) for j in range(N) for k in range(N)]
    Mp = {x for x in nodes if phi[x] < 0}
    Mm = {x for x in nodes if x not in Mp}

    def stencil(x):
        i, j, k = x
        return {(i, j, k), (i + 1, j, k), (i - 1, j, k), (i, j + 1, k), (i, j - 1, k), (i, j, k + 1), (i, j, k - 1)}

    Np = set().union(*(stencil(x) for x in Mp)) if Mp else set()
    Nm = set().union(*(stencil(x) for x in Mm)) if Mm else set()
    gamma = Np & Nm
    gp = gamma & Mp
    gm = gamma & Mm
    D = {n: sorted(y for y in stencil(n) - {n} if y not in Np) for n in gm}
    dn = set().union(*D.values()) if D else set()
    return dict(Mp=sorted(Mp), gm=sorted(gm), gp=sorted(gp), Np=sorted(Np), D=D, dnodes=sorted(dn))
