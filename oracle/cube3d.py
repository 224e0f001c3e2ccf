"""The method for d = 3 on box domains (oracle; test infrastructure, run only by tests/).

Section 2.1 admits shape-regular tetrahedral meshes for d = 3, and Section 4.2 builds the
level sequence by regular refinement into beta^d congruent children (beta = 2 here). The
steps of Algorithms 4.1 and 4.2 do not depend on d: this module builds the d = 3 hierarchy
and runs the multilevel oracle (multilevel.py; multiple.py for several eigenpairs) on it
unchanged. There is no GPU path for d = 3.

Readings (the paper runs no d = 3 case):
* T_H: the box of W.Box3 in cubes of side H, each cut into the six Kuhn (Freudenthal)
  tetrahedra around its main diagonal, with vertices c, c + e_a, c + e_a + e_b, c + (1, 1, 1)
  for the six orders (a, b, .) of the axes. Halving the lattice splits every Kuhn
  tetrahedron into 8 congruent Kuhn tetrahedra (Freudenthal's subdivision), so T_{h_k} is
  the regular refinement of T_{h_{k-1}} and the P1 spaces are nested; a fine node
  2p + s (s in {0, 1}^3) is the midpoint of the coarse edge from p to p + s.
* D_j: the parts^3 equal boxes of coarse cubes; Omega_j: D_j dilated by o cubes in every
  direction and clipped to the box; closed G_j: the free nodes of closure(D_j) at distance
  >= delta from every face of D_j inside the box (for a box D_j that is the Chebyshev
  distance to dD_j minus dOmega); delta a multiple of H/4, as for d = 2.
* Forms: a(u, v) = (grad u, grad v), b(u, v) = (u, v).
"""
from __future__ import annotations

from dataclasses import dataclass
from itertools import permutations

import numpy as np
import scipy.sparse as sp

import workloads as W

from . import multilevel as ML
from . import multiple as MU
from .partition import LevelPartition


@dataclass
class Level3:
    ell: int
    res: int                 # lattice cells per side of a coarse cube (2^ell)
    nx: int
    ny: int
    nz: int
    pts: np.ndarray          # (nv, 3) int64 lattice coordinates (x fastest in the node index)
    tets: np.ndarray         # (E, 4) node indices
    boundary: np.ndarray     # (nv,) bool: on the surface of the box

    @property
    def nv(self) -> int:
        return self.pts.shape[0]

    def index(self, q) -> np.ndarray:
        q = np.asarray(q, np.int64)
        return (q[..., 2] * (self.ny + 1) + q[..., 1]) * (self.nx + 1) + q[..., 0]


# the first two axes of each of the six orders of (x, y, z)
_KUHN = [(a, b) for a, b, _ in permutations(range(3))]


def build_level(box: W.Box3, ell: int) -> Level3:
    """Nodes, Kuhn tetrahedra and surface nodes of lattice level ell (h = H / 2^ell)."""
    res = 1 << ell
    nx, ny, nz = (n * res for n in box.nc)
    z, y, x = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.int64)
    top = np.array([nx, ny, nz])
    boundary = np.any((pts == 0) | (pts == top), axis=1)
    cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    corner = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1).astype(np.int64)
    lv = Level3(ell, res, nx, ny, nz, pts, np.empty((0, 4), np.int64), boundary)
    eye = np.eye(3, dtype=np.int64)
    tets = []
    for a, b in _KUHN:
        v1 = corner + eye[a]
        v2 = v1 + eye[b]
        tets.append(np.stack([lv.index(corner), lv.index(v1), lv.index(v2), lv.index(corner + 1)], axis=1))
    lv.tets = np.concatenate(tets)
    return lv


def assemble(lv: Level3, H: float):
    """P1 stiffness and mass over all nodes of a level: per tetrahedron with volume V and
    barycentric gradients g_i, K_e = V g_i . g_j and M_e = V (1 + delta_ij) / 20."""
    X = lv.pts[lv.tets].astype(np.float64) * (H / lv.res)           # (E, 4, 3)
    Ed = X[:, 1:] - X[:, :1]                                         # rows: edge vectors from vertex 0
    vol = np.abs(np.linalg.det(Ed)) / 6.0
    # x - X_0 = Ed^T xi, so the gradient of xi_i is column i of Ed^{-1}
    g = np.empty((Ed.shape[0], 4, 3))
    g[:, 1:] = np.transpose(np.linalg.inv(Ed), (0, 2, 1))
    g[:, 0] = -g[:, 1:].sum(axis=1)
    Ke = vol[:, None, None] * np.einsum("eid,ejd->eij", g, g)
    Me = (vol / 20.0)[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None]
    rows = np.repeat(lv.tets, 4, axis=1).ravel()
    cols = np.tile(lv.tets, (1, 4)).ravel()
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(lv.nv, lv.nv))
    M = sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(lv.nv, lv.nv))
    K.sum_duplicates()
    M.sum_duplicates()
    return K, M


def interpolation(coarse: Level3, fine: Level3) -> sp.csr_matrix:
    """Exact embedding V_{h_l} -> V_{h_{l+1}}: fine node 2p + s takes the mean of the coarse
    values at p and p + s (both p when s = 0)."""
    q = fine.pts
    s = q & 1
    cols = np.stack([coarse.index((q - s) >> 1), coarse.index((q + s) >> 1)], axis=1).ravel()
    rows = np.repeat(np.arange(fine.nv), 2)
    P = sp.csr_matrix((np.full(2 * fine.nv, 0.5), (rows, cols)), shape=(fine.nv, coarse.nv))
    P.sum_duplicates()
    return P


def subdomain_boxes(box: W.Box3):
    """(D_j low, D_j high, Omega_j low, Omega_j high) in coarse-cube coordinates, j = 0..parts^3-1."""
    nc = np.array(box.nc)
    w = nc // box.parts
    out = []
    for kz in range(box.parts):
        for ky in range(box.parts):
            for kx in range(box.parts):
                lo = np.array([kx, ky, kz]) * w
                hi = lo + w
                out.append((lo, hi, np.maximum(lo - box.overlap, 0), np.minimum(hi + box.overlap, nc)))
    return out


def level_partition(box: W.Box3, lv: Level3) -> LevelPartition:
    """Unknowns of every Omega_j, the closed G_j and the G_{m+1} unknowns on one level."""
    free = ~lv.boundary
    delta_lat = box.delta / box.H * lv.res
    if lv.ell >= 2 and abs(delta_lat - round(delta_lat)) > 1e-9:
        raise ValueError("delta must be a multiple of H/4")
    nc = np.array(box.nc)
    q = lv.pts
    local, gn = [], []
    in_g = np.full(lv.nv, -1, np.int64)
    for j, (lo, hi, olo, ohi) in enumerate(subdomain_boxes(box)):
        loc = np.nonzero(np.all((q > olo * lv.res) & (q < ohi * lv.res), axis=1))[0]
        d0, d1 = lo * lv.res, hi * lv.res
        in_d = np.all((q >= d0) & (q <= d1), axis=1) & free
        dist = np.full(lv.nv, np.inf)
        for ax in range(3):                     # faces of D_j that lie inside the box
            if lo[ax] > 0:
                dist = np.minimum(dist, q[:, ax] - d0[ax])
            if hi[ax] < nc[ax]:
                dist = np.minimum(dist, d1[ax] - q[:, ax])
        g = np.nonzero(in_d & (dist >= delta_lat - 1e-9))[0]
        if np.any(in_g[g] >= 0):
            raise ValueError("closed G_j overlap: delta too small for the partition")
        in_g[g] = j
        assert np.all(np.isin(g, loc)), "closed G_j must lie inside the unknowns of Omega_j"
        local.append(loc)
        gn.append(g)
    strip = np.nonzero(free & (in_g < 0))[0]
    return LevelPartition(free, local, gn, strip)


def build(box: W.Box3) -> ML.Hierarchy:
    """The d = 3 hierarchy T_H = T_{h_0}, ..., T_{h_n} in the form multilevel.py takes."""
    n = box.levels
    levels = [build_level(box, ell) for ell in range(n + 1)]
    K, M = [], []
    for lv in levels:
        k, m = assemble(lv, box.H)
        K.append(k)
        M.append(m)
    interp = [interpolation(levels[ell], levels[ell + 1]) for ell in range(n)]
    hier = ML.Hierarchy(box, 0, levels, K, M, interp)
    for ell in range(2, n + 1):
        hier.parts[ell] = level_partition(box, levels[ell])
    hier.ones_int = [np.asarray(m.sum(axis=1)).ravel() for m in M]
    return hier


@dataclass
class Result3:
    lam: float                 # lambda_{h_n}
    u: np.ndarray              # u_{h_n} over all nodes of level n (zero on the surface)
    lam_levels: list           # lambda_{h_k}, k = 1..n


def solve(box: W.Box3, hier: ML.Hierarchy | None = None) -> Result3:
    """Algorithm 4.2 in d = 3: the level-1 eigenproblem, then one correction per level."""
    hier = hier or build(box)
    lam, u = ML.global_eigpair(hier, 1)
    lams = [lam]
    for k in range(1, box.levels):
        lam, u = ML.correction(hier, k, lam, u)
        lams.append(lam)
    return Result3(lam, u, lams)


def solve_multi(box: W.Box3, q: int, hier: ML.Hierarchy | None = None):
    """The q smallest eigenpairs by the subspace form (multiple.py): (lams, U, lam_levels)."""
    hier = hier or build(box)
    lams, U = MU.global_eigpairs(hier, 1, q)
    levels = [lams]
    for k in range(1, box.levels):
        lams, U = MU.correction_multi(hier, k, lams, U)
        levels.append(lams)
    return lams, U, np.array(levels)
