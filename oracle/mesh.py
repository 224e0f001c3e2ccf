"""Triangulations T_H, T_{h_1}, ..., T_{h_n} and nodal interpolation (oracle).

Paper: Section 2.1 (shape-regular triangulation, P_k spaces), Section 4.2
(T_{h_1} from T_H by regular refinement, T_{h_k} from T_{h_{k-1}} by regular
refinement producing beta^d congruent elements, beta = 2), Section 6 (beta = 2,
"connecting the midpoints of each edge").

Reading (no mesh is given in the paper): T_H splits every in-domain square cell
of side H by its SW-NE diagonal. Points are kept as integer lattice coordinates
in units of H / 2^level from the grid origin, so all geometry is exact.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Level:
    ell: int                 # refinement level; 0 is T_H, k is T_{h_k} with h_k = H / 2^k
    res: int                 # lattice points per coarse cell side (2^ell)
    nx: int                  # lattice extent in x (ncx * res)
    ny: int
    tri_pts: np.ndarray      # (E, 3, 2) int64 lattice coordinates of each triangle, counter-clockwise
    tris: np.ndarray         # (E, 3) node indices
    pts: np.ndarray          # (Nv, 2) int64 lattice coordinates of the nodes
    cell: np.ndarray         # (E,) flat coarse cell index (cj * ncx + ci) of each triangle's T_H ancestor
    boundary: np.ndarray     # (Nv,) bool, node lies on the boundary of Omega
    h: float                 # mesh size (leg length) H / 2^ell

    @property
    def nv(self) -> int:
        return self.pts.shape[0]

    def key(self, p: np.ndarray) -> np.ndarray:
        return p[..., 1] * (self.nx + 1) + p[..., 0]

    def xy(self, x0: float, y0: float, H: float) -> np.ndarray:
        return np.stack([x0 + self.pts[:, 0] * (H / self.res), y0 + self.pts[:, 1] * (H / self.res)], axis=1)


def coarse_triangles(cell_in: np.ndarray):
    """Two triangles per in-domain cell: lower (ci,cj),(ci+1,cj),(ci+1,cj+1); upper (ci,cj),(ci+1,cj+1),(ci,cj+1)."""
    ncy, ncx = cell_in.shape
    cj, ci = np.nonzero(cell_in)
    flat = cj * ncx + ci
    p00 = np.stack([ci, cj], 1)
    p10 = np.stack([ci + 1, cj], 1)
    p11 = np.stack([ci + 1, cj + 1], 1)
    p01 = np.stack([ci, cj + 1], 1)
    lower = np.stack([p00, p10, p11], 1)
    upper = np.stack([p00, p11, p01], 1)
    tri = np.empty((2 * ci.size, 3, 2), np.int64)
    tri[0::2] = lower
    tri[1::2] = upper
    cell = np.repeat(flat, 2)
    return tri, cell


def red_refine(tri_pts: np.ndarray) -> np.ndarray:
    """Regular refinement: each triangle (A,B,C) -> 4 congruent children through the edge midpoints.

    Lattice resolution doubles, so A -> 2A and the midpoint of AB -> A + B. Child c of
    triangle e gets index 4e + c, children order: (A,ab,ca), (ab,B,bc), (ca,bc,C), (ab,bc,ca).
    """
    A, B, C = tri_pts[:, 0], tri_pts[:, 1], tri_pts[:, 2]
    A2, B2, C2 = 2 * A, 2 * B, 2 * C
    ab, bc, ca = A + B, B + C, C + A
    kids = np.stack([
        np.stack([A2, ab, ca], 1),
        np.stack([ab, B2, bc], 1),
        np.stack([ca, bc, C2], 1),
        np.stack([ab, bc, ca], 1),
    ], 1)  # (E, 4, 3, 2)
    return kids.reshape(-1, 3, 2)


def _edges(tris: np.ndarray):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]], 0)
    e.sort(axis=1)
    return e


def boundary_nodes(tris: np.ndarray, nv: int) -> np.ndarray:
    """Nodes on an edge that belongs to exactly one triangle of the collection."""
    e = _edges(tris)
    uniq, cnt = np.unique(e, axis=0, return_counts=True)
    bnd = np.zeros(nv, bool)
    bnd[uniq[cnt == 1].ravel()] = True
    return bnd


def _make_level(ell: int, ncx: int, ncy: int, tri_pts: np.ndarray, cell: np.ndarray, H: float) -> Level:
    res = 1 << ell
    nx, ny = ncx * res, ncy * res
    keys = tri_pts[..., 1] * (nx + 1) + tri_pts[..., 0]
    uk, inv = np.unique(keys.ravel(), return_inverse=True)
    tris = inv.reshape(-1, 3).astype(np.int64)
    pts = np.stack([uk % (nx + 1), uk // (nx + 1)], 1).astype(np.int64)
    bnd = boundary_nodes(tris, pts.shape[0])
    return Level(ell, res, nx, ny, tri_pts, tris, pts, cell, bnd, H / res)


def build_levels(cell_in: np.ndarray, n: int, H: float) -> list[Level]:
    """T_H (level 0) and its n successive regular refinements."""
    ncy, ncx = cell_in.shape
    tri, cell = coarse_triangles(cell_in)
    out = [_make_level(0, ncx, ncy, tri, cell, H)]
    for ell in range(1, n + 1):
        tri = red_refine(tri)
        cell = np.repeat(cell, 4)
        out.append(_make_level(ell, ncx, ncy, tri, cell, H))
    return out


def interpolation(coarse: Level, fine: Level) -> sp.csr_matrix:
    """Nodal interpolation V_{h_l} -> V_{h_{l+1}} (all nodes): exact for P1 because the spaces are nested.

    A fine node that is a coarse node keeps its value; a fine node at the midpoint of a
    coarse edge gets the mean of the edge's two end values (the P1 function is linear
    along the edge).
    """
    # coarse node c sits at fine lattice point 2 * pts[c]
    old_rows = node_index(fine, 2 * coarse.pts)
    e = np.unique(_edges(coarse.tris), axis=0)
    mid_rows = node_index(fine, coarse.pts[e[:, 0]] + coarse.pts[e[:, 1]])
    rows = np.concatenate([old_rows, mid_rows, mid_rows])
    cols = np.concatenate([np.arange(coarse.nv), e[:, 0], e[:, 1]])
    vals = np.concatenate([np.ones(coarse.nv), np.full(e.shape[0], 0.5), np.full(e.shape[0], 0.5)])
    assert np.unique(rows).size == fine.nv, "every fine node must be a coarse node or an edge midpoint"
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.nv, coarse.nv))


def node_index(lv: Level, p: np.ndarray) -> np.ndarray:
    """Index of the node at lattice point(s) p; raises if a point is not a node of the level."""
    keys = lv.key(lv.pts)  # sorted: nodes come out of np.unique
    q = lv.key(np.asarray(p, np.int64))
    idx = np.searchsorted(keys, q)
    if np.any(idx >= keys.size) or np.any(keys[np.minimum(idx, keys.size - 1)] != q):
        raise KeyError("lattice point is not a node of this level")
    return idx.astype(np.int64)


def node_grid_index(lv: Level) -> np.ndarray:
    """Flat index j * (nx + 1) + i of each node in the full (ny+1) x (nx+1) lattice."""
    return lv.key(lv.pts)
