"""P1 bilinear forms a(u,v) = (kappa grad u, grad v) and b(u,v) = (u, v) (oracle).

Paper: Section 2.2 (L u = -div(A grad u), a(u,v) = (A grad u, grad v); here A = kappa I
with kappa constant on each triangle), Section 3 (b(u,v) = (u,v)).

Element matrices are the textbook P1 ones: with the barycentric gradients g_i of a
triangle T of area |T|, K_T[i,j] = kappa_T |T| g_i . g_j and M_T[i,j] = |T| (1 + [i=j]) / 12.
The global matrices are assembled over ALL nodes; Dirichlet conditions are imposed by
restricting to the free (non-boundary) nodes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import workloads as W

from .mesh import Level


def element_geometry(coords: np.ndarray, tris: np.ndarray):
    """Signed-area determinant and barycentric gradients of every triangle."""
    p = coords[tris]  # (E, 3, 2)
    x1, y1 = p[:, 0, 0], p[:, 0, 1]
    x2, y2 = p[:, 1, 0], p[:, 1, 1]
    x3, y3 = p[:, 2, 0], p[:, 2, 1]
    det = (x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1)
    g = np.empty((tris.shape[0], 3, 2))
    g[:, 0, 0], g[:, 0, 1] = (y2 - y3) / det, (x3 - x2) / det
    g[:, 1, 0], g[:, 1, 1] = (y3 - y1) / det, (x1 - x3) / det
    g[:, 2, 0], g[:, 2, 1] = (y1 - y2) / det, (x2 - x1) / det
    return det, g


def assemble(lv: Level, kappa_elem: np.ndarray, H: float):
    """Global P1 stiffness K (with kappa per triangle) and consistent mass M over all nodes of lv."""
    coords = lv.pts.astype(np.float64) * (H / lv.res)
    det, g = element_geometry(coords, lv.tris)
    area = 0.5 * np.abs(det)
    Ke = (kappa_elem * area)[:, None, None] * np.einsum("eid,ejd->eij", g, g)
    Me = (area / 12.0)[:, None, None] * (np.ones((3, 3)) + np.eye(3))[None]
    rows = np.repeat(lv.tris, 3, axis=1).ravel()
    cols = np.tile(lv.tris, (1, 3)).ravel()
    n = lv.nv
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))
    M = sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(n, n))
    K.sum_duplicates()
    M.sum_duplicates()
    return K, M


def finest_elem_kappa(problem: W.Problem, lv: Level, b: int) -> np.ndarray:
    """kappa on each triangle of the level at which the problem's kappa is given."""
    if problem.kappa_kind == W.KAPPA_ONE:
        return np.ones(lv.tris.shape[0])
    if problem.kappa_kind == W.KAPPA_PER_COARSE_CELL:
        kc = problem.kappa[b].ravel()
        return kc[lv.cell]
    if problem.kappa_kind == W.KAPPA_PER_FINE_ELEM:
        # identify each finest triangle geometrically: its cell is the lattice square at the
        # minimum corner; it is the lower one iff it contains the cell's SE corner.
        tp = lv.tri_pts
        lo = tp.min(axis=1)
        se = lo + np.array([1, 0])
        is_lower = np.any(np.all(tp == se[:, None, :], axis=2), axis=1)
        t = np.where(is_lower, 0, 1)
        return problem.kappa[b][lo[:, 1], lo[:, 0], t]
    raise ValueError("unknown kappa kind")


def kappa_all_levels(problem: W.Problem, levels: list[Level], b: int) -> list[np.ndarray]:
    """kappa per triangle on every level.

    Reading of Section 2.2 / 4.2 for a coefficient given on T_{h_n}: the form a(.,.) is the
    exact one, so on a coarser triangle (whose P1 functions have constant gradient there)
    the effective coefficient is the area mean of kappa over the triangle's descendants.
    Regular refinement gives 4 children of equal area, so each level is the mean of its
    children on the next level (children of triangle e are 4e .. 4e+3).
    """
    n = len(levels) - 1
    out = [None] * (n + 1)
    if problem.kappa_kind == W.KAPPA_PER_FINE_ELEM:
        out[n] = finest_elem_kappa(problem, levels[n], b)
        for ell in range(n - 1, -1, -1):
            out[ell] = out[ell + 1].reshape(-1, 4).mean(axis=1)
    else:
        for ell in range(n + 1):
            out[ell] = finest_elem_kappa(problem, levels[ell], b)
    return out


def node_integrals(lv: Level, H: float) -> np.ndarray:
    """int_Omega phi_x for every nodal basis function (row sums of the consistent mass)."""
    _, M = assemble(lv, np.ones(lv.tris.shape[0]), H)
    return np.asarray(M.sum(axis=1)).ravel()
