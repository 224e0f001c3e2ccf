"""P2 (quadratic) elements for Example 1's forms (oracle; test infrastructure, run only by
tests/).

Section 6 runs Example 1 with linear and with quadratic elements: with P2 the algorithm keeps
its structure, the spaces V_{h_k}, V_{0H} and the local spaces become the quadratic Lagrange
spaces on the same triangulations, and the eigenvalue errors fall at O(h^4) (the paper's
figure for the quadratic element). Forms: a(u, v) = (grad u, grad v), b(u, v) = (u, v).

Construction: the P2 nodes of T_{h_l} (vertices and edge midpoints) are exactly the vertices of
the once-refined triangulation T_{h_{l+1}}, so P2 level l uses the node set (and Level object)
of lattice level l + 1. The partition's node sets (Omega_j, closed G_j, G_{m+1}) are taken on
that node set by the same geometric rules as for P1, and the multilevel oracles (multilevel.py,
multiple.py) run on the hierarchy unchanged.

Element matrices: the six quadratic Lagrange functions on a triangle in barycentric
coordinates, phi_i = l_i (2 l_i - 1) at the vertices and phi_ij = 4 l_i l_j at the edge
midpoints, integrated by Dunavant's rule of degree 4 (exact for the mass, degree 4, and the
stiffness, degree 2). Interpolation from level l to l + 1 evaluates the six functions of each
level-l triangle at the fine nodes it contains (exact: the spaces are nested).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import workloads as W

from . import multilevel as ML
from .fem import element_geometry
from .mesh import Level, build_levels, node_index
from .partition import level_partition, subdomains
from .tensor import QUAD_BARY, QUAD_W

# local node order of a triangle: vertices 0, 1, 2, then midpoints of edges 01, 12, 20
_EDGES = ((0, 1), (1, 2), (2, 0))


def shape(lam: np.ndarray):
    """Values (..., 6) of the six P2 functions at barycentric points lam (..., 3), and their
    derivatives (..., 6, 3) with respect to the three barycentric coordinates."""
    val = np.empty(lam.shape[:-1] + (6,))
    der = np.zeros(lam.shape[:-1] + (6, 3))
    for i in range(3):
        val[..., i] = lam[..., i] * (2.0 * lam[..., i] - 1.0)
        der[..., i, i] = 4.0 * lam[..., i] - 1.0
    for m, (a, b) in enumerate(_EDGES):
        val[..., 3 + m] = 4.0 * lam[..., a] * lam[..., b]
        der[..., 3 + m, a] = 4.0 * lam[..., b]
        der[..., 3 + m, b] = 4.0 * lam[..., a]
    return val, der


def element_nodes(coarse: Level, nodes: Level) -> np.ndarray:
    """(E, 6) indices in `nodes` (lattice level l + 1) of the P2 nodes of each triangle of
    `coarse` (lattice level l), in the local order above."""
    v = 2 * coarse.tri_pts                         # vertices in the finer lattice's coordinates
    mids = [coarse.tri_pts[:, a] + coarse.tri_pts[:, b] for a, b in _EDGES]
    pts = np.concatenate([v, np.stack(mids, axis=1)], axis=1)   # (E, 6, 2)
    return node_index(nodes, pts.reshape(-1, 2)).reshape(-1, 6)


def assemble(coarse: Level, nodes: Level, H: float):
    """Global P2 stiffness and mass over all P2 nodes of level l (the nodes of lattice level
    l + 1) from the triangles of lattice level l."""
    E = coarse.tri_pts.shape[0]
    coords = coarse.tri_pts.reshape(-1, 2).astype(np.float64) * (H / coarse.res)
    det, g = element_geometry(coords, np.arange(3 * E).reshape(E, 3))   # g: (E, 3, 2) grad of l_k
    area = 0.5 * np.abs(det)
    val, der = shape(QUAD_BARY)                                        # (Q, 6), (Q, 6, 3)
    grad = np.einsum("qak,ekd->eqad", der, g)                          # (E, Q, 6, 2)
    Ke = area[:, None, None] * np.einsum("q,eqad,eqbd->eab", QUAD_W, grad, grad)
    Me = area[:, None, None] * np.einsum("q,qa,qb->ab", QUAD_W, val, val)[None]
    idx = element_nodes(coarse, nodes)
    rows = np.repeat(idx, 6, axis=1).ravel()
    cols = np.tile(idx, (1, 6)).ravel()
    n = nodes.nv
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))
    M = sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(n, n))
    K.sum_duplicates()
    M.sum_duplicates()
    return K, M


def interpolation(coarse: Level, nodes: Level, fine_nodes: Level) -> sp.csr_matrix:
    """Interpolation from P2 on lattice level l (nodes: lattice l + 1) to P2 on level l + 1
    (nodes: lattice l + 2): every fine node inside a level-l triangle takes the value of that
    triangle's quadratic there (the 15 fine nodes of a triangle have barycentric coordinates
    (a, b, c) / 4, a + b + c = 4)."""
    idx = element_nodes(coarse, nodes)                                 # (E, 6)
    bary = np.array([(a, b, 4 - a - b) for a in range(5) for b in range(5 - a)], np.int64)  # (15, 3)
    val, _ = shape(bary / 4.0)                                         # (15, 6)
    pts4 = 4 * coarse.tri_pts                                          # vertices in lattice l + 2
    fine_pts = np.einsum("pk,ekd->epd", bary, pts4) // 4              # (E, 15, 2), exact integers
    frow = node_index(fine_nodes, fine_pts.reshape(-1, 2)).reshape(-1, 15)
    # a fine node on a shared edge or vertex gets the same value from every triangle: keep one
    first = np.unique(frow.ravel(), return_index=True)[1]
    e_of = first // 15
    p_of = first % 15
    assert first.size == fine_nodes.nv, "every fine node lies in some coarse triangle"
    rows = np.repeat(frow.ravel()[first], 6)
    cols = idx[e_of].ravel()
    vals = val[p_of].ravel()
    P = sp.csr_matrix((vals, (rows, cols)), shape=(fine_nodes.nv, nodes.nv))
    P.eliminate_zeros()
    return P


def build(problem: W.Problem) -> ML.Hierarchy:
    """The multilevel hierarchy of `problem` (kappa = 1 only) with P2 spaces: level l uses the
    triangles of lattice level l and the nodes of lattice level l + 1."""
    if problem.kappa_kind != W.KAPPA_ONE:
        raise ValueError("the P2 oracle takes kappa = 1 (Example 1)")
    n = problem.levels
    lat = build_levels(problem.cell_in, n + 2, problem.H)
    levels = [lat[l + 1] for l in range(n + 1)]
    K, M = [], []
    for l in range(n + 1):
        k, m = assemble(lat[l], lat[l + 1], problem.H)
        K.append(k)
        M.append(m)
    interp = [interpolation(lat[l], lat[l + 1], lat[l + 2]) for l in range(n)]
    hier = ML.Hierarchy(problem, 0, levels, K, M, interp)
    subs = subdomains(problem)
    for l in range(2, n + 1):
        hier.parts[l] = level_partition(problem, subs, levels[l])
    hier.ones_int = [np.asarray(m.sum(axis=1)).ravel() for m in M]
    return hier
