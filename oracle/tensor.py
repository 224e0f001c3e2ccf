"""Example 2 of Section 6: a full tensor coefficient and a weighted mass (oracle; test
infrastructure, run only by tests/).

Forms (Section 6, Example 2): a(u, v) = (A grad u, grad v) with a smooth symmetric positive
definite A(x) and b(u, v) = (phi u, v) with a smooth weight phi(x) > 0. P1 elements on the
same structured triangulation as every other workload. Neither form is piecewise constant,
so the element integrals are taken by quadrature:
  K_T[i, j] = |T| sum_q w_q g_i . A(x_q) g_j,   M_T[i, j] = |T| sum_q w_q phi(x_q) l_i(q) l_j(q),
with g_i the (constant) barycentric gradients, l_i(q) the barycentric coordinates of point q,
and the 6-point rule of degree 4 of Dunavant (1985, Int. J. Numer. Meth. Eng. 21) below:
exact for polynomials of degree <= 4, so the quadrature error stays below the O(h^2)
eigenvalue error of P1.

The multilevel oracle (multilevel.py, multiple.py) works on assembled matrices: build()
returns the same Hierarchy with these K and M, and the one- and several-eigenpair forms of
Algorithms 4.1 / 4.2 run on it unchanged.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import workloads as W

from . import multilevel as ML
from .fem import element_geometry
from .mesh import Level, build_levels, interpolation
from .partition import level_partition, subdomains

# Dunavant's degree-4 rule: barycentric points (a, b, b) with their permutations, weights
# relative to the triangle's area.
_A1, _B1, _W1 = 0.108103018168070, 0.445948490915965, 0.223381589678011
_A2, _B2, _W2 = 0.816847572980459, 0.091576213509771, 0.109951743655322
QUAD_BARY = np.array([[_A1, _B1, _B1], [_B1, _A1, _B1], [_B1, _B1, _A1],
                      [_A2, _B2, _B2], [_B2, _A2, _B2], [_B2, _B2, _A2]])
QUAD_W = np.array([_W1, _W1, _W1, _W2, _W2, _W2])


def assemble(lv: Level, x0: float, y0: float, H: float, tensor, weight):
    """Global P1 stiffness of (A grad u, grad v) and mass of (phi u, v) over all nodes of lv;
    tensor(x, y) -> (a11, a12, a22), weight(x, y) -> phi (vectorised)."""
    coords = lv.xy(x0, y0, H)
    det, g = element_geometry(coords, lv.tris)
    area = 0.5 * np.abs(det)
    p = coords[lv.tris]                                   # (E, 3, 2)
    xq = np.einsum("qk,ekd->eqd", QUAD_BARY, p)           # (E, Q, 2) quadrature points
    a11, a12, a22 = tensor(xq[..., 0], xq[..., 1])        # (E, Q) each
    phi = weight(xq[..., 0], xq[..., 1])
    # integral of A over T: |T| sum_q w_q A(x_q)
    i11 = area * (a11 @ QUAD_W)
    i12 = area * (a12 @ QUAD_W)
    i22 = area * (a22 @ QUAD_W)
    gx, gy = g[:, :, 0], g[:, :, 1]
    Ke = (i11[:, None, None] * gx[:, :, None] * gx[:, None, :]
          + i12[:, None, None] * (gx[:, :, None] * gy[:, None, :] + gy[:, :, None] * gx[:, None, :])
          + i22[:, None, None] * gy[:, :, None] * gy[:, None, :])
    ll = np.einsum("qi,qj->qij", QUAD_BARY, QUAD_BARY)    # (Q, 3, 3) products of barycentric coordinates
    Me = area[:, None, None] * np.einsum("eq,qij->eij", phi * QUAD_W[None, :], ll)
    rows = np.repeat(lv.tris, 3, axis=1).ravel()
    cols = np.tile(lv.tris, (1, 3)).ravel()
    n = lv.nv
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))
    M = sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(n, n))
    K.sum_duplicates()
    M.sum_duplicates()
    return K, M


def build(problem: W.Problem, tensor, weight) -> ML.Hierarchy:
    """The multilevel hierarchy of `problem`'s mesh and partition with these forms."""
    n = problem.levels
    levels = build_levels(problem.cell_in, n, problem.H)
    K, M = [], []
    for lv in levels:
        k, m = assemble(lv, problem.x0, problem.y0, problem.H, tensor, weight)
        K.append(k)
        M.append(m)
    interp = [interpolation(levels[i], levels[i + 1]) for i in range(n)]
    hier = ML.Hierarchy(problem, 0, levels, K, M, interp)
    subs = subdomains(problem)
    for ell in range(2, n + 1):
        hier.parts[ell] = level_partition(problem, subs, levels[ell])
    hier.ones_int = [np.asarray(m.sum(axis=1)).ravel() for m in M]
    return hier


def example2_hierarchy(levels: int = 4, parts: int = 4) -> ML.Hierarchy:
    return build(W.example2(levels, parts), W.example2_tensor, W.example2_weight)
