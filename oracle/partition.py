"""Domain decomposition D_j, Omega_j, G_j and G_{m+1} (oracle).

Paper: Section 4, the paragraph before Algorithm 4.1: disjoint D_1..D_m covering Omega;
Omega_j enlarges D_j and aligns with T_H; G_j is compactly contained in D_j
(G subset-subset D means dist(dD \\ dOmega, dG \\ dOmega) > 0, Section 2); and
G_{m+1} = Omega minus the union of the closed G_j.

Readings (the paper gives the sets only in a figure):
* Omega_j = in-domain coarse cells within Chebyshev cell distance o_j of D_j.
* G_j = { x in closure(D_j) : dist_inf(x, dD_j \\ dOmega) >= delta }, a closed set; delta is
  the paper's inset parameter of Section 6 and must be a multiple of H/4 so that G_j aligns
  with T_{h_2}, the first level on which a correction runs.
* A node of T_{h_k} belongs to closed G_j by the distance test above; the unknowns of the
  G_{m+1} problem are the free nodes of Omega that belong to no closed G_j.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import workloads as W

from .mesh import Level, boundary_nodes


def _dilate(mask: np.ndarray, r: int) -> np.ndarray:
    """Chebyshev dilation of a boolean cell mask by r cells (no wrap-around)."""
    out = mask.copy()
    ny, nx = mask.shape
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            src = mask[max(0, -dy):ny - max(0, dy), max(0, -dx):nx - max(0, dx)]
            out[max(0, dy):ny - max(0, -dy), max(0, dx):nx - max(0, -dx)] |= src
    return out


@dataclass
class Subdomain:
    j: int
    d_cells: np.ndarray        # bool [ncy, ncx]: D_j
    omega_cells: np.ndarray    # bool [ncy, ncx]: Omega_j
    interface: np.ndarray      # (s, 2, 2) int64 coarse-lattice segments of dD_j \ dOmega


def subdomains(p: W.Problem) -> list[Subdomain]:
    inside = p.cell_in.astype(bool)
    out = []
    ncy, ncx = inside.shape
    for j in range(p.m):
        d = p.cell_owner == j
        if not d.any():
            raise ValueError(f"subdomain {j} owns no cell")
        om = _dilate(d, int(p.overlap[j])) & inside
        segs = []
        cj, ci = np.nonzero(d)
        for x, y in zip(ci, cj):
            # the four sides of cell (x, y) with the neighbour across each side
            for (nxc, nyc), seg in (((x, y - 1), ((x, y), (x + 1, y))), ((x, y + 1), ((x, y + 1), (x + 1, y + 1))),
                                    ((x - 1, y), ((x, y), (x, y + 1))), ((x + 1, y), ((x + 1, y), (x + 1, y + 1)))):
                if 0 <= nxc < ncx and 0 <= nyc < ncy and inside[nyc, nxc] and not d[nyc, nxc]:
                    segs.append(seg)
        out.append(Subdomain(j, d, om, np.array(segs, np.int64).reshape(-1, 2, 2)))
    return out


def dist_inf_to_segments(pts: np.ndarray, segs: np.ndarray) -> np.ndarray:
    """Chebyshev distance from points to a union of axis-parallel segments (same lattice units)."""
    if segs.shape[0] == 0:
        return np.full(pts.shape[0], np.inf)
    px = pts[:, 0][:, None].astype(np.float64)
    py = pts[:, 1][:, None].astype(np.float64)
    ax, ay = segs[:, 0, 0][None], segs[:, 0, 1][None]
    bx, by = segs[:, 1, 0][None], segs[:, 1, 1][None]
    dx = np.maximum(np.maximum(np.minimum(ax, bx) - px, px - np.maximum(ax, bx)), 0.0)
    dy = np.maximum(np.maximum(np.minimum(ay, by) - py, py - np.maximum(ay, by)), 0.0)
    return np.maximum(dx, dy).min(axis=1)


@dataclass
class LevelPartition:
    free: np.ndarray              # (Nv,) bool: free nodes of Omega (not on dOmega)
    local: list[np.ndarray]       # per j: node indices of the free nodes of Omega_j (unknowns of step 1)
    g_nodes: list[np.ndarray]     # per j: node indices in closed G_j (excluding dOmega)
    strip: np.ndarray             # node indices of the unknowns of the G_{m+1} problem


def level_partition(p: W.Problem, subs: list[Subdomain], lv: Level) -> LevelPartition:
    free = ~lv.boundary
    ncx = p.ncx
    local, gn = [], []
    delta_lat = p.delta / p.H * lv.res
    if lv.ell >= 2 and abs(delta_lat - round(delta_lat)) > 1e-9:
        raise ValueError("delta must be a multiple of H/4")
    in_g = np.zeros(lv.nv, np.int64) - 1
    for s in subs:
        om = s.omega_cells.ravel()[lv.cell]
        tri_j = lv.tris[om]
        nodes_j = np.unique(tri_j)
        bnd_j = boundary_nodes(tri_j, lv.nv)
        loc = nodes_j[~bnd_j[nodes_j]]
        local.append(loc)
        dm = s.d_cells.ravel()[lv.cell]
        dn = np.unique(lv.tris[dm])                     # nodes of closure(D_j)
        dist = dist_inf_to_segments(lv.pts[dn], s.interface * lv.res)
        g = dn[(dist >= delta_lat - 1e-9) & free[dn]]
        if np.any(in_g[g] >= 0):
            raise ValueError("closed G_j overlap: delta too small for the partition")
        in_g[g] = s.j
        gn.append(g)
        assert np.all(np.isin(g, loc)), "closed G_j must lie inside the unknowns of Omega_j"
    strip = np.nonzero(free & (in_g < 0))[0]
    return LevelPartition(free, local, gn, strip)
