"""Seeded synthetic problem descriptions for the multilevel local-and-parallel
P1 eigensolver (Li, Han, Xie, You: Algorithm 4.1 / 4.2).

This module holds NO arithmetic of the method. It only generates the inputs that
both the CPU oracle and the CUDA path consume:

* a coarse background grid T_H of ``ncx x ncy`` square cells of side H with a
  cell mask (the domain Omega is the union of the in-domain cells; every cell is
  split by its SW-NE diagonal into two right triangles);
* the disjoint subdomains D_j as an owner index per coarse cell, the overlap
  ``o_j`` (in coarse cells) that enlarges D_j to Omega_j, and the inset delta that
  defines G_j (Section 4, the decomposition before Algorithm 4.1);
* the number of levels n (h_k = H / 2^k, Section 4.2), the batch size and the
  diffusion coefficient kappa of a(u, v) = (kappa grad u, grad v).

Random numbers come from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

KAPPA_ONE = 0             # kappa == 1: the Laplacian of Example 1
KAPPA_PER_COARSE_CELL = 1  # kappa[b, cj, ci] on coarse cells
KAPPA_PER_FINE_ELEM = 2    # kappa[b, cj, ci, t] on finest-level triangles, t=0 lower, t=1 upper

GLUE_PAPER = 0  # Algorithm 4.1 step 2: indicator of G_j plus the G_{m+1} boundary value problem
GLUE_PU = 1     # smooth partition of unity built from coarse hat functions


@dataclass
class Problem:
    """One (batched) eigenproblem description.

    Arrays are row-major with y (``cj``) as the slow index: ``cell_in[cj, ci]``.
    Fine-element kappa layout: ``kappa[b, cj, ci, 0]`` is the lower triangle of
    finest cell (ci, cj) with vertices (ci,cj),(ci+1,cj),(ci+1,cj+1);
    ``kappa[b, cj, ci, 1]`` the upper one with vertices (ci,cj),(ci+1,cj+1),(ci,cj+1).
    """

    name: str
    ncx: int
    ncy: int
    x0: float
    y0: float
    H: float
    cell_in: np.ndarray
    cell_owner: np.ndarray
    overlap: np.ndarray
    delta: float
    levels: int
    batch: int = 1
    kappa_kind: int = KAPPA_ONE
    kappa: np.ndarray | None = None
    glue_mode: int = GLUE_PAPER
    notes: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.overlap.shape[0])

    @property
    def fine_nx(self) -> int:
        return self.ncx << self.levels

    @property
    def fine_ny(self) -> int:
        return self.ncy << self.levels

    def with_levels(self, n: int) -> "Problem":
        """Same geometry and partition with n levels (fine kappa is only valid at its own n)."""
        if self.kappa_kind == KAPPA_PER_FINE_ELEM and n != self.levels:
            raise ValueError("per-element kappa is defined on the finest level only")
        return replace(self, levels=n, name=f"{self.name}-n{n}")

    def take_batch(self, idx) -> "Problem":
        idx = np.atleast_1d(np.asarray(idx, dtype=np.int64))
        kap = None if self.kappa is None else np.ascontiguousarray(self.kappa[idx])
        return replace(self, batch=int(idx.size), kappa=kap, name=f"{self.name}-b{idx.size}")


def _grid_owner(ncx: int, ncy: int, px: int, py: int) -> np.ndarray:
    """Owner index of each cell for a px x py tiling of the grid into equal blocks."""
    bx, by = ncx // px, ncy // py
    ci = np.arange(ncx) // bx
    cj = np.arange(ncy) // by
    return (cj[:, None] * px + ci[None, :]).astype(np.int32)


def unit_square(nc: int, parts: int, levels: int, overlap: int = 1, delta_in_H: float = 0.5,
                batch: int = 1, name: str | None = None) -> Problem:
    """(0,1)^2 with an nc x nc coarse grid split into parts x parts equal blocks D_j."""
    H = 1.0 / nc
    m = parts * parts
    return Problem(
        name=name or f"square{nc}-m{m}-n{levels}",
        ncx=nc, ncy=nc, x0=0.0, y0=0.0, H=H,
        cell_in=np.ones((nc, nc), np.uint8),
        cell_owner=_grid_owner(nc, nc, parts, parts),
        overlap=np.full(m, overlap, np.int32),
        delta=delta_in_H * H,
        levels=levels, batch=batch,
    )


def single_subdomain(nc: int, levels: int) -> Problem:
    """One subdomain D_1 = Omega_1 = Omega: Algorithm 4.1 reduces to one inverse-iteration step + RR."""
    p = unit_square(nc, 1, levels, overlap=0, name=f"square{nc}-single-n{levels}")
    return p


def _guillotine(rng: np.random.Generator, x: int, y: int, w: int, h: int, pieces: int):
    """Split the w x h cell rectangle at (x, y) into `pieces` rectangles by guillotine cuts.

    The piece to cut is drawn with probability proportional to its area (among the
    pieces wider or taller than one cell); the axis is drawn among the splittable
    ones; the cut line is uniform among the interior coarse grid lines.
    """
    if pieces > w * h:
        raise ValueError("more pieces than cells")
    rects = [(x, y, w, h)]
    while len(rects) < pieces:
        area = np.array([rw * rh if (rw > 1 or rh > 1) else 0 for (_, _, rw, rh) in rects], np.float64)
        i = int(rng.choice(len(rects), p=area / area.sum()))
        rx, ry, rw, rh = rects.pop(i)
        axes = [a for a, s in ((0, rw), (1, rh)) if s > 1]
        ax = axes[int(rng.integers(len(axes)))]
        if ax == 0:
            c = int(rng.integers(1, rw))
            rects += [(rx, ry, c, rh), (rx + c, ry, rw - c, rh)]
        else:
            c = int(rng.integers(1, rh))
            rects += [(rx, ry, rw, c), (rx, ry + c, rw, rh - c)]
    return rects


def lshape(levels: int = 8, seed: int = 3, pieces=(21, 21, 22), nc_half: int = 8) -> Problem:
    """L = (-1,1)^2 minus [0,1)x(-1,0]; coarse h = 1/nc_half; guillotine D_j; o_j ~ U{1,2}; delta = H/4."""
    nc = 2 * nc_half
    H = 2.0 / nc
    cell_in = np.ones((nc, nc), np.uint8)
    cell_in[:nc_half, nc_half:] = 0  # cj < nc_half (y < 0) and ci >= nc_half (x >= 0): removed quadrant
    rng = np.random.Generator(np.random.PCG64(seed))
    quads = [(0, nc_half), (nc_half, nc_half), (0, 0)]  # upper-left, upper-right, lower-left (ci0, cj0)
    rects = []
    for (qx, qy), k in zip(quads, pieces):
        rects += _guillotine(rng, qx, qy, nc_half, nc_half, k)
    rects.sort(key=lambda r: (r[1], r[0]))
    owner = np.full((nc, nc), -1, np.int32)
    for j, (rx, ry, rw, rh) in enumerate(rects):
        owner[ry:ry + rh, rx:rx + rw] = j
    assert np.all((owner >= 0) == (cell_in == 1))
    m = len(rects)
    overlap = rng.integers(1, 3, size=m).astype(np.int32)
    return Problem(
        name=f"lshape-h{nc_half}-m{m}-n{levels}-s{seed}",
        ncx=nc, ncy=nc, x0=-1.0, y0=-1.0, H=H,
        cell_in=cell_in, cell_owner=owner, overlap=overlap,
        delta=0.25 * H, levels=levels,
        notes={"rects": rects, "seed": seed},
    )


def kappa_coarse_batch(p: Problem, batch: int, seed: int, lo: float = 1.0, hi: float = 10.0) -> Problem:
    """kappa per coarse cell, log-uniform in [lo, hi], independent per problem of the batch."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kap = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(batch, p.ncy, p.ncx)))
    kap = kap * p.cell_in[None]
    return replace(p, batch=batch, kappa_kind=KAPPA_PER_COARSE_CELL, kappa=kap,
                   name=f"{p.name}-kc{batch}-s{seed}")


def kappa_fine_elem(p: Problem, seed: int, lo: float = 0.5, hi: float = 2.0, batch: int = 1) -> Problem:
    """kappa per finest-level triangle, log-uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ny, nx = p.fine_ny, p.fine_nx
    kap = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(batch, ny, nx, 2)))
    mask = np.repeat(np.repeat(p.cell_in, 1 << p.levels, axis=0), 1 << p.levels, axis=1)
    kap = kap * mask[None, :, :, None]
    return replace(p, batch=batch, kappa_kind=KAPPA_PER_FINE_ELEM, kappa=kap,
                   name=f"{p.name}-kf-s{seed}")


# --- the five workloads -----------------------------------------------------------------

def config1() -> Problem:
    """Unit square, 8x8 coarse cells, 2x2 subdomains (overlap 1), 3 refinements (finest h = 1/64)."""
    return unit_square(8, 2, 3, name="c1-square8-m4-n3")


def config2(levels: int = 6) -> Problem:
    """Unit square, 16x16 coarse cells, 4x4 subdomains, 6 levels (finest 1024x1024, 1,046,529 DOFs)."""
    return unit_square(16, 4, levels, name=f"c2-square16-m16-n{levels}")


def config3(levels: int = 8, seed: int = 3) -> Problem:
    """L-shape, coarse h = 1/8, 64 guillotine subdomains with overlap 1-2, 8 levels (h = 1/2048)."""
    p = lshape(levels=levels, seed=seed)
    p.name = f"c3-{p.name}"
    return p


def config4(batch: int = 256, levels: int = 4, seed: int = 4) -> Problem:
    """256 problems on the unit square, kappa per 16x16 coarse cell log-uniform in [1,10], finest 256^2."""
    p = kappa_coarse_batch(unit_square(16, 4, levels), batch, seed)
    p.name = f"c4-square16-m16-n{levels}-kc{batch}"
    return p


def config5(levels: int = 5, seed: int = 5) -> Problem:
    """Unit square, finest 512^2, kappa per fine element log-uniform in [0.5, 2]."""
    p = kappa_fine_elem(unit_square(16, 4, levels), seed)
    p.name = f"c5-square16-m16-n{levels}-kf"
    return p


CONFIGS = {"c1": config1, "c2": config2, "c3": config3, "c4": config4, "c5": config5}


# --- Example 2 of Section 6 (full tensor coefficient, weighted mass) ---------------------

def example2_tensor(x, y):
    """The coefficient matrix of Example 2 at (x, y): (a11, a12, a22) with a11 = exp(1 + x^2),
    a12 = a21 = exp(x y), a22 = exp(1 + y^2)."""
    return np.exp(1.0 + x * x), np.exp(x * y), np.exp(1.0 + y * y)


def example2_weight(x, y):
    """The weight of b(u, v) = (phi u, v) in Example 2: phi = (1 + x^2)(1 + y^2)."""
    return (1.0 + x * x) * (1.0 + y * y)


def example2(levels: int = 4, parts: int = 4) -> Problem:
    """Example 2's domain and decomposition: (-1,1)^2, H = 0.1 (a 20 x 20 coarse grid),
    delta = 0.1, parts x parts equal blocks D_j with overlap one coarse cell. The forms come
    from example2_tensor and example2_weight (the GPU path takes kappa I and the plain mass)."""
    nc = 20
    H = 2.0 / nc
    m = parts * parts
    return Problem(
        name=f"ex2-square20-m{m}-n{levels}",
        ncx=nc, ncy=nc, x0=-1.0, y0=-1.0, H=H,
        cell_in=np.ones((nc, nc), np.uint8),
        cell_owner=_grid_owner(nc, nc, parts, parts),
        overlap=np.full(m, 1, np.int32),
        delta=H,
        levels=levels,
        notes={"forms": "example2"},
    )


# --- d = 3 (Section 2.1 admits tetrahedra; the paper runs only d = 2) -----------------------

@dataclass
class Box3:
    """A box (0, ncx H) x (0, ncy H) x (0, ncz H) of coarse cubes of side H, split into
    parts^3 equal blocks D_j (a coarse-cube box each) with overlap o coarse cubes and inset
    delta; n levels h_k = H / 2^k. Only the oracle takes it (no GPU path for d = 3)."""
    name: str
    nc: tuple
    H: float
    levels: int
    parts: int
    overlap: int
    delta: float

    def with_levels(self, n: int) -> "Box3":
        return replace(self, levels=n, name=f"{self.name.rsplit('-n', 1)[0]}-n{n}")


def unit_cube(nc: int, parts: int, levels: int, overlap: int = 1, delta_in_H: float = 0.5) -> Box3:
    """The unit cube in nc^3 coarse cubes, parts^3 subdomain blocks (nc divisible by parts)."""
    if nc % parts:
        raise ValueError("nc must be a multiple of parts")
    H = 1.0 / nc
    return Box3(name=f"cube{nc}-m{parts ** 3}-o{overlap}-n{levels}", nc=(nc, nc, nc), H=H, levels=levels,
                parts=parts, overlap=overlap, delta=delta_in_H * H)
