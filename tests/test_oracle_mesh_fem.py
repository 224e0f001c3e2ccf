"""Pins of the oracle's mesh, interpolation and P1 forms against closed forms and brute force.

Paper anchors: Section 2.1 (P1 spaces on T_h), Section 2.2 (a(u,v)), Section 3 (b(u,v),
discrete eigenproblem, min-max upper bound), Section 4.2 (regular refinement, nested spaces).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import fem, mesh
from oracle import multilevel as ML


def _slash_mesh(nc, res):
    """Structured SW-NE diagonal mesh at lattice resolution res (independent construction)."""
    out = set()
    n = nc * res
    for j in range(n):
        for i in range(n):
            out.add(tuple(sorted([(i, j), (i + 1, j), (i + 1, j + 1)])))
            out.add(tuple(sorted([(i, j), (i + 1, j + 1), (i, j + 1)])))
    return out


def test_red_refinement_gives_slash_mesh():
    cell_in = np.ones((2, 2), np.uint8)
    lv = mesh.build_levels(cell_in, 3, 0.5)
    for ell in range(4):
        got = {tuple(sorted(map(tuple, t))) for t in lv[ell].tri_pts.tolist()}
        assert got == _slash_mesh(2, 1 << ell)
        # every triangle is counter-clockwise with area (1/2) lattice units
        p = lv[ell].tri_pts
        det = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
        assert np.all(det == 1)


def test_boundary_of_lshape():
    p = W.lshape(levels=2, nc_half=2, pieces=(2, 2, 2))
    lv = mesh.build_levels(p.cell_in, 2, p.H)[2]
    # lattice 16x16 at res 4; L-shape with removed quadrant x >= 8, y <= 8 (lattice units)
    x, y = lv.pts[:, 0], lv.pts[:, 1]
    expect = (x == 0) | (y == 16) | (x == 16) | (y == 0) | ((x >= 8) & (y == 8)) | ((x == 8) & (y <= 8))
    assert np.array_equal(lv.boundary, expect)
    assert not np.any((x > 8) & (y < 8))  # no nodes in the removed quadrant


def test_interpolation_reproduces_linear_functions():
    rng = np.random.default_rng(0)
    p = W.lshape(levels=2, nc_half=2, pieces=(2, 2, 2))
    lv = mesh.build_levels(p.cell_in, 2, p.H)
    a, b, c = rng.normal(size=3)
    for ell in range(2):
        I = mesh.interpolation(lv[ell], lv[ell + 1])
        fc = a + b * lv[ell].pts[:, 0] / lv[ell].res + c * lv[ell].pts[:, 1] / lv[ell].res
        ff = a + b * lv[ell + 1].pts[:, 0] / lv[ell + 1].res + c * lv[ell + 1].pts[:, 1] / lv[ell + 1].res
        assert np.allclose(I @ fc, ff, atol=1e-13)


def _row(A, lv, i, j):
    idx = mesh.node_index(lv, np.array([[i, j]]))[0]
    r = A.getrow(idx)
    out = {}
    for col, v in zip(r.indices, r.data):
        if abs(v) > 0:
            pi, pj = lv.pts[col]
            out[(int(pi - i), int(pj - j))] = v
    return out


def test_interior_stencils():
    """Closed forms on the SW-NE mesh: K row = [4; -1 x4], M row = h^2/12 [6; 1 on E,W,N,S,NE,SW]."""
    H = 0.25
    lv = mesh.build_levels(np.ones((4, 4), np.uint8), 2, H)[2]
    K, M = fem.assemble(lv, np.ones(lv.tris.shape[0]), H)
    h = H / 4
    k = _row(K, lv, 7, 9)
    assert set(k) == {(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)}
    assert k[(0, 0)] == pytest.approx(4.0, abs=1e-14)
    for d in [(1, 0), (-1, 0), (0, 1), (0, -1)]:
        assert k[d] == pytest.approx(-1.0, abs=1e-14)
    m = _row(M, lv, 7, 9)
    assert set(m) == {(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1)}
    assert m[(0, 0)] == pytest.approx(6 * h * h / 12, rel=1e-14)
    for d in [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1)]:
        assert m[d] == pytest.approx(h * h / 12, rel=1e-14)


def test_stiffness_row_with_a_different_kappa_on_each_of_six_triangles():
    """Hand-computed row, independent of the oracle's layout rule: node c = (3, 5) of the finest
    lattice touches six triangles, L(c) and U(c) of the cell NE of it, U of the cell SE, L of the
    cell NW, L and U of the cell SW (kappa[cj][ci][t], t = 0 the triangle with the cell's SE
    corner). On a right triangle with legs h the P1 stiffness couples the two legs' end nodes
    by -kappa/2 and the hypotenuse's by 0, so each axis edge of c gets the mean of the two
    triangles it is a leg of, and the diagonal edges nothing."""
    p = W.kappa_fine_elem(W.unit_square(2, 1, 2, overlap=0), seed=0)
    kap = np.ones_like(p.kappa)
    vals = {"Lc": 2.0, "Uc": 3.0, "Us": 5.0, "Lw": 7.0, "Lsw": 11.0, "Usw": 13.0}
    kap[0, 5, 3, 0], kap[0, 5, 3, 1] = vals["Lc"], vals["Uc"]
    kap[0, 4, 3, 1] = vals["Us"]
    kap[0, 5, 2, 0] = vals["Lw"]
    kap[0, 4, 2, 0], kap[0, 4, 2, 1] = vals["Lsw"], vals["Usw"]
    kap[0, 4, 3, 0] = kap[0, 5, 2, 1] = 17.0  # the two other triangles of those cells: not at c
    p.kappa = kap
    levels = mesh.build_levels(p.cell_in, p.levels, p.H)
    lv = levels[p.levels]
    K, _ = fem.assemble(lv, fem.kappa_all_levels(p, levels, 0)[p.levels], p.H)
    row = _row(K, lv, 3, 5)
    we, wn = (vals["Lc"] + vals["Us"]) / 2, (vals["Uc"] + vals["Lw"]) / 2
    ww, ws = (vals["Lw"] + vals["Usw"]) / 2, (vals["Us"] + vals["Lsw"]) / 2
    assert set(row) == {(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)}
    assert row[(0, 0)] == pytest.approx(we + wn + ww + ws, rel=1e-14)
    assert row[(1, 0)] == pytest.approx(-we, rel=1e-14) and row[(0, 1)] == pytest.approx(-wn, rel=1e-14)
    assert row[(-1, 0)] == pytest.approx(-ww, rel=1e-14) and row[(0, -1)] == pytest.approx(-ws, rel=1e-14)


def test_element_matrices_against_quadrature():
    """Brute force: gradients by finite differences of barycentrics, mass by a degree-2 exact rule."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        P = rng.normal(size=(3, 2))
        if np.linalg.det(np.c_[P, np.ones(3)]) < 0:
            P = P[[0, 2, 1]]
        det, g = fem.element_geometry(P, np.array([[0, 1, 2]]))
        T = np.c_[P, np.ones(3)]  # barycentric lambda(x) = [x, y, 1] @ inv(T)

        def bary(x):
            return np.array([x[0], x[1], 1.0]) @ np.linalg.inv(T)

        eps = 1e-6
        x0 = P.mean(axis=0)
        gfd = np.stack([(bary(x0 + eps * e) - bary(x0 - eps * e)) / (2 * eps) for e in np.eye(2)], 1)
        assert np.allclose(g[0], gfd, atol=1e-6 * max(1.0, np.abs(gfd).max()))
        area = abs(np.linalg.det(T)) / 2
        # edge-midpoint rule integrates quadratics exactly on triangles
        mids = [(P[0] + P[1]) / 2, (P[1] + P[2]) / 2, (P[2] + P[0]) / 2]
        Mq = sum(np.outer(bary(q), bary(q)) for q in mids) * area / 3
        Me = area / 12 * (np.ones((3, 3)) + np.eye(3))
        assert np.allclose(Mq, Me, rtol=1e-12, atol=1e-15)


def test_lumped_pencil_closed_form():
    """With mass lumped to its row sums (h^2 per interior node) the eigenvalues are
    (4/h^2)(sin^2(i pi h/2) + sin^2(j pi h/2)) on the unit square."""
    N = 8
    lv = mesh.build_levels(np.ones((N, N), np.uint8), 0, 1.0 / N)[0]
    K, M = fem.assemble(lv, np.ones(lv.tris.shape[0]), 1.0 / N)
    f = ~lv.boundary
    Kf = K[f][:, f].toarray()
    lump = np.asarray(M.sum(axis=1)).ravel()[f]
    h = 1.0 / N
    got = np.sort(sla.eigh(Kf, np.diag(lump), eigvals_only=True))
    ii = np.arange(1, N)
    want = np.sort(((4 / h ** 2) * (np.sin(ii[:, None] * np.pi * h / 2) ** 2 + np.sin(ii[None, :] * np.pi * h / 2) ** 2)).ravel())
    assert np.allclose(got, want, rtol=1e-12)


def test_consistent_eigenvalue_converges_to_2pi2():
    """lambda_1 = 2 pi^2 on (0,1)^2; P1 error is O(h^2) (Prop. 3.1 (ii)) and lies above (min-max)."""
    p = W.unit_square(16, 1, 3, overlap=0)
    h = ML.build(p)
    lam = [ML.global_eigpair(h, ell)[0] for ell in (1, 2, 3)]
    exact = 2 * np.pi ** 2
    assert all(l > exact for l in lam)
    e = [l - exact for l in lam]
    assert 3.8 < e[0] / e[1] < 4.2 and 3.8 < e[1] / e[2] < 4.2
    rich = (4 * lam[2] - lam[1]) / 3
    assert abs(rich - exact) < 1e-5
    # cross-check against independently computed values for N = 32, 64
    assert lam[0] == pytest.approx(19.7867922901912, rel=1e-11)
    assert lam[1] == pytest.approx(19.751100837039726, rel=1e-11)


def test_galerkin_identity_for_averaged_kappa():
    """With kappa averaged over descendants, P^T K_fine P equals K_coarse exactly (nested P1 spaces)."""
    p = W.kappa_fine_elem(W.unit_square(3, 1, 2, overlap=0), seed=11, lo=0.2, hi=5.0)
    h = ML.build(p)
    for ell in range(2):
        I = h.interp[ell]
        assert np.allclose((I.T @ h.K[ell + 1] @ I).toarray(), h.K[ell].toarray(), rtol=1e-12, atol=1e-12)
        assert np.allclose((I.T @ h.M[ell + 1] @ I).toarray(), h.M[ell].toarray(), rtol=1e-12, atol=1e-15)
    pc = W.kappa_coarse_batch(W.unit_square(4, 2, 2), batch=2, seed=3)
    h = ML.build(pc, b=1)
    I = h.interp[1] @ h.interp[0]
    assert np.allclose((I.T @ h.K[2] @ I).toarray(), h.K[0].toarray(), rtol=1e-12, atol=1e-12)


def test_rayleigh_quotient_error_identity():
    """Prop. 3.2 for the discrete pair: RQ(psi) - lambda = [a(u-psi,u-psi) - lambda b(u-psi,u-psi)] / b(psi,psi)."""
    p = W.kappa_coarse_batch(W.unit_square(4, 2, 2), batch=1, seed=7)
    h = ML.build(p)
    lam, u = ML.global_eigpair(h, 2)
    K, M = h.K[2], h.M[2]
    rng = np.random.default_rng(2)
    psi = u + 0.1 * rng.normal(size=u.size) * (~h.levels[2].boundary)
    lhs = (psi @ K @ psi) / (psi @ M @ psi) - lam
    d = u - psi
    rhs = (d @ K @ d - lam * (d @ M @ d)) / (psi @ M @ psi)
    assert lhs == pytest.approx(rhs, rel=1e-9)
    assert u @ M @ u == pytest.approx(1.0, rel=1e-13)
