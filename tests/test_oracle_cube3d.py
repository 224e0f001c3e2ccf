"""The d = 3 oracle (oracle/cube3d.py): Section 2.1 admits tetrahedral meshes for d = 3 and
Section 4.2 refines regularly into beta^d congruent children; the paper runs only d = 2.

Pins, none of which re-derives the construction from itself:
* refinement: each level has 6 Kuhn tetrahedra per lattice cube, all of volume h^3 / 6 (8
  congruent children per parent), and the level-to-level interpolation reproduces linear
  functions exactly (the spaces are nested);
* the P1 stiffness on the Kuhn mesh is the 7-point Laplacian scaled by h at interior nodes
  (a known property of this triangulation), and every interior row of the mass sums to the
  nodal volume h^3;
* with the lumped mass the smallest eigenvalue on the unit cube has the closed form
  (12 / h^2) sin^2(pi h / 2);
* the discrete eigenvalues approach 3 pi^2 at order 2, and the 6 pi^2 triple splits into a
  double eigenvalue and a single one (the mesh is symmetric under permutations of the axes,
  whose 2-dimensional representation keeps the pair exactly double);
* an exact discrete eigenpair is a fixed point of the correction (Algorithm 4.1), and the
  multilevel algorithm (Algorithm 4.2; the subspace form for several pairs) reaches the
  fine-mesh eigenvalues far inside the discretization error, from above.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import cube3d as C3
from oracle import multilevel as ML
from oracle import multiple as MU

PI2 = np.pi ** 2


def test_kuhn_refinement_is_congruent_and_nested():
    box = W.unit_cube(2, 1, 3)
    levels = [C3.build_level(box, ell) for ell in range(4)]
    for lv in levels:
        h = box.H / lv.res
        assert lv.tets.shape[0] == 6 * lv.nx * lv.ny * lv.nz
        X = lv.pts[lv.tets].astype(float) * h
        vol = np.abs(np.linalg.det(X[:, 1:] - X[:, :1])) / 6.0
        assert np.allclose(vol, h ** 3 / 6.0, rtol=1e-12)
        assert abs(vol.sum() - 1.0) < 1e-12
    for c, f in zip(levels[:-1], levels[1:]):
        P = C3.interpolation(c, f)
        xc = c.pts * (box.H / c.res)
        xf = f.pts * (box.H / f.res)
        for lin_c, lin_f in ((np.ones(c.nv), np.ones(f.nv)), (xc[:, 0], xf[:, 0]), (xc[:, 1], xf[:, 1]),
                             (xc[:, 2], xf[:, 2]), (xc @ [1.0, -2.0, 3.0], xf @ [1.0, -2.0, 3.0])):
            assert np.abs(P @ lin_c - lin_f).max() < 1e-13


def test_stiffness_is_the_seven_point_laplacian_and_mass_rows_the_nodal_volume():
    box = W.unit_cube(2, 1, 2)
    lv = C3.build_level(box, 2)
    K, M = C3.assemble(lv, box.H)
    h = box.H / lv.res
    inner = np.nonzero(np.all((lv.pts > 1) & (lv.pts < lv.nx - 1), axis=1))[0]
    axis = {(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)}
    for i in inner[::7]:
        row = K.getrow(i).toarray().ravel()
        for j in np.nonzero(np.abs(row) > 1e-14 * h)[0]:
            d = tuple(int(v) for v in lv.pts[j] - lv.pts[i])
            want = 6.0 * h if d == (0, 0, 0) else (-h if d in axis else 0.0)
            assert abs(row[j] - want) < 1e-13, (d, row[j])
        assert abs(row.sum()) < 1e-13
        assert np.count_nonzero(np.abs(row) > 1e-14 * h) == 7
        assert abs(M.getrow(i).sum() - h ** 3) < 1e-15


def test_lumped_pencil_closed_form():
    box = W.unit_cube(2, 1, 3)
    lv = C3.build_level(box, 3)
    K, _ = C3.assemble(lv, box.H)
    h = box.H / lv.res
    f = np.nonzero(~lv.boundary)[0]
    w = spla.eigsh(K[f][:, f].tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)
    lam = float(w[0]) / h ** 3
    assert lam == pytest.approx(12.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2, rel=1e-11)


def test_eigenvalues_converge_at_order_two_and_keep_the_symmetric_pair_double():
    h = C3.build(W.unit_cube(2, 1, 3))
    e = []
    for ell in (2, 3):
        lams, _ = MU.global_eigpairs(h, ell, 4)
        assert lams[0] > 3 * PI2 and np.all(lams[1:] > 6 * PI2)          # conforming: from above
        assert abs(lams[1] - lams[2]) <= 1e-10 * lams[1]                   # the 2-dimensional pair
        assert lams[3] - lams[2] > 1e-3 * lams[2]                          # the symmetric member splits off
        e.append(lams[0] - 3 * PI2)
    assert 3.7 < e[0] / e[1] < 4.3, e


@pytest.fixture(scope="module")
def cube8():
    box = W.unit_cube(4, 2, 2)          # 8 subdomains, overlap one coarse cube, delta = H/2
    h = C3.build(box)
    disc, Ud = MU.global_eigpairs(h, 2, 4)
    return box, h, disc, Ud


def test_partition_of_the_cube(cube8):
    box, h, _, _ = cube8
    part = h.parts[2]
    assert len(part.local) == 8
    # level 2 (h = H/4, 16^3 cells): Omega_j is a 12^3-cell box with 11^3 interior nodes;
    # closed G_j keeps the free nodes of the 8^3-cell D_j at least delta = 2 cells from its
    # three inner faces, 6 per axis; G_{m+1} takes the rest of the 15^3 free nodes
    assert [len(x) for x in part.local] == [11 ** 3] * 8
    assert [len(g) for g in part.g_nodes] == [6 ** 3] * 8
    assert len(part.strip) == 15 ** 3 - 8 * 6 ** 3
    nodes = np.sort(np.concatenate(part.g_nodes + [part.strip]))
    assert np.array_equal(nodes, np.nonzero(part.free)[0])                # closed G_j and G_{m+1} tile the free nodes
    with pytest.raises(ValueError):
        C3.level_partition(W.Box3("bad", (4, 4, 4), 0.25, 2, 2, 1, 0.3 * 0.25), h.levels[2])


def test_fixed_point_of_correction(cube8):
    _, h, _, _ = cube8
    lam_h, u_h = ML.global_eigpair(h, 2)
    lam, u, tr = ML.correction_on_level(h, 2, lam_h, u_h, trace=True)
    assert lam == pytest.approx(lam_h, rel=1e-10)
    assert np.abs(tr.u_tilde - u_h).max() < 1e-10 * np.abs(u_h).max()
    assert np.abs(u - u_h).max() < 1e-9 * np.abs(u_h).max()


def test_multilevel_reaches_the_fine_mesh_eigenvalues(cube8):
    box, h, disc, _ = cube8
    r = C3.solve(box, hier=h)
    assert r.lam >= disc[0] - 1e-12                                         # a Ritz value (min-max)
    assert r.lam - disc[0] <= 1e-2 * (disc[0] - 3 * PI2)
    lams, _, _ = C3.solve_multi(box, 3, hier=h)
    assert abs(lams[1] - lams[2]) <= 1e-10 * lams[1]
    exact = PI2 * np.array([3.0, 6.0, 6.0])
    assert np.all(lams >= disc[:3] - 1e-12)
    assert np.all(lams - disc[:3] <= 2e-2 * (disc[:3] - exact)), (lams, disc)
