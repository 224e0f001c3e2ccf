"""Quadratic (P2) elements in the oracle (oracle/p2.py): Section 6 runs Example 1 with linear
and with quadratic elements, the latter converging at O(h^4) (the paper's figure for the
quadratic element).

Pins, none of which re-derives the construction from itself:
* the six shape functions are a partition of unity and take the value 1 at their own node,
  0 at the other five;
* the level-to-level interpolation reproduces quadratics exactly (the spaces are nested);
* the forms are exact on quadratics: u^T K v = int grad u . grad v and u^T M v = int u v on
  the unit square for u, v in {x^2, y^2, xy} (closed forms);
* the discrete eigenvalues of the unit-square Laplacian approach pi^2 (k^2 + l^2) with errors
  falling by 16x per level (order 4);
* the multilevel algorithm with P2 spaces (one pair, and the 6 smallest by the subspace form)
  reaches the fine-mesh discrete eigenvalues, far inside the discretization error.
"""
import numpy as np

import workloads as W
from oracle import multilevel as ML
from oracle import multiple as MU
from oracle import p2 as P2
from oracle.mesh import build_levels

EXACT = np.pi ** 2 * np.array([2.0, 5.0, 5.0, 8.0, 10.0, 10.0])


def test_shape_functions():
    nodes = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [.5, .5, 0], [0, .5, .5], [.5, 0, .5]])
    val, der = P2.shape(nodes)
    assert np.allclose(val, np.eye(6), atol=1e-15)
    rng = np.random.default_rng(1)
    lam = rng.dirichlet(np.ones(3), size=20)
    v, d = P2.shape(lam)
    assert np.allclose(v.sum(axis=1), 1.0, atol=1e-14)
    # the derivative of the sum along any direction tangent to the simplex vanishes
    t = np.array([1.0, -1.0, 0.0])
    assert np.allclose(np.einsum("qak,k->q", d, t), 0.0, atol=1e-13)


def _quadratics(xy):
    x, y = xy[:, 0], xy[:, 1]
    return {"xx": x * x, "yy": y * y, "xy": x * y}


def test_interpolation_reproduces_quadratics():
    lat = build_levels(np.ones((2, 2), np.uint8), 4, 0.5)
    P = P2.interpolation(lat[1], lat[2], lat[3])
    qc = _quadratics(lat[2].xy(0.0, 0.0, 0.5))
    qf = _quadratics(lat[3].xy(0.0, 0.0, 0.5))
    for k in qc:
        assert np.abs(P @ qc[k] - qf[k]).max() <= 1e-14


def test_forms_exact_on_quadratics():
    p = W.unit_square(2, 1, 2, overlap=0)
    lat = build_levels(p.cell_in, 3, p.H)
    K, M = P2.assemble(lat[2], lat[3], p.H)
    q = _quadratics(lat[3].xy(0.0, 0.0, p.H))
    # int over (0,1)^2: grad x^2 = (2x, 0), grad y^2 = (0, 2y), grad xy = (y, x)
    exact_k = {("xx", "xx"): 4 / 3, ("yy", "yy"): 4 / 3, ("xx", "yy"): 0.0, ("xy", "xy"): 2 / 3,
               ("xx", "xy"): 2 * 0.25, ("yy", "xy"): 2 * 0.25}
    exact_m = {("xx", "xx"): 1 / 5, ("xx", "yy"): 1 / 9, ("xy", "xy"): 1 / 9, ("xx", "xy"): 1 / 8}
    for (a, b), v in exact_k.items():
        assert abs(q[a] @ (K @ q[b]) - v) <= 1e-12, (a, b)
    for (a, b), v in exact_m.items():
        assert abs(q[a] @ (M @ q[b]) - v) <= 1e-13, (a, b)


def test_eigenvalues_converge_at_order_four():
    h = P2.build(W.unit_square(4, 2, 4))
    e3 = MU.global_eigpairs(h, 3, 5)[0] - EXACT[:5]
    e4 = MU.global_eigpairs(h, 4, 5)[0] - EXACT[:5]
    assert np.all(e3 > 0) and np.all(e4 > 0)                  # conforming: from above
    ratio = e3 / e4
    assert np.all((ratio > 15.0) & (ratio < 17.0)), ratio


def test_multilevel_with_p2_reaches_the_fine_mesh_eigenvalues():
    p = W.unit_square(4, 2, 3)
    h = P2.build(p)
    disc = MU.global_eigpairs(h, 3, 7)[0]
    one = ML.solve(p, hier=h)
    assert abs(one.lam - disc[0]) <= 1e-9 * disc[0]
    r = MU.solve_multi(p, 6, hier=h)
    ml_err = np.abs(r.lams - disc[:6])
    fe_err = disc[:6] - EXACT
    assert np.all(ml_err <= 1e-2 * fe_err), (ml_err, fe_err)
    # the level values fall at order 4 towards the limit
    lv = r.lam_levels[:, 0] - EXACT[0]
    assert np.all(lv[:-1] / lv[1:] > 14.0), lv
