"""Example 2 of Section 6 in the oracle (oracle/tensor.py): full tensor A(x), weighted mass.

Pins, none of which re-derives the assembly from itself:
* the quadrature rule integrates every monomial of degree <= 4 exactly on the reference
  triangle (closed form a! b! / (a + b + 2)!);
* with A = I and phi = 1 the assembly equals the pinned Laplacian assembly (oracle/fem.py);
* for constant A and linear functions p, q the discrete form equals the exact integral
  (grad p . A grad q) |Omega| (the a12 coupling, its sign and the diagonal terms), and the
  weighted mass of polynomial pairs equals the closed-form integral of phi p q;
* Richardson extrapolation of the discrete eigenvalues on h = 0.0125 and 0.00625 reproduces
  the six eigenvalues the paper prints for Example 2 (tests/golden/example2_paper.json) to
  their 8 printed digits;
* the multilevel algorithm (Algorithm 4.2 with the subspace correction, q = 6, H = delta =
  0.1 as in the paper) reaches the fine-mesh discrete eigenvalues, far inside the
  discretization error, which falls at O(h^2) (the paper's Figure for Example 2).
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import fem
from oracle import multiple as MU
from oracle import tensor as T
from oracle.mesh import build_levels

HERE = os.path.dirname(os.path.abspath(__file__))


def _paper():
    with open(os.path.join(HERE, "golden", "example2_paper.json")) as f:
        return np.array(json.load(f)["eigenvalues"])


def test_quadrature_is_exact_to_degree_four():
    # reference triangle (0,0), (1,0), (0,1): point x = b1, y = b2 for barycentric (b0, b1, b2)
    x, y = T.QUAD_BARY[:, 1], T.QUAD_BARY[:, 2]
    assert abs(T.QUAD_W.sum() - 1.0) <= 1e-14
    for a in range(5):
        for b in range(5 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = 0.5 * np.sum(T.QUAD_W * x ** a * y ** b)  # area 1/2
            assert abs(got - exact) <= 1e-14 * max(1.0, exact) + 1e-15, (a, b, got, exact)


def test_identity_forms_reduce_to_the_laplacian_assembly():
    p = W.example2(levels=2)
    lv = build_levels(p.cell_in, 2, p.H)[2]
    K, M = T.assemble(lv, p.x0, p.y0, p.H, lambda x, y: (np.ones_like(x), np.zeros_like(x), np.ones_like(x)),
                      lambda x, y: np.ones_like(x))
    K0, M0 = fem.assemble(lv, np.ones(lv.tris.shape[0]), p.H)
    assert abs(K - K0).max() <= 1e-12 and abs(M - M0).max() <= 1e-15


def test_forms_on_linear_and_polynomial_functions():
    p = W.example2(levels=1)
    lv = build_levels(p.cell_in, 1, p.H)[1]
    a, b, c = 1.7, -0.4, 2.3
    K, _ = T.assemble(lv, p.x0, p.y0, p.H, lambda x, y: (a + 0 * x, b + 0 * x, c + 0 * x), lambda x, y: 1 + 0 * x)
    xy = lv.xy(p.x0, p.y0, p.H)
    px, py = xy[:, 0], xy[:, 1]
    area = 4.0  # (-1,1)^2
    assert abs(px @ (K @ px) - a * area) <= 1e-12
    assert abs(px @ (K @ py) - b * area) <= 1e-12
    assert abs(py @ (K @ py) - c * area) <= 1e-12
    # integrands of degree <= 4, which the rule integrates exactly on every triangle
    _, M = T.assemble(lv, p.x0, p.y0, p.H, W.example2_tensor, W.example2_weight)
    one = np.ones(lv.nv)
    assert abs(one @ (M @ one) - 64.0 / 9.0) <= 1e-12        # int phi = (2 + 2/3)^2
    _, M2 = T.assemble(lv, p.x0, p.y0, p.H, W.example2_tensor, lambda x, y: 1.0 + x * x)
    assert abs(px @ (M2 @ px) - 32.0 / 15.0) <= 1e-12        # int (1 + x^2) x^2 = 2 (2/3 + 2/5)
    assert abs(one @ (M2 @ py)) <= 1e-12                     # int (1 + x^2) y = 0


def test_extrapolated_eigenvalues_match_the_paper():
    h = T.example2_hierarchy(levels=4)
    l3 = MU.global_eigpairs(h, 3, 6)[0]
    l4 = MU.global_eigpairs(h, 4, 6)[0]
    ratio = (l3 - _paper()) / (l4 - _paper())
    assert np.all((ratio > 3.8) & (ratio < 4.2)), ratio       # O(h^2) discretization error
    rich = (4.0 * l4 - l3) / 3.0
    rel = np.abs(rich - _paper()) / _paper()
    assert np.all(rel <= 1e-7), rel                           # 8 printed digits


@pytest.mark.parametrize("levels", [3])
def test_multilevel_reaches_the_fine_mesh_eigenvalues(levels):
    p = W.example2(levels=levels)
    h = T.build(p, W.example2_tensor, W.example2_weight)
    r = MU.solve_multi(p, 6, hier=h)
    disc = MU.global_eigpairs(h, levels, 7)[0]
    assert disc[6] - disc[5] > 1e-3 * disc[6]                 # q = 6 stops at a gap
    ml_err = np.abs(r.lams - disc[:6]) / disc[:6]
    fe_err = np.abs(disc[:6] - _paper()) / _paper()
    assert np.all(ml_err <= 1e-7), ml_err
    assert np.all(ml_err <= 1e-3 * fe_err), (ml_err, fe_err)
    # every level's first eigenvalue decreases towards the limit (min-max on nested spaces)
    assert np.all(np.diff(r.lam_levels[:, 0]) < 0)
