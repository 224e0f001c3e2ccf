"""Pins of the several-eigenpairs oracle (oracle/multiple.py) against special cases, bounds and rates.

Paper anchors: Section 4 (the correction step; the multiple-eigenvalue version "in the
similar way"), Section 6 Table 1 (the first five eigenvalues converge at order 2, the second
and third being equal), Section 3 (min-max: Ritz values on a subspace of V_{0h} bound the
discrete eigenvalues from above, index by index).
"""
import numpy as np
import pytest

import workloads as W
from oracle import multilevel as ML
from oracle import multiple as MU

SQUARE = np.pi ** 2 * np.array([2.0, 5.0, 5.0, 8.0, 10.0])  # first five eigenvalues on (0,1)^2


def test_one_eigenpair_is_the_single_algorithm():
    p = W.config1()
    r = MU.solve_multi(p, 1)
    r1 = ML.solve(p)
    assert r.lams[0] == pytest.approx(r1.lam, rel=1e-13)
    assert np.allclose(r.lam_levels[:, 0], r1.lam_levels, rtol=1e-13)
    assert np.abs(r.u[0] - r1.u).max() < 1e-10


def test_first_five_converge_at_order_two():
    """Table 1's experiment on the unit square (H = 1/8, 2 x 2 subdomains, 5 levels): every one of
    lambda_1 .. lambda_5 has error order ~2 per level against the exact pi^2 (k^2 + l^2)."""
    p = W.unit_square(8, 2, 5)
    r = MU.solve_multi(p, 5)
    err = r.lam_levels - SQUARE[None, :]
    assert np.all(err > 0)
    orders = np.log2(err[:-1] / err[1:])
    assert np.all((orders > 1.95) & (orders < 2.05)), orders
    # the double eigenvalue 5 pi^2: both approximations converge to it
    assert abs(r.lams[1] - SQUARE[1]) < 5e-3 and abs(r.lams[2] - SQUARE[2]) < 5e-3


def test_min_max_index_by_index():
    """lambda_{i,alg} >= lambda_{i,h} on every level (Ritz values of a subspace of V_{0h}), and the
    gap is far below the discretisation error (a few per cent of it for the last index, whose
    subspace direction converges at the ratio lambda_q / lambda_{q+1})."""
    p = W.unit_square(8, 2, 4)
    q = 4
    r = MU.solve_multi(p, q)
    h = ML.build(p)
    for ell in (2, 3, 4):
        lam_h, _ = MU.global_eigpairs(h, ell, q)
        assert np.all(r.lam_levels[ell - 1] >= lam_h - 1e-10), (ell, r.lam_levels[ell - 1], lam_h)
        assert np.all(r.lam_levels[ell - 1] - lam_h < 5e-2 * (lam_h - SQUARE[:q])), ell


def test_single_subdomain_is_block_inverse_iteration_plus_rr():
    """One subdomain Omega_1 = Omega: step 1 gives u~_i = lambda_i K^{-1} M u_i, and step 3 is the
    Ritz problem on span{coarse hats, u~_1 .. u~_q}; both recomputed with dense LAPACK."""
    p = W.single_subdomain(4, 3)
    q = 3
    h = ML.build(p)
    lams1, U1 = MU.global_eigpairs(h, 1, q)
    lams, U = MU.correction_multi(h, 1, lams1, U1)
    f = ML.free(h, 2)
    K = h.K[2][f][:, f].toarray()
    M = h.M[2][f][:, f].toarray()
    UT = np.stack([lams1[i] * np.linalg.solve(K, M @ (h.interp[1] @ U1[:, i])[f]) for i in range(q)], axis=1)
    P = ML.coarse_basis(h, 2)[f].toarray()
    Q = np.c_[P, UT]
    A, B = Q.T @ K @ Q, Q.T @ M @ Q
    Li = np.linalg.inv(np.linalg.cholesky(B))
    w = np.linalg.eigvalsh(Li @ A @ Li.T)[:q]
    assert np.allclose(lams, w, rtol=1e-10)


def test_discrete_eigenpairs_are_a_fixed_point():
    """If the q input pairs are the exact discrete eigenpairs of the next level, every e^j is 0,
    every u~_i is u_i and the Ritz step returns them."""
    p = W.config1().with_levels(3)
    h = ML.build(p)
    q = 3
    lam_h, U_h = MU.global_eigpairs(h, 3, q)
    f = ML.free(h, 3)
    UT = np.zeros_like(U_h)
    for i in range(q):
        UT[:, i], _ = ML.glued(h, 3, lam_h[i], U_h[:, i])
        assert np.abs(UT[f, i] - U_h[f, i]).max() < 1e-9 * np.abs(U_h[:, i]).max()
    lams, U = MU.rayleigh_ritz(h, 3, UT, q)
    assert np.allclose(lams, lam_h, rtol=1e-10)


def test_orthonormal_with_the_sign_rule():
    p = W.lshape(levels=3, seed=7)
    q = 3
    h = ML.build(p)
    r = MU.solve_multi(p, q, hier=h)
    lv = h.levels[3]
    U = np.stack([r.u[i].ravel()[lv.key(lv.pts)] for i in range(q)], axis=1)
    G = U.T @ (h.M[3] @ U)
    assert np.allclose(G, np.eye(q), atol=1e-11)
    w = MU.sign_weight(h, 3)
    assert np.all(U.T @ (h.M[3] @ w) > 0)
    assert np.all(np.diff(r.lams) > 0)
