"""Pins of the oracle's Algorithms 4.1 / 4.2 against special cases, invariants and rates.

Paper anchors: Algorithm 4.1 (one correction step), Algorithm 4.2 (multilevel scheme),
Theorem 4.2 (|lambda - lambda_{h_n}| <~ h_n^2), Table 1 (orders ~2 for lambda_1),
Section 3 (min-max: the Ritz value on a subspace of V_{0h} bounds lambda_{1,h} from above).
"""
import numpy as np
import pytest

import workloads as W
from oracle import multilevel as ML
from oracle import partition


def test_partition_counts_config1():
    """Config 1 at h_2 = 1/32: quadrants D_j, delta = 1/16; G_j are 14x14 node blocks and the
    strip is the cross of three node lines each way (hand count)."""
    p = W.config1().with_levels(2)
    h = ML.build(p)
    part = h.parts[2]
    assert [g.size for g in part.g_nodes] == [196] * 4
    assert part.strip.size == 3 * 31 * 2 - 9
    assert [loc.size for loc in part.local] == [19 * 19] * 4
    lv = h.levels[2]
    x, y = lv.pts[part.strip, 0], lv.pts[part.strip, 1]
    assert np.all(((x >= 15) & (x <= 17)) | ((y >= 15) & (y <= 17)))
    g0 = lv.pts[part.g_nodes[0]]
    assert g0[:, 0].max() == 14 and g0[:, 1].max() == 14 and g0.min() == 1


def test_partition_rejects_bad_delta():
    p = W.unit_square(4, 2, 2)
    p.delta = 0.3 * p.H
    with pytest.raises(ValueError):
        ML.build(p)


def test_lshape_partition_is_valid():
    p = W.lshape(levels=3)
    assert p.m == 64
    subs = partition.subdomains(p)
    h = ML.build(p.with_levels(2))
    part = h.parts[2]
    covered = np.zeros(h.levels[2].nv, int)
    for g in part.g_nodes:
        covered[g] += 1
    covered[part.strip] += 1
    assert np.array_equal(covered, (~h.levels[2].boundary).astype(int))
    assert all(s.omega_cells.sum() >= s.d_cells.sum() for s in subs)


def test_fixed_point_of_correction():
    """If (lambda_k, u_k) is already the discrete eigenpair of V_{0h_{k+1}}, step 1 gives e^j = 0,
    the G_{m+1} problem reproduces u_k, and RR returns the same pair (Algorithm 4.1)."""
    for p in (W.config1().with_levels(3), W.kappa_coarse_batch(W.unit_square(8, 2, 3), 1, seed=9)):
        h = ML.build(p)
        lam_h, u_h = ML.global_eigpair(h, 3)
        lam, u, tr = ML.correction_on_level(h, 3, lam_h, u_h, trace=True)
        # dense LAPACK gets lambda_h only to ~eps * lambda_max / lambda_1 ~ 1e-12 relative here
        assert lam == pytest.approx(lam_h, rel=1e-10)
        assert np.abs(tr.u_tilde - u_h).max() < 1e-10 * np.abs(u_h).max()
        assert np.abs(u - u_h).max() < 1e-9 * np.abs(u_h).max()


def test_single_subdomain_is_inverse_iteration_plus_rr():
    """With one subdomain Omega_1 = Omega (no G_{m+1}), step 1 gives u~ = lambda_k K^{-1} M u_k, and
    step 3 is the Ritz problem on span{coarse hats, u~}; both recomputed here with dense LAPACK."""
    p = W.single_subdomain(4, 3)
    h = ML.build(p)
    lam1, u1 = ML.global_eigpair(h, 1)
    k = 1
    lam, u, tr = ML.correction(h, k, lam1, u1, trace=True)
    f = ML.free(h, 2)
    K = h.K[2][f][:, f].toarray()
    M = h.M[2][f][:, f].toarray()
    uk = (h.interp[1] @ u1)[f]
    ut = lam1 * np.linalg.solve(K, M @ uk)
    assert np.allclose(tr.u_tilde[f], ut, rtol=1e-10, atol=1e-12)
    P = ML.coarse_basis(h, 2)[f].toarray()
    Q = np.c_[P, ut]
    A, B = Q.T @ K @ Q, Q.T @ M @ Q
    Lc = np.linalg.cholesky(B)
    Li = np.linalg.inv(Lc)
    w = np.linalg.eigvalsh(Li @ A @ Li.T)
    assert lam == pytest.approx(w[0], rel=1e-11)


def test_min_max_and_paper_orders():
    """lambda_{h_n} >= lambda_{1,h_n} (Ritz value on a subspace) and lambda errors decay at order 2
    (Theorem 4.2; Table 1 reports orders 1.99, 1.99, 2.00, 2.00 for the first eigenvalue)."""
    exact = 2 * np.pi ** 2
    p = W.unit_square(8, 2, 5)
    r = ML.solve(p)
    h = ML.build(p.with_levels(4))
    for ell in (2, 3, 4):
        lam_fine, _ = ML.global_eigpair(h, ell)
        assert r.lam_levels[ell - 1] >= lam_fine - 1e-12
        assert r.lam_levels[ell - 1] - lam_fine < 1e-3 * (lam_fine - exact)
    err = np.array(r.lam_levels) - exact
    orders = np.log2(err[:-1] / err[1:])
    assert np.all((orders > 1.9) & (orders < 2.1)), orders


def test_batch_members_are_independent():
    p = W.kappa_coarse_batch(W.unit_square(4, 2, 3), batch=3, seed=5)
    r1 = ML.solve(p, b=1)
    r1b = ML.solve(p.take_batch([1]), b=0)
    assert r1.lam == r1b.lam
    # kappa scales lambda: every step is 1-homogeneous in kappa
    p2 = W.kappa_coarse_batch(W.unit_square(4, 2, 3), batch=3, seed=5)
    p2.kappa = 3.0 * p2.kappa
    assert ML.solve(p2, b=1).lam == pytest.approx(3.0 * r1.lam, rel=1e-12)


def test_eigenvector_normalisation_and_sign():
    r = ML.solve(W.config1())
    h = ML.build(W.config1())
    lv = h.levels[3]
    u = r.u.ravel()[lv.key(lv.pts)]
    assert u @ h.M[3] @ u == pytest.approx(1.0, rel=1e-13)
    assert u @ h.ones_int[3] > 0
    assert np.all(u >= -1e-12)  # first eigenfunction of the Laplacian is positive
