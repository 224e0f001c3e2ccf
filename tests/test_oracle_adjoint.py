"""Pins of the oracle's reverse-mode d lambda_{h_n} / d kappa (Algorithm 4.2 differentiated).

Checks against what the mathematics fixes, independently of the adjoint's own algebra:
central finite differences of the oracle's forward on a small mesh (per element and along a
random direction over all elements), and Euler's identity sum_e kappa_e dlambda/dkappa_e =
lambda (every step of Algorithms 4.1/4.2 is 1-homogeneous in kappa).
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD
from oracle import multilevel as ML


def _small(seed=21):
    return W.kappa_fine_elem(W.unit_square(4, 2, 3), seed=seed)


def _lam(p):
    return ML.solve(p).lam


def test_adjoint_matches_central_differences_per_element():
    p = _small()
    g, lam = AD.grad_kappa(p)
    assert lam == pytest.approx(_lam(p), rel=1e-13)
    rng = np.random.default_rng(0)
    ny, nx, _ = g.shape
    for _ in range(8):
        j, i, t = rng.integers(ny), rng.integers(nx), rng.integers(2)
        h = 1e-3 * p.kappa[0, j, i, t]   # central FD: truncation ~1e-10 here, rounding grows below
        pp, pm = _small(), _small()
        pp.kappa = p.kappa.copy(); pp.kappa[0, j, i, t] += h
        pm.kappa = p.kappa.copy(); pm.kappa[0, j, i, t] -= h
        fd = (_lam(pp) - _lam(pm)) / (2 * h)
        assert abs(fd - g[j, i, t]) <= 1e-6 * abs(g[j, i, t]) + 1e-9, (j, i, t, fd, g[j, i, t])


def test_adjoint_directional_derivative_and_euler_identity():
    p = _small(seed=4)
    g, lam = AD.grad_kappa(p)
    # Euler: lambda(t kappa) = t lambda(kappa)  =>  sum kappa * grad = lambda
    assert np.sum(p.kappa[0] * g) == pytest.approx(lam, rel=1e-10)
    rng = np.random.default_rng(1)
    d = rng.choice([-1.0, 1.0], size=p.kappa.shape) * p.kappa
    eps = 1e-4
    pp, pm = _small(seed=4), _small(seed=4)
    pp.kappa = p.kappa + eps * d
    pm.kappa = p.kappa - eps * d
    fd = (_lam(pp) - _lam(pm)) / (2 * eps)
    assert fd == pytest.approx(np.sum(g * d[0]), rel=1e-7)


def test_adjoint_close_to_hellmann_feynman():
    """The algorithm's derivative differs from the Hellmann-Feynman gradient of the final
    eigenfunction only through the sensitivity of u~; on a converged run they are close."""
    p = W.kappa_fine_elem(W.unit_square(4, 2, 4), seed=3)
    g, lam = AD.grad_kappa(p)
    r = ML.solve(p)
    hf = AD.hellmann_feynman(p, r.u)
    rel = np.linalg.norm(g - hf) / np.linalg.norm(hf)
    assert rel < 0.05, rel


@pytest.mark.parametrize("make", [
    lambda: W.lshape(levels=3, seed=7),
    lambda: W.kappa_coarse_batch(W.unit_square(6, 3, 3, overlap=2, delta_in_H=0.25), batch=2, seed=9),
])
def test_adjoint_directional_on_uneven_partitions(make):
    """L-shape with uneven subdomains and a wide strip; overlap 2 with delta = H/4."""
    p = make()
    b = p.batch - 1
    g, lam = AD.grad_kappa(p, b=b)
    assert lam == pytest.approx(ML.solve(p, b=b).lam, rel=1e-13)
    base = AD.finest_kappa(p, b)
    assert np.sum(base * g) == pytest.approx(lam, rel=1e-10)
    rng = np.random.default_rng(2)
    d = rng.uniform(-1.0, 1.0, size=base.shape) * base
    eps = 1e-4
    lp = AD.solve_with_fine_kappa(p, base + eps * d)
    lm = AD.solve_with_fine_kappa(p, base - eps * d)
    assert (lp - lm) / (2 * eps) == pytest.approx(np.sum(g * d), rel=1e-7)
