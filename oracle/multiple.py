"""Several eigenpairs: the subspace form of Algorithms 4.1 / 4.2 (oracle; test infrastructure).

Section 4 states the correction step for one simple eigenvalue and says the version for
several or multiple eigenvalues follows in the same way; Section 6 runs it for the first
five eigenvalues of the Laplacian, among them the double lambda_2 = lambda_3 (Table 1), and
the concluding remarks repeat that the simple-eigenvalue algorithm extends to that case.

Reading used here (the paper gives no formulas for it):
* Level 1 (Algorithm 4.2 step 1): the q smallest eigenpairs (lambda_{i,h_1}, u_{i,h_1}) of
  the pencil on V_{0h_1}, b-orthonormal.
* Correction (Algorithm 4.1) for i = 1..q: steps 1 and 2 exactly as for one eigenpair, with
  the right-hand sides lambda_{i,h_k} b(u_{i,h_k}, v) - a(u_{i,h_k}, v) and
  lambda_{i,h_k} b(u_{i,h_k}, v), giving q glued functions u~_i.
* Step 3 on the one space V_{H,h_{k+1}} = V_{0H} + span{u~_1, ..., u~_q} (dimension N_H + q):
  its q smallest Ritz pairs are (lambda_{i,h_{k+1}}, u_{i,h_{k+1}}), b-orthonormal.
  For a group of equal eigenvalues the span of the u~_i does not depend on the basis
  chosen for their eigenspace (steps 1 and 2 are linear in u for a fixed lambda).
* Sign of each u_i (the paper fixes none): b(u_i, W) > 0 for the T_H function
  W = sum_k omega_k phi_k over the free coarse nodes, omega at the coarse node (X, Y) being
  1 + frac(0.6180339887498949 k) with k = Y (ncx + 1) + X (a fixed, positive, irregular
  weight: a low-order polynomial weight is orthogonal to eigenfunctions that are odd under
  a symmetry of the domain, for example sin(pi x) sin(3 pi y) - sin(3 pi x) sin(pi y) on the
  square). W >= 0, so for the first eigenfunction (positive) this is the convention int u > 0
  of the one-eigenpair oracle. (A T_H function makes b(u_i, W) a combination of the step-3
  quantities P_H^T M u, which the Rayleigh-Ritz step has at hand.) Signs on the intermediate
  levels do not change the result: steps 1 and 2 are linear in u.

Every step is plain: sparse direct solves (SuperLU) for the local and G_{m+1} problems,
dense scipy.linalg.eigh for both eigenproblems.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W

from . import multilevel as ML


def sign_weight(hier: ML.Hierarchy, ell: int) -> np.ndarray:
    """Nodal values on level ell (all nodes) of the sign function W = sum of omega_k phi_k over
    the free coarse nodes (the coarse hats embedded by exact interpolation)."""
    c0 = hier.levels[0]
    f = ML.free(hier, 0)
    k = (c0.pts[f, 1] * (c0.nx + 1) + c0.pts[f, 0]).astype(np.float64)
    x = k * 0.6180339887498949
    omega = 1.0 + (x - np.floor(x))
    return ML.coarse_basis(hier, ell) @ omega


def normalize_columns(hier: ML.Hierarchy, ell: int, U: np.ndarray) -> np.ndarray:
    """Scale every column to b(u, u) = 1 and b(u, w) > 0."""
    M = hier.M[ell]
    w = sign_weight(hier, ell)
    out = U.copy()
    for i in range(U.shape[1]):
        u = out[:, i]
        u = u / np.sqrt(u @ (M @ u))
        if u @ (M @ w) < 0:
            u = -u
        out[:, i] = u
    return out


def global_eigpairs(hier: ML.Hierarchy, ell: int, q: int):
    """The q smallest eigenpairs of the discrete problem on V_{0h_ell}: (lams [q], U [nodes, q])."""
    f = ML.free(hier, ell)
    K, M = hier.K[ell][f][:, f], hier.M[ell][f][:, f]
    if K.shape[0] <= 4000:
        w, v = sla.eigh(K.toarray(), M.toarray(), subset_by_index=[0, q - 1])
    else:
        w, v = spla.eigsh(K.tocsc(), k=q, M=M.tocsc(), sigma=0.0, which="LM", tol=1e-14)
        order = np.argsort(w)
        w, v = w[order], v[:, order]
    U = np.zeros((hier.levels[ell].nv, q))
    U[f] = v
    return np.asarray(w, float), normalize_columns(hier, ell, U)


def rayleigh_ritz(hier: ML.Hierarchy, L: int, UT: np.ndarray, q: int):
    """Step 3 on V_{0H} + span{u~_1..u~_q}: the q smallest Ritz pairs (dense eigh of the raw pencil)."""
    K, M = hier.K[L], hier.M[L]
    f = ML.free(hier, L)
    P = ML.coarse_basis(hier, L)[f]
    Q = sp.hstack([P, sp.csr_matrix(UT[f])]).tocsr()
    Kf, Mf = K[f][:, f], M[f][:, f]
    A = (Q.T @ (Kf @ Q)).toarray()
    B = (Q.T @ (Mf @ Q)).toarray()
    A = 0.5 * (A + A.T)
    B = 0.5 * (B + B.T)
    w, c = sla.eigh(A, B, subset_by_index=[0, q - 1])
    U = np.zeros((hier.levels[L].nv, q))
    U[f] = Q @ c
    return np.asarray(w, float), normalize_columns(hier, L, U)


def correction_multi(hier: ML.Hierarchy, k: int, lams: np.ndarray, U: np.ndarray, mapper=map):
    """Algorithm 4.1 for q eigenpairs: level k -> k + 1 (see the module reading)."""
    q = U.shape[1]
    L = k + 1
    UT = np.zeros((hier.levels[L].nv, q))
    for i in range(q):
        u = hier.interp[k] @ U[:, i]               # u_{i,h_k} embedded in V_{h_{k+1}}
        UT[:, i], _ = ML.glued(hier, L, float(lams[i]), u, mapper)
    return rayleigh_ritz(hier, L, UT, q)


@dataclass
class MultiResult:
    lams: np.ndarray           # lambda_{i,h_n}, i = 1..q
    u: np.ndarray              # [q, ny+1, nx+1] u_{i,h_n} on the node lattice
    lam_levels: np.ndarray     # [n, q] lambda_{i,h_k}


def solve_multi(problem: W.Problem, q: int, b: int = 0, hier: ML.Hierarchy | None = None,
                mapper=map) -> MultiResult:
    """Algorithm 4.2 for the q smallest eigenpairs of batch member b."""
    hier = hier or ML.build(problem, b)
    n = problem.levels
    lams, U = global_eigpairs(hier, 1, q)
    levels = [lams]
    for k in range(1, n):
        lams, U = correction_multi(hier, k, lams, U, mapper)
        levels.append(lams)
    grids = np.stack([ML.to_grid(hier, n, U[:, i]) for i in range(q)])
    return MultiResult(lams, grids, np.array(levels))
