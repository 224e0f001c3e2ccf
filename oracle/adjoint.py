"""Reverse-mode derivative d lambda_{h_n} / d kappa of Algorithm 4.2 (oracle).

The forward map is the oracle's own Algorithm 4.2 (``multilevel.solve``); every step is
differentiated exactly (implicit differentiation of each linear solve and eigensolve):

* eigenpair (lambda, c) of a symmetric-definite pencil (A, B) with c^T B c = 1:
  d lambda = c^T (dA - lambda dB) c and dc = -G (dA - lambda dB) c - 1/2 (c^T dB c) c,
  G = (A - lambda B)^+ on the B-orthogonal complement of c. For adjoints (lam_bar, c_bar):
  z = G c_bar, A_bar = lam_bar c c^T - (c z^T + z c^T)/2, B_bar = -lambda A_bar - (c^T c_bar)/2 c c^T.
  Applied to the level-1 eigenproblem (Algorithm 4.2 step 1) and to the Rayleigh-Ritz
  problem of Algorithm 4.1 step 3 (A = Q^T K Q, B = Q^T M Q, Q = [coarse hats, u~]).
* every linear solve S x = f: the adjoint solves S^T x_bar_rhs = x_bar (S is symmetric).
* a(.,.) is linear in the per-triangle coefficient, and a coarser triangle's coefficient is
  the mean of its four children (the averaging the forward uses), so a derivative with
  respect to a level-L triangle spreads to each of its finest descendants with weight
  4^{L-n}.

Parity status: pinned by central finite differences on small meshes, by a directional
finite difference over all elements, and by Euler's identity sum_e kappa_e dlambda/dkappa_e
= lambda (every step is 1-homogeneous in kappa) - see tests/test_oracle_adjoint.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W

from . import fem
from .multilevel import Hierarchy, build, coarse_basis, free, global_eigpair, normalize


def element_form(hier: Hierarchy, ell: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """x_T^T K_T^{(1)} y_T for every triangle T of level ell (element stiffness with kappa = 1)."""
    lv = hier.levels[ell]
    coords = lv.pts.astype(np.float64) * (hier.problem.H / lv.res)
    det, g = fem.element_geometry(coords, lv.tris)
    area = 0.5 * np.abs(det)
    gx = np.einsum("eid,ei->ed", g, x[lv.tris])
    gy = np.einsum("eid,ei->ed", g, y[lv.tris])
    return area * np.einsum("ed,ed->e", gx, gy)


def pencil_adjoint(A, B, lam, c, lam_bar, c_bar):
    """(A_bar, B_bar) for the eigenpair (lam, c) of (A, B) with c^T B c = 1 (see module doc)."""
    n = A.shape[0]
    Bc = B @ c
    rhs = c_bar - Bc * (c @ c_bar)
    big = np.zeros((n + 1, n + 1))
    big[:n, :n] = A - lam * B
    big[:n, n] = Bc
    big[n, :n] = Bc
    z = np.linalg.solve(big, np.r_[rhs, 0.0])[:n]
    A_bar = lam_bar * np.outer(c, c) - 0.5 * (np.outer(c, z) + np.outer(z, c))
    B_bar = -lam * A_bar - 0.5 * (c @ c_bar) * np.outer(c, c)
    return A_bar, B_bar, z


def _forward_trace(hier: Hierarchy):
    """Algorithm 4.2 forward keeping what the reverse sweep needs at every level."""
    n = hier.problem.levels
    lam, u = global_eigpair(hier, 1)
    rec = {"lam1": lam, "u1": u, "levels": []}
    for k in range(1, n):
        L = k + 1
        K, M = hier.K[L], hier.M[L]
        part = hier.parts[L]
        uL = hier.interp[k] @ u
        r = lam * (M @ uL) - K @ uL
        lus, es = [], []
        for loc in part.local:
            lu = spla.splu(K[loc][:, loc].tocsc())
            e = np.zeros_like(uL)
            e[loc] = lu.solve(r[loc])
            lus.append(lu)
            es.append(e)
        ut = np.zeros_like(uL)
        for j, gset in enumerate(part.g_nodes):
            ut[gset] = uL[gset] + es[j][gset]
        S = part.strip
        lu_s = None
        if S.size:
            lu_s = spla.splu(K[S][:, S].tocsc())
            rhs_s = lam * (M @ uL)[S] - (K[S] @ ut)
            ut[S] = lu_s.solve(rhs_s)
        f = free(hier, L)
        P = coarse_basis(hier, L)[f]
        Q = sp.hstack([P, sp.csr_matrix(ut[f][:, None])]).tocsr()
        Kf, Mf = K[f][:, f], M[f][:, f]
        A = (Q.T @ (Kf @ Q)).toarray()
        B = (Q.T @ (Mf @ Q)).toarray()
        A = 0.5 * (A + A.T)
        B = 0.5 * (B + B.T)
        w, cm = sla.eigh(A, B, subset_by_index=[0, 0])
        c = cm[:, 0] / np.sqrt(cm[:, 0] @ B @ cm[:, 0])
        un = np.zeros_like(uL)
        un[f] = Q @ c
        if un @ hier.ones_int[L] < 0:   # the sign choice of the forward, a locally constant factor
            c, un = -c, -un
        rec["levels"].append(dict(L=L, lam_k=lam, u_in=uL, r=r, lus=lus, es=es, ut=ut, lu_s=lu_s,
                                  f=f, P=P, Q=Q, A=A, B=B, c=c, lam=float(w[0]), u=un))
        lam, u = float(w[0]), un
    rec["lam"] = lam
    return rec


def grad_kappa_levels(hier: Hierarchy):
    """dlambda_{h_n}/d(kappa on each triangle of level ell), for every ell, and lambda_{h_n}."""
    n = hier.problem.levels
    rec = _forward_trace(hier)
    G = {ell: np.zeros(hier.levels[ell].tris.shape[0]) for ell in range(1, n + 1)}
    lam_bar = 1.0
    u_bar = np.zeros(hier.levels[n].nv)
    for st in reversed(rec["levels"]):
        L = st["L"]
        K, M = hier.K[L], hier.M[L]
        part = hier.parts[L]
        f, Q, A, B, c, lam = st["f"], st["Q"], st["A"], st["B"], st["c"], st["lam"]
        # (8) u' = Q c and (7) the Rayleigh-Ritz eigenpair
        c_bar = Q.T @ u_bar[f]
        A_bar, B_bar, z = pencil_adjoint(A, B, lam, c, lam_bar, c_bar)
        uprime = np.zeros_like(u_bar)
        uprime[f] = Q @ c
        wz = np.zeros_like(u_bar)
        wz[f] = Q @ z
        G[L] += lam_bar * element_form(hier, L, uprime, uprime) - element_form(hier, L, uprime, wz)
        # (6) A = Q^T K Q, B = Q^T M Q: adjoint of the u~ column of Q, plus (8)'s Q_bar = u_bar c^T
        qa = np.zeros_like(u_bar)
        qa[f] = Q @ A_bar[:, -1]
        qb = np.zeros_like(u_bar)
        qb[f] = Q @ B_bar[:, -1]
        ut_bar = u_bar * c[-1] + 2.0 * (K @ qa) + 2.0 * (M @ qb)
        ut_bar[~part.free] = 0.0
        lam_k = st["lam_k"]
        uL = st["u_in"]
        ut = st["ut"]
        uin_bar = np.zeros_like(u_bar)
        lamk_bar = 0.0
        # (5) G_{m+1} problem: K_SS u~_S = lam_k (M u)_S - K_S,rest u~_rest
        S = part.strip
        if S.size:
            sbar = np.zeros_like(u_bar)
            sbar[S] = st["lu_s"].solve(ut_bar[S])
            lamk_bar += sbar[S] @ (M @ uL)[S]
            uin_bar += lam_k * (M @ sbar)
            ks = K @ sbar
            ut_bar = ut_bar - ks         # adjoint of the known values feeding the strip
            ut_bar[S] = 0.0
            G[L] += -element_form(hier, L, sbar, ut)
        # (4) gluing: u~ = u_in + e^j on closed G_j
        r_bar = np.zeros_like(u_bar)
        for j, gset in enumerate(part.g_nodes):
            uin_bar[gset] += ut_bar[gset]
            ebar = np.zeros_like(u_bar)
            ebar[gset] = ut_bar[gset]
            loc = part.local[j]
            # (3) e^j = A_j^{-1} r|Omega_j: adjoint solve with the same (symmetric) A_j
            t = np.zeros_like(u_bar)
            t[loc] = st["lus"][j].solve(ebar[loc])
            r_bar += t
            G[L] += -element_form(hier, L, t, st["es"][j])
        # (2) r = lam_k M u - K u
        lamk_bar += r_bar @ (M @ uL)
        uin_bar += lam_k * (M @ r_bar) - K @ r_bar
        G[L] += -element_form(hier, L, r_bar, uL)
        uin_bar[~part.free] = 0.0
        # (1) u = I u_k
        u_bar = hier.interp[L - 1].T @ uin_bar
        u_bar[hier.levels[L - 1].boundary] = 0.0
        lam_bar = lamk_bar
    # level 1: eigenpair of (K_1, M_1) on the free nodes
    f1 = free(hier, 1)
    K1 = hier.K[1][f1][:, f1].toarray()
    M1 = hier.M[1][f1][:, f1].toarray()
    u1 = rec["u1"][f1]
    _, _, z1 = pencil_adjoint(K1, M1, rec["lam1"], u1, lam_bar, u_bar[f1])
    # K1_bar = lam_bar u u^T - (u z^T + z u^T) / 2 in the nodal basis
    u1f = np.zeros(hier.levels[1].nv)
    u1f[f1] = u1
    z1f = np.zeros(hier.levels[1].nv)
    z1f[f1] = z1
    G[1] += lam_bar * element_form(hier, 1, u1f, u1f) - element_form(hier, 1, u1f, z1f)
    return G, rec["lam"]


def grad_kappa(problem: W.Problem, b: int = 0):
    """dlambda_{h_n}/dkappa_e for the finest-level triangles, shaped like the problem's kappa
    array ([ny][nx][2], lower then upper), and lambda_{h_n}."""
    hier = build(problem, b)
    G, lam = grad_kappa_levels(hier)
    n = problem.levels
    lv = hier.levels[n]
    E = lv.tris.shape[0]
    g = np.zeros(E)
    for ell in range(1, n + 1):
        # triangle e of level n descends from triangle e // 4^(n-ell) of level ell
        g += G[ell][np.arange(E) // (4 ** (n - ell))] * (4.0 ** (ell - n))
    tp = lv.tri_pts
    lo = tp.min(axis=1)
    se = lo + np.array([1, 0])
    t = np.where(np.any(np.all(tp == se[:, None, :], axis=2), axis=1), 0, 1)
    out = np.zeros((lv.ny, lv.nx, 2))
    out[lo[:, 1], lo[:, 0], t] = g
    return out, lam


def hellmann_feynman(problem: W.Problem, u_grid: np.ndarray):
    """Reference gradient int_T |grad u|^2 / int u^2 for a nodal field u on the finest level."""
    hier = build(problem)
    n = problem.levels
    lv = hier.levels[n]
    u = u_grid.ravel()[lv.key(lv.pts)]
    g = element_form(hier, n, u, u) / (u @ (hier.M[n] @ u))
    tp = lv.tri_pts
    lo = tp.min(axis=1)
    se = lo + np.array([1, 0])
    t = np.where(np.any(np.all(tp == se[:, None, :], axis=2), axis=1), 0, 1)
    out = np.zeros((lv.ny, lv.nx, 2))
    out[lo[:, 1], lo[:, 0], t] = g
    return out


def finest_kappa(problem: W.Problem, b: int = 0) -> np.ndarray:
    """Member b's kappa on every finest-level triangle, shaped [ny][nx][2] (lower, upper);
    zero outside the domain."""
    n = problem.levels
    ny, nx = problem.fine_ny, problem.fine_nx
    if problem.kappa_kind == W.KAPPA_PER_FINE_ELEM:
        return np.array(problem.kappa[b], dtype=np.float64)
    r = 1 << n
    mask = np.repeat(np.repeat(problem.cell_in, r, axis=0), r, axis=1).astype(np.float64)
    if problem.kappa_kind == W.KAPPA_ONE:
        kc = mask
    else:
        kc = np.repeat(np.repeat(np.asarray(problem.kappa[b], np.float64), r, axis=0), r, axis=1) * mask
    return np.repeat(kc[:, :, None], 2, axis=2).reshape(ny, nx, 2)


def solve_with_fine_kappa(problem: W.Problem, kappa_fine: np.ndarray) -> float:
    """lambda_{h_n} of Algorithm 4.2 for the problem's geometry with kappa given per finest
    triangle ([ny][nx][2])."""
    from dataclasses import replace

    from .multilevel import solve

    p = replace(problem, batch=1, kappa_kind=W.KAPPA_PER_FINE_ELEM, kappa=np.asarray(kappa_fine)[None])
    return solve(p).lam
