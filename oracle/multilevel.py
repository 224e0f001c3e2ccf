"""Algorithm 4.2 (multilevel correction) with Algorithm 4.1 (one correction step) - oracle.

Notation follows Section 4: (lambda_{h_k}, u_{h_k}) is the eigenpair approximation on
level k (mesh size h_k = H / 2^k), V_{0H} the coarse space on T_H, e^j_{h_{k+1}} the
solution of the auxiliary problem (Eq. Aux_Problem) on Omega_j, u~^j = u_{h_k} + e^j,
u~ the glued function (step 2, with the G_{m+1} problem, Eq. G_m+1_Problem) and the
final Rayleigh-Ritz problem on V_{H,h_{k+1}} = V_{0H} + span{u~} (Eq. Eigen_Augment_Problem).

Readings where the paper is silent (listed in full in the design notes):
* h_k = H / 2^k, k = 1..n (T_{h_1} is one regular refinement of T_H).
* Normalisation b(u,u) = 1 (Section 3) and sign int_Omega u > 0.
* Step 2's right-hand side is lambda_{h_k} b(u_{h_k}, v) only: the unknown there is the
  whole function u~^{m+1}, not a correction.
* Interpolating u_{h_k} into V_{h_{k+1}} is exact (nested spaces, Section 4.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W

from . import fem
from .mesh import Level, build_levels, interpolation
from .partition import LevelPartition, level_partition, subdomains


@dataclass
class Hierarchy:
    problem: W.Problem
    b: int
    levels: list[Level]
    K: list[sp.csr_matrix]          # stiffness over all nodes, per level
    M: list[sp.csr_matrix]          # mass over all nodes, per level
    interp: list[sp.csr_matrix]     # interp[l]: level l -> l+1, all nodes
    parts: dict = field(default_factory=dict)
    ones_int: list = field(default_factory=list)


def build(problem: W.Problem, b: int = 0) -> Hierarchy:
    n = problem.levels
    levels = build_levels(problem.cell_in, n, problem.H)
    kap = fem.kappa_all_levels(problem, levels, b)
    K, M = [], []
    for ell, lv in enumerate(levels):
        k, m = fem.assemble(lv, kap[ell], problem.H)
        K.append(k)
        M.append(m)
    interp = [interpolation(levels[i], levels[i + 1]) for i in range(n)]
    hier = Hierarchy(problem, b, levels, K, M, interp)
    subs = subdomains(problem)
    for ell in range(2, n + 1):
        hier.parts[ell] = level_partition(problem, subs, levels[ell])
    hier.ones_int = [np.asarray(m.sum(axis=1)).ravel() for m in M]  # int phi_x per node
    return hier


def free(hier: Hierarchy, ell: int) -> np.ndarray:
    return np.nonzero(~hier.levels[ell].boundary)[0]


def coarse_basis(hier: Hierarchy, ell: int) -> sp.csr_matrix:
    """Columns: the hat functions of the free coarse nodes of T_H, as nodal vectors on level ell.

    These are the basis of V_{0H} embedded in V_{h_ell} by repeated exact interpolation.
    """
    P = sp.identity(hier.levels[0].nv, format="csr")
    for i in range(ell):
        P = hier.interp[i] @ P
    return P.tocsr()[:, free(hier, 0)]


def normalize(hier: Hierarchy, ell: int, u: np.ndarray) -> np.ndarray:
    """Scale a full nodal vector to b(u,u) = 1 and int_Omega u > 0."""
    M = hier.M[ell]
    u = u / np.sqrt(u @ (M @ u))
    if u @ hier.ones_int[ell] < 0:
        u = -u
    return u


def smallest_eigpair(K: sp.spmatrix, M: sp.spmatrix):
    """Smallest eigenpair of K x = lambda M x (dense LAPACK for small sizes, shift-invert otherwise)."""
    n = K.shape[0]
    if n <= 4000:
        w, v = sla.eigh(K.toarray(), M.toarray(), subset_by_index=[0, 0])
        return float(w[0]), v[:, 0]
    w, v = spla.eigsh(K.tocsc(), k=1, M=M.tocsc(), sigma=0.0, which="LM", tol=1e-14)
    return float(w[0]), v[:, 0]


def global_eigpair(hier: Hierarchy, ell: int):
    """Discrete eigenproblem (Eq. Discrete_Weak_Eigen_Problem) on V_{0h_ell}; full nodal vector."""
    f = free(hier, ell)
    lam, x = smallest_eigpair(hier.K[ell][f][:, f], hier.M[ell][f][:, f])
    u = np.zeros(hier.levels[ell].nv)
    u[f] = x
    return lam, normalize(hier, ell, u)


@dataclass
class StepTrace:
    lam: float
    u_tilde: np.ndarray
    e_local: list
    coeff: np.ndarray


def local_solve(args):
    """One auxiliary problem of step 1: the sparse direct solve A_j e = rhs_j (a top-level
    function, so a process pool can run the m independent solves of a level)."""
    A, rhs = args
    return spla.splu(A).solve(rhs)


def correction(hier: Hierarchy, k: int, lam_k: float, u_k: np.ndarray, trace: bool = False, mapper=map):
    """Algorithm 4.1: (lambda_{h_{k+1}}, u_{h_{k+1}}) = Correction(V_{0H}, lambda_{h_k}, u_{h_k}, V_{0h_{k+1}}).

    u_k is the full nodal vector on level k (zero on dOmega); returns the level-(k+1) pair.
    `mapper(fn, items)` runs the m independent local solves of step 1 (the built-in map by
    default; a process pool's map gives the paper's one-processor-per-subdomain model).
    """
    u = hier.interp[k] @ u_k                      # u_{h_k} as an element of V_{h_{k+1}} (exact embedding)
    return correction_on_level(hier, k + 1, lam_k, u, trace, mapper)


def correction_on_level(hier: Hierarchy, L: int, lam_k: float, u: np.ndarray, trace: bool = False, mapper=map):
    """Steps 1-3 of Algorithm 4.1 on level L for a given pair (lambda_{h_k}, u_{h_k}) already in V_{h_L}."""
    K, M = hier.K[L], hier.M[L]
    ut, e_list = glued(hier, L, lam_k, u, mapper)
    # Step 3 (Eq. Eigen_Augment_Problem): Rayleigh-Ritz on V_{0H} + span{u~}.
    f = free(hier, L)
    P = coarse_basis(hier, L)[f]
    Q = sp.hstack([P, sp.csr_matrix(ut[f][:, None])]).tocsr()
    Kf, Mf = K[f][:, f], M[f][:, f]
    A = (Q.T @ (Kf @ Q)).toarray()
    B = (Q.T @ (Mf @ Q)).toarray()
    A = 0.5 * (A + A.T)
    B = 0.5 * (B + B.T)
    w, c = sla.eigh(A, B, subset_by_index=[0, 0])
    un = np.zeros_like(u)
    un[f] = Q @ c[:, 0]
    un = normalize(hier, L, un)
    lam = float(w[0])
    if trace:
        return lam, un, StepTrace(lam, ut, e_list, c[:, 0])
    return lam, un


def glued(hier: Hierarchy, L: int, lam_k: float, u: np.ndarray, mapper=map):
    """Steps 1 and 2 of Algorithm 4.1 on level L: the local solutions and the glued function
    u~ (with the G_{m+1} problem) for the pair (lambda_{h_k}, u_{h_k}) already in V_{h_L}.
    Returns (u~, [e^j])."""
    K, M = hier.K[L], hier.M[L]
    part: LevelPartition = hier.parts[L]
    Mu = M @ u
    Ku = K @ u
    # Step 1 (Eq. Aux_Problem): a(e^j, v) = lambda_k b(u_k, v) - a(u_k, v) for v in V_{0h_{k+1}}(Omega_j)
    rhs = lam_k * Mu - Ku
    u_tilde_j, e_list = [], []
    sols = mapper(local_solve, [(K[loc][:, loc].tocsc(), rhs[loc]) for loc in part.local])
    for loc, x in zip(part.local, sols):
        e = np.zeros_like(u)
        e[loc] = x
        e_list.append(e)
        u_tilde_j.append(u + e)                    # u~^j = u_{h_k} + e^j on Omega_j
    # Step 2: u~ = u~^j on closed G_j, and on G_{m+1} solve Eq. G_m+1_Problem with Dirichlet data u~^j.
    ut = np.zeros_like(u)
    for j, g in enumerate(part.g_nodes):
        ut[g] = u_tilde_j[j][g]
    S = part.strip
    if S.size:
        # a(u~^{m+1}, v) = lambda_k b(u_k, v), v in V_{0h}(G_{m+1}); known values of u~ move to the right.
        rhs_s = lam_k * Mu[S] - (K[S] @ ut)        # ut is zero on S here
        ut[S] = spla.splu(K[S][:, S].tocsc()).solve(rhs_s)
    return ut, e_list


@dataclass
class Result:
    lam: float                 # lambda_{h_n}
    u: np.ndarray              # u_{h_n} on the full (ny+1) x (nx+1) node lattice, zero outside/on dOmega
    lam_levels: list           # lambda_{h_k}, k = 1..n
    traces: list = field(default_factory=list)


def to_grid(hier: Hierarchy, ell: int, u: np.ndarray) -> np.ndarray:
    lv = hier.levels[ell]
    g = np.zeros((lv.ny + 1) * (lv.nx + 1))
    g[lv.key(lv.pts)] = u
    return g.reshape(lv.ny + 1, lv.nx + 1)


def solve(problem: W.Problem, b: int = 0, trace: bool = False, hier: Hierarchy | None = None,
          mapper=map) -> Result:
    """Algorithm 4.2 for batch member b (`mapper` runs the local solves, see `correction`)."""
    hier = hier or build(problem, b)
    n = problem.levels
    lam, u = global_eigpair(hier, 1)               # step 1: eigenproblem in V_{0h_1}
    lams = [lam]
    traces = []
    for k in range(1, n):                          # step 3: k = 1 .. n-1
        out = correction(hier, k, lam, u, trace=trace, mapper=mapper)
        lam, u = out[0], out[1]
        if trace:
            traces.append(out[2])
        lams.append(lam)
    return Result(lam, to_grid(hier, n, u), lams, traces)
