"""Write the oracle's results for the full-size workloads to tests/golden/*.json.

Calls only the CPU oracle (oracle/) on the seeded inputs of workloads/; nothing here
comes from the CUDA path. Each file holds lambda_{h_k} for k = 1..n, u_{h_n} sampled
on a coarse sub-lattice (every `stride`-th node in x and y) and the moments
(phi_i, u_{h_n}) = b(phi_i, u_{h_n}) of u_{h_n} against every hat function phi_i of the
level-`MOMENT_LEVEL` mesh (a whole-field pin: every fine node enters some moment); the
gradient file holds the
oracle adjoint dlambda_{h_n}/dkappa on 20 seeded finest triangles, its maximum modulus and
the Euler sum sum_e kappa_e g_e; the several-eigenpairs file holds lambda_{i,h_k} for the
q smallest eigenpairs.

Usage: python tests/golden/make_golden.py [name ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import multilevel as ML  # noqa: E402


MOMENT_LEVEL = 2


def hat_moments(hier, n, u_grid, level=MOMENT_LEVEL):
    """b(phi_i, u) for the hats phi_i of the free nodes of T_{h_level}, u a level-n nodal grid."""
    lv = hier.levels[n]
    u = u_grid.ravel()[lv.key(lv.pts)]
    v = hier.M[n] @ u
    for k in range(n - 1, level - 1, -1):  # apply the transposed embeddings, level n -> level
        v = hier.interp[k].T @ v
    return v[ML.free(hier, level)]


def record(p, members, stride, moments=True):
    out = {"problem": p.name, "levels": p.levels, "batch": p.batch, "stride": stride, "members": {},
           "moment_level": MOMENT_LEVEL if moments else None}
    for b in members:
        t = time.time()
        hier = ML.build(p, b=b)
        r = ML.solve(p, b=b, hier=hier)
        out["members"][str(b)] = {
            "lam": r.lam,
            "lam_levels": r.lam_levels,
            "u_samples": r.u[::stride, ::stride].tolist(),
            "oracle_seconds": time.time() - t,
        }
        if moments:
            out["members"][str(b)]["moments"] = hat_moments(hier, p.levels, r.u).tolist()
        print(p.name, b, r.lam, "%.1fs" % (time.time() - t), flush=True)
    return out


def record_grad(p, n_el=20, seed=20):
    from oracle import adjoint as AD

    t = time.time()
    g, lam = AD.grad_kappa(p, b=0)
    rng = np.random.default_rng(seed)
    ny, nx, _ = g.shape
    els = []
    while len(els) < n_el:  # elements inside the domain (kappa > 0)
        j, i, tt = int(rng.integers(ny)), int(rng.integers(nx)), int(rng.integers(2))
        if p.kappa[0, j, i, tt] > 0 and (j, i, tt) not in [e[:3] for e in els]:
            els.append((j, i, tt, float(g[j, i, tt])))
    out = {"problem": p.name, "lam": lam, "elements": els, "max_abs": float(np.abs(g).max()),
           "euler_sum": float(np.sum(p.kappa[0] * g)), "oracle_seconds": time.time() - t}
    print(p.name, "grad", lam, "%.1fs" % (time.time() - t), flush=True)
    return out


def record_multi(p, q):
    """The q smallest eigenvalues of the subspace form (oracle/multiple.py), every level."""
    from oracle import multiple as MU

    t = time.time()
    r = MU.solve_multi(p, q)
    out = {"problem": p.name, "levels": p.levels, "q": q, "lams": r.lams.tolist(),
           "lam_levels": r.lam_levels.tolist(), "oracle_seconds": time.time() - t}
    print(p.name, "q =", q, r.lams, "%.1fs" % (time.time() - t), flush=True)
    return out


JOBS = {
    "c2": lambda: record(W.config2(), [0], 64),
    "c4": lambda: record(W.config4(), list(range(0, 256, 37)), 16),
    "c5": lambda: record(W.config5(), [0], 32),
    "c3n5": lambda: record(W.config3(levels=5), [0], 32),
    "c3n6": lambda: record(W.config3(levels=6), [0], 64),
    "c3": lambda: record(W.config3(), [0], 256, moments=False),
    "grad_c5": lambda: record_grad(W.config5()),
    "c2_q6": lambda: record_multi(W.config2(), 6),
}

if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for name in names:
        data = JOBS[name]()
        with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as f:
            json.dump(data, f)
