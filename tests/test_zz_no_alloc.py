"""The workspace-free entry point (mlev_solve_noalloc) against the workspace one.

mlev_solve_noalloc exists for callers that may not allocate device memory (a plugin whose
host owns every device allocation, or a loop that must never enter the CUDA allocator);
it runs the same kernels with a fixed array compiled into the library as workspace. This
file is collected last so that a run stopping at its first failure has run every other
test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import workloads as W
from oracle import multilevel as ML

pytestmark = pytest.mark.gpu


def _b_norm(p, d_grid):
    h = ML.build(p)
    lv = h.levels[p.levels]
    d = d_grid.ravel()[lv.key(lv.pts)]
    return float(np.sqrt(max(d @ (h.M[p.levels] @ d), 0.0)))


@pytest.mark.parametrize("make", [lambda: W.config1(),
                                  lambda: W.kappa_coarse_batch(W.unit_square(8, 2, 3), batch=2, seed=6)])
def test_noalloc_matches_workspace_entry_point_twice(make):
    from paper_1401_4969_gb300 import mlev

    p = make()
    s = mlev.Solver(p)
    o = mlev.default_opts()
    lam_ref, u_ref, _ = s.solve(o, want_u=True)
    lam_ref, u_ref = lam_ref.cpu().numpy(), u_ref.cpu().numpy()
    for call in range(2):  # the shared array keeps the previous call's contents
        lam, u = s.alloc_outputs(want_u=True)
        rep = s.solve_noalloc(o, lam, u, report=True)
        assert rep["status_flags"] == 0
        lam, u = lam.cpu().numpy(), u.cpu().numpy()
        for b in range(p.batch):
            assert abs(lam[b] - lam_ref[b]) <= 1e-8 * abs(lam_ref[b]), (call, b)
            assert _b_norm(p, u[b] - u_ref[b]) <= 1e-6, (call, b)
    s.close()


@pytest.mark.parametrize("graph", [0, 1])
def test_noalloc_contexts_take_turns_on_the_shared_array(graph):
    """Two contexts with different problems alternate on the one array (A, B, A, B): each
    call must bring its own plan tables back in, whether the solve is replayed from a
    graph or launched directly, and match mlev_solve on a workspace of its own."""
    from paper_1401_4969_gb300 import mlev

    probs = {"A": W.config1(), "B": W.kappa_coarse_batch(W.unit_square(8, 4, 3, overlap=1), batch=3, seed=11)}
    solvers = {k: mlev.Solver(p) for k, p in probs.items()}
    o = mlev.default_opts(use_graph=graph)
    ref = {}
    for k, s in solvers.items():
        lam, u, _ = s.solve(mlev.default_opts(), want_u=True)
        ref[k] = (lam.cpu().numpy(), u.cpu().numpy())
    for k in ("A", "B", "A", "B", "A"):
        s, p = solvers[k], probs[k]
        lam, u = s.alloc_outputs(want_u=True)
        s.solve_noalloc(o, lam, u)
        rep = s.solve_noalloc(o, lam, u, report=True)  # a warm call right after: no table copy
        assert rep["status_flags"] == 0 and rep["h2d_bytes"] == 0, (k, rep["h2d_bytes"])
        lam, u = lam.cpu().numpy(), u.cpu().numpy()
        for b in range(p.batch):
            assert abs(lam[b] - ref[k][0][b]) <= 1e-8 * abs(ref[k][0][b]), (k, b)
            assert _b_norm(p, u[b] - ref[k][1][b]) <= 1e-6, (k, b)
    for s in solvers.values():
        s.close()


def test_noalloc_rejects_problems_above_its_limit():
    from paper_1401_4969_gb300 import mlev

    p = W.config2()  # 1024^2 fine grid: its workspace is far above the fixed array
    s = mlev.Solver(p)
    assert s.workspace_bytes(mlev.default_opts()) > mlev.NOALLOC_WORKSPACE_BYTES
    lam, _ = s.alloc_outputs()
    with pytest.raises(mlev.MlevError) as e:
        s.solve_noalloc(mlev.default_opts(), lam)
    assert e.value.code == -2 and "at most" in str(e.value)
    s.close()
