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
