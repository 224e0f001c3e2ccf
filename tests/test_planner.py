"""Host planner (C++ side of the ABI) against the oracle's decomposition sets, on CPU.

The planner derives Omega_j, the closed G_j and the G_{m+1} unknowns from the
description of Section 4 independently of the oracle; the unknown counts must agree.
"""
import numpy as np
import pytest

import workloads as W
from oracle import multilevel as ML
from paper_1401_4969_gb300 import mlev


def _counts_oracle(p):
    h = ML.build(p)
    part = h.parts[p.levels]
    return {
        "n_fine": int((~h.levels[p.levels].boundary).sum()),
        "n_local_fine": int(sum(loc.size for loc in part.local)),
        "n_strip_fine": int(part.strip.size),
        "n_coarse": int((~h.levels[0].boundary).sum()),
    }


@pytest.mark.parametrize("make", [
    lambda: W.config1(),
    lambda: W.config2(levels=3),
    lambda: W.lshape(levels=3),
    lambda: W.lshape(levels=3, seed=7),
    lambda: W.unit_square(6, 3, 3, overlap=2, delta_in_H=0.25),
])
def test_planner_counts_match_oracle(make):
    p = make()
    s = mlev.Solver(p, device=-1)
    assert s.info() == _counts_oracle(p)
    assert s.workspace_bytes(mlev.default_opts()) > 0
    s.close()


def test_planner_rejects_bad_inputs():
    p = W.unit_square(4, 2, 3)
    p.delta = 0.3 * p.H
    with pytest.raises(mlev.MlevError) as e:
        mlev.Solver(p, device=-1)
    assert e.value.code == -1
    q = W.unit_square(4, 2, 3)
    q.cell_owner = q.cell_owner.copy()
    q.cell_owner[0, 0] = 3  # D_3 no longer a rectangle
    with pytest.raises(mlev.MlevError) as e:
        mlev.Solver(q, device=-1)
    assert e.value.code == -6
    r = W.unit_square(4, 2, 3)
    r.delta = 2.0 * r.H  # G_j would be empty
    with pytest.raises(mlev.MlevError):
        mlev.Solver(r, device=-1)


def test_planning_context_cannot_solve():
    s = mlev.Solver(W.config1(), device=-1)
    with pytest.raises(Exception):
        s.solve()
