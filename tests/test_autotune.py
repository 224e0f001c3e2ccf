"""Autotuner search logic and cache (CPU, with a model evaluator), and one GPU tuning run."""
import numpy as np
import pytest

import workloads as W
from paper_1401_4969_gb300 import autotune as AT


def _model(o):
    """Synthetic cost/accuracy model: error falls geometrically with cycles, time grows with them."""
    cyc = o["vcycles"] * o["refine_passes"]
    scyc = o["strip_vcycles"] * o["refine_passes"]
    err = 1e-3 * 0.03 ** min(cyc, scyc + 1) * (3.0 if o["pre_smooth"] == 1 else 1.0) + 1e-3 * o["level1_tol"]
    ms = (1.0 + 0.5 * cyc + 0.3 * scyc + 0.01 * o["coarse_sweeps"] + 0.2 * o["pre_smooth"] + (0.4 if not o["fused"] else 0)
          - 0.05 * np.log10(o["level1_tol"]))
    return ms, err


def test_search_picks_the_fastest_schedule_within_target():
    res = AT.search(_model, target_rel=1e-8)
    bar = AT.SAFETY * 1e-8
    assert all(t.err <= bar for t in res.trials if t.ok)
    ms, err = _model({**res.opts})
    assert err <= bar
    # no accepted trial is faster than the result
    assert min(t.ms for t in res.trials if t.ok) == pytest.approx(res.ms)
    # the model's error does not depend on the coarsest sweeps: the cheapest candidate wins
    assert res.opts["fused"] == 1 and res.opts["coarse_sweeps"] == 5
    # the level-1 target was loosened, and the next looser candidate broke the bar
    chosen = res.opts["level1_tol"]
    assert chosen in AT.LEVEL1_TOLS
    i = AT.LEVEL1_TOLS.index(chosen)
    if i + 1 < len(AT.LEVEL1_TOLS):
        looser = [t for t in res.trials if t.opts["level1_tol"] == AT.LEVEL1_TOLS[i + 1]]
        assert looser and not any(t.ok for t in looser)


def test_apply_keeps_float_keys():
    class O:
        pass

    o = AT.apply(O(), {"vcycles": 2.0, "level1_tol": 1e-6})
    assert o.vcycles == 2 and isinstance(o.vcycles, int) and o.level1_tol == 1e-6


def test_search_raises_when_nothing_meets_the_target():
    with pytest.raises(RuntimeError):
        AT.search(lambda o: (1.0, 1.0), target_rel=1e-8)


def test_candidates_are_in_increasing_work_order():
    c = AT.cycle_candidates()
    work = [x["vcycles"] * x["refine_passes"] + 0.5 * x["strip_vcycles"] * x["refine_passes"] for x in c]
    assert work == sorted(work)
    assert {"vcycles": 2, "refine_passes": 1, "strip_vcycles": 2} in c


def test_signature_changes_with_coefficient_and_geometry():
    a = W.kappa_coarse_batch(W.unit_square(8, 2, 3), batch=2, seed=1)
    b = W.kappa_coarse_batch(W.unit_square(8, 2, 3), batch=2, seed=2)
    c = W.kappa_coarse_batch(W.unit_square(8, 2, 4), batch=2, seed=1)
    assert len({AT.problem_signature(x) for x in (a, b, c)}) == 3
    assert AT.problem_signature(a) == AT.problem_signature(W.kappa_coarse_batch(W.unit_square(8, 2, 3), batch=2, seed=1))


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "t.json")
    AT._store_cache(path, {"k": {"opts": {"vcycles": 2}, "ms": 1.0, "err": 0.0}})
    assert AT._load_cache(path)["k"]["opts"]["vcycles"] == 2
    assert AT._load_cache(str(tmp_path / "missing.json")) == {}


@pytest.mark.gpu
def test_tuned_schedule_meets_target_against_oracle(tmp_path):
    from oracle import multilevel as ML
    from paper_1401_4969_gb300 import mlev

    p = W.kappa_coarse_batch(W.unit_square(8, 2, 4), batch=2, seed=3)
    res = AT.tune(p, target_rel=1e-8, cache_path=str(tmp_path / "tune.json"), reps=2)
    assert not res.cached
    again = AT.tune(p, target_rel=1e-8, cache_path=str(tmp_path / "tune.json"))
    assert again.cached and again.opts == res.opts
    s = mlev.Solver(p)
    lam, _, _ = s.solve(AT.apply(mlev.default_opts(), res.opts))
    s.close()
    lam = lam.cpu().numpy()
    for b in range(p.batch):
        ref = ML.solve(p, b=b).lam
        assert abs(lam[b] - ref) / ref <= 1e-8
