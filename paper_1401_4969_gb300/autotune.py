"""Autotuner for the solver's schedule: iteration counts and sweep counts per workload.

The paper takes every local and G_{m+1} solve as exact (Algorithm 4.1); the GPU path
replaces them by a fixed number of multigrid cycles, so how many cycles a workload needs
for a given eigenvalue accuracy is an empirical property of the problem (geometry, levels,
coefficient). The tuner measures it on the device:

1. a reference eigenvalue from a conservative FP64 solve (6 V-cycles, 2 passes),
2. candidate schedules timed with CUDA events (graph replay) and accepted when every batch
   member's eigenvalue is within `safety * target_rel` of the reference,
3. a staged search: first the cycle counts (vcycles, refine_passes, strip_vcycles) in
   increasing order of work, then the smoothing sweeps and coarsest-grid sweeps of the
   cheapest accepted schedule, then the residual target of the level-1 eigensolver (each
   correction step of Algorithm 4.1 contracts the error of the previous level's
   eigenvector, so level 1 need not be solved to rounding), then the size of the one-block
   tail of the fused V-cycle and the fused / unfused multigrid kernels.

The fastest accepted schedule is cached in a JSON file keyed by the problem's signature,
the precision, the target and the device name.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass, field

import numpy as np

TUNE_KEYS = ("vcycles", "refine_passes", "strip_vcycles", "pre_smooth", "post_smooth", "coarse_sweeps", "fused",
             "tail_nodes", "reg_depths", "level1_tol")
FLOAT_KEYS = ("level1_tol",)
# A schedule is accepted when every eigenvalue is within SAFETY * target_rel of the reference
# (a 4x margin to the target for what the reference itself and other inputs may add).
SAFETY = 0.25
LEVEL1_TOLS = (1e-8, 1e-6, 1e-4, 1e-3, 1e-2, 3e-2, 1e-1)  # level-1 residual targets tried, tightest first


def default_cache_path() -> str:
    p = os.environ.get("MLEV_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "mlev", "tune.json")


def problem_signature(problem) -> str:
    """Hash of everything that changes the solver's convergence: geometry, partition,
    levels, batch and coefficient values."""
    h = hashlib.sha256()
    for name in ("ncx", "ncy", "H", "delta", "levels", "batch", "kappa_kind"):
        h.update(repr(getattr(problem, name)).encode())
    for name in ("cell_in", "cell_owner", "overlap"):
        h.update(np.ascontiguousarray(getattr(problem, name)).tobytes())
    if getattr(problem, "kappa", None) is not None:
        h.update(np.ascontiguousarray(problem.kappa, dtype=np.float64).tobytes())
    return h.hexdigest()[:24]


def cycle_candidates() -> list[dict]:
    """(vcycles, refine_passes, strip_vcycles) in increasing order of V-cycle work."""
    out = []
    for vc in (1, 2, 3, 4, 5, 6, 8):
        for rp in (1, 2):
            for svc in (1, 2, 3, 4, 6, 8):
                if svc > vc + 2:
                    continue
                out.append({"vcycles": vc, "refine_passes": rp, "strip_vcycles": svc})
    out.sort(key=lambda c: (c["vcycles"] * c["refine_passes"] + 0.5 * c["strip_vcycles"] * c["refine_passes"],
                            c["refine_passes"]))
    return out


@dataclass
class Trial:
    opts: dict
    ms: float
    err: float
    ok: bool


@dataclass
class TuneResult:
    opts: dict
    ms: float
    err: float
    target_rel: float
    trials: list = field(default_factory=list)
    cached: bool = False

    def as_dict(self):
        return {"opts": self.opts, "ms": self.ms, "err": self.err, "target_rel": self.target_rel,
                "trials": [t.__dict__ for t in self.trials]}


def search(evaluate, target_rel: float, safety: float = SAFETY, base: dict | None = None,
           max_accept: int = 3, reg_legs: bool = True) -> TuneResult:
    """Staged search with an evaluator evaluate(opts dict) -> (ms, max relative error).

    Stage 1 walks the cycle candidates in increasing work and stops after `max_accept`
    accepted schedules; stage 2 lowers the smoothing and coarsest sweeps of the fastest
    accepted one and loosens the level-1 residual target; stage 3 compares the fused and
    unfused multigrid kernels, and for the hybrid the register-blocked legs on its finest
    one or two depths."""
    base = dict(base or {"pre_smooth": 2, "post_smooth": 2, "coarse_sweeps": 40, "fused": 1, "tail_nodes": 0,
                         "level1_tol": 1e-10})
    tol = safety * target_rel
    trials: list[Trial] = []

    def run(o):
        ms, err = evaluate(o)
        t = Trial(dict(o), float(ms), float(err), bool(err <= tol))
        trials.append(t)
        return t

    accepted = []
    for c in cycle_candidates():
        t = run({**base, **c})
        if t.ok:
            accepted.append(t)
            if len(accepted) >= max_accept:
                break
    if not accepted:
        raise RuntimeError(f"no schedule reached relative error {tol:g}; best trials: "
                           f"{sorted(trials, key=lambda t: t.err)[:3]}")
    best = min(accepted, key=lambda t: t.ms)
    for key, values in (("coarse_sweeps", (20, 10, 5)), ("pre_smooth", (1,)), ("post_smooth", (1,)),
                        ("level1_tol", LEVEL1_TOLS)):
        for v in values:
            t = run({**best.opts, key: v})
            if t.ok and t.ms < best.ms:
                best = t
    # kernel choice: fused tiles, one launch per operation, or the hybrid (per-operation
    # kernels on large grids, the one-block tail below tail_nodes), and the tail's size
    for fused, tn in ((0, 0), (2, 4096), (2, 1024), (2, 256), (1, 4096), (1, 1024)):
        t = run({**best.opts, "fused": fused, "tail_nodes": tn})
        if t.ok and t.ms < best.ms:
            best = t
    # the hybrid with the register-blocked legs (FP32 only) on its finest depths
    if reg_legs and best.opts.get("fused") == 2:
        for rd in (1, 2):
            t = run({**best.opts, "reg_depths": rd})
            if t.ok and t.ms < best.ms:
                best = t
    return TuneResult(opts={k: best.opts[k] for k in TUNE_KEYS if k in best.opts}, ms=best.ms, err=best.err,
                      target_rel=target_rel, trials=trials)


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(path, data):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cache_key(problem, precision: int, target_rel: float, device_name: str) -> str:
    return f"{problem_signature(problem)}/p{precision}/t{target_rel:g}/{device_name}"


def tune(problem, precision: int = 1, target_rel: float = 1e-8, device: int = 0, cache_path: str | None = None,
         use_cache: bool = True, reps: int = 5, solver=None) -> TuneResult:
    """Fastest schedule for `problem` whose eigenvalues stay within SAFETY * target_rel of a
    conservative FP64 reference solve on the same device. Results are cached."""
    import torch

    from . import mlev

    dev_name = torch.cuda.get_device_name(device)
    path = cache_path or default_cache_path()
    key = cache_key(problem, precision, target_rel, dev_name)
    if use_cache:
        hit = _load_cache(path).get(key)
        if hit:
            return TuneResult(opts=hit["opts"], ms=hit["ms"], err=hit["err"], target_rel=target_rel, cached=True)
    own = solver is None
    s = solver or mlev.Solver(problem, device=device)
    try:
        lam, _ = s.alloc_outputs()
        ref = mlev.default_opts(precision=mlev.PREC_FP64, vcycles=6, refine_passes=2, strip_vcycles=6)
        s.solve_into(ref, lam)
        lam_ref = lam.cpu().numpy().copy()
        stream = torch.cuda.current_stream(device)

        def evaluate(o):
            opts = mlev.default_opts(precision=precision, use_graph=1, **o)
            try:
                for _ in range(2):
                    s.solve_into(opts, lam, None, stream)
                torch.cuda.synchronize(device)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    s.solve_into(opts, lam, None, stream)
                e1.record(stream)
                torch.cuda.synchronize(device)
            except mlev.MlevError:
                return float("inf"), float("inf")
            err = float(np.max(np.abs(lam.cpu().numpy() - lam_ref) / np.abs(lam_ref)))
            return e0.elapsed_time(e1) / reps, err

        res = search(evaluate, target_rel, reg_legs=precision == mlev.PREC_MIXED)
    finally:
        if own:
            s.close()
    if use_cache:
        data = _load_cache(path)
        data[key] = {"opts": res.opts, "ms": res.ms, "err": res.err}
        _store_cache(path, data)
    return res


def apply(opts_struct, tuned: dict):
    """Copy a tuned schedule into an mlev Opts structure."""
    for k, v in tuned.items():
        setattr(opts_struct, k, float(v) if k in FLOAT_KEYS else int(v))
    return opts_struct


# ------------------------------------------------------------------ committed schedules
COMMITTED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "schedules.json")


def committed_key(workload: str, precision: int, target_rel: float, device_name: str) -> str:
    return f"{workload}/p{precision}/t{target_rel:g}/{device_name}"


def committed(workload: str, problem, precision: int, target_rel: float, device_name: str,
              path: str | None = None) -> dict | None:
    """The schedule this tuner chose for a named workload on a device and stored in
    schedules.json (None if absent, or if the workload's inputs changed since)."""
    entry = _load_cache(path or COMMITTED).get(committed_key(workload, precision, target_rel, device_name))
    if not entry or entry.get("signature") != problem_signature(problem):
        return None
    return entry


def tune_committed(workloads, out: str, target_rel: float = 1e-8, device: int = 0):
    """Tune each named workload of workloads.CONFIGS in both precisions and store the results
    (opts, time, error, problem signature) in `out`, keyed as committed() reads them."""
    import torch

    import workloads as W

    from . import mlev

    dev_name = torch.cuda.get_device_name(device)
    data = _load_cache(out)
    for name in workloads:
        p = W.CONFIGS[name]()
        s = mlev.Solver(p, device=device)
        try:
            for prec in (mlev.PREC_MIXED, mlev.PREC_FP64):
                r = tune(p, precision=prec, target_rel=target_rel, device=device, use_cache=False, solver=s)
                data[committed_key(name, prec, target_rel, dev_name)] = {
                    "opts": r.opts, "ms": r.ms, "err": r.err, "signature": problem_signature(p), "problem": p.name,
                    "trials": len(r.trials)}
                print(name, prec, r.opts, "%.3f ms" % r.ms, "err %.2e" % r.err, flush=True)
        finally:
            s.close()
        _store_cache(out, data)
    return data


if __name__ == "__main__":
    import argparse
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser(description="tune named workloads and store their schedules")
    ap.add_argument("workloads", nargs="+")
    ap.add_argument("--out", default=COMMITTED)
    ap.add_argument("--target", type=float, default=1e-8)
    a = ap.parse_args()
    tune_committed(a.workloads, a.out, a.target)
