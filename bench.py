#!/usr/bin/env python3
"""Benchmark of the multilevel local-and-parallel P1 eigensolver on GB300.

A step is one whole multilevel eigensolve (Algorithm 4.2: the level-1 eigenproblem,
then every correction step of Algorithm 4.1 with its local problems, gluing, G_{m+1}
problem and Rayleigh-Ritz) of the unit-square workload with a 16x16 coarse grid, 4x4
overlapping subdomains and 6 levels (finest 1024x1024, 1,046,529 unknowns), computed
in the mixed form (FP32 multigrid local solves + FP64 residual refinement).

Metric: fine-mesh DOF/s = unknowns of T_{h_n} / seconds per solve, whole job (all ranks).
Also reported: the same solve in plain FP64 on the GPU, the end-to-end rate through the
host-buffer C call, the roofline of the dominant kernel and the CPU oracle's rate.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mlev|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine-mesh DOF/s per multilevel eigensolve at rel lambda err <=1e-8, vs plain FP64 GPU; HBM %"
WORKLOAD = "c2: unit square, coarse 16x16, 4x4 subdomains (overlap 1, delta=H/2), 6 levels, finest 1024x1024"
REL_TOL = 1e-8


# Schedules (cycle and sweep counts) come from the autotuner: the fastest schedule whose
# eigenvalue stays within 0.25 x the 1e-8 bar of a conservative FP64 GPU solve, tuned
# separately for the mixed path and for the plain FP64 comparator (equal accuracy target).
# The timed result is then checked against the stored oracle eigenvalue.
TUNED = {"mixed": None, "fp64": None}


def autotune_safety():
    from paper_1401_4969_gb300 import autotune

    return autotune.SAFETY


def mixed_opts(mlev, graph=1):
    from paper_1401_4969_gb300 import autotune

    return autotune.apply(mlev.default_opts(precision=mlev.PREC_MIXED, use_graph=graph), TUNED["mixed"].opts)


def fp64_opts(mlev, graph=1):
    from paper_1401_4969_gb300 import autotune

    return autotune.apply(mlev.default_opts(precision=mlev.PREC_FP64, use_graph=graph), TUNED["fp64"].opts)


# ------------------------------------------------------------------ helpers
def dist_env():
    from paper_1401_4969_gb300 import replicas

    return replicas.env_ranks()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def start_clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def stop_clock_sampler(proc, fh, path, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    fh.close()
    rows = []
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != gpu_index:
            continue
        try:
            rows.append({"sm": float(parts[1]), "max": float(parts[2]), "power": float(parts[3]),
                         "hw": parts[5], "hwt": parts[6], "swt": parts[7], "pcap": parts[8]})
        except ValueError:
            continue
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
    top = max(r["power"] for r in rows)
    load = [r for r in rows if r["power"] >= 0.5 * top] or rows
    reasons = set()
    for r in load:
        for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                          ("pcap", "sw_power_cap")):
            if r[key].lower() == "active":
                reasons.add(name)
    return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["max"] for r in rows),
            "reasons": sorted(reasons), "samples": len(load)}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kern_mg.cu", "kern_mgfused.cu", "kern_common.cuh", "kern_blk.cuh"):
        with open(os.path.join(ROOT, "paper_1401_4969_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it still matches the source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch_full_size")


def golden_lambda():
    path = os.path.join(ROOT, "tests", "golden", "oracle_c2.json")
    with open(path) as f:
        return json.load(f)["members"]["0"]["lam"]


# ------------------------------------------------------------------ CPU oracle legs
ORACLE_SAMPLE_LEVELS = {"cpu_baseline": 5, "reference": 4}


def oracle_sample_cmd(levels):
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "import workloads as W\n"
        "from oracle import multilevel as ML\n"
        "p = W.config2(levels=%d)\n"
        "t = time.perf_counter(); h = ML.build(p); r = ML.solve(p, hier=h); dt = time.perf_counter() - t\n"
        "n = int((~h.levels[p.levels].boundary).sum())\n"
        "print(json.dumps({'seconds': dt, 'dofs': n, 'lam': r.lam}))\n" % (ROOT, levels))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    return [sys.executable, "-c", code], env


def run_oracle_sample(levels):
    cmd, env = oracle_sample_cmd(levels)
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def reference_arm(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    lv = ORACLE_SAMPLE_LEVELS["reference"]
    for _ in range(args.warmup):
        run_oracle_sample(lv)
    times, dofs = [], None
    for _ in range(args.steps):
        r = run_oracle_sample(lv)
        times.append(r["seconds"])
        dofs = r["dofs"]
    ms = 1e3 * statistics.mean(times)
    value = dofs / (ms / 1e3)
    sample = (f"oracle (FP64 NumPy/SciPy, sparse LU local/strip solves, dense Rayleigh-Ritz) on the same "
              f"geometry truncated to {lv} levels ({dofs} unknowns), one process, BLAS threads = 1")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + f" (sample: {lv} levels)", "global_batch": 1, "flush": "none (CPU)"},
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_adjoint(mlev, W, torch, reps=5):
    """dlambda/dkappa on the 512 x 512 per-triangle-kappa workload: forward solve time and
    mlev_grad_kappa time (forward with level checkpoints + reverse sweep), default mixed opts."""
    p = W.config5()
    s = mlev.Solver(p)
    o = mlev.default_opts(precision=mlev.PREC_MIXED)
    lam, _ = s.alloc_outputs()

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    fwd = timed(lambda: s.solve_into(o, lam))
    grad = timed(lambda: s.grad_kappa(o))
    s.close()
    return {"workload": "c5: unit square 16x16, 4x4 subdomains, 5 levels (512x512), kappa per finest triangle",
            "opts": "library defaults (mixed)", "forward_ms": fwd, "grad_ms": grad, "grad_over_forward": grad / fwd,
            "dofs": 511 * 511}


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mlev", choices=["mlev", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-kernel profiled pass")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing (512x512 kappa workload)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    args.warmup = max(args.warmup, 3)

    rank, local_rank, world = dist_env()
    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    cpu_base = None
    if rank == 0 and not args.no_cpu_baseline:
        # spawned before any CUDA work of this process matters; its own process, no CUDA
        cpu_base = subprocess.Popen(oracle_sample_cmd(ORACLE_SAMPLE_LEVELS["cpu_baseline"])[0],
                                    env=oracle_sample_cmd(ORACLE_SAMPLE_LEVELS["cpu_baseline"])[1],
                                    stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)

    import workloads as W
    from paper_1401_4969_gb300 import autotune, mlev, replicas

    p = W.config2()
    solver = mlev.Solver(p, device=local_rank)
    info = solver.info()
    # untimed: pick the schedules (cached per problem / precision / target / device)
    TUNED["mixed"] = autotune.tune(p, precision=mlev.PREC_MIXED, target_rel=REL_TOL, device=local_rank,
                                   solver=solver)
    if not args.no_fp64:
        TUNED["fp64"] = autotune.tune(p, precision=mlev.PREC_FP64, target_rel=REL_TOL, device=local_rank,
                                      solver=solver)
    n_units = info["n_fine"] * p.batch
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    lam, _ = solver.alloc_outputs(want_u=False)

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(opts, steps, warmup):
        for w in range(warmup):
            flush.fill_(w & 0xFF)
            solver.solve_into(opts, lam, None, stream)
        barrier()
        torch.cuda.synchronize()
        evs = []
        for k in range(steps):
            flush.fill_(k & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.solve_into(opts, lam, None, stream)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        barrier()
        ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        return replicas.max_over_ranks(ms, dist, "cuda")

    om = mixed_opts(mlev)
    rep = solver.solve_into(mixed_opts(mlev, graph=0), lam, None, stream, report=True)
    launches_per_step = rep["kernel_launches"]
    # nvidia-smi samples of the timed region (MLEV_BENCH_OUT: keep them in that directory)
    clk_path = os.path.join(os.environ.get("MLEV_BENCH_OUT", tempfile.gettempdir()), f"bench_clocks_r{rank}.csv")
    sampler, fh = start_clock_sampler(clk_path)
    ms_mixed = timed(om, args.steps, args.warmup)
    clocks = stop_clock_sampler(sampler, fh, clk_path, local_rank)
    value = world * n_units / (ms_mixed / 1e3)
    lam_mixed = float(lam[0].item())

    ms_fp64 = None
    lam_fp64 = None
    if not args.no_fp64:
        of = fp64_opts(mlev)
        ms_fp64 = timed(of, max(3, args.steps // 4), 2)
        lam_fp64 = float(lam[0].item())

    if args.no_e2e or args.no_profile:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": ms_mixed, "partial": "e2e/profile legs skipped",
                              "gpu_launches": launches_per_step * args.steps}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # end to end through the host-buffer entry point: plan tables in, lambda and u_{h_n} out
    ny, nx = solver.grid_shape()
    lam_h = torch.empty(p.batch, dtype=torch.float64, pin_memory=True).numpy()
    u_h = torch.empty((p.batch, ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    oh = mixed_opts(mlev, graph=1)  # graph replay, as in the device-timed leg
    io = solver.solve_host(oh, lam_h, u_h, report=True)
    solver.solve_host(oh, lam_h, u_h)
    e2e_t = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.solve_host(oh, lam_h, u_h)
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = replicas.max_over_ranks(1e3 * statistics.mean(e2e_t), dist, "cuda")
    e2e_lambda = float(lam_h[0])
    h2d, d2h = int(io["h2d_bytes"]), int(io["d2h_bytes"])

    # profiled pass: per-kernel-family CUDA-event times on the solve's stream
    op = mixed_opts(mlev, graph=0)
    op.profile = 1
    prof = None
    for _ in range(2):
        flush.fill_(1)
        solver.solve_into(op, lam, None, stream)
        prof = mlev.profile_read(solver)
    torch.cuda.synchronize()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    adjoint = None if args.no_adjoint else time_adjoint(mlev, W, torch)
    peak, peak_kind = measured_peaks()
    dom = max(prof, key=lambda r: r["ms"])
    with_bytes = [r for r in prof if r["bytes"] > 0]
    dom_hbm = max(with_bytes, key=lambda r: r["ms"])
    ach = (dom_hbm["bytes"] / dom_hbm["launches"]) / (dom_hbm["ms"] / dom_hbm["launches"] / 1e3) / 1e9
    traffic = ncu_traffic(dom_hbm["name"])
    total_prof_ms = sum(r["ms"] for r in prof)
    roofline = {"bound": "hbm", "kernel": dom_hbm["name"], "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": traffic, "launches_per_step": dom_hbm["launches"],
                "algorithmic_bytes_per_launch": dom_hbm["bytes"] / dom_hbm["launches"],
                "avg_launch_us": 1e3 * dom_hbm["ms"] / dom_hbm["launches"],
                "share_of_step": dom_hbm["ms"] / total_prof_ms,
                "top_kernel_by_time": dom["name"],
                "note": "working set of this workload (~90 MB) is L2-resident (129 MB L2); achieved is "
                        "algorithmic bytes over event time, so it can exceed the HBM peak"}

    gold = golden_lambda()
    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": p.batch * world, "dofs_per_problem": info["n_fine"],
                   "parallelism": f"replicas{world}" if world > 1 else "single", "precision": "mixed",
                   "flush": "L2 flushed (512 MB write) before every timed step",
                   "opts": dict(TUNED["mixed"].opts),
                   "opts_fp64": None if TUNED["fp64"] is None else dict(TUNED["fp64"].opts),
                   "autotune": {"target_rel": REL_TOL, "safety": autotune_safety(),
                                "reference": "FP64 GPU solve, 6 V-cycles x 2 passes",
                                "mixed_trials": len(TUNED["mixed"].trials),
                                "mixed_err_vs_reference": TUNED["mixed"].err,
                                "fp64_err_vs_reference": None if TUNED["fp64"] is None else TUNED["fp64"].err}},
        "accuracy": {"lambda": lam_mixed, "lambda_oracle": gold, "rel_err": abs(lam_mixed - gold) / gold,
                     "tol": REL_TOL,
                     "fp64_rel_err": None if lam_fp64 is None else abs(lam_fp64 - gold) / gold},
        "fp64_gpu": None if ms_fp64 is None else {"value": world * n_units / (ms_fp64 / 1e3), "unit": "DOF/s",
                                                  "ms_per_step": ms_fp64,
                                                  "speedup_mixed_over_fp64": ms_fp64 / ms_mixed},
        "e2e": {"value": world * n_units / (e2e_ms / 1e3), "unit": "DOF/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "call": "mlev_solve_host (plan tables H2D, graph-replayed solve, lambda + u_{h_n} D2H, pinned host buffers)",
                "lambda_matches_device_path": e2e_lambda == lam_mixed},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline,
        "profile": [{k: r[k] for k in ("name", "launches", "ms", "bytes")} for r in prof if r["launches"]],
        "clocks": clocks,
        "adjoint": adjoint,
    }
    if cpu_base is not None:
        out, err = cpu_base.communicate()
        try:
            r = json.loads(out.strip().splitlines()[-1])
            line["cpu_baseline"] = {
                "value": r["dofs"] / r["seconds"], "unit": "DOF/s", "cores": 1, "kind": "oracle",
                "sample": f"oracle Algorithm 4.2 on the same geometry truncated to "
                          f"{ORACLE_SAMPLE_LEVELS['cpu_baseline']} levels ({r['dofs']} unknowns), "
                          f"{r['seconds']:.1f} s, one process, BLAS threads = 1"}
        except Exception as e:  # report, do not hide
            line["cpu_baseline"] = {"error": f"{e}: {err[-300:]}"}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
