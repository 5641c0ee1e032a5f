#!/usr/bin/env python
"""Benchmark: quasi-static load steps per second of the single-edge notched square on a
1024 x 1024 crossed P1 mesh (6.3M dofs, AT1, ell = 4h, ORAM omega = 1.5, 50 load steps to
t = 0.6), mixed precision (FP32 inner solves, FP64 residuals and decisions) against the plain
FP64 GPU path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one load step (Algorithm 2 to convergence).  The W warm-up steps are the first W
steps of the schedule; the K timed steps are the next K (capped at the end of the schedule).
Replicas only: under torchrun every rank solves its own copy (no collective on the data path);
the time is the max over ranks and the value counts the steps of all ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "load steps/s at 1024^2 mesh (notched square, ORAM omega=1.5), mixed vs FP64 GPU"
UNIT = "load_steps/s"
L2_BYTES = 126.5e6
# load steps (1-based) of the 50-step schedule in which the damage grows: the crack starts from
# the notch at step 33, grows slowly to a near-critical state at step 34 and runs through the
# ligament at step 35; every timed sample holds them
GROWTH_STEPS = (33, 34, 35, 36)
# steps repeated in plain FP64 to measure the mixed-precision error on damage-growth steps
FP64_STEPS = (33, 36)
# iteration cap of alternate minimization: near-critical steps need well over 2000 iterations at
# 1024^2 (the paper's own AM counts reach 3382, Table 3)
AM_MAXIT = 20000


def select_steps(nsched: int, first: int, k: int, growth) -> list:
    """K schedule indices (0-based) from first .. nsched-1: all of them if K covers the range,
    else the damage-growth steps plus evenly spaced others, sorted."""
    avail = list(range(first, nsched))
    if k >= len(avail):
        return avail
    g = [s - 1 for s in growth if first <= s - 1 < nsched][:k]
    rest = [s for s in avail if s not in g]
    m = k - len(g)
    pick = set()
    for i in range(m):
        pick.add(rest[int(round(i * (len(rest) - 1) / max(m - 1, 1)))] if m > 1 else rest[0])
    for s in rest:  # rounding may have picked one twice
        if len(pick) >= m:
            break
        pick.add(s)
    return sorted(set(g) | pick)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=47)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--algo", choices=["ORAM", "ORAM_N"], default="ORAM",
                    help="ORAM (Algorithm 2) or ORAM-N (Algorithm 3)")
    ap.add_argument("--growth-steps", default=",".join(map(str, GROWTH_STEPS)),
                    help="comma-separated load steps always timed ('' : none; then one timed "
                         "step is the first after the warm-up)")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="damage-growth steps repeated in plain FP64 (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graphs", action="store_true",
                    help="host-driven CG loops (per-kernel profilers cannot see inside graphs)")
    ap.add_argument("--quiet", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=32,
                    help="jobs in the serving sample (0: no serving leg)")
    ap.add_argument("--serve-rate", type=float, default=8.0, help="Poisson arrivals per second")
    ap.add_argument("--serve-max-n", type=int, default=1024, help="largest serving mesh N")
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--serve-arena-gb", type=float, default=16.0)
    ap.add_argument("--serve-only", action="store_true", help="run the serving leg alone")
    ap.add_argument("--batch-instances", type=int, default=256,
                    help="instances in the batch leg (0: no batch leg)")
    ap.add_argument("--batch-workers", type=int, default=8)
    ap.add_argument("--configs", action="store_true",
                    help="whole schedules of the bar 128x16, the notched square 512^2 and the "
                         "thermal slab 1024x256, FP64 and mixed, then exit")
    ap.add_argument("--omega-sweep", action="store_true",
                    help="alternate-minimization iterations versus omega (Tables 1-3) on the "
                         "surfing, bar and thermal workloads, then exit")
    return ap.parse_args()


def log(args, *a):
    if not args.quiet:
        print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------------
class Clocks:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        smax = max((num(r[1]) or 0) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        loaded = [s for s in sm if s >= 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on a bounded sample
# ---------------------------------------------------------------------------------------------
ORACLE_SAMPLE = r"""
import sys, time, json
sys.path.insert(0, sys.argv[1])
import workloads as W
from oracle import am
from oracle.problem import Problem
out = {}
for n in (128, 256):
    w = W.notched_square(n=n)
    p = Problem(w)
    am.begin_step(p, *w.loads[int(sys.argv[2])])
    t0 = time.perf_counter()
    am.oram_iteration(p, w.omega, 0.0)
    out[n] = time.perf_counter() - t0
print(json.dumps(out))
"""


def oracle_iteration_seconds(target_n: int, step_index: int):
    """Seconds per ORAM iteration of the oracle at target_n^2, extrapolated with the size
    exponent fitted between one iteration at 128^2 and one at 256^2 (single thread)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", ORACLE_SAMPLE, ROOT, str(step_index)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    t = {int(k): v for k, v in json.loads(r.stdout.strip().splitlines()[-1]).items()}
    p = math.log(t[256] / t[128]) / math.log(4.0)  # node count grows 4x per refinement
    ratio = (target_n / 256.0) ** 2
    return t[256] * ratio ** p, t, p


def iterations_lower_bound(omega: float, tol: float) -> int:
    """ORAM iterations of a load step in which the damage does not move: the over-relaxed
    u-update contracts the error by |1 - omega| per iteration (Section 2.1)."""
    return int(math.ceil(math.log(tol) / math.log(abs(1.0 - omega)))) + 1


BAR_FULL_RUN = r"""
import sys, time, json
sys.path.insert(0, sys.argv[1])
import workloads as W
from oracle import am
from oracle.problem import Problem
w = W.bar()
p = Problem(w)
t0 = time.perf_counter()
its = 0
for (t, dT) in w.loads:
    r = am.load_step(p, t, dT, omega=w.omega, tol=1e-6)
    its += r["its"]
print(json.dumps({"seconds": time.perf_counter() - t0, "steps": len(w.loads), "its": its}))
"""


def oracle_bar_full_run():
    """Full oracle run of the 128 x 16 bar (Section 4.2, 20 load steps, AM, tol 1e-6), single
    thread: seconds, steps and AM iterations."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", BAR_FULL_RUN, ROOT], capture_output=True, text=True,
                       env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_record(size: int, step_index: int, am_iters_per_step: float):
    """The oracle (FP64, sparse LU, single thread) on the metric's workload: its time per ORAM
    iteration at size^2 extrapolated from one iteration at 128^2 and 256^2, times the mean AM
    iteration count per timed load step that the GPU run measured.  A full measured oracle run of
    the 128 x 16 bar is reported beside it."""
    it_s, t, p = oracle_iteration_seconds(size, step_index)
    bar = oracle_bar_full_run()
    return {"value": 1.0 / (it_s * am_iters_per_step), "unit": UNIT, "cores": 1, "kind": "oracle",
            "extrapolated": True, "host_cores": os.cpu_count(),
            "bar_128x16_full_run": {"seconds": bar["seconds"], "load_steps": bar["steps"],
                                    "am_iters": bar["its"],
                                    "load_steps_per_s": bar["steps"] / bar["seconds"]},
            "sample": (f"one ORAM iteration of the FP64 oracle (sparse LU solves) at 128^2 "
                       f"({t[128]:.1f}s) and 256^2 ({t[256]:.1f}s), load step {step_index + 1}; "
                       f"time per iteration extrapolated to {size}^2 with the fitted size exponent "
                       f"{p:.2f} ({it_s:.0f}s), times the GPU run's mean of "
                       f"{am_iters_per_step:.1f} AM iterations per timed load step; extrapolated. "
                       f"Measured in full: the 128x16 bar, 20 load steps, {bar['its']} AM "
                       f"iterations in {bar['seconds']:.1f}s")}


# ---------------------------------------------------------------------------------------------
# reference arm: the oracle timed on the host cores
# ---------------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import workloads as W
    from oracle import am
    from oracle.problem import Problem

    os.environ.setdefault("OMP_NUM_THREADS", "1")
    w = W.notched_square(n=args.size)
    t_big, t, p = oracle_iteration_seconds(args.size, args.warmup)
    n_small = 128
    ws = W.notched_square(n=n_small)
    prob = Problem(ws)
    scale = ((args.size / n_small) ** 2) ** p
    n_it = iterations_lower_bound(w.omega, 1e-6)
    nsteps = min(args.steps, len(w.loads) - args.warmup)
    for k in range(args.warmup):  # warm-up samples
        am.begin_step(prob, *ws.loads[k])
        am.oram_iteration(prob, ws.omega, 0.0)
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + nsteps):
        am.begin_step(prob, *ws.loads[k])
        am.oram_iteration(prob, ws.omega, 0.0)
    el = time.perf_counter() - t0
    per_it = el / nsteps * scale
    value = 1.0 / (per_it * n_it)
    sample = (f"each step: one ORAM iteration of the FP64 oracle at {n_small}^2 on load step k, "
              f"scaled to {args.size}^2 by the size exponent {p:.2f} fitted from 128^2/256^2 "
              f"iterations, times {n_it} iterations per load step (lower bound); extrapolated")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": nsteps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"notched_square_{args.size}_crossed_AT1_ORAM_omega1.5",
                       "mesh": f"{args.size}x{args.size} crossed P1", "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "host_cores": os.cpu_count(), "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------
def aggregate_max(value: float) -> float:
    """Max of a per-rank scalar over all ranks (1 rank: identity)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def traffic_from_profiles(kclass: str):
    """DRAM bytes per launch of a kernel class from the committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) >= 2 and parts[0] == kclass and not line.startswith("#"):
                try:
                    return float(parts[1])
                except ValueError:
                    return None
    return None


def serve_record(args, ctx):
    """Serving leg: a seeded Poisson stream of notched-square and bar jobs (N log-uniform on
    [32, serve_max_n], 10-60 load steps each, mixed precision) through the libpf request loop;
    per-load-step latency = end of the step minus the moment it became ready (arrival for the
    first step), so admission and worker queueing are included.  Jobs with N <= 64 are run again
    alone in plain FP64 afterwards, and their per-step energies compared."""
    import numpy as np

    import workloads as W
    from paper_1511_08463_gb300 import sim as S

    jobs = W.serving_stream(n_jobs=args.serve_jobs, rate=args.serve_rate, seed=0, lo=32,
                            hi=args.serve_max_n)
    arena = int(args.serve_arena_gb * 1e9)
    srv = S.Server(arena, workers=args.serve_workers, ctx=ctx)
    t0 = srv.now()
    mk = lambda w, prec: S.make_opts(omega=w.omega, precision=prec, am_maxit=AM_MAXIT)
    ids = [srv.submit(j.workload, opts=mk(j.workload, "mixed"), arrival=t0 + j.arrival,
                      fields=False) for j in jobs]
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    lat = np.concatenate([r["latency"] for r in res])
    ok = [r["status"] == 0 for r in res]
    lat_ok = np.concatenate([r["latency"] for r, g in zip(res, ok) if g] or [np.zeros(0)])
    svc = np.array([rep["seconds"] for r in res for rep in r["reports"]])
    makespan = max(r["finished"] for r in res) - t0
    last_arrival = max(r["arrival"] for r in res) - t0
    failed = []
    for j, r in zip(jobs, res):
        if r["status"] != 0:
            bad = [k for k, rep in enumerate(r["reports"]) if rep["status"] != 0]
            failed.append({"job": j.job_id, "workload": j.workload.name, "status": r["status"],
                           "steps_done": r["steps_done"], "steps": len(j.workload.loads),
                           "first_failing_step": bad[0] + 1 if bad else None})
    # FP64 reference runs of the small jobs, alone and in order
    errs = []
    for j, r in zip(jobs, res):
        w = j.workload
        if max(w.nx, w.ny) > 64 or r["status"] != 0:
            continue
        g = S.Sim(w, ctx)
        o = mk(w, "fp64")
        e = []
        for rep, ld in zip(r["reports"], w.loads):
            r64 = g.load_step(*ld, o, allow_notconv=True)
            e.append(abs(rep["energy"][2] - r64["energy"][2]) / abs(r64["energy"][2]))
        g.close()
        errs.append(max(e))
    pct = lambda a, q: float(np.percentile(a, q) * 1e3) if a.size else None
    return {
        "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
        "p50_ms_converged_jobs": pct(lat_ok, 50), "p99_ms_converged_jobs": pct(lat_ok, 99),
        "service_p50_ms": pct(svc, 50), "service_p99_ms": pct(svc, 99),
        "steps": int(lat.size), "steps_per_s": float(lat.size / makespan),
        "makespan_s": makespan, "last_arrival_s": last_arrival, "jobs": len(jobs),
        "jobs_not_ok": len(failed), "failed_jobs": failed,
        "max_rel_energy_err_vs_fp64": max(errs) if errs else None,
        "fp64_checked_jobs": len(errs),
        "workers": st["workers"], "max_active": st["max_active"],
        "arena_gb": st["arena_bytes"] / 1e9, "arena_peak_gb": st["arena_peak"] / 1e9,
        "sizes": sorted(max(j.workload.nx, j.workload.ny) for j in jobs),
        "sample": f"{len(jobs)} jobs, Poisson rate {args.serve_rate}/s (seed 0), notched squares "
                  f"and bars, N log-uniform 32..{args.serve_max_n} (multiple of 16), 10-60 load "
                  f"steps each, mixed precision, default tolerances, am_maxit {AM_MAXIT}; "
                  f"energy error: every step of each converged job with N <= 64 against the same "
                  f"job run alone in plain FP64",
    }


def configs_record(ctx):
    """Whole load schedules of the other configurations in mixed precision, and their steps before
    damage growth in plain FP64: load steps/s, AM iterations, steps not converged, the FP64/mixed
    time ratio over the same steps and the largest relative energy difference of mixed against
    FP64 over those steps."""
    import workloads as W
    from paper_1511_08463_gb300 import sim as S

    cases = {"bar_128x16_AT1_AM": W.bar(),
             "notched_512_crossed_AT1_ORAM_omega1.5": W.notched_square(n=512),
             "thermal_1024x256_AT1_ORAM_omega1.6": W.thermal_shock()}
    FP64_CONFIG_STEPS = {"bar_128x16_AT1_AM": 20, "notched_512_crossed_AT1_ORAM_omega1.5": 30,
                         "thermal_1024x256_AT1_ORAM_omega1.6": 9}
    out = {}
    for name, w in cases.items():
        rec = {}
        energies = {}
        for prec in ("fp64", "mixed"):
            g = S.Sim(w, ctx)
            o = S.make_opts(omega=w.omega, precision=prec, am_maxit=AM_MAXIT)
            # plain FP64 runs the steps before damage growth only (the growth steps take
            # minutes in FP64 at these sizes); mixed runs the whole schedule
            loads = w.loads if prec == "mixed" else w.loads[:FP64_CONFIG_STEPS[name]]
            t0 = time.perf_counter()
            reps = [g.load_step(*ld, o, allow_notconv=True) for ld in loads]
            dt = time.perf_counter() - t0
            g.close()
            energies[prec] = [r["energy"][2] for r in reps]
            if prec == "mixed":
                mixed_secs = [r["seconds"] for r in reps]
            rec[prec] = {"load_steps": len(reps), "seconds": dt, "load_steps_per_s": len(reps) / dt,
                         "am_iters": sum(r["am_iters"] for r in reps),
                         "max_am_iters_per_step": max(r["am_iters"] for r in reps),
                         "not_ok": sum(1 for r in reps if r["status"] != 0)}
        nf = len(energies["fp64"])
        rec["mixed_speedup_same_steps"] = (rec["fp64"]["seconds"] /
                                           sum(mixed_secs[:nf]))
        rec["max_rel_energy_diff_mixed_vs_fp64"] = max(
            abs(a - b) / max(abs(b), 1e-300) for a, b in zip(energies["mixed"], energies["fp64"]))
        out[name] = rec
    return out


def omega_sweep_record(ctx):
    """AM iterations and time of whole schedules for fixed omega in 1.0 .. 1.8 and the automated
    omega, on the three workloads of the paper's over-relaxation tables: surfing (Table 1), the
    bar (Table 2) and the thermal shock (Table 3), mixed precision, default tolerances."""
    import workloads as W
    from paper_1511_08463_gb300 import sim as S

    cases = {"surfing_52x26_ell0.2": W.surfing(nx=52, ny=26, ell=0.2, n_steps=8, t_max=1.2),
             "bar_128x16": W.bar(),
             "thermal_128x32": W.thermal_shock(nx=128, ny=32, n_steps=20)}
    out = {}
    for name, w in cases.items():
        rows = {}
        for om in (1.0, 1.2, 1.4, 1.6, 1.8, "auto"):
            opts = S.make_opts(omega=1.0 if om == "auto" else om, omega_auto=int(om == "auto"),
                               precision="mixed", am_maxit=AM_MAXIT)
            g = S.Sim(w, ctx)
            its, secs, bad = 0, 0.0, 0
            for ld in w.loads:
                r = g.load_step(*ld, opts, allow_notconv=True)
                its += r["am_iters"]
                secs += r["seconds"]
                bad += r["status"] != 0
            g.close()
            rows[str(om)] = {"am_iters": its, "seconds": round(secs, 3), "not_ok": bad}
        out[name] = rows
    return out


def batch_record(args, ctx):
    """Batch leg: seeded notched squares (N log-uniform on [64, 256] in multiples of 16, ell in
    [2h, 8h], nu in [0.2, 0.35]), one load step each from rest to t ~ U[0.5, 1] (before crack
    initiation, near t = 1.3 on these meshes), all through one pf_solve_batch call (concurrent
    host threads, one stream each), mixed precision."""
    import numpy as np
    import torch

    import workloads as W
    from paper_1511_08463_gb300 import sim as S

    ws = W.batch_of_notched(n_instances=args.batch_instances, seed=0, t_max=1.0)
    sims = [S.Sim(w, ctx) for w in ws]
    opts = S.make_opts(omega=ws[0].omega, precision="mixed", batch_workers=args.batch_workers)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, reps = S.solve_batch(sims, [w.loads[0] for w in ws], opts=opts, ctx=ctx)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    secs = np.array([r["seconds"] for r in reps])
    nodes = sum(g.n_nodes for g in sims)
    for g in sims:
        g.close()
    return {
        "instances": len(ws), "seconds": dt, "instances_per_s": len(ws) / dt,
        "workers": args.batch_workers, "worst_status": int(st),
        "not_converged": sum(1 for r in reps if r["status"] != 0),
        "step_p50_ms": float(np.percentile(secs, 50) * 1e3),
        "step_p99_ms": float(np.percentile(secs, 99) * 1e3),
        "mean_nodes": nodes / len(ws),
        "sample": f"{len(ws)} notched squares (seed 0), N log-uniform 64..256 (multiple of 16), "
                  f"ell ~ U[2h, 8h], nu ~ U[0.2, 0.35], one load step each from rest to "
                  f"t ~ U[0.5, 1] (pre-initiation), omega 1.6, mixed precision, one "
                  f"pf_solve_batch call with {args.batch_workers} host threads",
    }


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1511_08463_gb300 import _build

    if rank == 0:
        _build.build()
    barrier()
    import workloads as W
    from paper_1511_08463_gb300 import binding as B
    from paper_1511_08463_gb300 import sim as S

    lib = B.load()
    if args.configs:
        rec = configs_record(S.Context(local))
        if rank == 0:
            print(json.dumps({"configs": rec}), flush=True)
        return 0
    if args.omega_sweep:
        rec = omega_sweep_record(S.Context(local))
        if rank == 0:
            print(json.dumps({"omega_sweep": rec}), flush=True)
        return 0
    if args.serve_only:
        rec = serve_record(args, S.Context(local))
        if rank == 0:
            print(json.dumps({"serving": rec}), flush=True)
        return 0
    w = W.notched_square(n=args.size)
    nsched = len(w.loads)
    W0 = min(args.warmup, nsched - 1)
    K = max(1, min(args.steps, nsched - W0))
    ctx = S.Context(local)
    sim = S.Sim(w, ctx)
    opts = S.make_opts(algo=args.algo, omega=w.omega, precision=args.precision,
                       use_graphs=0 if args.no_graphs else 1, am_maxit=AM_MAXIT)
    log(args, f"[rank {rank}] nodes {sim.n_nodes} levels {sim.levels} workspace "
              f"{sim.workspace_bytes / 1e9:.2f} GB; warm-up {W0} steps")
    # warm-up: the first W0 steps
    for k in range(W0):
        sim.load_step(*w.loads[k], opts, allow_notconv=True)
    snap = sim.get_fields()
    torch.cuda.synchronize()

    # ---- kernel timing replay: load step W0+1 with graph capture off, every class timed with
    # CUDA events on the launching stream (events cannot bracket single launches in a graph)
    lib.pf_prof_reset()
    lib.pf_prof_enable(1, -1)
    popts = S.make_opts(algo=args.algo, omega=w.omega, precision=args.precision, use_graphs=0,
                        am_maxit=AM_MAXIT)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    sim.load_step(*w.loads[W0], popts, allow_notconv=True)
    p1.record()
    torch.cuda.synchronize()
    lib.pf_prof_enable(0, -1)
    prof_tab = B.prof_table()
    replay_s = p0.elapsed_time(p1) / 1e3
    dominant = max(prof_tab.items(), key=lambda kv: kv[1]["ms"])[0] if prof_tab else None
    sim.set_fields(*snap)
    torch.cuda.synchronize()
    # the FP64-data kernels: the same load step replayed on the FP64 path, per-launch times of
    # its FP64 kernels against the mixed path's double-float ones
    df_vs_fp64 = None
    if args.precision == "mixed" and world == 1:
        lib.pf_prof_reset()
        lib.pf_prof_enable(1, -1)
        sim.load_step(*w.loads[W0], S.make_opts(algo=args.algo, omega=w.omega, precision="fp64",
                                               use_graphs=0, am_maxit=AM_MAXIT),
                      allow_notconv=True)
        torch.cuda.synchronize()
        lib.pf_prof_enable(0, -1)
        tab64 = B.prof_table()
        sim.set_fields(*snap)
        torch.cuda.synchronize()
        pairs = [("elastic_resid_df_f64_l0", "elastic_resid_f64_l0"),
                 ("damage_grad_df_f64_l0", "damage_grad_f64_l0"),
                 ("damage_trial_df_f64_l0", "damage_trial_f64_l0"),
                 ("damage_q_df_f64_l0", "damage_q_f64_l0")]
        df_vs_fp64 = {}
        for a, b in pairs:
            if a in prof_tab and b in tab64 and prof_tab[a]["timed"] and tab64[b]["timed"]:
                ua = prof_tab[a]["ms"] * 1e3 / prof_tab[a]["timed"]
                ub = tab64[b]["ms"] * 1e3 / tab64[b]["timed"]
                df_vs_fp64[a] = {"df_us_per_launch": round(ua, 1), "fp64_kernel": b,
                                 "fp64_us_per_launch": round(ub, 1), "speedup": round(ub / ua, 2)}

    # ---- main pass over the schedule (CUDA graphs on) -------------------------------------------
    # Every step from W0+1 on runs in order, so each step starts from the state its predecessor
    # left.  The K timed steps are a stratified sample that always holds the damage-growth steps
    # (select_steps).  A timed step: copy the state in from pinned host memory (e2e only), the
    # load step, copy the state back (e2e only).  value: sum of the device-event intervals around
    # the timed load steps alone (state resident); e2e: events around copy-in, step and copy-out.
    growth = tuple(int(x) for x in args.growth_steps.split(",") if x.strip())
    timed = select_steps(nsched, W0, K, growth)
    last = max(timed)
    fp64_at = [k - 1 for k in FP64_STEPS if W0 <= k - 1 <= last] or [timed[0]]
    n = sim.n_nodes
    hu = torch.empty((n, 2), dtype=torch.float64, pin_memory=True)
    ha = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hp = torch.empty(n, dtype=torch.float64, pin_memory=True)
    lib.pf_prof_reset()
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    ev = {k: [torch.cuda.Event(enable_timing=True) for _ in range(4)] for k in timed}
    launches0 = lib.pf_launch_count()
    reps = {}
    before, after = {}, {}  # states around the steps the FP64 leg repeats
    synced = False  # the pinned host copy holds the current state
    for k in range(W0, last + 1):
        if k in fp64_at:
            before[k] = sim.get_fields()
        if k in ev:
            if not synced:  # refresh the host copy (outside the timed region)
                B.check(lib.pf_get_fields(sim.h, hu.data_ptr(), ha.data_ptr(), hp.data_ptr()))
            e = ev[k]
            e[0].record()
            B.check(lib.pf_set_fields(sim.h, hu.data_ptr(), ha.data_ptr(), hp.data_ptr()))
            e[1].record()
            reps[k] = sim.load_step(*w.loads[k], opts, allow_notconv=True)
            e[2].record()
            B.check(lib.pf_get_fields(sim.h, hu.data_ptr(), ha.data_ptr(), hp.data_ptr()))
            e[3].record()
            synced = True
        else:
            reps[k] = sim.load_step(*w.loads[k], opts, allow_notconv=True)
            synced = False
        if k in fp64_at:
            after[k] = sim.get_fields()
        log(args, f"[rank {rank}] step {k + 1}: {reps[k]['am_iters']} AM iterations, "
                  f"{reps[k]['seconds']:.2f} s, status {reps[k]['status']}"
                  f"{' (timed)' if k in ev else ''}")
    torch.cuda.synchronize()
    barrier()
    launches = lib.pf_launch_count() - launches0
    clk = clocks.stop()
    elapsed = sum(ev[k][1].elapsed_time(ev[k][2]) for k in timed) / 1e3
    elapsed_max = aggregate_max(elapsed)
    value = K * world / elapsed_max
    e2e_el = aggregate_max(sum(ev[k][0].elapsed_time(ev[k][3]) for k in timed) / 1e3)
    e2e_value = K * world / e2e_el
    run_steps = list(range(W0, last + 1))
    sched_s = sum(reps[k]["seconds"] for k in run_steps)

    # roofline of the dominant kernel class (from the timing replay)
    import json as _json

    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as fh:
            peaks = _json.load(fh)
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "of measured" if hbm_peak else "of fallback"
    hbm_peak = hbm_peak or 6800.0
    roof = None
    if dominant and prof_tab[dominant]["timed"]:
        d = prof_tab[dominant]
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        per_launch = d["bytes"] / d["timed"]
        traffic = traffic_from_profiles(dominant)
        roof = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "peak_source": peak_src,
                "traffic": traffic, "algorithmic_bytes_per_launch": per_launch,
                "avg_launch_us": d["ms"] * 1e3 / d["timed"], "launches": d["timed"],
                "share_of_replay_step": d["ms"] / 1e3 / replay_s,
                "measured_on": f"replay of load step {W0 + 1} with graph capture off"}

    # ---- FP64 GPU path on damage-growth steps ------------------------------------------------
    # Each repeated step starts from the state the mixed run started it from; reported per step:
    # both times, the relative energy difference and the max-norm field differences.
    # (extra legs run on single-GPU runs only; a failing extra leg reports its error in the line
    # instead of taking the measured metric with it)
    fp = None
    try:
        if world == 1 and args.fp64_steps > 0:
            o64 = S.make_opts(algo=args.algo, omega=w.omega, precision="fp64",
                              use_graphs=0 if args.no_graphs else 1, am_maxit=AM_MAXIT)
            rows = []
            for k in fp64_at[:args.fp64_steps]:
                sim.set_fields(*before[k])
                torch.cuda.synchronize()
                r64 = sim.load_step(*w.loads[k], o64, allow_notconv=True)
                u64, a64, _ = sim.get_fields()
                um, am_, _ = after[k]
                rm = reps[k]
                rows.append({
                    "step": k + 1, "fp64_s": r64["seconds"], "mixed_s": rm["seconds"],
                    "mixed_speedup": r64["seconds"] / rm["seconds"],
                    "am_iters_fp64": r64["am_iters"], "am_iters_mixed": rm["am_iters"],
                    "status_fp64": r64["status"], "status_mixed": rm["status"],
                    "rel_energy_diff": abs(rm["energy"][2] - r64["energy"][2]) / abs(r64["energy"][2]),
                    "u_maxnorm_rel_diff": float(np.abs(um - u64).max() / np.abs(u64).max()),
                    "alpha_maxnorm_diff": float(np.abs(am_ - a64).max())})
            fp = {"steps": [r["step"] for r in rows], "per_step": rows,
                  "fp64_steps_per_s": len(rows) / sum(r["fp64_s"] for r in rows),
                  "mixed_steps_per_s": len(rows) / sum(r["mixed_s"] for r in rows),
                  "mixed_speedup": sum(r["fp64_s"] for r in rows) / sum(r["mixed_s"] for r in rows),
                  "max_rel_energy_diff_mixed_vs_fp64": max(r["rel_energy_diff"] for r in rows),
                  "max_u_maxnorm_rel_diff": max(r["u_maxnorm_rel_diff"] for r in rows),
                  "max_alpha_maxnorm_diff": max(r["alpha_maxnorm_diff"] for r in rows)}
    except Exception as e:  # report, never fake
        fp = {"error": f"{type(e).__name__}: {e!s}"[:300]}

    # ---- CPU baseline -------------------------------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            mean_its = sum(reps[k]["am_iters"] for k in timed) / len(timed)
            cpu = cpu_baseline_record(args.size, W0, mean_its)
        except Exception as e:  # report, never fake
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"failed: {e!s}"[:300]}

    # ---- serving and batch legs (rank-local; rank 0 reports) ----------------------------------
    serving = batch = None
    n_dofs, ws_gb = 3 * sim.n_nodes, sim.workspace_bytes / 1e9
    do_serve = args.serve_jobs > 0 and world == 1
    do_batch = args.batch_instances > 0 and world == 1
    if do_serve or do_batch:
        sim.close()  # release the 1024^2 workspace first
        del sim
        torch.cuda.empty_cache()
    if do_serve:
        try:
            serving = serve_record(args, ctx)
        except Exception as e:  # report, never fake
            serving = {"error": f"{type(e).__name__}: {e!s}"[:300]}
    if do_batch:
        try:
            batch = batch_record(args, ctx)
        except Exception as e:  # report, never fake
            batch = {"error": f"{type(e).__name__}: {e!s}"[:300]}
        torch.cuda.empty_cache()

    if rank == 0:
        tr = [reps[k] for k in timed]
        run = [reps[k] for k in run_steps]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W0, "ms_per_step": elapsed_max / K * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {
                "workload": f"notched_square_{args.size}_crossed_AT1_{args.algo}_omega1.5",
                "mesh": f"{args.size}x{args.size} crossed P1", "dofs": n_dofs,
                "load_steps": (f"{len(timed)} timed of steps {W0 + 1}-{last + 1} of {nsched} "
                               f"(t up to {w.loads[-1][0]}): {[k + 1 for k in timed]}; the "
                               f"damage-growth steps {list(growth)} are always timed"),
                "precision": args.precision, "parallelism": f"replicas x{world}",
                "cuda_graphs": not args.no_graphs, "am_maxit": AM_MAXIT,
                "l2": f"inputs larger than L2: resident state + work buffers "
                      f"{ws_gb:.2f} GB per replica"},
            "clocks": clk, "gpu_launches": int(launches),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 32 * n,
                    "d2h_bytes_per_step": 32 * n, "steps": K,
                    "how": "per timed step: state copied in from pinned host memory, the load step, "
                           "state copied out, all inside the CUDA-event interval"},
            "schedule": {"steps": f"{W0 + 1}-{last + 1}", "load_steps_per_s": len(run_steps) / sched_s,
                         "seconds": sched_s, "not_ok": sum(1 for r in run if r["status"] != 0),
                         "how": "every step of the range run in order; host clock around each "
                                "pf_load_step"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "fp64_window": fp,
            "serving": serving,
            "batch": batch,
            "solver": {"algo": args.algo, "timed_steps": [k + 1 for k in timed],
                       "am_iters_per_step": [r["am_iters"] for r in tr],
                       "newton_iters_per_step": [r["newton_iters"] for r in tr],
                       "seconds_per_step": [round(r["seconds"], 3) for r in tr],
                       "status_per_step": [r["status"] for r in tr],
                       "phi_rel_per_step": [r["phi_norm"] / r["phi_start"] if r["phi_start"] > 0
                                            else 0.0 for r in tr],
                       "omega_bar_min_per_step": [r["omega_bar_min"] for r in tr],
                       "minres_iters": sum(r["krylov_iters_newton"] for r in tr),
                       "cg_u": sum(r["cg_iters_u"] for r in tr),
                       "cg_alpha": sum(r["cg_iters_alpha"] for r in tr),
                       "rs_iters": sum(r["rs_iters"] for r in tr),
                       "u_solves_reused": sum(r["u_solves_reused"] for r in tr),
                       "subproblems_not_converged": sum(r["u_notconv"] + r["alpha_notconv"]
                                                        for r in run),
                       "not_converged_steps": sum(1 for r in run if r["status"] != 0),
                       "final_energy": reps[last]["energy"]},
            "kernel_classes_replay_step": {k: {"ms": round(v["ms"], 3),
                                               "launches": v["launches"]}
                                           for k, v in sorted(prof_tab.items(),
                                                              key=lambda kv: -kv[1]["ms"])
                                           if v["ms"] >= 1.0 or "_df" in k},
            "df_kernels_vs_fp64": df_vs_fp64,
            "replay_step_seconds_no_graphs": replay_s,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
