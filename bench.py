#!/usr/bin/env python
"""Benchmark of the restarted-PDHG hot path on one GB300 (or N replicas).

A step is one pass of the whole hot path over one synthetic LP: pdhg_create
(transpose, scaling, power iteration), pdhg_solve to eps_rel = 1e-4, pdhg_get
(float64 residual report) and pdhg_warmstart_point (Algorithm 1), with the
LP's arrays already resident on the device.  L2 is flushed (512 MiB write)
between steps, outside the timed events.

Prints ONE JSON line (rank 0).  ``value`` = PDHG iterations per second of the
whole job (all ranks' iterations / the slowest rank's summed step time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PDHG time-to-1e-4 KKT & iters/s; HBM GB/s vs peak; FP32-mix vs FP64 plain"
EPS = 1e-4
MAX_ITER = 2_000_000
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "powerlaw": ("planted LP m=200000 n=1000000 nnz=5000000, power-law row lengths "
                 "(exponent 2.1, 4..20000), 1% of rows x1e3, CSR int32, seed 0"),
    "powerlaw50m": ("planted LP m=2000000 n=10000000 nnz=50000000, power-law row lengths "
                    "(exponent 2.1, 4..20000), 1% of rows x1e3, CSR int32, seed 0"),
    "transport": ("balanced transportation LP 2000 supply x 2000 demand, m=4000 "
                  "n=4000000 nnz=8000000, seed 0"),
    "small": "planted LP m=200 n=500, 5 nnz per column, seed 0",
    "batch": ("512 planted LPs, m ~ floor(exp(U[ln 50, ln 5000])) (seed 0), n = floor(2.5 m), "
              "5 nnz per column, LP i seeded i (sum m=617840, sum n=1544469, sum nnz=7722345)"),
    "adjoint": ("64 planted LPs m=2000 n=5000, 5 nnz per column, seeds 0..63, targets "
                "U[0,1] seeded 1000+i; loss ||x - x_target||^2"),
    "hybrid": ("15 LPs: planted m in {500, 1000, 2000} (n = 2.5m, 5 nnz per column) x seeds "
               "0..2; transportation 20x30, 30x40, 40x60; power-law m=1000 n=5000 nnz=25000 "
               "(seeds 0, 1) and m=2000 n=10000 nnz=60000 (seed 0)"),
}


def hybrid_lps():
    from paper_2603_03150_gb300 import lpgen
    lps = [lpgen.planted_lp(m, int(2.5 * m), seed=s) for m in (500, 1000, 2000) for s in range(3)]
    lps += [lpgen.transportation_lp(a, b) for a, b in ((20, 30), (30, 40), (40, 60))]
    lps += [lpgen.powerlaw_lp(m=1000, n=5000, nnz=25000, k_max=500, seed=s) for s in (0, 1)]
    lps.append(lpgen.powerlaw_lp(m=2000, n=10000, nnz=60000, k_max=1000, seed=0))
    return lps


def make_lp(name):
    from paper_2603_03150_gb300 import lpgen
    if name == "powerlaw":
        return lpgen.powerlaw_lp()
    if name == "powerlaw50m":
        return lpgen.powerlaw_lp(m=2_000_000, n=10_000_000, nnz=50_000_000)
    if name == "transport":
        return lpgen.transportation_lp()
    return lpgen.planted_lp(200, 500, seed=0)


# ---------------------------------------------------------------------------
def shard_lps(weights, world_size):
    """Greedy balance of independent LPs over ranks by weight (nonzeros),
    heaviest first; returns sorted index lists, one per rank."""
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0] * world_size
    parts = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += weights[i]
    return [sorted(p) for p in parts]


def reduce_over_ranks(total_ms, units, device):
    """Max of the timed milliseconds and sum of the work units over ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None
        # raw samples beside the run (the summary goes into the JSON line)
        out_dir = os.environ.get("PDHG_BENCH_OUT", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return FALLBACK_HBM_GBS, "of fallback"


def kernel_source_sha():
    """Hash of the iteration kernels' sources with comments and blank space
    removed (a comment edit does not invalidate a measurement)."""
    import re
    h = hashlib.sha256()
    for f in ["spmv_tile.cuh", "iter_kernels.cu", "common.cuh", "epilogues.cuh", "panel.cu"]:
        src = open(os.path.join(ROOT, "paper_2603_03150_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, precision: str, workload: str, e_per_thread: int):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources and the same schedule variant (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(f"{workload}/{precision}/{kernel}/E{e_per_thread}")
    if not e or e.get("source_sha") != kernel_source_sha():
        return None
    return e.get("bytes_per_launch")


def algorithmic_bytes(m, n, nnz, s):
    """Bytes each kernel must move per launch (each matrix once, each dense
    vector once, gathered vector once).
      primal (rows of A^T): A^T col+val, row_ptr; gather y; read x, c, x_avg;
                            write x, x_avg
      dual   (rows of A):   A col+val, row_ptr; gather x; read y, b, Ax, y_avg,
                            Ax_avg; write y, Ax, y_avg, Ax_avg"""
    primal = nnz * (4 + s) + 4 * (n + 1) + s * (m + 5 * n)
    dual = nnz * (4 + s) + 4 * (m + 1) + s * (n + 9 * m)
    return {"primal": primal, "dual": dual}


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2603_03150_gb300 import build as B
    from paper_2603_03150_gb300 import pdhg

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)
    lp = make_lp(args.workload)
    m, n, nnz = lp.m, lp.n, lp.nnz
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(lp, k))) for k in
            ["row_ptr", "col", "val", "b", "c"]}
    devt = {k: v.to(dev) for k, v in host.items()}
    pinned = {k: v.pin_memory() for k, v in host.items()}
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run_steps(precision, k, w, device_io=True, method=None, omega_rule=None):
        """k timed steps after w untimed ones; each step's GPU timeline split
        by events on the solver's stream: create | solve | get + Algorithm 1."""
        outs = None
        if not device_io:
            mk = lambda L: torch.empty(L, dtype=torch.float64).pin_memory()
            outs = ((mk(n), mk(m), mk(n)), (mk(n), mk(m), mk(n)))
        src = devt if device_io else pinned
        rec = []
        for i in range(w + k):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            stream.synchronize()
            ev[0].record(stream)
            s = pdhg.Solver(m, n, src["row_ptr"], src["col"], src["val"], src["b"], src["c"],
                            precision=precision, device_io=device_io, stream=stream.cuda_stream,
                            method=method or args.method, spmv_layout=args.layout,
                            omega_rule=omega_rule or args.omega_rule, step_rule=args.step_rule)
            ev[1].record(stream)
            st = s.solve(EPS, args.max_iter)
            ev[2].record(stream)
            g = s.get(out=outs[0] if outs else None)
            s.warmstart_point(unscaled=True, out=outs[1] if outs else None)
            ev[3].record(stream)
            stream.synchronize()
            # outside the timed region: counters, the Section 4.3 violation
            info = s.info(violation=True)
            launches = s.launch_count()
            checks = s.fp64_checks()
            sched = s.schedule()
            layout = s.layout()
            s.close()
            if i >= w:
                rec.append(dict(ms=ev[0].elapsed_time(ev[3]), create_ms=ev[0].elapsed_time(ev[1]),
                                solve_ms=ev[1].elapsed_time(ev[2]),
                                get_ms=ev[2].elapsed_time(ev[3]), iters=info["iters"], status=st,
                                r_P=g["r_P"], r_D=g["r_D"], gap=g["gap"],
                                max_violation=info["max_violation"], launches=launches,
                                fp64_checks=checks, sched=sched, layout=layout,
                                obj=float(torch.dot(torch.as_tensor(g["x"]).to(dev),
                                                    devt["c"]).item())))
        return rec

    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        rec = run_steps(args.precision, args.steps, args.warmup)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    total_ms = sum(r["ms"] for r in rec)
    total_it = sum(r["iters"] for r in rec)
    solve_ms = sum(r["solve_ms"] for r in rec)
    if ws > 1:
        total_ms, total_it_all = reduce_over_ranks(total_ms, total_it, dev)
    else:
        total_it_all = float(total_it)
    value = total_it_all / (total_ms / 1e3)

    # end to end: host (pinned) inputs and outputs through the C ABI
    e2e_rec = run_steps(args.precision, max(1, args.steps), 1, device_io=False)
    e2e_ms = sum(r["ms"] for r in e2e_rec)
    e2e_val = sum(r["iters"] for r in e2e_rec) / (e2e_ms / 1e3) * ws
    h2d = 4 * (m + 1) + 4 * nnz + 8 * nnz + 8 * m + 8 * n
    d2h = 2 * 8 * (2 * n + m)

    # FP64 plain on the same GPU
    fp64 = None
    if args.fp64_steps > 0 and args.precision != "fp64":
        r64 = run_steps("fp64", args.fp64_steps, 1)
        fp64 = dict(time_to_eps_s=float(np.mean([r["ms"] for r in r64]) / 1e3),
                    create_ms=float(np.mean([r["create_ms"] for r in r64])),
                    solve_ms=float(np.mean([r["solve_ms"] for r in r64])),
                    iters=int(np.mean([r["iters"] for r in r64])),
                    iter_per_s=sum(r["iters"] for r in r64) / (sum(r["ms"] for r in r64) / 1e3),
                    solve_iter_per_s=sum(r["iters"] for r in r64) /
                    (sum(r["solve_ms"] for r in r64) / 1e3),
                    status=[pdhg.STATUS_NAMES.get(r["status"], r["status"]) for r in r64],
                    max_violation=max(r["max_violation"] for r in r64), objective=r64[-1]["obj"])

    # cuPDLP+'s PID primal weight, with the averaged and the Halpern iteration,
    # on the same workload and precision (not the default: the timed steps
    # above run the options the parity tests pin)
    variants = {}
    if (args.variant_steps > 0 and args.method == "averaged" and args.omega_rule == "smooth" and
            args.step_rule == "constant"):
        for name, meth in (("pid", "averaged"), ("halpern_pid", "halpern")):
            rv = run_steps(args.precision, args.variant_steps, 1, method=meth, omega_rule="pid")
            variants[name] = dict(
                method=meth, omega_rule="pid",
                time_to_eps_s=float(np.mean([r["ms"] for r in rv]) / 1e3),
                create_ms=float(np.mean([r["create_ms"] for r in rv])),
                solve_ms=float(np.mean([r["solve_ms"] for r in rv])),
                iters=int(np.mean([r["iters"] for r in rv])),
                iter_per_s=sum(r["iters"] for r in rv) / (sum(r["ms"] for r in rv) / 1e3),
                status=[pdhg.STATUS_NAMES.get(r["status"], r["status"]) for r in rv],
                max_violation=max(r["max_violation"] for r in rv), objective=rv[-1]["obj"])

    # roofline of the dominant half-step: back-to-back launches of each
    # half-step on a solved iterate of the same LP (pdhg_time_kernels: CUDA
    # events around the run, none between launches), after the timed steps.
    # On the CSR tiles a half-step is one fused kernel; on the column panels
    # it is the panel SpMV plus the row pass, and the pair is the unit whose
    # algorithmic bytes are counted (the panel partial sums are not).
    s_bytes = 4 if args.precision == "fp32" else 8
    ab = algorithmic_bytes(m, n, nnz, s_bytes)
    with torch.cuda.stream(stream):
        sk = pdhg.Solver(m, n, devt["row_ptr"], devt["col"], devt["val"], devt["b"], devt["c"],
                         precision=args.precision, device_io=True, stream=stream.cuda_stream,
                         method=args.method, spmv_layout=args.layout, omega_rule=args.omega_rule,
                         step_rule=args.step_rule)
        sk.solve(EPS, args.max_iter)
        kt = sk.time_kernels(args.kernel_reps)
        gf = {"dual": sk.gather_floor(True, 20), "primal": sk.gather_floor(False, 20)}
        lay = sk.layout()
        sched = sk.schedule()
        sk.close()
    on_panels = {"primal": lay["at"]["panels"] > 0, "dual": lay["a"]["panels"] > 0}
    half = {"primal": kt["primal_ms"], "dual": kt["dual_ms"]}
    spmv = {"primal": kt["primal_spmv_ms"], "dual": kt["dual_spmv_ms"]}
    names = {"primal": ("k_panel_spmv + k_panel_primal" if on_panels["primal"] else "k_primal"),
             "dual": ("k_panel_spmv + k_panel_dual" if on_panels["dual"] else "k_dual")}
    dom = "primal" if half["primal"] >= half["dual"] else "dual"
    oth = "dual" if dom == "primal" else "primal"
    dur = half[dom]
    peak, peak_src = peaks()
    ach = ab[dom] / (dur / 1e3) / 1e9 if dur > 0 else 0.0
    variant = sched["at_variant" if dom == "primal" else "a_variant"]
    it_bytes = ab["primal"] + ab["dual"]
    it_ms = kt["iteration_ms"]
    solve_it_ms = solve_ms / max(total_it, 1)
    roofline = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4),
                "traffic": ncu_traffic(("panel_" + dom) if on_panels[dom] else
                                       ("k_primal" if dom == "primal" else "k_dual"),
                                       args.precision, args.workload,
                                       "panels" if on_panels[dom] else variant),
                "kernel": names[dom], "half_step": dom,
                "layout": "column panels" if on_panels[dom] else "CSR tiles",
                "peak_source": peak_src, "algorithmic_bytes_per_launch": ab[dom],
                "mean_launch_ms": round(dur, 5),
                "timing": f"pdhg_time_kernels: {args.kernel_reps} back-to-back launches of each "
                          "half-step on a solved iterate of the same LP, CUDA events on the "
                          "launching stream around the run",
                "kernels_ms": {"spmv_or_fused": round(spmv[dom] if on_panels[dom] else dur, 5),
                               "row_pass": round(dur - spmv[dom], 5) if on_panels[dom] else None},
                "other": {"kernel": names[oth], "mean_launch_ms": round(half[oth], 5),
                          "achieved_gbs": round(ab[oth] / (max(half[oth], 1e-9) / 1e3) / 1e9, 1),
                          "spmv_ms": round(spmv[oth], 5) if on_panels[oth] else None},
                "iteration": {"algorithmic_bytes": it_bytes, "ms": round(it_ms, 5),
                              "achieved_gbs": round(it_bytes / (it_ms / 1e3) / 1e9, 1) if it_ms else None,
                              "frac": round(it_bytes / (it_ms / 1e3) / 1e9 / peak, 4) if it_ms else None,
                              "in_solve_ms": round(solve_it_ms, 5),
                              "in_solve_frac": round(it_bytes / (solve_it_ms / 1e3) / 1e9 / peak, 4),
                              "note": "in_solve: the timed steps' pdhg_solve time / iterations "
                                      "(evaluations, restarts and float64 checks included)"}}
    roofline["gather_floor"] = {
        "what": "mean ms of a pass over the same nonzeros keeping only the index/value loads, "
                "the random gathers and one FMA each (no row logic, scan or epilogue)",
        "dual_ms": round(gf["dual"], 5), "primal_ms": round(gf["primal"], 5),
        "frac": round(gf[dom] / dur, 4) if dur > 0 else None,
        "note": "frac > 1: the half-step beats the cost of L1/L2 gathers (column panels "
                "gather from shared memory)"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(lp, args.cpu_iters, args.method, args.omega_rule, args.step_rule)

    if rank == 0:
        ms_step = total_ms / max(len(rec), 1)
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "iter/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "precision": args.precision +
                       ("_mixed (f64 norms, gap, restart rule, step/weight updates)" if args.precision == "fp32" else ""),
                       "eps_rel": EPS, "method": args.method, "omega_rule": args.omega_rule,
                       "step_rule": args.step_rule,
                       "layout": args.layout,
                       "step": "create + solve to eps + get + warmstart_point (create and "
                               "solve also reported apart)",
                       "l2": "flushed between steps (512 MiB write), inputs resident in HBM",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "schedule": rec[0]["sched"]},
            "time_to_eps_s": round(ms_step / 1e3, 5),
            "create_ms": round(float(np.mean([r["create_ms"] for r in rec])), 3),
            "solve_ms": round(solve_ms / max(len(rec), 1), 3),
            "solve_iter_per_s": round(total_it / (solve_ms / 1e3), 2),
            "get_and_warmstart_ms": round(float(np.mean([r["get_ms"] for r in rec])), 3),
            "iters_to_eps": int(np.mean([r["iters"] for r in rec])),
            "max_violation": max(r["max_violation"] for r in rec),
            "fp64_checks": {"run": int(sum(r["fp64_checks"][0] for r in rec)),
                            "rejected": int(sum(r["fp64_checks"][1] for r in rec))},
            "status": [pdhg.STATUS_NAMES.get(r["status"], r["status"]) for r in rec],
            "kkt_at_exit": {"r_P": rec[-1]["r_P"], "r_D": rec[-1]["r_D"], "gap": rec[-1]["gap"]},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_val, 2), "unit": "iter/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms / len(e2e_rec), 3)},
            "gpu_launches": int(sum(r["launches"] for r in rec)),
            "clocks": clk.summary(),
        }
        if lp.x_star is not None:
            obj = float(lp.c @ lp.x_star)
            line["objective_rel_err_vs_planted"] = abs(rec[-1]["obj"] - obj) / (1 + abs(obj))
            if fp64:
                fp64["objective_rel_err_vs_planted"] = abs(fp64["objective"] - obj) / (1 + abs(obj))
        for v in variants.values():
            if lp.x_star is not None:
                obj = float(lp.c @ lp.x_star)
                v["objective_rel_err_vs_planted"] = abs(v["objective"] - obj) / (1 + abs(obj))
            if fp64:
                v["objective_rel_err_vs_fp64"] = (abs(v["objective"] - fp64["objective"]) /
                                                  (1 + abs(fp64["objective"])))
        if variants:
            line["variants"] = variants
        if fp64:
            line["fp64"] = fp64
            line["objective_rel_err_vs_fp64"] = (abs(rec[-1]["obj"] - fp64["objective"]) /
                                                 (1 + abs(fp64["objective"])))
            line["fp32_vs_fp64_time_speedup"] = round(fp64["time_to_eps_s"] / (ms_step / 1e3), 3)
            line["fp32_vs_fp64_solve_speedup"] = round(fp64["solve_ms"] / (solve_ms / max(len(rec), 1)), 3)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_batch(args):
    """Batched solve of the 512-LP workload (FP32-mixed and FP64) against 512
    sequential FP64 single-LP solves on the same GPU.  Ranks take disjoint
    shards of the LPs (no collective on the data path)."""
    import torch
    import torch.distributed as dist

    from paper_2603_03150_gb300 import build as B
    from paper_2603_03150_gb300 import lpgen, pdhg

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)
    all_lps = lpgen.planted_batch(512)
    mine = shard_lps([lp.nnz for lp in all_lps], ws)[rank]
    lps = [all_lps[i] for i in mine]
    # inputs resident in HBM before the timed region (as the headline line);
    # the e2e figure below starts from the Python LP objects on the host
    host = dict(m=np.array([lp.m for lp in lps], dtype=np.int32),
                n=np.array([lp.n for lp in lps], dtype=np.int32),
                row_ptr=np.concatenate([np.asarray(lp.row_ptr, np.int32) for lp in lps]),
                col=np.concatenate([np.asarray(lp.col, np.int32) for lp in lps]),
                val=np.concatenate([np.asarray(lp.val, np.float64) for lp in lps]),
                b=np.concatenate([np.asarray(lp.b, np.float64) for lp in lps]),
                c=np.concatenate([np.asarray(lp.c, np.float64) for lp in lps]))
    dev_arrays = {k: (v if k in ("m", "n") else torch.from_numpy(v).to(dev)) for k, v in host.items()}
    dev_lps = [{k: torch.from_numpy(np.ascontiguousarray(getattr(lp, k))).to(dev)
                for k in ("row_ptr", "col", "val", "b", "c")} for lp in lps]

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    def batched(precision, from_host=False, persistent=0):
        if from_host:
            s = pdhg.BatchSolver(lps, precision=precision)
        else:
            s = pdhg.BatchSolver(arrays=dev_arrays, precision=precision, device_io=True,
                                 persistent=persistent)
        st = s.solve(EPS, args.max_iter)
        g = s.get()
        n_launch = s.launch_count()
        s.close()
        return st, g, n_launch

    res = {}
    # graph of per-half-step launches (default) and one persistent cooperative launch
    for prec, persistent in (("fp32", 0), ("fp64", 0), ("fp32", 1), ("fp64", 1)):
        for _ in range(max(1, args.warmup - 2)):
            batched(prec, persistent=persistent)
        ms = []
        for _ in range(args.steps):
            t, (st, g, nl) = timed(lambda: batched(prec, persistent=persistent))
            ms.append(t)
        res[prec + ("_persistent" if persistent else "")] = dict(
            ms=float(np.mean(ms)), status=int(st), iters_max=int(g["iters"].max()),
            iters_median=int(np.median(g["iters"])),
            max_violation_max=float(g["max_violation"].max()), kernel_launches=int(nl))

    def sequential():
        it = []
        for lp, d in zip(lps, dev_lps):
            with pdhg.Solver(lp.m, lp.n, d["row_ptr"], d["col"], d["val"], d["b"], d["c"],
                             device_io=True) as s1:
                s1.solve(EPS, args.max_iter)
                s1.get()
                it.append(s1.info(violation=False)["iters"])
        return it

    t_seq, seq_it = timed(sequential)
    e2e_ms = float(np.mean([timed(lambda: batched("fp32", from_host=True))[0]
                            for _ in range(args.steps)]))
    total_ms = res["fp32"]["ms"]
    units = len(lps)
    if ws > 1:
        total_ms, units = reduce_over_ranks(total_ms, units, dev)
    if rank == 0:
        line = {"metric": "LPs solved to eps_rel=1e-4 per second (batched, FP32-mixed)",
                "value": round(units / (total_ms / 1e3), 2), "unit": "LP/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms, 2),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": {"workload": WORKLOADS["batch"], "eps_rel": EPS,
                                                "step": "batch create + solve + get, inputs "
                                                        "resident in HBM",
                                                "parallelism": f"LP shards x{ws}"},
                "e2e": {"value": round(units / (e2e_ms / 1e3), 2), "unit": "LP/s",
                        "from": "Python LP objects on the host (concatenation and upload timed)",
                        "ms_per_step": round(e2e_ms, 2)},
                "batched_fp32": res["fp32"], "batched_fp64": res["fp64"],
                "batched_fp32_persistent": res["fp32_persistent"],
                "batched_fp64_persistent": res["fp64_persistent"],
                "persistent_vs_graph_fp32_speedup": round(res["fp32"]["ms"] / res["fp32_persistent"]["ms"], 3),
                "sequential_fp64_ms": round(t_seq, 2),
                "sequential_fp64_iters_median": int(np.median(seq_it)),
                "batched_fp64_vs_sequential_fp64_speedup": round(t_seq / res["fp64"]["ms"], 2),
                "batched_fp32_vs_sequential_fp64_speedup": round(t_seq / res["fp32"]["ms"], 2)}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_adjoint(args):
    """64 LPs of 2000 x 5000, loss = ||x*(b, c) - t||^2 through torch.autograd
    (forward: batched solve + active-set polish; backward: the adjoint).
    value: the device path -- one BatchLP (A's context built once, before the
    timed steps), b, c, t CUDA tensors, forward + backward per step.
    e2e: the same step from host arrays through lp_solution with a context
    per call (A, b, c copied in and x, dL/db, dL/dc copied out every step)."""
    import torch

    from oracle import adjoint_ref as R
    from paper_2603_03150_gb300 import build as B
    from paper_2603_03150_gb300 import lpgen
    from paper_2603_03150_gb300.autograd import BatchLP, lp_solution

    B.build()
    lps, targets = lpgen.adjoint_batch(64, 2000, 5000)
    st = dict(m=np.array([lp.m for lp in lps], np.int32), n=np.array([lp.n for lp in lps], np.int32),
              row_ptr=np.concatenate([lp.row_ptr for lp in lps]),
              col=np.concatenate([lp.col for lp in lps]), val=np.concatenate([lp.val for lp in lps]))
    b0 = np.concatenate([lp.b for lp in lps])
    c0 = np.concatenate([lp.c for lp in lps])
    tcat = np.concatenate(targets)
    dev = torch.device("cuda", 0)
    bt, ct, tt = (torch.tensor(a, device=dev) for a in (b0, c0, tcat))
    blp = BatchLP(st, device="cuda")

    def step(b_src, c_src, t_src, lp):
        b = b_src.clone().requires_grad_(True)
        c = c_src.clone().requires_grad_(True)
        x = lp_solution(b, c, lp, eps_rel=EPS, max_iter=args.max_iter)
        ((x - t_src) ** 2).sum().backward()
        return x, b.grad, c.grad

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        ms, out = [], None
        for _ in range(k):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t0) * 1e3)
        return float(np.mean(ms)), out

    with Clocks(0) as clk:
        ms_step, (x, gb, gc) = timed(lambda: step(bt, ct, tt, blp), args.steps, args.warmup)
    bh, ch, th = (torch.from_numpy(a) for a in (b0, c0, tcat))
    e2e_ms, (xh, gbh, _) = timed(lambda: step(bh, ch, th, st), max(1, args.steps), 1)
    blp.close()
    lp = lps[0]
    xs = x.detach().cpu().numpy()[:lp.n]
    gr = R.grad_b(lp.dense(), xs > 0, 2.0 * (xs - targets[0]))
    err = float(np.linalg.norm(gb.cpu().numpy()[:lp.m] - gr) / np.linalg.norm(gr))
    err_h = float(np.linalg.norm(gbh.numpy()[:lp.m] - gb.cpu().numpy()[:lp.m]) /
                  np.linalg.norm(gb.cpu().numpy()[:lp.m]))
    sm, sn, nnz = int(st["m"].sum()), int(st["n"].sum()), int(st["val"].size)
    h2d = 4 * (sm + len(lps)) + 12 * nnz + 8 * sm + 8 * sn
    d2h = 8 * sn + 8 * sm + 8 * sn
    line = {"metric": "gradients dL/db, dL/dc per second (64 LPs, batched solve + polish + adjoint)",
            "value": round(64 / (ms_step / 1e3), 2), "unit": "LP-gradients/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["adjoint"], "eps_rel": EPS,
                       "step": "autograd forward (solve + polish) and backward (adjoint) on one "
                               "BatchLP; b, c, x and the gradients CUDA tensors"},
            "e2e": {"value": round(64 / (e2e_ms / 1e3), 2), "unit": "LP-gradients/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": round(e2e_ms, 2),
                    "step": "host arrays through lp_solution, a context per call"},
            "grad_b_rel_err_vs_dense_lp0": err, "grad_b_host_vs_device_rel": err_h,
            "polished_support_sizes": sorted(set(blp_active_sizes(x, st))),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def blp_active_sizes(x, st):
    """Positive entries per LP of a polished x."""
    xs = x.detach().cpu().numpy()
    off = np.concatenate([[0], np.cumsum(st["n"])])
    return [int((xs[off[i]:off[i + 1]] > 0).sum()) for i in range(len(st["n"]))]


def run_sweep(args):
    """Tolerance sweep (eps_rel = 1e-4, 1e-6, 1e-8) on one LP, FP64 plain and
    FP32-mixed: time to the Section 2 test, iterations and the maximum
    violation of the returned point on the original model (Section 4.3).
    One warm-up and `--steps` timed solves per (precision, eps); the ratio of
    each time to the eps = 1e-4 time is the shape of the paper's tradeoff."""
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2603_03150_gb300 import pdhg
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    lp = make_lp(args.workload)
    devt = {k: torch.from_numpy(np.ascontiguousarray(getattr(lp, k))).to(dev)
            for k in ["row_ptr", "col", "val", "b", "c"]}
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {}
    launches = 0
    with Clocks(local) as clk:
        for prec in args.sweep_precisions.split(","):
            rows = []
            for eps in (1e-4, 1e-6, 1e-8):
                ms, its, sts, viol = [], [], [], []
                for i in range(1 + args.steps):
                    with torch.cuda.stream(stream):
                        flush.fill_(float(i))
                    stream.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    s = pdhg.Solver(lp.m, lp.n, devt["row_ptr"], devt["col"], devt["val"],
                                    devt["b"], devt["c"], precision=prec, device_io=True,
                                    stream=stream.cuda_stream, method=args.method,
                                    spmv_layout=args.layout, omega_rule=args.omega_rule)
                    st = s.solve(eps, args.max_iter)
                    s.get()
                    e1.record(stream)
                    stream.synchronize()
                    info = s.info(violation=True)
                    launches += s.launch_count()
                    s.close()
                    if i >= 1:
                        ms.append(e0.elapsed_time(e1))
                        its.append(info["iters"])
                        sts.append(pdhg.STATUS_NAMES.get(st, st))
                        viol.append(info["max_violation"])
                rows.append(dict(eps_rel=eps, time_s=round(float(np.mean(ms)) / 1e3, 5),
                                 iters=int(np.mean(its)), status=sts,
                                 max_violation=float(np.max(viol))))
            t0 = rows[0]["time_s"]
            for r in rows:
                r["time_vs_1e-4"] = round(r["time_s"] / t0, 3) if t0 > 0 else None
            out[prec] = rows
    head = "fp64" if "fp64" in out else next(iter(out))
    value = out[head][-1]["time_s"]
    line = {"metric": "tolerance sweep: time to eps_rel and max violation (FP64, FP32-mixed)",
            "value": value, "unit": f"s ({head.upper()}, eps_rel = 1e-8)", "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if head == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "method": args.method,
                       "omega_rule": args.omega_rule, "layout": args.layout,
                       "step": "create + solve to eps + get", "max_iter": args.max_iter,
                       "l2": "flushed between solves (512 MiB write)"},
            "sweep": out, "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_hybrid(args):
    """PDHG on the GPU to eps_rel = 1e-4 and 1e-6, Algorithm 1's start point
    (scaled model) from the GPU, then the host interior-point method warm
    (with the bump loop) and cold on the same scaled LP: success rate, the
    geometric mean of warm/cold interior-point iterations over LPs both
    solve, and how many solve in <= 10 iterations (the statistics of the
    paper's Section 4.6 tables)."""
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import scipy.sparse as sp
    from paper_2603_03150_gb300 import hybrid_ipm as H
    from paper_2603_03150_gb300 import pdhg
    torch.cuda.set_device(local)
    prec = args.precision if args.precision_set else "fp64"
    rows, launches = [], 0
    with Clocks(local) as clk:
        for lp in hybrid_lps():
            A = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
            row = {"lp": lp.name, "m": lp.m, "n": lp.n, "nnz": int(lp.nnz)}
            scaled = None
            for eps in (1e-4, 1e-6):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                with pdhg.Solver.from_lp(lp, precision=prec, method=args.method) as s:
                    st = s.solve(eps, args.max_iter)
                    xp, y, zp, _ = s.warmstart_point(unscaled=False)
                    its = s.info(violation=False)["iters"]
                    if scaled is None:
                        sc = s.scaling()
                        Dr, Dc = np.asarray(sc["D_r"]), np.asarray(sc["D_c"])
                        scaled = (sp.diags(Dr) @ A @ sp.diags(Dc)).tocsr(), Dr * lp.b, Dc * lp.c
                    launches += s.launch_count()
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                As, bs, cs = scaled
                rw = H.warm_start(As, bs, cs, np.asarray(xp), np.asarray(y), np.asarray(zp))
                t2 = time.perf_counter()
                row[f"{eps:.0e}"] = {"pdhg_status": pdhg.STATUS_NAMES.get(st, st),
                                     "pdhg_iters": its, "pdhg_s": round(t1 - t0, 4),
                                     "ipm_status": rw["status"], "ipm_iters": rw["iters"],
                                     "bumps": rw["bumps"], "ipm_s": round(t2 - t1, 3)}
            t2 = time.perf_counter()
            rc = H.mehrotra(*scaled)
            row["cold"] = {"ipm_status": rc["status"], "ipm_iters": rc["iters"],
                           "ipm_s": round(time.perf_counter() - t2, 3)}
            rows.append(row)
    summary = {}
    cold_ok = [r for r in rows if r["cold"]["ipm_status"] == "optimal"]
    summary["cold"] = {"tried": len(rows), "solved": len(cold_ok),
                       "solved_in_10": sum(r["cold"]["ipm_iters"] <= 10 for r in cold_ok)}
    for key in ("1e-04", "1e-06"):
        tried = [r for r in rows if r[key]["pdhg_status"] == "converged"]
        ok = [r for r in tried if r[key]["ipm_status"] == "optimal"]
        both = [r for r in ok if r["cold"]["ipm_status"] == "optimal"]
        ratio = (float(np.exp(np.mean([np.log(max(r[key]["ipm_iters"], 1) /
                                              max(r["cold"]["ipm_iters"], 1)) for r in both])))
                 if both else None)
        summary[key] = {"tried": len(tried), "solved": len(ok),
                        "success_rate": round(len(ok) / max(len(tried), 1), 3),
                        "ipm_iteration_ratio_geomean": round(ratio, 3) if ratio else None,
                        "solved_in_10": sum(r[key]["ipm_iters"] <= 10 for r in ok)}
    line = {"metric": "IPM iterations warm (PDHG eps 1e-4 + Algorithm 1) / cold, geometric mean",
            "value": summary["1e-04"]["ipm_iteration_ratio_geomean"], "unit": "ratio",
            "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS["hybrid"], "pdhg_precision": prec,
                       "method": args.method, "ipm": "host Mehrotra predictor-corrector, dense "
                       "normal equations, Section 2 test at 1e-8, scaled model",
                       "algorithm1": "mu_min = alpha_min = 1e-6, delta_max = 1e-4, bump loop "
                       "at first step < 1e-6"},
            "summary": summary, "paper_section_4_6": {"1e-04": {"success_rate": [0.81, 0.83],
                                                          "ipm_iteration_ratio": [0.51, 0.55]},
                                                "1e-06": {"success_rate": [0.88, 0.87],
                                                          "ipm_iteration_ratio": [0.30, 0.35]}},
            "per_lp": rows, "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """A short fixed run for profilers (ncu): one context on --workload, then
    --profile-run iterations with eps_rel = 0 (no test can end it early).
    Prints the iterations done and the layout of each half-step."""
    from paper_2603_03150_gb300 import build as B
    from paper_2603_03150_gb300 import pdhg
    B.build()
    lp = make_lp(args.workload)
    layout = args.layout
    with pdhg.Solver.from_lp(lp, precision=args.precision, spmv_layout=layout,
                             method=args.method, omega_rule=args.omega_rule,
                             step_rule=args.step_rule) as s:
        s.solve(0.0, args.profile_run)
        print(json.dumps({"iters": s.info(violation=False)["iters"], "layout": s.layout(),
                          "schedule": s.schedule(), "launches": s.launch_count()}), flush=True)


def cpu_baseline(lp, iters, method="averaged", omega_rule="smooth", step_rule="constant"):
    """The oracle as it stands, timed on this host: its set-up once (timed
    apart), then `iters` PDHG iterations (steady-state iterations per second)."""
    from oracle import pdhg_oracle as O
    t0 = time.perf_counter()
    S = O.setup(lp)
    t1 = time.perf_counter()
    O.solve(lp, EPS, iters, opts=O.Options(method=method, omega_rule=omega_rule,
                                           step_rule=step_rule), S=S)
    t2 = time.perf_counter()
    return {"value": round(iters / (t2 - t1), 3), "unit": "iter/s", "cores": 1, "kind": "oracle",
            "sample": f"{iters} iterations of the float64 numpy/scipy oracle on the same LP after "
                      f"its set-up (scaling + power iteration, {t1 - t0:.1f} s, not counted)",
            "setup_s": round(t1 - t0, 2)}


def run_reference(args):
    """The oracle on the same workload: set-up once (untimed), then each step
    runs `ref_iters` more PDHG iterations and Algorithm 1 on the current iterate."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import pdhg_oracle as O
    lp = make_lp(args.workload)
    t0 = time.perf_counter()
    S = O.setup(lp)
    setup_s = time.perf_counter() - t0
    st = O.initial_state(S)
    times, its = [], 0
    k = 0
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        k += args.ref_iters
        r = O.solve(lp, EPS, k, opts=O.Options(method=args.method, omega_rule=args.omega_rule,
                                               step_rule=args.step_rule), S=S, state=st)
        st = r.state
        zs = np.maximum(0.0, S.c_t - S.At.T @ st.y)
        O.centered_start_point(st.x, zs)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
            its += args.ref_iters
    total = sum(times)
    val = its / total
    line = {"metric": METRIC, "value": round(val, 3), "unit": "iter/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / len(times) * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOADS[args.workload], "precision": "fp64", "eps_rel": EPS,
                       "step": f"{args.ref_iters} oracle iterations + Algorithm 1"},
            "cpu_baseline": {"value": round(val, 3), "unit": "iter/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps of {args.ref_iters} iterations after the "
                                       f"oracle's set-up ({setup_s:.1f} s, not counted)"},
            "e2e": {"value": round(val, 3), "unit": "iter/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="powerlaw")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--sweep-precisions", default="fp64,fp32",
                    help="precisions of --eps-sweep, comma-separated")
    ap.add_argument("--layout", choices=["auto", "csr", "panels"], default="auto",
                    help="FP32 half-step layout: autotuned (default), CSR tiles or column panels")
    ap.add_argument("--method", choices=["averaged", "halpern"], default="averaged",
                    help="PDHG iteration: restarted averaged (default) or reflected Halpern")
    ap.add_argument("--omega-rule", choices=["smooth", "pid"], default="smooth",
                    help="primal weight at restarts: smoothed ratio (default) or PID control")
    ap.add_argument("--step-rule", choices=["constant", "adaptive"], default="constant",
                    help="step size: constant (default) or PDLP's adaptive step")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--variant-steps", type=int, default=2,
                    help="steps of each PID primal-weight variant reported beside the default")
    ap.add_argument("--cpu-iters", type=int, default=128)
    ap.add_argument("--kernel-reps", type=int, default=50,
                    help="back-to-back launches per half-step for the roofline timing")
    ap.add_argument("--ref-iters", type=int, default=64)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--max-iter", type=int, default=MAX_ITER,
                    help="iteration cap per solve (profiling runs use a small cap)")
    ap.add_argument("--profile-run", type=int, default=0, metavar="ITERS",
                    help="profiling mode: ITERS iterations on --workload with eps_rel = 0, "
                         "no timing (for ncu)")
    ap.add_argument("--eps-sweep", action="store_true",
                    help="tolerance sweep 1e-4 / 1e-6 / 1e-8 on --workload (FP64 and FP32-mixed)")
    args = ap.parse_args()
    args.precision_set = any(a.startswith("--precision") for a in sys.argv[1:])
    if args.warmup < 3 and args.profile_run == 0:
        ap.error("--warmup must be >= 3")
    if args.profile_run > 0:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "hybrid":
        run_hybrid(args)
    elif args.eps_sweep:
        if args.max_iter == MAX_ITER:
            args.max_iter = 200_000  # FP32-mixed stalls above its precision: bound the sweep
        run_sweep(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
