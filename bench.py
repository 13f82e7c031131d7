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
    "transport": ("balanced transportation LP 2000 supply x 2000 demand, m=4000 "
                  "n=4000000 nnz=8000000, seed 0"),
    "small": "planted LP m=200 n=500, 5 nnz per column, seed 0",
}


def make_lp(name):
    from paper_2603_03150_gb300 import lpgen
    if name == "powerlaw":
        return lpgen.powerlaw_lp()
    if name == "transport":
        return lpgen.transportation_lp()
    return lpgen.planted_lp(200, 500, seed=0)


# ---------------------------------------------------------------------------
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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

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
    h = hashlib.sha256()
    for f in ["spmv_tile.cuh", "iter_kernels.cu", "common.cuh"]:
        h.update(open(os.path.join(ROOT, "paper_2603_03150_gb300", "csrc", f), "rb").read())
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

    def step(precision, device_io=True, timing=False, outs=None):
        src = devt if device_io else pinned
        s = pdhg.Solver(m, n, src["row_ptr"], src["col"], src["val"], src["b"], src["c"],
                        precision=precision, device_io=device_io, stream=stream.cuda_stream,
                        kernel_timing=timing)
        st = s.solve(EPS, args.max_iter)
        g = s.get(out=outs[0] if outs else None)
        w = s.warmstart_point(unscaled=True, out=outs[1] if outs else None)
        return s, st, g, w

    def run_steps(precision, k, w, device_io=True, timing=False):
        outs = None
        if not device_io:
            mk = lambda L: torch.empty(L, dtype=torch.float64).pin_memory()
            outs = ((mk(n), mk(m), mk(n)), (mk(n), mk(m), mk(n)))
        rec = []
        for i in range(w + k):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            stream.synchronize()
            e0.record(stream)
            s, st, g, wp = step(precision, device_io, timing, outs)
            e1.record(stream)
            stream.synchronize()
            info = s.info(violation=False)
            kt = s.kernel_timing() if timing else None
            launches = s.launch_count()
            sched = s.schedule()
            s.close()
            if i >= w:
                rec.append(dict(ms=e0.elapsed_time(e1), iters=info["iters"], status=st,
                                r_P=g["r_P"], r_D=g["r_D"], gap=g["gap"], kt=kt,
                                launches=launches, sched=sched,
                                obj=float(torch.dot(torch.as_tensor(g["x"]).to(dev),
                                                    devt["c"]).item())))
        return rec

    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        rec = run_steps(args.precision, args.steps, args.warmup, timing=True)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    total_ms = sum(r["ms"] for r in rec)
    total_it = sum(r["iters"] for r in rec)
    if ws > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        it = torch.tensor([total_it], dtype=torch.float64, device=dev)
        dist.all_reduce(it, op=dist.ReduceOp.SUM)
        total_ms, total_it_all = float(t.item()), float(it.item())
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
                    iters=int(np.mean([r["iters"] for r in r64])),
                    iter_per_s=sum(r["iters"] for r in r64) / (sum(r["ms"] for r in r64) / 1e3),
                    status=[r["status"] for r in r64])

    # roofline of the dominant kernel (sampled CUDA-event durations)
    s_bytes = 4 if args.precision == "fp32" else 8
    ab = algorithmic_bytes(m, n, nnz, s_bytes)
    ns = sum(r["kt"]["samples"] for r in rec)
    pm = sum(r["kt"]["primal_ms"] * r["kt"]["samples"] for r in rec) / max(ns, 1)
    dm = sum(r["kt"]["dual_ms"] * r["kt"]["samples"] for r in rec) / max(ns, 1)
    dom, dur = ("primal", pm) if pm >= dm else ("dual", dm)
    peak, peak_src = peaks()
    ach = ab[dom] / (dur / 1e3) / 1e9 if dur > 0 else 0.0
    roofline = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4),
                "traffic": ncu_traffic("k_primal" if dom == "primal" else "k_dual", args.precision,
                                       args.workload,
                                       (rec[0]["sched"]["at_tile_nnz" if dom == "primal" else "a_tile_nnz"] + 4) // 256),
                "kernel": "k_primal" if dom == "primal" else "k_dual",
                "peak_source": peak_src, "algorithmic_bytes_per_launch": ab[dom],
                "mean_launch_ms": round(dur, 5), "samples": ns,
                "other": {"kernel": "k_dual" if dom == "primal" else "k_primal",
                          "mean_launch_ms": round(dm if dom == "primal" else pm, 5),
                          "achieved_gbs": round(ab["dual" if dom == "primal" else "primal"] /
                                                (max(dm if dom == "primal" else pm, 1e-9) / 1e3) / 1e9, 1)}}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(lp, args.cpu_iters)

    if rank == 0:
        ms_step = total_ms / max(len(rec), 1)
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "iter/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "precision": args.precision +
                       ("_mixed (f64 norms, gap, restart rule, step/weight updates)" if args.precision == "fp32" else ""),
                       "eps_rel": EPS, "step": "create + solve to eps + get + warmstart_point",
                       "l2": "flushed between steps (512 MiB write), inputs resident in HBM",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "schedule": rec[0]["sched"]},
            "time_to_eps_s": round(ms_step / 1e3, 5),
            "iters_to_eps": int(np.mean([r["iters"] for r in rec])),
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
            line["fp64"] = fp64
            line["fp32_vs_fp64_time_speedup"] = round(fp64["time_to_eps_s"] / (ms_step / 1e3), 3)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def cpu_baseline(lp, iters):
    """The oracle as it stands, timed on this host: its set-up once (timed
    apart), then `iters` PDHG iterations (steady-state iterations per second)."""
    from oracle import pdhg_oracle as O
    t0 = time.perf_counter()
    S = O.setup(lp)
    t1 = time.perf_counter()
    O.solve(lp, EPS, iters, S=S)
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
        r = O.solve(lp, EPS, k, S=S, state=st)
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
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--cpu-iters", type=int, default=128)
    ap.add_argument("--ref-iters", type=int, default=64)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--max-iter", type=int, default=MAX_ITER,
                    help="iteration cap per solve (profiling runs use a small cap)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
