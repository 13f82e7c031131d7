"""A short, fixed PDHG run for profilers: create a context on one of the
bench workloads and run a given number of iterations (no termination test
is allowed to end it early: eps_rel = 0).  Prints the iterations done and the
layout of each half-step.

    python -m paper_2603_03150_gb300.profile_run --workload powerlaw \\
        --precision fp32 --layout panels --iters 128
"""
import argparse
import json

from . import lpgen, pdhg

WORKLOADS = {
    "powerlaw": lambda: lpgen.powerlaw_lp(seed=0),
    "powerlaw50m": lambda: lpgen.powerlaw_lp(m=2_000_000, n=10_000_000, nnz=50_000_000, seed=0),
    "transport": lambda: lpgen.transportation_lp(2000, 2000),
    "small": lambda: lpgen.planted_lp(200, 500, seed=0),
}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="powerlaw")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--layout", choices=["auto", "csr", "panels"], default="panels")
    ap.add_argument("--method", choices=["averaged", "halpern"], default="averaged")
    ap.add_argument("--iters", type=int, default=128)
    a = ap.parse_args(argv)
    lp = WORKLOADS[a.workload]()
    with pdhg.Solver.from_lp(lp, precision=a.precision, spmv_layout=a.layout,
                             method=a.method) as s:
        s.solve(0.0, a.iters)
        print(json.dumps({"iters": s.info(violation=False)["iters"], "layout": s.layout(),
                          "schedule": s.schedule()}))


if __name__ == "__main__":
    main()
