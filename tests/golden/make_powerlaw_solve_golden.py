"""Writes powerlaw_solve_1e-4.json: the float64 oracle's full solve of the
power-law planted LP (m = 200,000, n = 1,000,000, 5,000,000 nonzeros, seed 0)
to eps_rel = 1e-4 under the default options -- iteration and restart counts,
the returned iterate's choice, residuals, objective and Section 4.3 maximum
violation.  It calls only the oracle and the seeded input generator; one run
takes several minutes on one core, so the tests read the stored values.

    python tests/golden/make_powerlaw_solve_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import pdhg_oracle as O  # noqa: E402
from paper_2603_03150_gb300 import lpgen  # noqa: E402


def main():
    lp = lpgen.powerlaw_lp(seed=0)
    t0 = time.perf_counter()
    r = O.solve(lp, 1e-4, 2_000_000)
    dt = time.perf_counter() - t0
    out = {
        "source": "float64 oracle (oracle/pdhg_oracle.py, default options), lpgen.powerlaw_lp(seed=0), "
                  "eps_rel = 1e-4; written by tests/golden/make_powerlaw_solve_golden.py",
        "eps_rel": 1e-4,
        "status": int(r.status),
        "iters": int(r.iters),
        "restarts": int(r.restarts),
        "chosen": r.chosen,
        "r_P": float(r.r_P),
        "r_D": float(r.r_D),
        "gap": float(r.gap),
        "objective": float(lp.c @ r.x),
        "max_violation": float(r.max_violation),
        "oracle_seconds": round(dt, 1),
    }
    with open(os.path.join(HERE, "powerlaw_solve_1e-4.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
