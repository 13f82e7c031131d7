"""GPU parity of the optional reflected Halpern iteration (method 1) against
the oracle's ``method="halpern"``, through the C ABI.

Tolerances as for the averaged method: FP64 iterates after 100 iterations
within 1e-9 relative with identical restart logs; full FP64 solves with the
oracle's iteration and restart counts; FP32-mixed solves pass the Section 2
test re-evaluated in float64 and match the FP64 oracle objective to 1e-3.
"""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2603_03150_gb300 import build as B
from paper_2603_03150_gb300 import lpgen
from paper_2603_03150_gb300 import pdhg

from test_gpu_parity import gappy_lp, heavy_row_lp, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _opts(rho):
    return O.Options(method="halpern", reflection=rho)


def _compare(st, ost, tol):
    # x_avg / y_avg hold T(z) in this method
    for k in ["x", "y", "x_avg", "y_avg", "x_last", "y_last"]:
        assert rel_inf(st[k], getattr(ost, k)) < tol, k
    assert st["k"] == ost.k and st["t"] == ost.t and st["restarts"] == ost.restarts
    assert abs(st["omega"] - ost.omega) <= tol * ost.omega


@pytest.mark.parametrize("tile_nnz", [0, 3000, -4])
@pytest.mark.parametrize("rho", [1.0, 0.5])
@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(200, 500, seed=0), heavy_row_lp,
                                   gappy_lp, lambda: lpgen.transportation_lp(40, 50)])
def test_halpern_fp64_iterates_after_100(maker, rho, tile_nnz):
    lp = maker()
    r = O.solve(lp, 1e-12, 100, opts=_opts(rho))
    with pdhg.Solver.from_lp(lp, tile_nnz=tile_nnz, method="halpern", reflection=rho) as s:
        assert s.solve(1e-12, 100) == pdhg.PDHG_MAX_ITER
        _compare(s.state(), r.state, 1e-9)
        lg = s.log()
    assert [(e["k"], e["restart"], e["cand"]) for e in lg] == \
           [(e["k"], e["restart"], e["cand"]) for e in r.log]


@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(200, 500, seed=0),
                                   lambda: lpgen.transportation_lp(30, 40)])
def test_halpern_fp64_solve_matches_oracle(maker):
    lp = maker()
    r = O.solve(lp, 1e-4, 100_000, opts=_opts(1.0))
    with pdhg.Solver.from_lp(lp, method="halpern") as s:
        assert s.solve(1e-4, 100_000) == pdhg.PDHG_CONVERGED
        g = s.get()
        info = s.info()
        lg = s.log()
    assert info["iters"] == r.iters and info["restarts"] == r.restarts
    assert info["chosen_average"] == (r.chosen == "average")
    assert [(e["k"], e["restart"], e["cand"]) for e in lg] == \
           [(e["k"], e["restart"], e["cand"]) for e in r.log]
    obj = float(lp.c @ r.x)
    assert abs(float(lp.c @ g["x"]) - obj) <= 1e-8 * (1 + abs(obj))
    assert abs(g["r_P"] - r.r_P) <= 1e-8 * (1 + r.r_P)
    assert abs(g["gap"] - r.gap) <= 1e-8 * (1 + abs(obj))
    if lp.x_star is not None:  # planted: x is unique
        assert rel_inf(g["x"], r.x) < 1e-8
    # the returned iterate is x >= 0 whichever candidate won (T(z) always is)
    if info["chosen_average"]:
        assert np.min(g["x"]) >= 0.0


@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(1000, 2500, seed=3),
                                   lambda: lpgen.transportation_lp(40, 50)])
def test_halpern_fp32_mixed_converges_and_holds_in_fp64(maker):
    lp = maker()
    r = O.solve(lp, 1e-4, 200_000, opts=_opts(1.0))
    with pdhg.Solver.from_lp(lp, precision="fp32", method="halpern") as s:
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        g = s.get()
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, g["x"], g["y"], 1e-4)
    assert ok, (rp, rd, gap)
    obj = float(lp.c @ r.x)
    assert abs(float(lp.c @ g["x"]) - obj) <= 1e-3 * (1 + abs(obj))


def test_halpern_checkpoint_resume_matches_uninterrupted_run():
    """The checkpoint holds the anchor (x_last, y_last); resuming recomputes
    A~ times the anchor, so the resumed run continues the same iteration."""
    lp = lpgen.planted_lp(200, 500, seed=2)
    with pdhg.Solver.from_lp(lp, method="halpern") as s:
        s.solve(1e-12, 192)
        ref = s.state()
    with pdhg.Solver.from_lp(lp, method="halpern") as s1:
        s1.solve(1e-12, 100)
        ck = s1.state()
    with pdhg.Solver.from_lp(lp, method="halpern") as s2:
        s2.set_state(ck)
        s2.solve(1e-12, 192)
        got = s2.state()
    for k in ["x", "y", "x_avg", "y_avg", "x_last", "y_last"]:
        assert rel_inf(got[k], ref[k]) < 1e-12, k
    assert got["k"] == ref["k"] == 192 and got["restarts"] == ref["restarts"]


def test_halpern_options_are_checked():
    lp = lpgen.planted_lp(20, 50, seed=1)
    with pytest.raises(pdhg.PDHGError):
        pdhg.Solver.from_lp(lp, method="halpern", reflection=1.5)
    with pytest.raises(pdhg.PDHGError):
        pdhg.BatchSolver([lp, lp], method=1)
