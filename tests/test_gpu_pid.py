"""PID primal-weight control (options.omega_rule = 1, the reading of
cuPDLP+'s primal-weight controller) against the oracle's omega_update_pid:
float64 iterates, weights and controller state after several restarts, the
restart logs, full solves' iteration counts, and checkpoint/resume with the
controller's state."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2603_03150_gb300 import build as B
from paper_2603_03150_gb300 import lpgen, pdhg

from test_gpu_parity import heavy_row_lp, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


GAINS = [(0.99, 0.01, 0.0), (0.5, 0.2, 0.3)]


@pytest.mark.parametrize("gains", GAINS)
@pytest.mark.parametrize("method", ["averaged", "halpern"])
@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(200, 500, seed=0), heavy_row_lp,
                                   lambda: lpgen.transportation_lp(40, 50)])
def test_pid_iterates_after_640_match_oracle(maker, method, gains):
    lp = maker()
    kp, ki, kd = gains
    opts = O.Options(method=method, omega_rule="pid", pid_kp=kp, pid_ki=ki, pid_kd=kd)
    r = O.solve(lp, 1e-12, 640, opts=opts)
    assert r.state.restarts >= 2
    with pdhg.Solver.from_lp(lp, method=method, omega_rule="pid", pid_kp=kp, pid_ki=ki,
                             pid_kd=kd) as s:
        assert s.solve(1e-12, 640) == pdhg.PDHG_MAX_ITER
        st = s.state()
        lg = s.log()
    for key in ("x", "y", "x_avg", "y_avg"):
        assert rel_inf(st[key], getattr(r.state, key)) < 1e-9, key
    assert st["restarts"] == r.state.restarts and st["t"] == r.state.t
    assert abs(st["omega"] - r.state.omega) <= 1e-9 * r.state.omega
    assert abs(st["pid_integral"] - r.state.pid_integral) <= 1e-9 * (1 + abs(r.state.pid_integral))
    assert abs(st["pid_prev"] - r.state.pid_prev) <= 1e-9 * (1 + abs(r.state.pid_prev))
    assert [(e["k"], e["restart"], e["cand"]) for e in lg] == \
           [(e["k"], e["restart"], e["cand"]) for e in r.log]
    for e, o in zip(lg, r.log):
        assert abs(e["omega"] - o["omega"]) <= 1e-9 * o["omega"]


def test_pid_full_solve_matches_oracle_and_differs_from_smoothing():
    lp = lpgen.planted_lp(200, 500, seed=0)
    r = O.solve(lp, 1e-4, 200_000, opts=O.Options(omega_rule="pid"))
    assert r.status == O.STATUS_CONVERGED
    with pdhg.Solver.from_lp(lp, omega_rule="pid") as s:
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        info = s.info()
        g = s.get()
        w_pid = s.state()["omega"]
    assert info["iters"] == r.iters and info["restarts"] == r.restarts
    assert rel_inf(g["x"], r.x) < 1e-8
    with pdhg.Solver.from_lp(lp) as s2:
        s2.solve(1e-4, 200_000)
        w_smooth = s2.state()["omega"]
    assert w_pid != w_smooth


def test_pid_checkpoint_resume_equals_uninterrupted():
    lp = heavy_row_lp(2)
    kw = dict(omega_rule="pid", pid_kp=0.7, pid_ki=0.1, pid_kd=0.2)
    with pdhg.Solver.from_lp(lp, **kw) as s:
        s.solve(1e-12, 700)
        ref = s.state()
    with pdhg.Solver.from_lp(lp, **kw) as s1:
        s1.solve(1e-12, 300)
        ck = s1.state()
        assert ck["pid_integral"] != 0.0
    with pdhg.Solver.from_lp(lp, **kw) as s2:
        s2.set_state(ck)
        s2.solve(1e-12, 700)
        got = s2.state()
    for key in ("x", "y", "x_avg", "y_avg"):
        assert rel_inf(got[key], ref[key]) < 1e-12, key
    assert got["pid_integral"] == pytest.approx(ref["pid_integral"], rel=1e-12, abs=1e-15)
    assert got["omega"] == pytest.approx(ref["omega"], rel=1e-12)


def test_invalid_omega_rule_rejected():
    lp = lpgen.planted_lp(20, 50, seed=0)
    with pytest.raises(ValueError):
        pdhg.Solver.from_lp(lp, omega_rule="bogus")
    o = pdhg.Options()
    pdhg.lib().pdhg_default_options(o)
    assert (o.omega_rule, o.pid_kp, o.pid_ki, o.pid_kd) == (0, 0.99, 0.01, 0.0)
