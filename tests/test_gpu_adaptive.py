"""PDLP's adaptive step (options.step_rule = 1) against the oracle's
adaptive_step: float64 iterates, step-weighted averages, step state and
restart logs after several restarts; a forced rejection (a first step 100x
the constant one) undone on the device exactly as in the oracle; full solves
with the oracle's attempt, restart and rejection counts; the float64 test
for float32-mixed solves; checkpoint/resume of the step state; and the
combinations the option does not support rejected.

The adaptive rule feeds each attempt's rounding into the next step size,
so differences between two correct implementations grow along the
trajectory (measured: the step sizes agree to about 1e-13 after 64
attempts, 1e-11 to 1e-8 after 128 depending on the LP, and the trajectories part within
a few hundred).  These tests therefore start the oracle from the context's
own scaling, sigma_max, step and primal weight (its setup built from
pdhg_get_scaling), so that only the order of the floating-point sums
differs, compare iterates after 72 attempts (the restart at 64 and eight more; the
forced case adds a rejection), and compare full solves by their outcome."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg_oracle as O
from paper_2603_03150_gb300 import build as B
from paper_2603_03150_gb300 import lpgen, pdhg

from test_gpu_parity import gappy_lp, heavy_row_lp, mid_column_lp, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _setup_from(s, lp):
    """The oracle's Setup with the context's D_r, D_c, sigma_max, eta and omega_0."""
    sc = s.scaling()
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    Dr, Dc = np.array(sc["D_r"], dtype=np.float64), np.array(sc["D_c"], dtype=np.float64)
    At = (sp.diags(Dr) @ A @ sp.diags(Dc)).tocsr()
    b, c = np.asarray(lp.b, float), np.asarray(lp.c, float)
    return O.Setup(A, b, c, Dr, Dc, At, Dr * b, Dc * c, sc["sigma_max"], sc["power_iters"],
                   sc["eta"], sc["omega0"])


def _compare(st, r):
    for key in ("x", "y", "x_avg", "y_avg", "x_last", "y_last"):
        assert rel_inf(st[key], getattr(r.state, key)) < 1e-9, key
    assert st["k"] == r.state.k and st["t"] == r.state.t
    assert st["restarts"] == r.state.restarts
    assert abs(st["omega"] - r.state.omega) <= 1e-9 * r.state.omega
    assert abs(st["step_eta"] - r.state.eta) <= 1e-9 * r.state.eta
    assert abs(st["eta_sum"] - r.state.eta_sum) <= 1e-9 * (1 + r.state.eta_sum)
    assert st["step_rejects"] == r.state.step_rejects


MAKERS = [lambda: lpgen.planted_lp(200, 500, seed=0), heavy_row_lp,
          lambda: lpgen.transportation_lp(40, 50), gappy_lp]


@pytest.mark.parametrize("maker", MAKERS)
def test_adaptive_iterates_after_72_match_oracle(maker):
    lp = maker()
    opts = O.Options(step_rule="adaptive")
    with pdhg.Solver.from_lp(lp, step_rule="adaptive") as s:
        r = O.solve(lp, 1e-12, 72, opts=opts, S=_setup_from(s, lp))
        assert r.state.restarts >= 1
        assert s.solve(1e-12, 72) == pdhg.PDHG_MAX_ITER
        st = s.state()
        lg = s.log()
    _compare(st, r)
    assert [(e["k"], e["restart"], e["cand"]) for e in lg] == \
           [(e["k"], e["restart"], e["cand"]) for e in r.log]


@pytest.mark.parametrize("maker", [mid_column_lp, gappy_lp])
def test_adaptive_split_rows_at_a_small_tile_capacity(maker):
    """tile_nnz = 100 splits rows of both matrices across tiles (rows of A~^T
    of 150 to 1500 entries on the first LP): every split row's terms of the
    attempt's sums have a record of their own; iterates after 72 attempts as
    in the oracle."""
    lp = maker()
    opts = O.Options(step_rule="adaptive")
    with pdhg.Solver.from_lp(lp, step_rule="adaptive", tile_nnz=100) as s:
        r = O.solve(lp, 1e-12, 72, opts=opts, S=_setup_from(s, lp))
        assert s.solve(1e-12, 72) == pdhg.PDHG_MAX_ITER
        st = s.state()
    _compare(st, r)


def test_forced_rejection_is_undone_as_in_the_oracle():
    lp = lpgen.planted_lp(200, 500, seed=0)
    opts = O.Options(step_rule="adaptive")
    with pdhg.Solver.from_lp(lp, step_rule="adaptive") as s:
        S = _setup_from(s, lp)
        st0 = O.initial_state(S)
        st0.eta = 100.0 * S.eta
        r = O.solve(lp, 1e-12, 72, opts=opts, S=S, state=st0)
        assert r.state.step_rejects >= 1
        s0 = s.step_state()
        assert s0["step_rejects"] == 0 and s0["eta_sum"] == 0.0
        assert s0["step_eta"] == S.eta
        s.set_state(dict(s.state(), step_eta=100.0 * s0["step_eta"], eta_sum=0.0))
        assert s.solve(1e-12, 1) == pdhg.PDHG_MAX_ITER
        one = s.state()
        assert one["step_rejects"] == 1 and one["eta_sum"] == 0.0
        assert not np.any(one["x"]) and not np.any(one["y"])  # nothing moved
        assert s.solve(1e-12, 72) == pdhg.PDHG_MAX_ITER
        st = s.state()
    _compare(st, r)


@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(500, 1250, seed=2),
                                   lambda: lpgen.transportation_lp(20, 30), gappy_lp])
def test_adaptive_full_solve_reaches_the_oracles_optimum(maker):
    """Full solves to 1e-4: the returned point passes the Section 2 test as
    the oracle evaluates it, its objective is within 1e-2 of the oracle's
    adaptive solve (two points that pass the relative test at 1e-4 can differ
    by 1e-3 in objective on these LPs), and on the transportation LP the
    adaptive step needs fewer attempts than the constant one."""
    lp = maker()
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    with pdhg.Solver.from_lp(lp, step_rule="adaptive") as s:
        r = O.solve(lp, 1e-4, 200_000, opts=O.Options(step_rule="adaptive"), S=_setup_from(s, lp))
        assert r.status == O.STATUS_CONVERGED
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        info = s.info()
        g = s.get()
    ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, g["x"], g["y"], 1e-4)
    assert ok, (rp, rd, gap)
    obj, ref = float(lp.c @ g["x"]), float(lp.c @ r.x)
    assert abs(obj - ref) <= 1e-2 * (1 + abs(ref))
    if lp.m == 50:  # the transportation LP
        with pdhg.Solver.from_lp(lp) as s2:
            assert s2.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
            assert info["iters"] < s2.info()["iters"]


def test_adaptive_fp32_mixed_passes_the_test_in_fp64():
    lp = gappy_lp()
    eps = 1e-4
    with pdhg.Solver.from_lp(lp, precision="fp32", step_rule="adaptive") as s:
        assert s.solve(eps, 200_000) == pdhg.PDHG_CONVERGED
        g = s.get()
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, g["x"], g["y"], eps)
    assert ok, (rp, rd, gap)


def test_adaptive_checkpoint_resume_equals_uninterrupted():
    lp = gappy_lp()
    with pdhg.Solver.from_lp(lp, step_rule="adaptive") as s:
        s.solve(1e-12, 1000)
        ref = s.state()
    with pdhg.Solver.from_lp(lp, step_rule="adaptive") as s1:
        s1.solve(1e-12, 500)
        ck = s1.state()
    with pdhg.Solver.from_lp(lp, step_rule="adaptive") as s2:
        s2.set_state(ck)
        s2.solve(1e-12, 1000)
        got = s2.state()
    for key in ("x", "y", "x_avg", "y_avg"):
        np.testing.assert_array_equal(got[key], ref[key])
    assert got["step_eta"] == ref["step_eta"] and got["eta_sum"] == ref["eta_sum"]


def test_unsupported_combinations_are_rejected():
    lp = lpgen.planted_lp(20, 50, seed=0)
    for kw in (dict(method="halpern"), dict(precision="fp32", spmv_layout="panels")):
        with pytest.raises(pdhg.PDHGError):
            pdhg.Solver.from_lp(lp, step_rule="adaptive", **kw)
    o = pdhg.Options()
    pdhg.lib().pdhg_default_options(pdhg.ctypes.byref(o))
    assert o.step_rule == 0
    with pytest.raises(pdhg.PDHGError):
        pdhg.BatchSolver([lp, lp], step_rule=1)
