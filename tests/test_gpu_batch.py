"""Batched solves (block-diagonal batch with per-LP state) against the oracle
run LP by LP.  Same tolerances as the single-LP parity tests: FP64 iterates
1e-9 relative after 100 iterations; FP32-mixed must pass the test in float64."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2603_03150_gb300 import build as B
from paper_2603_03150_gb300 import lpgen
from paper_2603_03150_gb300 import pdhg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def rel_inf(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def mixed_batch():
    lps = [lpgen.planted_lp(m, int(2.5 * m), 5, seed=s)
           for s, m in enumerate([20, 57, 200, 333, 600, 41])]
    # one LP with rows longer than a tile (split rows inside a batch)
    lps.insert(3, lpgen.powerlaw_lp(m=300, n=3000, nnz=15000, k_max=2500, seed=5))
    return lps


def test_batch_iterates_match_oracle_after_100():
    lps = mixed_batch()
    with pdhg.BatchSolver(lps) as s:
        assert s.solve(1e-12, 100) == pdhg.PDHG_MAX_ITER
        g = s.get()
    xs, ys = s.split(g["x"], "n"), s.split(g["y"], "m")
    for i, lp in enumerate(lps):
        r = O.solve(lp, 1e-12, 100)
        assert g["iters"][i] == 100
        assert rel_inf(xs[i], r.x) < 1e-9, i
        assert rel_inf(ys[i], r.y) < 1e-9, i


def test_batch_fp64_solve_matches_oracle_per_lp():
    lps = mixed_batch()[:5]
    with pdhg.BatchSolver(lps) as s:
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        g = s.get()
    xs = s.split(g["x"], "n")
    for i, lp in enumerate(lps):
        r = O.solve(lp, 1e-4, 200_000)
        assert r.status == O.STATUS_CONVERGED
        assert g["iters"][i] == r.iters, (i, g["iters"][i], r.iters)
        assert rel_inf(xs[i], r.x) < 1e-8
        assert abs(g["r_P"][i] - r.r_P) <= 1e-8 * (1 + r.r_P)
        assert abs(g["max_violation"][i] - r.max_violation) <= 1e-8 * (1 + r.max_violation)


def test_batch_fp32_mixed_all_converge():
    lps = lpgen.planted_batch(count=24, m_lo=50, m_hi=800)
    with pdhg.BatchSolver(lps, precision="fp32") as s:
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        assert np.all(s.lp_status == 0)
        g = s.get()
    xs, ys = s.split(g["x"], "n"), s.split(g["y"], "m")
    for i, lp in enumerate(lps):
        A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
        ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, xs[i], ys[i], 1e-4)
        assert ok, (i, rp, rd, gap)
        assert abs(rp - g["r_P"][i]) <= 1e-9 * (1 + rp)
        obj = float(lp.c @ lp.x_star)
        assert abs(float(lp.c @ xs[i]) - obj) <= 1e-3 * (1 + abs(obj))


def test_batch_fp32_screen_rejections_per_lp():
    """With a loose float32 screen (100 eps) every LP's early candidates are
    re-evaluated in float64 and rejected; each LP still ends on a candidate
    that meets the Section 2 test at eps."""
    lps = lpgen.planted_batch(count=12, m_lo=50, m_hi=600)
    with pdhg.BatchSolver(lps, precision="fp32", fp32_screen=100.0) as s:
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        g = s.get()
        checks, rejects = s.fp64_checks()
    assert rejects >= 1 and checks == rejects + len(lps)
    xs, ys = s.split(g["x"], "n"), s.split(g["y"], "m")
    for i, lp in enumerate(lps):
        A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
        ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, xs[i], ys[i], 1e-4)
        assert ok, (i, rp, rd, gap)


def test_batch_of_one_equals_single_lp_path():
    lp = lpgen.planted_lp(200, 500, seed=0)
    with pdhg.BatchSolver([lp]) as s:
        s.solve(1e-4, 100_000)
        gb = s.get()
    with pdhg.Solver.from_lp(lp) as t:
        t.solve(1e-4, 100_000)
        gs = t.get()
        it = t.info()["iters"]
    assert gb["iters"][0] == it
    assert rel_inf(gb["x"], gs["x"]) < 1e-12 and rel_inf(gb["y"], gs["y"]) < 1e-12


def test_batch_warmstart_matches_oracle():
    lps = mixed_batch()[:4]
    with pdhg.BatchSolver(lps) as s:
        s.solve(1e-4, 200_000)
        g = s.get()
        xw, yw, zw, mu = s.warmstart_point()
    xs, ys = s.split(g["x"], "n"), s.split(g["y"], "m")
    xws, zws = s.split(xw, "n"), s.split(zw, "n")
    for i, lp in enumerate(lps):
        S = O.setup(lp)
        x_t, y_t = xs[i] / S.D_c, ys[i] / S.D_r
        z_t = np.maximum(0.0, S.c_t - S.At.T @ y_t)
        ox, oz, omu = O.centered_start_point(x_t, z_t)
        assert abs(mu[i] - omu) <= 1e-9 * omu, i
        assert rel_inf(xws[i], ox) < 1e-8 and rel_inf(zws[i], oz) < 1e-8, i


def test_batch_invalid_local_column_rejected():
    lps = mixed_batch()[:2]
    lps[1].col = lps[1].col.copy()
    lps[1].col[0] = lps[1].n  # out of its own LP's range (inside the next block's)
    with pytest.raises(pdhg.PDHGError) as e:
        pdhg.BatchSolver(lps)
    assert e.value.status == pdhg.PDHG_INVALID_ARG


# ---------------------------------------------------------------- persistent launch
def test_persistent_batch_equals_the_graph_path():
    """One cooperative launch for the whole batched solve (options.persistent)
    runs the same kernels in the same order as the graph of per-half-step
    launches on the same schedules (8 nonzeros per thread, full tiles): the
    float64 solves agree bit for bit, LP by LP."""
    lps = lpgen.planted_batch(count=16, m_lo=50, m_hi=600)
    out = {}
    for persistent in (0, 1):
        with pdhg.BatchSolver(lps, persistent=persistent, tile_nnz=2044) as s:
            assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
            g = s.get()
            out[persistent] = (np.asarray(g["x"]).copy(), np.asarray(g["y"]).copy(), g["iters"].copy())
    assert np.array_equal(out[0][2], out[1][2])
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_persistent_batch_iterates_match_oracle():
    lps = lpgen.planted_batch(count=8, m_lo=50, m_hi=400)
    with pdhg.BatchSolver(lps, persistent=1) as s:
        s.solve(1e-4, 100_000)
        g = s.get()
    xs = s.split(g["x"], "n")
    for i, lp in enumerate(lps):
        r = O.solve(lp, 1e-4, 100_000)
        assert g["iters"][i] == r.iters
        assert rel_inf(xs[i], r.x) < 1e-8


def test_persistent_fp32_batch_meets_the_test_in_fp64():
    lps = lpgen.planted_batch(count=12, m_lo=50, m_hi=600)
    with pdhg.BatchSolver(lps, precision="fp32", persistent=1) as s:
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        g = s.get()
        checks, rejects = s.fp64_checks()
    assert checks - rejects == len(lps)
    xs, ys = s.split(g["x"], "n"), s.split(g["y"], "m")
    for i, lp in enumerate(lps):
        A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
        ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, xs[i], ys[i], 1e-4)
        assert ok, (i, rp, rd, gap)


def test_persistent_barrier_wait_runs_out_to_timeout():
    """A grid barrier that waits for an arrival nothing makes (options.wait_test)
    gives up after wait_limit_ms: every block returns, the solve reports
    PDHG_TIMEOUT, and the GPU goes on working (a fresh batch then solves)."""
    import time
    lps = lpgen.planted_batch(count=4, m_lo=50, m_hi=200)
    with pdhg.BatchSolver(lps, persistent=1, wait_test=1, wait_limit_ms=50) as s:
        t0 = time.perf_counter()
        st = s.solve(1e-4, 10_000)
        dt = time.perf_counter() - t0
        msg = pdhg.lib().pdhg_last_error().decode()
    assert st == pdhg.PDHG_TIMEOUT
    assert np.all(s.lp_status == pdhg.PDHG_TIMEOUT)
    assert 0.04 <= dt < 30.0, dt
    assert "grid barrier" in msg
    with pdhg.BatchSolver(lps, persistent=1) as s2:
        assert s2.solve(1e-4, 100_000) == pdhg.PDHG_CONVERGED
