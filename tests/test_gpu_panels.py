"""Column-panel half-steps (FP32-mixed, single LP) against the CPU oracle.

The panel path computes the same products A~^T y and A~ x+ of the PDHG
iteration (Section 2) as the CSR tiles, summed per panel and then across
panels, so:
  * the layout's pseudo-row count (distinct (panel, row) pairs of the
    nonzeros) is checked exactly against a host count;
  * after 10 iterations (one evaluation, at k = 10) the float32 iterates
    agree with the float64 oracle to 1e-5 relative in the infinity norm:
    each entry is a few float32 products and sums away from the oracle's,
    and a wrong index, sign or dropped term is an O(1) error;
  * after 100 iterations (evaluations at 64 and 100) the restart log equals
    the oracle's and the iterates agree to 1e-4 relative;
  * full solves pass the Section 2 test re-evaluated in float64 and the
    objective matches the FP64 oracle's to 1e-3 relative (as for the CSR
    FP32-mixed path).
Small panel widths give several panels at test sizes, long pseudo-rows
(more than 256 nonzeros of a row inside one panel), panels without any
nonzero and rows without nonzeros in a panel.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg_oracle as O
from paper_2603_03150_gb300 import build as B
from paper_2603_03150_gb300 import lpgen
from paper_2603_03150_gb300 import pdhg

from test_gpu_parity import dense_column_lp, gappy_lp, heavy_row_lp, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


# (maker, panel width asked for) -- widths chosen so every case has several
# panels on both matrices and the dense partial sums stay within the limit
CASES = [
    ("planted", lambda: lpgen.planted_lp(200, 500, seed=0), 64),
    ("planted_1panel", lambda: lpgen.planted_lp(200, 500, seed=0), 0),
    ("heavy_rows", heavy_row_lp, 2048),
    ("gappy", gappy_lp, 1024),
    ("dense_columns", dense_column_lp, 128),
    ("transport", lambda: lpgen.transportation_lp(40, 50), 256),
    # 100,000 columns of A~ at the widest width: tiles capped at 128
    # pseudo-rows (2 panels of 50,000 columns; the 256 cap would give 3)
    ("wide_128cap", lambda: lpgen.powerlaw_lp(m=10_000, n=100_000, nnz=500_000, k_max=2000,
                                               seed=4), 0),
]
IDS = [c[0] for c in CASES]


def pseudo_rows(rp, col, rows, P):
    """Distinct (panel, row) pairs among the nonzeros of a CSR matrix."""
    r = np.repeat(np.arange(rows), np.diff(rp))
    return len(set(zip((np.asarray(col) // P).tolist(), r.tolist())))


@pytest.mark.parametrize("name,maker,width", CASES, ids=IDS)
def test_layout_counts(name, maker, width):
    lp = maker()
    with pdhg.Solver.from_lp(lp, precision="fp32", spmv_layout="panels", panel_width=width) as s:
        L = s.layout()
    A = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    At = A.T.tocsr()
    At.sort_indices()
    for side, M, rows, cols in (("a", A, lp.m, lp.n), ("at", At, lp.n, lp.m)):
        d = L[side]
        assert d["panels"] > 0, (side, d)
        P = d["panel_width"]
        assert P % 8 == 0 and d["panels"] == -(-cols // P)
        if width:
            assert P <= width
        assert d["pseudo_rows"] == pseudo_rows(M.indptr, M.indices, rows, P)
        assert d["tiles"] >= 1


def test_wide_matrix_takes_the_128_pseudo_row_cap():
    """A~ with 100,000 columns and pseudo-rows of about 17 nonzeros: 256-nonzero
    tiles would hold far fewer than 96 pseudo-rows, so the layout caps tiles at
    128 pseudo-rows, which widens the panels: 2 of 50,000 columns (the 256 cap's
    shared-memory staging leaves room for 3 of 33,336).  A~^T (10,000 columns)
    fits one panel either way."""
    lp = CASES[IDS.index("wide_128cap")][1]()
    with pdhg.Solver.from_lp(lp, precision="fp32", spmv_layout="panels") as s:
        L = s.layout()
    assert L["a"]["panels"] == 2 and L["a"]["panel_width"] == 50_000, L["a"]
    assert L["at"]["panels"] == 1, L["at"]


def _state_close(st, ost, tol):
    assert rel_inf(st["x"], ost.x) < tol
    assert rel_inf(st["y"], ost.y) < tol
    assert rel_inf(st["x_avg"], ost.x_avg) < tol
    assert rel_inf(st["y_avg"], ost.y_avg) < tol
    assert st["k"] == ost.k and st["t"] == ost.t and st["restarts"] == ost.restarts


@pytest.mark.parametrize("method", ["averaged", "halpern"])
@pytest.mark.parametrize("name,maker,width", CASES, ids=IDS)
def test_iterates_match_oracle(name, maker, width, method):
    lp = maker()
    opts = O.Options(method=method)
    st = {}
    for k in (10, 100):  # fresh contexts: an evaluation happens at every solve's end
        with pdhg.Solver.from_lp(lp, precision="fp32", spmv_layout="panels", panel_width=width,
                                 method=method) as s:
            assert s.layout()["a"]["panels"] > 0 and s.layout()["at"]["panels"] > 0
            s.solve(1e-12, k)
            st[k] = s.state()
            lg = s.log()
    st10, st100 = st[10], st[100]
    r10 = O.solve(lp, 1e-12, 10, opts=opts)
    _state_close(st10, r10.state, 1e-5)
    r100 = O.solve(lp, 1e-12, 100, opts=opts)
    _state_close(st100, r100.state, 1e-4)
    assert [(e["k"], e["restart"], e["cand"]) for e in lg] == \
           [(e["k"], e["restart"], e["cand"]) for e in r100.log]


@pytest.mark.parametrize("name,maker,width", CASES, ids=IDS)
def test_panels_match_csr_tiles(name, maker, width):
    """The two float32 layouts differ only in the order of the sums."""
    lp = maker()
    out = {}
    for lay in ("csr", "panels"):
        with pdhg.Solver.from_lp(lp, precision="fp32", spmv_layout=lay, panel_width=width) as s:
            s.solve(1e-12, 100)
            out[lay] = (s.state(), s.layout())
    assert out["csr"][1]["a"]["panels"] == 0 and out["csr"][1]["at"]["panels"] == 0
    a, b = out["csr"][0], out["panels"][0]
    for k in ("x", "y", "x_avg", "y_avg"):
        assert rel_inf(b[k], a[k]) < 1e-4, k


@pytest.mark.parametrize("method", ["averaged", "halpern"])
@pytest.mark.parametrize("maker,width", [(lambda: lpgen.planted_lp(1000, 2500, seed=3), 256),
                                         (lambda: lpgen.transportation_lp(40, 50), 256),
                                         (heavy_row_lp, 2048)])
def test_panel_solve_holds_in_fp64(maker, width, method):
    lp = maker()
    r = O.solve(lp, 1e-4, 200_000)
    assert r.status == O.STATUS_CONVERGED
    with pdhg.Solver.from_lp(lp, precision="fp32", spmv_layout="panels", panel_width=width,
                             method=method) as s:
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        g = s.get()
    eps = 1e-4
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, g["x"], g["y"], eps)
    assert ok, (rp, rd, gap)
    obj = float(lp.c @ r.x)
    assert abs(float(lp.c @ g["x"]) - obj) <= 1e-3 * (1 + abs(obj))


def _edge_lps():
    rng = np.random.default_rng(11)
    out = []
    # one row
    out.append(lpgen.planted_lp(1, 40, seed=1))
    # one column per panel of width 8, rows of one nonzero
    m, n = 64, 64
    A = sp.identity(n, format="csr") * 2.0
    x = rng.uniform(0.5, 2, n) * (rng.random(n) < 0.5)
    y = rng.standard_normal(m)
    z = np.where(x > 0, 0.0, rng.uniform(0.5, 2, n))
    out.append(lpgen.LP(m, n, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.copy(),
                        A @ x, A.T @ y + z, x, y, z, name="diagonal"))
    # a dense row of 700 entries inside one panel of width 1024 (a long
    # pseudo-row) next to short rows
    m, n = 50, 1000
    rows = [np.zeros(700, int)]
    cols = [rng.choice(n, 700, replace=False)]
    for i in range(1, m):
        k = int(rng.integers(1, 9))
        rows.append(np.full(k, i))
        cols.append(rng.choice(n, k, replace=False))
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    A = sp.coo_matrix((rng.standard_normal(rows.size), (rows, cols)), shape=(m, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    x = rng.uniform(0.5, 2, n) * (rng.random(n) < 0.3)
    y = rng.standard_normal(m)
    z = np.where(x > 0, 0.0, rng.uniform(0.5, 2, n))
    out.append(lpgen.LP(m, n, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.copy(),
                        A @ x, A.T @ y + z, x, y, z, name="long_pseudo_row"))
    return out


@pytest.mark.parametrize("idx", range(3))
@pytest.mark.parametrize("width", [8, 1024])
def test_edge_shapes(idx, width):
    lp = _edge_lps()[idx]
    with pdhg.Solver.from_lp(lp, precision="fp32", spmv_layout="panels", panel_width=width) as s:
        L = s.layout()
        s.solve(1e-12, 10)
        st = s.state()
    r = O.solve(lp, 1e-12, 10)
    if L["a"]["panels"] == 0 and L["at"]["panels"] == 0:
        pytest.skip("panels do not apply to this shape")
    _state_close(st, r.state, 1e-5)


def test_auto_layout_reports_consistently_and_converges():
    lp = heavy_row_lp(2)
    with pdhg.Solver.from_lp(lp, precision="fp32") as s:
        L = s.layout()
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        g = s.get()
    for side in ("a", "at"):
        d = L[side]
        assert (d["panels"] == 0) == (d["panel_width"] == 0) == (d["tiles"] == 0)
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, g["x"], g["y"], 1e-4)
    assert ok, (rp, rd, gap)


def test_fp64_and_batches_ignore_panels():
    lp = lpgen.planted_lp(200, 500, seed=0)
    with pdhg.Solver.from_lp(lp, spmv_layout="panels", panel_width=64) as s:
        L = s.layout()
    assert L["a"]["panels"] == 0 and L["at"]["panels"] == 0


def test_full_size_powerlaw_matches_oracle():
    """The bench's power-law LP (m = 200k, n = 1M, 5M nonzeros) at full size:
    3 float32 iterations with the layout the bench runs (autotuned) and with
    column panels forced agree with 3 float64 oracle iterations to 1e-4
    relative over the whole vectors, with the same restart decision."""
    lp = lpgen.powerlaw_lp(seed=0)
    r = O.solve(lp, 1e-12, 3)
    for lay in ("auto", "panels"):
        with pdhg.Solver.from_lp(lp, precision="fp32", spmv_layout=lay) as s:
            L = s.layout()
            s.solve(1e-12, 3)
            st = s.state()
            lg = s.log()
        if lay == "panels":
            assert L["a"]["panels"] > 0 and L["at"]["panels"] > 0
        _state_close(st, r.state, 1e-4)
        assert [(e["k"], e["restart"], e["cand"]) for e in lg] == \
               [(e["k"], e["restart"], e["cand"]) for e in r.log]


def test_panels_are_deterministic_and_resume_from_a_checkpoint():
    """The panel sums have a fixed order: two contexts give bit-identical
    iterates, and a run checkpointed at k = 100 (iterates, averages, restart
    point, scalars and the A~x caches) and resumed in a new context repeats
    the uninterrupted run bit for bit.  (A solve that reaches max_iter stops
    before that evaluation's restart decision, so a checkpoint is taken off
    the evaluation points k = 64 j, where the uninterrupted run does not
    evaluate.)"""
    lp = heavy_row_lp(3)
    kw = dict(precision="fp32", spmv_layout="panels", panel_width=2048)
    runs = []
    for _ in range(2):
        with pdhg.Solver.from_lp(lp, **kw) as s:
            s.solve(1e-12, 320)
            runs.append(s.state())
    for k in ("x", "y", "x_avg", "y_avg", "Ax", "Ax_avg"):
        assert np.array_equal(runs[0][k], runs[1][k]), k
    with pdhg.Solver.from_lp(lp, **kw) as s1:
        s1.solve(1e-12, 100)
        ck = s1.state()
    with pdhg.Solver.from_lp(lp, **kw) as s2:
        s2.set_state(ck)
        s2.solve(1e-12, 320)
        got = s2.state()
    for k in ("x", "y", "x_avg", "y_avg", "Ax", "Ax_avg"):
        assert np.array_equal(got[k], runs[0][k]), k
    assert got["k"] == runs[0]["k"] == 320 and got["restarts"] == runs[0]["restarts"]


@pytest.mark.parametrize("layout", ["csr", "panels"])
def test_time_kernels_times_real_work_and_leaves_the_state(layout):
    """pdhg_time_kernels runs each half-step back to back on the current
    iterate (as mid-solve, also after a finished solve) and restores the
    state: the state after the call is bit-identical, a continued solve
    repeats an uninterrupted one, and every timed kernel did work (a
    half-step is slower than its panel SpMV alone; an iteration costs at
    least the slower half-step)."""
    lp = heavy_row_lp(3)
    kw = dict(precision="fp32", spmv_layout=layout, panel_width=2048)
    with pdhg.Solver.from_lp(lp, **kw) as s:
        s.solve(1e-12, 100)
        before = s.state()
        ms = s.time_kernels(20)
        after = s.state()
        for k in ("x", "y", "x_avg", "y_avg", "Ax", "Ax_avg"):
            assert np.array_equal(before[k], after[k]), k
        assert (before["k"], before["t"], before["omega"]) == (after["k"], after["t"], after["omega"])
        s.solve(1e-12, 200)
        cont = s.state()
    with pdhg.Solver.from_lp(lp, **kw) as s2:
        s2.solve(1e-12, 200)
        ref = s2.state()
    for k in ("x", "y", "x_avg", "y_avg"):
        assert np.array_equal(cont[k], ref[k]), k
    assert ms["primal_ms"] > 0 and ms["dual_ms"] > 0
    assert ms["iteration_ms"] >= 0.8 * max(ms["primal_ms"], ms["dual_ms"])
    if layout == "panels":
        assert 0 < ms["primal_spmv_ms"] < ms["primal_ms"] and 0 < ms["dual_spmv_ms"] < ms["dual_ms"]
    else:
        assert ms["primal_spmv_ms"] == 0 and ms["dual_spmv_ms"] == 0
    # after a finished solve the kernels are still timed as mid-solve
    with pdhg.Solver.from_lp(lpgen.planted_lp(200, 500, seed=0), **kw) as s3:
        assert s3.solve(1e-4, 100_000) == pdhg.PDHG_CONVERGED
        ms3 = s3.time_kernels(20)
        ms3b = s3.time_kernels(20)
        assert s3.info(violation=False)["status"] == pdhg.PDHG_CONVERGED
    assert ms3["dual_ms"] > 0 and ms3b["dual_ms"] > 0


def test_panel_load_wait_runs_out_to_timeout():
    """options.wait_test makes every panel load expect 16 bytes more than its
    bulk copies deliver, so its transaction barrier never completes: each
    block gives up after wait_limit_ms, flags the error and returns.  The
    solve reports PDHG_TIMEOUT with the reason, and the GPU goes on working
    (a context without the test bytes then solves)."""
    import time
    lp = lpgen.planted_lp(200, 500, seed=0)
    with pdhg.Solver.from_lp(lp, precision="fp32", spmv_layout="panels", wait_test=True,
                             wait_limit_ms=2, eval_freq=8) as s:
        t0 = time.perf_counter()
        st = s.solve(1e-4, 8)
        dt = time.perf_counter() - t0
        msg = pdhg.lib().pdhg_last_error().decode()
    assert st == pdhg.PDHG_TIMEOUT
    assert "column-panel" in msg
    # 8 iterations x 2 half-steps, each block waiting twice for 2 ms
    assert 0.03 <= dt < 30.0, dt
    with pdhg.Solver.from_lp(lp, precision="fp32", spmv_layout="panels") as s2:
        assert s2.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED


def test_wait_options_are_validated():
    lp = lpgen.planted_lp(20, 50, seed=0)
    for limit in (0, -5):
        with pytest.raises(pdhg.PDHGError):
            pdhg.Solver.from_lp(lp, precision="fp32", wait_limit_ms=limit)
