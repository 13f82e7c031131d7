"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances:
  * transpose: bit-exact (index work and copied values);
  * scaling D_r, D_c: 1e-12 relative (only the order of float64 products
    differs: the oracle divides round by round, the device multiplies
    accumulated factors);
  * FP64 iterates after 100 iterations: 1e-9 relative in the infinity norm;
  * FP32-mixed: no iterate parity; the termination test must hold when
    re-evaluated in float64, and the objective must agree with the FP64
    oracle to 1e-3 relative (the test at eps = 1e-4 bounds the relative gap
    by 1e-4; a 10x margin covers float32 residual evaluation).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg_oracle as O
from paper_2603_03150_gb300 import build as B
from paper_2603_03150_gb300 import lpgen
from paper_2603_03150_gb300 import pdhg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def rel_inf(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b)))) if b.size else 0.0


def dense_column_lp(seed=0):
    """An LP whose A^T has rows of every length class: 1, ~5, 40, 3000 and
    9000 entries (columns of A), exercising every per-column sort path."""
    rng = np.random.default_rng(seed)
    m, n = 9500, 300
    rows, cols = [], []
    for j in range(n):
        k = [1, 5, 40, 3000, 9000][j % 5] if j < 10 else int(rng.integers(1, 8))
        r = rng.choice(m, size=k, replace=False)
        rows.append(r)
        cols.append(np.full(k, j))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = rng.standard_normal(rows.size)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
    A.sort_indices()
    x = rng.uniform(0.5, 2, n) * (rng.random(n) < 0.3)
    y = rng.standard_normal(m)
    z = np.where(x > 0, 0.0, rng.uniform(0.5, 2, n))
    b = A @ x
    c = A.T @ y + z
    return lpgen.LP(m, n, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.copy(), b, c,
                    x, y, z, name="dense_columns")


def mid_column_lp(seed=0):
    """Columns of 150 to 1500 entries: shorter than a full tile of 8
    nonzeros per thread (2044), longer than the reduced tile capacities a
    forced tile_nnz may ask for, so those schedules split rows of A^T that
    the full capacity keeps whole (the split records of the evaluation must
    cover them)."""
    rng = np.random.default_rng(seed)
    m, n = 3000, 400
    rows, cols = [], []
    for j in range(n):
        k = [150, 600, 1500][j % 3] if j < 60 else int(rng.integers(2, 7))
        rows.append(rng.choice(m, size=k, replace=False))
        cols.append(np.full(k, j))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    A = sp.csr_matrix((rng.standard_normal(rows.size), (rows, cols)), shape=(m, n))
    A.sort_indices()
    x = rng.uniform(0.5, 2, n) * (rng.random(n) < 0.3)
    y = rng.standard_normal(m)
    z = np.where(x > 0, 0.0, rng.uniform(0.5, 2, n))
    return lpgen.LP(m, n, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.copy(),
                    A @ x, A.T @ y + z, x, y, z, name="mid_columns")


def heavy_row_lp(seed=0):
    """Power-law rows with some rows longer than every tile size (split rows)."""
    return lpgen.powerlaw_lp(m=3000, n=12000, nnz=90000, k_max=9000, seed=seed)


def gappy_lp(seed=0):
    """Runs of empty rows and empty columns (1200 / 1500 in a row: longer than
    a tile's row limit), rows and columns longer than any tile (split rows in
    A and A^T), single-entry rows, and a planted optimum."""
    rng = np.random.default_rng(seed)
    m, n = 4500, 6000
    live_r = np.r_[0:100, 1300:m]
    live_c = np.r_[0:2000, 3500:n]
    rows, cols = [], []
    for j in live_c:  # ~3 entries per live column
        k = int(rng.integers(1, 6))
        rows.append(rng.choice(live_r, size=k, replace=False))
        cols.append(np.full(k, j))
    rows.append(np.full(4500, 1500))  # a row of 4500 entries
    cols.append(rng.choice(live_c, size=4500, replace=False))
    rows.append(rng.choice(live_r, size=2500, replace=False))  # a column of 2500 entries
    cols.append(np.full(2500, 10))
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    A = sp.coo_matrix((rng.standard_normal(rows.size), (rows, cols)), shape=(m, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    x = rng.uniform(0.5, 2, n) * (rng.random(n) < 0.3)
    y = rng.standard_normal(m)
    z = np.where(x > 0, 0.0, rng.uniform(0.5, 2, n))
    b = A @ x
    c = A.T @ y + z
    return lpgen.LP(m, n, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.copy(), b, c,
                    x, y, z, name="gappy")


# ----------------------------------------------------------------- a1
@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(200, 500, seed=0), dense_column_lp,
                                   heavy_row_lp])
def test_transpose_bit_exact(maker):
    lp = maker()
    with pdhg.Solver.from_lp(lp) as s:
        rp, ci, v = s.transpose(lp.nnz)
    orp, oci, ov = O.transpose_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    np.testing.assert_array_equal(v, ov)


# ----------------------------------------------------------------- a2 + a3
@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(200, 500, seed=0), heavy_row_lp,
                                   lambda: lpgen.transportation_lp(40, 50)])
def test_scaling_and_step_parity(maker):
    lp = maker()
    S = O.setup(lp)
    with pdhg.Solver.from_lp(lp) as s:
        d = s.scaling()
    assert rel_inf(d["D_r"], S.D_r) < 1e-12
    assert rel_inf(d["D_c"], S.D_c) < 1e-12
    assert abs(d["sigma_max"] - S.sigma_max) <= 1e-10 * S.sigma_max
    assert abs(d["eta"] - S.eta) <= 1e-10 * S.eta
    assert abs(d["omega0"] - S.omega0) <= 1e-12 * S.omega0
    assert d["power_iters"] == S.power_iters


# ----------------------------------------------------------------- a4-a8, FP64
def _compare_state(st, ost, tol):
    assert rel_inf(st["x"], ost.x) < tol
    assert rel_inf(st["y"], ost.y) < tol
    assert rel_inf(st["x_avg"], ost.x_avg) < tol
    assert rel_inf(st["y_avg"], ost.y_avg) < tol
    assert st["k"] == ost.k and st["t"] == ost.t and st["restarts"] == ost.restarts
    assert abs(st["omega"] - ost.omega) <= tol * ost.omega


# tile_nnz: autotuned; 8 nonzeros per thread at reduced capacities (100: most
# rows split); 16 per thread (3000); 32 per thread, 64-bit window words (8000);
# the vector variant (falls back to segmented where rows exceed 256)
@pytest.mark.parametrize("tile_nnz", [0, 100, 512, 1371, 3000, 8000, -4, -8])
@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(200, 500, seed=0), heavy_row_lp,
                                   dense_column_lp, gappy_lp, mid_column_lp])
def test_fp64_iterates_after_100(maker, tile_nnz):
    lp = maker()
    r = O.solve(lp, 1e-12, 100)
    with pdhg.Solver.from_lp(lp, tile_nnz=tile_nnz) as s:
        st = s.solve(1e-12, 100)
        assert st == pdhg.PDHG_MAX_ITER
        _compare_state(s.state(), r.state, 1e-9)
        lg = s.log()
    assert [(e["k"], e["restart"], e["cand"]) for e in lg] == \
           [(e["k"], e["restart"], e["cand"]) for e in r.log]


@pytest.mark.parametrize("graphs", [True, False])
def test_fp64_solve_matches_oracle(graphs):
    lp = lpgen.planted_lp(200, 500, seed=0)
    r = O.solve(lp, 1e-4, 100_000)
    with pdhg.Solver.from_lp(lp, use_graphs=graphs) as s:
        assert s.solve(1e-4, 100_000) == pdhg.PDHG_CONVERGED
        g = s.get()
        info = s.info()
        lg = s.log()
    assert info["iters"] == r.iters and info["restarts"] == r.restarts
    assert info["chosen_average"] == (r.chosen == "average")
    assert [(e["k"], e["restart"], e["cand"]) for e in lg] == \
           [(e["k"], e["restart"], e["cand"]) for e in r.log]
    assert rel_inf(g["x"], r.x) < 1e-8 and rel_inf(g["y"], r.y) < 1e-8
    obj = float(lp.c @ r.x)
    assert abs(float(lp.c @ g["x"]) - obj) <= 1e-4 * abs(obj)
    eps = 1e-4
    assert g["r_P"] <= eps * (1 + np.linalg.norm(lp.b))
    assert g["r_D"] <= eps * (1 + np.linalg.norm(lp.c))
    assert abs(g["r_P"] - r.r_P) <= 1e-8 * (1 + r.r_P)
    assert abs(g["gap"] - r.gap) <= 1e-8 * (1 + abs(obj))
    assert abs(info["max_violation"] - r.max_violation) <= 1e-8 * (1 + r.max_violation)


def test_report_matches_oracle_residuals_on_gpu_iterate():
    lp = heavy_row_lp(1)
    with pdhg.Solver.from_lp(lp) as s:
        s.solve(1e-4, 640)
        g = s.get()
        info = s.info()
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    _, rp, rd, gap = O.termination_test(A, lp.b, lp.c, g["x"], g["y"], 1e-4)
    _, _, z = O.residuals(A, lp.b, lp.c, g["x"], g["y"])
    assert abs(g["r_P"] - rp) <= 1e-9 * (1 + rp)
    assert abs(g["r_D"] - rd) <= 1e-9 * (1 + rd)
    assert abs(g["gap"] - gap) <= 1e-9 * (1 + abs(float(lp.c @ g["x"])))
    assert rel_inf(g["z"], z) < 1e-9
    assert abs(info["max_violation"] - O.max_violation(A, lp.b, lp.c, g["x"], g["y"])) <= \
        1e-9 * (1 + info["max_violation"])


# ----------------------------------------------------------------- FP32-mixed
@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(200, 500, seed=0),
                                   lambda: lpgen.planted_lp(1000, 2500, seed=3),
                                   lambda: lpgen.transportation_lp(40, 50)])
def test_fp32_mixed_converges_and_holds_in_fp64(maker):
    lp = maker()
    r = O.solve(lp, 1e-4, 200_000)
    assert r.status == O.STATUS_CONVERGED
    with pdhg.Solver.from_lp(lp, precision="fp32") as s:
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        g = s.get()
        checks, rejects = s.fp64_checks()
    eps = 1e-4
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    # the float64 check decides convergence: the Section 2 test holds at eps itself
    ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, g["x"], g["y"], eps)
    assert ok, (rp, rd, gap)
    assert checks - rejects == 1
    obj = float(lp.c @ r.x)
    assert abs(float(lp.c @ g["x"]) - obj) <= 1e-3 * (1 + abs(obj))


@pytest.mark.parametrize("layout", ["csr", "panels"])
def test_fp32_screen_rejections_continue_the_solve(layout):
    """A loose float32 screen (100 eps) passes long before the iterate meets
    the test: each screened candidate is re-evaluated in float64, the early
    ones are rejected and the solve goes on, and the one accepted meets the
    Section 2 test at eps when the oracle re-evaluates it."""
    lp = lpgen.planted_lp(1000, 2500, seed=3)
    eps = 1e-4
    kw = dict(spmv_layout=layout, panel_width=512) if layout == "panels" else dict(spmv_layout="csr")
    with pdhg.Solver.from_lp(lp, precision="fp32", fp32_screen=100.0, **kw) as s:
        if layout == "panels" and s.layout()["a"]["panels"] == 0:
            pytest.skip("column panels do not apply to this LP")
        assert s.solve(eps, 200_000) == pdhg.PDHG_CONVERGED
        g = s.get()
        checks, rejects = s.fp64_checks()
        log = s.log()
    assert rejects >= 1 and checks == rejects + 1
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, g["x"], g["y"], eps)
    assert ok, (rp, rd, gap)
    # a rejected evaluation still applies the restart rule (it is logged)
    assert len(log) >= rejects


def test_fp64_context_runs_no_fp64_checks():
    lp = lpgen.planted_lp(200, 500, seed=0)
    with pdhg.Solver.from_lp(lp) as s:
        assert s.solve(1e-4, 100_000) == pdhg.PDHG_CONVERGED
        assert s.fp64_checks() == (0, 0)


# ----------------------------------------------------------------- a9
def test_warmstart_point_matches_oracle_on_gpu_iterate():
    lp = lpgen.planted_lp(200, 500, seed=0)
    S = O.setup(lp)
    with pdhg.Solver.from_lp(lp) as s:
        s.solve(1e-4, 100_000)
        info = s.info()
        st = s.state()
        xw, yw, zw, mu = s.warmstart_point()
        xu, yu, zu, mu2 = s.warmstart_point(unscaled=True)
    xs = st["x_avg"] if info["chosen_average"] else st["x"]
    ys = st["y_avg"] if info["chosen_average"] else st["y"]
    zs = np.maximum(0.0, S.c_t - S.At.T @ ys)
    ox, oz, omu = O.centered_start_point(xs, zs)
    assert abs(mu - omu) <= 1e-10 * omu and mu == mu2
    assert rel_inf(xw, ox) < 1e-9 and rel_inf(zw, oz) < 1e-9
    np.testing.assert_array_equal(yw, ys)
    assert rel_inf(xu, S.D_c * ox) < 1e-9 and rel_inf(zu, oz / S.D_c) < 1e-9
    assert rel_inf(yu, S.D_r * ys) < 1e-12


def test_warmstart_point_golden_cases_on_device():
    """Algorithm 1 hand cases through the device: an identity LP has
    D_r = D_c = 1 exactly, so setting x~ = x and y~ = 0 makes z~ = max(0, c)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "alg1_cases.json")))
    for case in g["cases"]:
        n = len(case["x"])
        I = sp.identity(n, format="csr")
        c = np.array(case["z"], dtype=float)
        b = np.ones(n)
        with pdhg.Solver(n, n, I.indptr, I.indices, I.data, b, c) as s:
            sc = s.scaling()
            assert np.all(sc["D_r"] == 1.0) and np.all(sc["D_c"] == 1.0)
            st = s.state()
            st.update(x=np.array(case["x"], float), y=np.zeros(n), x_avg=np.zeros(n),
                      y_avg=np.zeros(n), x_last=np.zeros(n), y_last=np.zeros(n))
            s.set_state(st)
            xw, yw, zw, mu = s.warmstart_point(case["mu_min"], case["delta_max"], case["alpha_min"])
        assert abs(mu - case["mu"]) <= 1e-15 * max(1.0, case["mu"]), case["name"]
        np.testing.assert_allclose(xw, case["x_out"], rtol=1e-12, err_msg=case["name"])
        np.testing.assert_allclose(zw, case["z_out"], rtol=1e-12, err_msg=case["name"])


# ----------------------------------------------------------------- checkpoint
def test_checkpoint_resume_matches_uninterrupted_run():
    lp = lpgen.planted_lp(200, 500, seed=2)
    with pdhg.Solver.from_lp(lp) as s:
        s.solve(1e-12, 192)
        ref = s.state()
    with pdhg.Solver.from_lp(lp) as s1:
        s1.solve(1e-12, 100)
        ck = s1.state()
    with pdhg.Solver.from_lp(lp) as s2:
        s2.set_state(ck)
        s2.solve(1e-12, 192)
        got = s2.state()
    for k in ["x", "y", "x_avg", "y_avg"]:
        assert rel_inf(got[k], ref[k]) < 1e-12, k
    assert got["k"] == ref["k"] == 192 and got["restarts"] == ref["restarts"]


# ----------------------------------------------------------------- edge cases
def test_edge_shapes_match_oracle():
    """One row; one column; an empty row (b_i = 0); ragged sizes."""
    rng = np.random.default_rng(7)
    cases = []
    # m = 1
    A = sp.csr_matrix(rng.uniform(0.5, 1.5, (1, 7)))
    cases.append(lpgen.LP(1, 7, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data,
                          np.array([3.0]), rng.uniform(0.5, 2, 7)))
    # n = 1
    A = sp.csr_matrix(rng.uniform(0.5, 1.5, (3, 1)))
    cases.append(lpgen.LP(3, 1, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data,
                          A.toarray().ravel() * 2.0, np.array([1.0])))
    # an empty row and an empty column
    D = rng.standard_normal((6, 9)) * (rng.random((6, 9)) < 0.5)
    D[2, :] = 0.0
    D[:, 4] = 0.0
    A = sp.csr_matrix(D)
    x0 = rng.uniform(0.5, 1, 9)
    cases.append(lpgen.LP(6, 9, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data,
                          D @ x0, rng.uniform(0.5, 2, 9)))
    for lp in cases:
        r = O.solve(lp, 1e-12, 130)
        with pdhg.Solver.from_lp(lp) as s:
            s.solve(1e-12, 130)
            _compare_state(s.state(), r.state, 1e-9)


@pytest.mark.parametrize("bad", ["rowptr", "col_range", "col_order", "nan_val", "nan_b"])
def test_invalid_input_is_rejected(bad):
    lp = lpgen.planted_lp(20, 50, seed=1)
    rp, col, val, b = lp.row_ptr.copy(), lp.col.copy(), lp.val.copy(), lp.b.copy()
    if bad == "rowptr":
        rp[5] = rp[6] + 1
    elif bad == "col_range":
        col[3] = lp.n
    elif bad == "col_order":
        s0 = rp[2]
        col[s0], col[s0 + 1] = col[s0 + 1], col[s0]
    elif bad == "nan_val":
        val[7] = np.nan
    else:
        b[0] = np.inf
    with pytest.raises(pdhg.PDHGError) as e:
        pdhg.Solver(lp.m, lp.n, rp, col, val, b, lp.c)
    assert e.value.status == pdhg.PDHG_INVALID_ARG


def test_device_io_with_torch_tensors():
    """Same schedule (tile_nnz pinned; autotuned contexts may pick different
    schedules and differ in the last bits), device vs host I/O: bit-equal."""
    import torch
    lp = lpgen.planted_lp(200, 500, seed=0)
    t = {k: torch.from_numpy(np.asarray(getattr(lp, k))).cuda()
         for k in ["row_ptr", "col", "val", "b", "c"]}
    stream = torch.cuda.Stream()
    with pdhg.Solver(lp.m, lp.n, t["row_ptr"], t["col"], t["val"], t["b"], t["c"],
                     device_io=True, stream=stream.cuda_stream, tile_nnz=2048) as s:
        assert s.solve(1e-4, 100_000) == pdhg.PDHG_CONVERGED
        g = s.get()
    with pdhg.Solver.from_lp(lp, tile_nnz=2048) as h:
        h.solve(1e-4, 100_000)
        gh = h.get()
    assert g["x"].is_cuda
    np.testing.assert_array_equal(g["x"].cpu().numpy(), gh["x"])
    np.testing.assert_array_equal(g["y"].cpu().numpy(), gh["y"])


def test_kernel_timing_samples():
    lp = lpgen.planted_lp(1000, 2500, seed=1)
    with pdhg.Solver.from_lp(lp, kernel_timing=True) as s:
        s.solve(1e-6, 640)
        t = s.kernel_timing()
    assert t["samples"] >= 5 and t["primal_ms"] > 0 and t["dual_ms"] > 0


# ----------------------------------------------------------------- tolerance sweep
def test_tolerance_sweep_matches_oracle():
    """eps_rel = 1e-4, 1e-6, 1e-8 (FP64): the oracle's iteration counts, the
    maximum violation of the returned point (Section 4.3) as the oracle computes
    it, and violations that shrink with eps."""
    lp = lpgen.planted_lp(200, 500, seed=0)
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    viols = []
    for eps in (1e-4, 1e-6, 1e-8):
        r = O.solve(lp, eps, 200_000)
        with pdhg.Solver.from_lp(lp) as s:
            assert s.solve(eps, 200_000) == pdhg.PDHG_CONVERGED
            g = s.get()
            info = s.info()
        assert info["iters"] == r.iters and info["restarts"] == r.restarts
        mv = O.max_violation(A, lp.b, lp.c, g["x"], g["y"])
        assert abs(info["max_violation"] - mv) <= 1e-9 * (1 + mv)
        assert abs(info["max_violation"] - r.max_violation) <= 1e-7 * (1 + r.max_violation)
        viols.append(info["max_violation"])
    assert viols[2] < viols[0]


# ----------------------------------------------------------------- no optimum
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["infeasible", "unbounded"])
def test_lp_without_optimum_ends_cleanly(kind, precision):
    """PDHG (this reading) has no infeasibility certificate: an LP without an
    optimum runs to the iteration limit or stops on a non-finite evaluation,
    never faults, and the context stays usable (get and the warm-start point
    answer; a second solve call continues)."""
    rng = np.random.default_rng(3)
    m, n = 30, 80
    D = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.3)
    if kind == "infeasible":
        D[0, :] = np.abs(D[0, :]) + 0.1      # sum of positive terms ...
        b = np.abs(rng.standard_normal(m))
        b[0] = -1.0                           # ... equal to -1: no x >= 0
        c = rng.uniform(0.5, 2.0, n)
    else:
        D[:, 0] = 0.0                         # column 0 free of constraints
        D[0, 0] = 0.0
        x0 = rng.uniform(0.5, 1.0, n)
        b = D @ x0
        c = rng.uniform(0.5, 2.0, n)
        c[0] = -1.0                           # and of negative cost: unbounded
    A = sp.csr_matrix(D)
    lp = lpgen.LP(m, n, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.copy(), b, c)
    with pdhg.Solver.from_lp(lp, precision=precision) as s:
        st = s.solve(1e-6, 3000)
        assert st in (pdhg.PDHG_MAX_ITER, pdhg.PDHG_NUMERICAL_ERROR)
        g = s.get()
        assert g["x"].shape == (n,)
        s.warmstart_point()
        st2 = s.solve(1e-6, 3200)
        assert st2 in (pdhg.PDHG_MAX_ITER, pdhg.PDHG_NUMERICAL_ERROR)
        assert s.info(violation=False)["iters"] <= 3200


def test_gather_floor_diagnostic_runs_and_leaves_state():
    lp = heavy_row_lp(0)
    with pdhg.Solver.from_lp(lp, precision="fp32") as s:
        s.solve(1e-12, 64)
        before = s.state()
        t_a, t_t = s.gather_floor(True, 3), s.gather_floor(False, 3)
        assert t_a > 0 and t_t > 0
        after = s.state()
        for k in ["x", "y", "x_avg", "y_avg"]:
            np.testing.assert_array_equal(before[k], after[k])
