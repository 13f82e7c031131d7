"""Pins for the CPU oracle against facts fixed outside it: hand-derived
values, closed forms, invariants, brute force and an independent LP solver.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
flipped sign, a transposed operand, a wrong update order) breaks at least one.
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg_oracle as O
from paper_2603_03150_gb300 import lpgen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --------------------------------------------------------------- a1 transpose
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_transpose_matches_dense_and_is_stable(seed):
    rng = np.random.default_rng(seed)
    m, n = 37, 53
    D = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.15)
    rows, cols = np.nonzero(D)
    A = sp.csr_matrix((D[rows, cols], (rows, cols)), shape=(m, n))
    rp, ci, v = O.transpose_csr(m, n, A.indptr, A.indices, A.data)
    T = np.zeros((n, m))
    for j in range(n):
        T[j, ci[rp[j]:rp[j + 1]]] = v[rp[j]:rp[j + 1]]
        # stable: the rows of column j come in increasing order
        assert np.all(np.diff(ci[rp[j]:rp[j + 1]]) > 0)
    np.testing.assert_array_equal(T, D.T)


# --------------------------------------------------------------- a2 scaling
def test_ruiz_one_round_by_hand():
    # A = [[4,0],[1,9]]: row max [4,9] -> r=[2,3]; col max [4,9] -> s=[2,3]
    A = sp.csr_matrix(np.array([[4.0, 0.0], [1.0, 9.0]]))
    D_r, D_c, At = O.scale(A, ruiz_iters=1, pock_chambolle=False)
    np.testing.assert_allclose(D_r, [0.5, 1 / 3], rtol=1e-15)
    np.testing.assert_allclose(D_c, [0.5, 1 / 3], rtol=1e-15)
    np.testing.assert_allclose(At.toarray(), [[1.0, 0.0], [1 / 6, 1.0]], rtol=1e-15)


def test_pock_chambolle_by_hand():
    # A = [[4,0],[1,9]]: row 1-norms [4,10] -> r=[2,sqrt10]; col 1-norms [5,9] -> s=[sqrt5,3]
    A = sp.csr_matrix(np.array([[4.0, 0.0], [1.0, 9.0]]))
    D_r, D_c, At = O.scale(A, ruiz_iters=0, pock_chambolle=True)
    np.testing.assert_allclose(D_r, [0.5, 1 / np.sqrt(10)], rtol=1e-15)
    np.testing.assert_allclose(D_c, [1 / np.sqrt(5), 1 / 3], rtol=1e-15)
    np.testing.assert_allclose(At.toarray(), [[2 / np.sqrt(5), 0.0],
                                              [1 / np.sqrt(50), 3 / np.sqrt(10)]], rtol=1e-14)


def test_scaling_reconstructs_and_equilibrates():
    lp = lpgen.powerlaw_lp(m=2000, n=10000, nnz=50000, k_max=2000, seed=3)
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    D_r, D_c, At = O.scale(A, 10, True)
    R = sp.diags(D_r) @ A @ sp.diags(D_c)
    np.testing.assert_allclose(At.toarray(), R.toarray(), rtol=1e-12, atol=0)
    # Ruiz alone drives every row and column infinity norm to 1
    _, _, Ar = O.scale(A, 10, False)
    for v in (O._row_absmax(Ar), O._col_absmax(Ar)):
        assert v.min() >= 1 - 1e-2 and v.max() <= 1 + 1e-12
    _, _, Ar = O.scale(A, 20, False)
    for v in (O._row_absmax(Ar), O._col_absmax(Ar)):
        assert v.min() >= 1 - 1e-4 and v.max() <= 1 + 1e-12


def test_scaling_empty_row_and_column_keep_factor_one():
    A = sp.csr_matrix(np.array([[2.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 8.0]]))
    D_r, D_c, At = O.scale(A, 10, True)
    assert D_r[1] == 1.0 and D_c[1] == 1.0


# --------------------------------------------------------------- a3 step size
def test_power_iteration_closed_form_diagonal():
    A = sp.csr_matrix(np.diag([3.0, 1.0, 2.0]))
    s, k = O.power_iteration(A, 200, 1e-10)
    assert abs(s - 3.0) < 1e-9 and k < 200


@pytest.mark.parametrize("seed", [0, 1])
def test_power_iteration_vs_svd(seed):
    lp = lpgen.planted_lp(60, 150, 5, seed=seed)
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    _, _, At = O.scale(A)
    s, _ = O.power_iteration(At, 200, 1e-10)
    true = np.linalg.norm(At.toarray(), 2)
    assert s <= true * (1 + 1e-12)
    assert s >= true * (1 - 1e-3)


def test_initial_omega():
    assert O.initial_omega(np.array([3.0, 4.0]), np.array([0.0, 10.0])) == 2.0
    assert O.initial_omega(np.zeros(2), np.ones(2)) == 1.0


# --------------------------------------------------------------- a4/a5 step
def test_pdhg_step_by_hand():
    g = _load("small_lp_hand.json")
    A = sp.csr_matrix(np.array(g["A"]))
    s = g["step"]
    x1, y1 = O.pdhg_step(A, np.array(g["b"]), np.array(g["c"]), np.array(s["x"]),
                         np.array(s["y"]), s["tau"], s["sigma"])
    np.testing.assert_allclose(x1, s["x_new"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(y1, s["y_new"], rtol=0, atol=1e-15)


@pytest.mark.parametrize("tau,sigma", [(0.1, 10.0), (1.0, 1.0), (3.0, 0.01)])
def test_pdhg_fixed_point_at_planted_optimum(tau, sigma):
    """A strictly complementary optimum is a fixed point of one step for any
    tau, sigma > 0: on supp(x*), z* = 0 leaves x*; off it, x* - tau z* < 0
    projects to 0; and b - A x* = 0 leaves y*."""
    lp = lpgen.planted_lp(200, 500, seed=4)
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    x1, y1 = O.pdhg_step(A, lp.b, lp.c, lp.x_star, lp.y_star, tau, sigma)
    np.testing.assert_allclose(x1, lp.x_star, rtol=0, atol=1e-12 * (1 + tau))
    np.testing.assert_allclose(y1, lp.y_star, rtol=0, atol=1e-12 * (1 + sigma) * 10)


# --------------------------------------------------------------- a7 residuals
def test_kkt_termination_violation_by_hand():
    g = _load("small_lp_hand.json")
    A = sp.csr_matrix(np.array(g["A"]))
    b, c = np.array(g["b"]), np.array(g["c"])
    k = g["kkt"]
    assert abs(O.kkt_error(A, b, c, np.array(k["x"]), np.array(k["y"]), k["omega"])
               - k["value"]) < 1e-13
    t = g["term"]
    x, y = np.array(t["x"]), np.array(t["y"])
    ok1, rp, rd, gap = O.termination_test(A, b, c, x, y, 1.0)
    ok2 = O.termination_test(A, b, c, x, y, 2.0)[0]
    assert ok1 == t["converged_eps_1"] and ok2 == t["converged_eps_2"]
    assert abs(rp - t["r_P"]) < 1e-13 and abs(rd - t["r_D"]) < 1e-13 and abs(gap - t["gap"]) < 1e-13
    v = g["violation"]
    assert abs(O.max_violation(A, b, c, np.array(v["x"]), np.array(v["y"])) - v["value"]) < 1e-13


def test_optimality_conditions_at_planted_point():
    """Section 2: at the planted optimum the residuals vanish, x,z >= 0, and
    the gap c^T x - b^T y vanishes (equivalently x^T z = 0)."""
    lp = lpgen.planted_lp(200, 500, seed=0)
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    ok, rp, rd, gap = O.termination_test(A, lp.b, lp.c, lp.x_star, lp.y_star, 1e-12)
    assert ok and rp < 1e-12 and rd < 1e-12 and gap < 1e-10
    assert O.max_violation(A, lp.b, lp.c, lp.x_star, lp.y_star) < 1e-12


# --------------------------------------------------------------- a9 Algorithm 1
def test_algorithm1_hand_cases():
    for case in _load("alg1_cases.json")["cases"]:
        xp, zp, mu = O.centered_start_point(np.array(case["x"]), np.array(case["z"]),
                                            case["mu_min"], case["delta_max"], case["alpha_min"])
        assert abs(mu - case["mu"]) <= 1e-15 * max(1.0, case["mu"]), case["name"]
        np.testing.assert_allclose(xp, case["x_out"], rtol=1e-12, err_msg=case["name"])
        np.testing.assert_allclose(zp, case["z_out"], rtol=1e-12, err_msg=case["name"])


def test_algorithm1_centering_with_wide_delta():
    """With delta_max large enough that no clamp binds, the second update of
    each pair lands exactly on x'_j z'_j = mu_target."""
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 2, 400) * (rng.random(400) < 0.5)
    z = rng.uniform(0, 2, 400) * (rng.random(400) < 0.5)
    xp, zp, mu = O.centered_start_point(x, z, 1e-6, 1e6, 1e-6)
    np.testing.assert_allclose(xp * zp, mu, rtol=1e-12)
    assert np.all(xp > 0) and np.all(zp > 0)


# --------------------------------------------------------------- full solve
def test_solve_planted_small_converges_to_planted_optimum():
    lp = lpgen.planted_lp(200, 500, seed=0)
    r = O.solve(lp, 1e-4, 100_000)
    assert r.status == O.STATUS_CONVERGED
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    assert O.termination_test(A, lp.b, lp.c, r.x, r.y, 1e-4)[0]
    assert np.all(r.x >= 0) and np.all(r.z >= 0)
    obj = float(lp.c @ lp.x_star)
    assert abs(float(lp.c @ r.x) - obj) <= 1e-4 * (1 + abs(obj))
    r8 = O.solve(lp, 1e-8, 400_000)
    assert r8.status == O.STATUS_CONVERGED
    assert np.max(np.abs(r8.x - lp.x_star)) < 1e-5


def _brute_force_vertex_min(A, b, c):
    m, n = A.shape
    best = np.inf
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if abs(np.linalg.det(AB)) < 1e-10:
            continue
        xB = np.linalg.solve(AB, b)
        if np.all(xB >= -1e-10):
            best = min(best, float(c[list(B)] @ xB))
    return best


@pytest.mark.parametrize("m,n,seed", [(3, 7, 0), (4, 9, 1), (5, 10, 2), (6, 12, 3), (4, 8, 4)])
def test_solve_matches_vertex_enumeration(m, n, seed):
    lp = lpgen.tiny_feasible_lp(m, n, seed)
    A = lp.dense()
    best = _brute_force_vertex_min(A, lp.b, lp.c)
    r = O.solve(lp, 1e-9, 2_000_000)
    assert r.status == O.STATUS_CONVERGED
    assert abs(float(lp.c @ r.x) - best) <= 1e-6 * (1 + abs(best))


@pytest.mark.parametrize("m,n,seed", [(4, 9, 10), (5, 11, 11)])
def test_planted_tiny_matches_vertex_enumeration(m, n, seed):
    lp = lpgen.planted_lp(m, n, 3, seed=seed, n_pos=2)
    best = _brute_force_vertex_min(lp.dense(), lp.b, lp.c)
    assert abs(best - float(lp.c @ lp.x_star)) <= 1e-9 * (1 + abs(best))
    r = O.solve(lp, 1e-9, 2_000_000)
    assert abs(float(lp.c @ r.x) - best) <= 1e-6 * (1 + abs(best))


def test_solve_matches_highs_on_planted_and_transportation():
    from scipy.optimize import linprog
    for lp in (lpgen.planted_lp(200, 500, seed=1), lpgen.transportation_lp(30, 40, seed=0)):
        A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
        h = linprog(lp.c, A_eq=A, b_eq=lp.b, bounds=(0, None), method="highs")
        assert h.status == 0
        r = O.solve(lp, 1e-4, 200_000)
        assert r.status == O.STATUS_CONVERGED
        assert abs(float(lp.c @ r.x) - h.fun) <= 2e-4 * (1 + abs(h.fun)), lp.name


def test_max_iter_stops_without_restart_and_counts():
    lp = lpgen.planted_lp(200, 500, seed=0)
    r = O.solve(lp, 1e-12, 100)
    assert r.status == O.STATUS_MAX_ITER and r.iters == 100
    # one evaluation of the restart rule at k = 64 (k = 100 only tests termination)
    assert [e["k"] for e in r.log] == [64]
    r2 = O.solve(lp, 1e-12, 128)
    assert [e["k"] for e in r2.log] == [64]  # k = 128 = max_iter: no restart rule


def test_termination_primal_bound_uses_norm_b():
    g = _load("small_lp_hand.json")
    A = sp.csr_matrix(np.array(g["A"]))
    b, c = np.array(g["b"]), np.array(g["c"])
    t = g["term_primal_binding"]
    x, y = np.array(t["x"]), np.array(t["y"])
    ok8, rp, rd, gap = O.termination_test(A, b, c, x, y, 0.8)
    assert ok8 == t["converged_eps_0.8"]
    assert O.termination_test(A, b, c, x, y, 0.7)[0] == t["converged_eps_0.7"]
    assert abs(rp - t["r_P"]) < 1e-13 and rd == t["r_D"] and abs(gap - t["gap"]) < 1e-13


def test_running_average_is_mean_of_iterates():
    """Before the first evaluation the averages are the plain means of the
    iterates x^1..x^k, y^1..y^k produced by repeated single steps."""
    lp = lpgen.planted_lp(200, 500, seed=2)
    S = O.setup(lp)
    r = O.solve(lp, 1e-12, 50, S=S)
    tau, sigma = S.eta / S.omega0, S.eta * S.omega0
    x, y = np.zeros(lp.n), np.zeros(lp.m)
    xs, ys = [], []
    for _ in range(50):
        x, y = O.pdhg_step(S.At, S.b_t, S.c_t, x, y, tau, sigma)
        xs.append(x)
        ys.append(y)
    np.testing.assert_allclose(r.state.x, x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(r.state.x_avg, np.mean(xs, axis=0), rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.state.y_avg, np.mean(ys, axis=0), rtol=0, atol=1e-12)


# ------------------------------------------------------ reflected Halpern (optional)
def _m_norm2(A, tau, sigma, x, y):
    """||(x, y)||_M^2 for the PDHG metric M = [[I/tau, A^T], [A, I/sigma]] of
    the update x+ = P(x - tau(c - A^T y)), y+ = y + sigma(b - A(2x+ - x))
    (A is the scaled m x n matrix)."""
    return float(x @ x / tau + y @ y / sigma + 2.0 * (y @ (A @ x)))


def _m_inner(A, tau, sigma, u, v):
    (ux, uy), (vx, vy) = u, v
    return float(ux @ vx / tau + uy @ vy / sigma + uy @ (A @ vx) + vy @ (A @ ux))


def test_pdhg_step_is_firmly_nonexpansive_in_the_pdhg_metric():
    """The PDHG map is the resolvent of a monotone operator in the metric M:
    ||Tz - Tw||_M^2 <= <Tz - Tw, z - w>_M for any z, w.  A sign slip in the
    extrapolation or a transposed product breaks it for some pair."""
    lp = lpgen.planted_lp(40, 90, seed=3)
    S = O.setup(lp)
    At, b_t, c_t = S.At, S.b_t, S.c_t
    m, n = At.shape
    tau, sigma = S.eta / S.omega0, S.eta * S.omega0
    rng = np.random.default_rng(0)
    for _ in range(50):
        z = (rng.standard_normal(n), rng.standard_normal(m))
        w = (rng.standard_normal(n), rng.standard_normal(m))
        Tz = O.pdhg_step(At, b_t, c_t, *z, tau, sigma)
        Tw = O.pdhg_step(At, b_t, c_t, *w, tau, sigma)
        d = (Tz[0] - Tw[0], Tz[1] - Tw[1])
        lhs = _m_norm2(At, tau, sigma, *d)
        rhs = _m_inner(At, tau, sigma, d, (z[0] - w[0], z[1] - w[1]))
        assert lhs <= rhs * (1 + 1e-12) + 1e-12


def test_halpern_first_step_with_full_reflection_is_one_pdhg_step():
    """rho = 1, t = 0: lam = 1/2 and z1 = (2 T(z0) - z0)/2 + z0/2 = T(z0)."""
    lp = lpgen.planted_lp(30, 70, seed=1)
    ra = O.solve(lp, 1e-15, 1)
    rh = O.solve(lp, 1e-15, 1, opts=O.Options(method="halpern", reflection=1.0))
    np.testing.assert_allclose(rh.state.x, ra.state.x, rtol=0, atol=1e-15)
    np.testing.assert_allclose(rh.state.y, ra.state.y, rtol=0, atol=1e-15)


@pytest.mark.parametrize("start", ["zero", "restart_point"])
@pytest.mark.parametrize("rho", [0.0, 0.5, 1.0])
def test_halpern_fixed_point_residual_bound(rho, start):
    """Without restarts, Halpern's iteration on the nonexpansive operator
    R = (1 + rho) T - rho I with lam_t = (t+1)/(t+2) satisfies
    ||z_t - R z_t||_M <= 2 ||z_0 - z*||_M / (t + 1); since z - Rz = (1+rho)(z - Tz)
    this is ||z_t - T z_t||_M <= 2 ||z_0 - z*||_M / ((1 + rho)(t + 1)) for every
    saddle point z* (here the planted one, scaled).  A wrong weight, a missing
    anchor term or a wrong reflection breaks it within the first iterations."""
    lp = lpgen.planted_lp(60, 150, seed=2)
    opts = O.Options(method="halpern", reflection=rho, beta_sufficient=0.0,
                     beta_necessary=0.0, beta_artificial=1e30)
    S = O.setup(lp, opts)
    At, b_t, c_t = S.At, S.b_t, S.c_t
    tau, sigma = S.eta / S.omega0, S.eta * S.omega0
    xs, ys = lp.x_star / S.D_c, lp.y_star / S.D_r
    # z* is a fixed point of T (the planted pair is a saddle point)
    Tx, Ty = O.pdhg_step(At, b_t, c_t, xs, ys, tau, sigma)
    assert np.max(np.abs(Tx - xs)) < 1e-9 and np.max(np.abs(Ty - ys)) < 1e-9
    st = O.initial_state(S)
    if start == "restart_point":  # as right after a restart: z = z0 = anchor != 0
        rng = np.random.default_rng(5)
        st.x = st.x_last = rng.uniform(0.0, 2.0, st.x.size)
        st.y = st.y_last = rng.standard_normal(st.y.size)
    r0 = np.sqrt(_m_norm2(At, tau, sigma, st.x - xs, st.y - ys))
    for t in range(1, 201):
        res = O.solve(lp, 1e-300, t, opts=opts, S=S, state=st)
        st = res.state
        assert st.restarts == 0 and st.t == t
        Tx, Ty = O.pdhg_step(At, b_t, c_t, st.x, st.y, tau, sigma)
        g = np.sqrt(max(0.0, _m_norm2(At, tau, sigma, st.x - Tx, st.y - Ty)))
        assert g <= 2.0 * r0 / ((1.0 + rho) * (t + 1)) * (1 + 1e-9), t


def test_halpern_solve_reaches_the_planted_optimum():
    lp = lpgen.planted_lp(200, 500, seed=0)
    r = O.solve(lp, 1e-8, 200_000, opts=O.Options(method="halpern"))
    assert r.status == O.STATUS_CONVERGED
    opt = float(lp.c @ lp.x_star)
    assert abs(float(lp.c @ r.x) - opt) <= 1e-6 * (1 + abs(opt))
    assert np.max(np.abs(r.x - lp.x_star)) < 1e-5


def test_halpern_second_candidate_is_the_projected_pdhg_output():
    """The reflected iterate leaves the cone x >= 0 (2 x^ - x < 0 where x^ = 0 <
    x), the PDHG output T(z) never does: the evaluation's second candidate
    (and any iterate returned as 'average') is T(z), not z."""
    lp = lpgen.planted_lp(200, 500, seed=4)
    r = O.solve(lp, 1e-300, 100, opts=O.Options(method="halpern", reflection=1.0))
    assert np.min(r.state.x) < 0.0           # the iterate itself is outside
    assert np.min(r.state.x_avg) >= 0.0      # the candidate is inside
    r2 = O.solve(lp, 1e-4, 200_000, opts=O.Options(method="halpern", reflection=1.0))
    if r2.chosen == "average":
        assert np.min(r2.x_scaled) >= 0.0


# --------------------------------------------------------------- a8 restart rule and omega
_RR = None


def _rr():
    global _RR
    if _RR is None:
        _RR = _load("restart_rule_cases.json")
    return _RR


def _decision_failures(decide):
    """Names of the hand cases that `decide` (restart_decision's signature)
    gets wrong."""
    g = _rr()
    opts = O.Options(**g["betas"])
    bad = []
    for c in g["decisions"]:
        d = decide(c["kkt_cur"], c["kkt_avg"], c["kkt_last"], c["kkt_prev"], c["t"], c["k"], opts)
        if any(d[key] != c[key] for key in ("use_avg", "k_cand", "r1", "r2", "r3", "restart")):
            bad.append(c["name"])
    return bad


def _omega_failures(update):
    bad = []
    for c in _rr()["omega"]:
        w = update(c["dx"], c["dy"], c["omega"], c["theta"], 1e-10)
        if abs(w - c["omega_new"]) > 1e-14 * c["omega_new"]:
            bad.append(c["name"])
    return bad


def test_restart_decision_hand_cases():
    assert _decision_failures(O.restart_decision) == []


def test_omega_update_hand_cases():
    assert _omega_failures(O.omega_update) == []


def test_restart_bookkeeping_trace_by_hand():
    g = _rr()
    tr = g["trace"]
    opts = O.Options(**g["betas"])
    last, prev = tr["start"]["kkt_last"], tr["start"]["kkt_prev"]
    for e in tr["evals"]:
        d = O.restart_decision(e["kkt_cur"], e["kkt_avg"], last, prev, e["t"], e["k"], opts)
        for key in ("use_avg", "restart", "r1", "r2", "r3"):
            assert d[key] == e[key], (e["k"], key)
        last, prev = O.advance_restart_kkts(last, d["k_cand"], d["restart"])
        assert (last, prev) == (e["kkt_last"], e["kkt_prev"]), e["k"]


def _mutant_decision(kind):
    def decide(kc, ka, kl, kp, t, k, opts):
        use_avg = (ka <= kc) if kind == "tie_to_average" else (ka < kc)
        cand = ka if use_avg else kc
        r1 = cand <= opts.beta_sufficient * kl
        if kind == "r2_against_last":
            r2 = cand <= opts.beta_necessary * kl and cand > kl
        elif kind == "r2_ge":
            r2 = cand <= opts.beta_necessary * kl and cand >= kp
        elif kind == "r2_against_current":
            r2 = cand <= opts.beta_necessary * kl and kc > kp
        else:
            r2 = cand <= opts.beta_necessary * kl and cand > kp
        r3 = (t > opts.beta_artificial * k) if kind == "r3_strict" else (t >= opts.beta_artificial * k)
        if kind == "cand_is_current":
            cand = kc
            r1 = cand <= opts.beta_sufficient * kl
        return dict(use_avg=use_avg, k_cand=cand, r1=r1, r2=r2, r3=r3, restart=r1 or r2 or r3)
    return decide


@pytest.mark.parametrize("kind", ["tie_to_average", "r2_against_last", "r2_ge", "r2_against_current",
                                  "r3_strict", "cand_is_current"])
def test_restart_pins_catch_planted_slips(kind):
    """Each plausible slip in the rule, planted in a copy on the CPU, fails a
    named hand case."""
    assert _decision_failures(_mutant_decision(kind)) != []


@pytest.mark.parametrize("kind", ["swap_dx_dy", "swap_theta", "no_old_weight", "guard_ge"])
def test_omega_pins_catch_planted_slips(kind):
    def update(dx, dy, w, theta, mn):
        if kind == "guard_ge":
            ok = dx >= mn and dy >= mn
        else:
            ok = dx > mn and dy > mn
        if not ok:
            return w
        if kind == "swap_dx_dy":
            dx, dy = dy, dx
        if kind == "swap_theta":
            theta = 1.0 - theta
        if kind == "no_old_weight":
            return float(np.exp(theta * np.log(dy / dx)))
        return float(np.exp(theta * np.log(dy / dx) + (1.0 - theta) * np.log(w)))
    assert _omega_failures(update) != []


def test_solve_applies_the_rule_it_logs():
    """The loop feeds the rule the right references: every logged evaluation
    equals restart_decision on the logged inputs, kkt_last / kkt_prev move as
    the bookkeeping says, and omega moves by omega_update on the logged
    distances (wiring check of the loop around the pinned functions)."""
    lp = lpgen.planted_lp(m=60, n=150, nnz_per_col=4, seed=5)
    res = O.solve(lp, eps_rel=1e-7, max_iter=64 * 40)
    opts = O.Options()
    assert len(res.log) >= 5 and any(e["restart"] for e in res.log)
    assert any(e["restart"] and not e["r3"] for e in res.log)
    for e, nxt in zip(res.log, res.log[1:] + [None]):
        d = O.restart_decision(e["kkt_cur"], e["kkt_avg"], e["kkt_last"], e["kkt_prev"],
                               e["t"], e["k"], opts)
        assert (d["restart"], d["r1"], d["r2"], d["r3"]) == (e["restart"], e["r1"], e["r2"], e["r3"])
        assert e["cand"] == ("average" if d["use_avg"] else "current")
        last, prev = O.advance_restart_kkts(e["kkt_last"], d["k_cand"], d["restart"])
        if e["restart"]:
            w = O.omega_update(e["dx"], e["dy"], e["omega"], opts.theta, opts.omega_update_min)
            assert e["omega_new"] == w
        if nxt is not None:
            assert (nxt["kkt_last"], nxt["kkt_prev"]) == (last, prev)
            assert nxt["omega"] == (e["omega_new"] if e["restart"] else e["omega"])
            assert nxt["t"] == (nxt["k"] - e["k"] if e["restart"] else e["t"] + nxt["k"] - e["k"])


@pytest.mark.parametrize("kind", ["prev_only_on_restart", "last_always", "prev_is_current"])
def test_bookkeeping_trace_catches_planted_slips(kind):
    g = _rr()
    tr = g["trace"]
    opts = O.Options(**g["betas"])
    last, prev = tr["start"]["kkt_last"], tr["start"]["kkt_prev"]
    wrong = False
    for e in tr["evals"]:
        d = O.restart_decision(e["kkt_cur"], e["kkt_avg"], last, prev, e["t"], e["k"], opts)
        if kind == "prev_only_on_restart":
            last, prev = (d["k_cand"], d["k_cand"]) if d["restart"] else (last, prev)
        elif kind == "last_always":
            last, prev = d["k_cand"], d["k_cand"]
        else:
            last, prev = (d["k_cand"] if d["restart"] else last), e["kkt_cur"]
        wrong |= (last, prev) != (e["kkt_last"], e["kkt_prev"])
    assert wrong


# --------------------------------------------------------------- PID primal weight
def _pid_failures(update):
    """Names of the hand-worked PID traces that `update`
    (omega_update_pid's signature) gets wrong."""
    bad = []
    for tr in _load("pid_weight_cases.json")["traces"]:
        w, I, e = tr["omega0"], tr["integral0"], tr["prev0"]
        for st in tr["steps"]:
            w, I, e = update(st["dx"], st["dy"], w, I, e, tr["kp"], tr["ki"], tr["kd"], 1e-10)
            if (abs(w - st["omega"]) > 1e-14 * st["omega"] or abs(I - st["integral"]) > 1e-14
                    or abs(e - st["error"]) > 1e-14):
                bad.append(tr["name"])
                break
    return bad


def test_pid_weight_hand_traces():
    assert _pid_failures(O.omega_update_pid) == []


def test_pid_with_kp_only_is_the_smoothing_rule():
    rng = np.random.default_rng(3)
    for _ in range(50):
        dx, dy, w, th = rng.uniform(0.1, 10), rng.uniform(0.1, 10), rng.uniform(0.1, 10), rng.uniform(0, 1)
        a = O.omega_update_pid(dx, dy, w, 0.0, 0.0, th, 0.0, 0.0)[0]
        assert abs(a - O.omega_update(dx, dy, w, th)) <= 1e-13 * a


def test_pid_default_gains_converge_to_a_constant_ratio():
    """With the distances' ratio fixed at rho, the loop's fixed point is
    omega = rho with no accumulated error (the integral returns to 0); with
    the default gains the integral decays by about ki = 1% per restart."""
    for rho, w in ((5.0, 1.0), (0.01, 30.0)):
        I = e = 0.0
        for _ in range(4000):
            w, I, e = O.omega_update_pid(1.0, rho, w, I, e)
        assert abs(np.log(w / rho)) < 1e-10 and abs(I) < 1e-8


@pytest.mark.parametrize("kind", ["error_sign", "integral_before_update", "derivative_reversed",
                                  "derivative_on_error"])
def test_pid_traces_catch_planted_slips(kind):
    def update(dx, dy, w, I, ep, kp, ki, kd, mn):
        if not (dx > mn and dy > mn):
            return w, I, ep
        e = np.log(dy / dx) - np.log(w)
        if kind == "error_sign":
            e = -e
        I_new = I + e
        Iu = I if kind == "integral_before_update" else I_new
        d = (ep - e) if kind == "derivative_reversed" else (e if kind == "derivative_on_error" else e - ep)
        return float(np.exp(np.log(w) + kp * e + ki * Iu + kd * d)), float(I_new), float(e)
    assert _pid_failures(update) != []


def test_pid_solve_reaches_the_planted_optimum():
    lp = lpgen.planted_lp(200, 500, seed=0)
    r = O.solve(lp, 1e-6, 200_000, opts=O.Options(omega_rule="pid"))
    assert r.status == O.STATUS_CONVERGED
    obj = float(lp.c @ lp.x_star)
    assert abs(float(lp.c @ r.x) - obj) <= 1e-5 * (1 + abs(obj))
    assert any("pid_integral" in e for e in r.log)


# ----------------------------------------------------- adaptive step (PDLP)
ADAPT = json.load(open(os.path.join(GOLD, "adaptive_step_cases.json")))


def _adapt_case_ok(fn, c):
    a = fn(np.array(c["dx"]), np.array(c["dy"]), np.array(c["A_dx"]), c["eta"], c["omega"], c["j"])
    em = float("inf") if c["eta_max"] == "inf" else c["eta_max"]
    return (a["accept"] == c["accept"] and a["eta_max"] == pytest.approx(em, rel=1e-14)
            and a["eta_next"] == pytest.approx(c["eta_next"], rel=1e-14))


def test_adaptive_step_hand_cases():
    for c in ADAPT["cases"]:
        assert _adapt_case_ok(O.adaptive_step, c), c["name"]


def _adaptive_slip(kind):
    def f(dx, dy, A_dx, eta, omega, j):
        inter = float(np.dot(dy, A_dx)) if kind == "no_abs" else abs(float(np.dot(dy, A_dx)))
        if kind == "omega_swapped":
            num = float(np.dot(dx, dx)) / omega + omega * float(np.dot(dy, dy))
        else:
            num = omega * float(np.dot(dx, dx)) + float(np.dot(dy, dy)) / omega
        two = 1.0 if kind == "no_two" else 2.0
        em = num / (two * inter) if inter != 0.0 else float("inf")
        jj = j if kind == "j_excludes_current" else j + 1.0
        p1, p2 = (-0.6, -0.3) if kind == "exponents_swapped" else (-0.3, -0.6)
        nxt = min((1.0 - jj ** p1) * em, (1.0 + jj ** p2) * eta)
        return dict(accept=eta <= em, eta_max=em, eta_next=nxt)
    return f


@pytest.mark.parametrize("kind", ["no_abs", "omega_swapped", "no_two", "j_excludes_current",
                                  "exponents_swapped"])
def test_adaptive_step_pins_catch_planted_slips(kind):
    slip = _adaptive_slip(kind)
    assert not all(_adapt_case_ok(slip, c) for c in ADAPT["cases"]), kind


def test_step_weighted_average_by_hand():
    g = ADAPT["weighted_average"]
    avg, total = np.zeros(1), 0.0
    for x, eta, want, s in zip(g["x"], g["eta"], g["averages"], g["sums"]):
        avg, total = O.step_weighted_average(avg, np.array([x]), eta, total)
        assert avg[0] == pytest.approx(want, rel=1e-15) and total == s


def test_small_steps_are_always_accepted():
    """|dy^T A dx| <= ||A|| ||dx|| ||dy|| <= ||A|| (omega ||dx||^2 + ||dy||^2 / omega) / 2,
    so eta_max >= 1 / ||A||_2 for every move: a step at 1 / ||A||_2 is never
    rejected, while large steps are."""
    rng = np.random.default_rng(11)
    rejected = 0
    for _ in range(200):
        A = rng.normal(size=(7, 5))
        dx, dy = rng.normal(size=5), rng.normal(size=7)
        omega = float(np.exp(rng.uniform(-2, 2)))
        s = float(np.linalg.norm(A, 2))
        assert O.adaptive_step(dx, dy, A @ dx, 1.0 / s, omega, 5)["accept"]
        rejected += not O.adaptive_step(dx, dy, A @ dx, 100.0 / s, omega, 5)["accept"]
    assert rejected > 0


def test_adaptive_rejection_leaves_the_iterate_and_averages():
    """From the start with a step 100x the constant one: the attempt is
    rejected (nothing but the step and the counters moves, the step shrinks);
    attempts go on shrinking it until one is accepted, which moves the
    iterate, and the accepted step then satisfies eta <= eta_max."""
    lp = lpgen.planted_lp(200, 500, seed=0)
    opts = O.Options(step_rule="adaptive")
    S = O.setup(lp, opts)
    st = O.initial_state(S)
    st.eta = 100.0 * S.eta
    x0, y0, xa0 = st.x.copy(), st.y.copy(), st.x_avg.copy()
    r = O.solve(lp, 1e-12, 1, opts=opts, S=S, state=st)
    st = r.state
    assert st.step_rejects == 1 and st.k == 1 and st.t == 1 and st.eta < 100.0 * S.eta
    assert np.array_equal(st.x, x0) and np.array_equal(st.y, y0) and np.array_equal(st.x_avg, xa0)
    assert st.eta_sum == 0.0
    for k in range(2, 40):
        eta, rej = st.eta, st.step_rejects
        st = O.solve(lp, 1e-12, k, opts=opts, S=S, state=st).state
        if st.step_rejects == rej:  # accepted: the iterate moved with step eta
            assert not np.array_equal(st.x, x0) and st.eta_sum == eta
            assert np.array_equal(st.x_avg, st.x)  # the first accepted iterate is the average
            break
    else:
        raise AssertionError("no attempt accepted")


def test_adaptive_solve_reaches_the_planted_optimum():
    for lp in (lpgen.planted_lp(200, 500, seed=0), lpgen.planted_lp(500, 1250, seed=2)):
        r = O.solve(lp, 1e-6, 100_000, opts=O.Options(step_rule="adaptive"))
        assert r.status == O.STATUS_CONVERGED
        obj = float(lp.c @ lp.x_star)
        assert abs(float(lp.c @ r.x) - obj) <= 1e-5 * (1 + abs(obj))
    with pytest.raises(ValueError):
        O.solve(lpgen.planted_lp(20, 50, seed=0), 1e-4, 10,
                opts=O.Options(step_rule="adaptive", method="halpern"))
