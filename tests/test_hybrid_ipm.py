"""The host-side interior-point consumer of the warm-start point (Algorithm 1's
bump loop, Section 3.1): pinned against HiGHS (scipy.optimize.linprog) and
the Section 2 test; the bump loop's mechanics; warm starts from the oracle's
PDHG point."""
import numpy as np
import pytest
import scipy.optimize as so

from oracle import pdhg_oracle as O
from paper_2603_03150_gb300 import hybrid_ipm as H
from paper_2603_03150_gb300 import lpgen


def _scaled(lp):
    S = O.setup(lp)
    return S, S.At, S.b_t, S.c_t


def _highs(A, b, c):
    r = so.linprog(c, A_eq=A, b_eq=b, bounds=(0, None), method="highs")
    assert r.status == 0
    return r.fun


@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(200, 500, seed=0),
                                   lambda: lpgen.transportation_lp(20, 30),
                                   lambda: lpgen.tiny_feasible_lp(5, 10, 0),
                                   lambda: lpgen.tiny_feasible_lp(6, 12, 3)])
def test_cold_ipm_reaches_the_highs_optimum(maker):
    lp = maker()
    _, A, b, c = _scaled(lp)
    r = H.mehrotra(A, b, c)
    assert r["status"] == "optimal"
    ref = _highs(A, b, c)
    assert abs(float(c @ r["x"]) - ref) <= 1e-7 * (1 + abs(ref))
    # the Section 2 test at the interior-point tolerance, and an interior point
    assert H._converged(A, b, c, r["x"], r["y"], r["z"], 1e-8)
    assert np.min(r["x"]) > 0 and np.min(r["z"]) > 0


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_warm_start_from_the_pdhg_point(eps):
    """Algorithm 1's point from a PDHG solution at eps: the warm-started
    method reaches the same optimum, here in fewer iterations than cold."""
    lp = lpgen.planted_lp(200, 500, seed=0)
    res = O.solve(lp, eps, 100_000)
    S, A, b, c = _scaled(lp)
    xp, y, zp, _ = O.warmstart_point(res)
    rw = H.warm_start(A, b, c, xp, y, zp)
    rc = H.mehrotra(A, b, c)
    ref = _highs(A, b, c)
    assert rw["status"] == "optimal" and rw["bumps"] == 0
    assert abs(float(c @ rw["x"]) - ref) <= 1e-7 * (1 + abs(ref))
    assert rw["iters"] < rc["iters"]


def test_bump_loop_raises_alpha_min_tenfold_until_the_step_is_long_enough():
    lp = lpgen.planted_lp(60, 150, seed=1)
    res = O.solve(lp, 1e-4, 100_000)
    _, A, b, c = _scaled(lp)
    xp, y, zp, _ = O.warmstart_point(res)
    # a minimum step the method cannot take (steps stop at 0.99 of the way to
    # the boundary): every attempt is rejected and alpha_min grows to the cap
    r = H.warm_start(A, b, c, xp, y, zp, alpha_min=1e-6, min_step=0.995, max_bumps=4)
    assert r["status"] == "stuck" and r["bumps"] == 4
    assert r["alpha_min"] == pytest.approx(1e-6 * 10 ** 4)
    assert r["iters"] == 0
    # an attainable minimum step: no bump, and the start is left as given
    r = H.warm_start(A, b, c, xp, y, zp, alpha_min=1e-6, min_step=1e-6)
    assert r["bumps"] == 0 and r["status"] == "optimal"
    assert r["first_step"] >= 1e-6


def test_start_point_must_be_interior():
    lp = lpgen.tiny_feasible_lp(4, 8, 1)
    _, A, b, c = _scaled(lp)
    x = np.ones(lp.n)
    x[0] = 0.0
    with pytest.raises(ValueError):
        H.mehrotra(A, b, c, start=(x, np.zeros(lp.m), np.ones(lp.n)))
