"""The hand-over chain on the GPU (Algorithm 1, Section 3.1; Section 4.6's
warm-start statistics): pdhg_solve to eps_rel on the device, the start point
of pdhg_warmstart_point in the scaled model, then the host interior-point
consumer (a Mehrotra predictor-corrector with Algorithm 1's bump loop)
warm-started from it.  The consumer must reach the HiGHS optimum of the same
scaled LP (scipy.optimize.linprog) and, from a PDHG point, in fewer
iterations than from its cold start; a start whose first interior-point step
is below the paper's minimum (1e-6) must drive the bump loop."""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

from paper_2603_03150_gb300 import build as B
from paper_2603_03150_gb300 import hybrid_ipm as H
from paper_2603_03150_gb300 import lpgen, pdhg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _scaled_lp(lp, sc):
    """A~ = D_r A D_c, b~ = D_r b, c~ = D_c c from the context's own scaling."""
    Dr, Dc = np.asarray(sc["D_r"]), np.asarray(sc["D_c"])
    A = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    return (sp.diags(Dr) @ A @ sp.diags(Dc)).tocsr(), Dr * lp.b, Dc * lp.c


def _highs(A, b, c):
    r = so.linprog(c, A_eq=A, b_eq=b, bounds=(0, None), method="highs")
    assert r.status == 0
    return r.fun


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("eps", [1e-4, 1e-6])
@pytest.mark.parametrize("maker", [lambda: lpgen.planted_lp(200, 500, seed=0),
                                   lambda: lpgen.planted_lp(500, 1250, seed=2),
                                   lambda: lpgen.transportation_lp(20, 30)])
def test_gpu_start_point_warm_starts_the_interior_point_method(maker, eps, precision):
    lp = maker()
    if precision == "fp32" and eps < 1e-4:
        pytest.skip("float32-mixed is used at the hand-over tolerance 1e-4")
    with pdhg.Solver.from_lp(lp, precision=precision) as s:
        assert s.solve(eps, 500_000) == pdhg.PDHG_CONVERGED
        xp, y, zp, mu = s.warmstart_point()
        sc = s.scaling()
    A, b, c = _scaled_lp(lp, sc)
    assert np.all(xp > 0) and np.all(zp > 0) and mu >= 1e-6
    rw = H.warm_start(A, b, c, np.asarray(xp), np.asarray(y), np.asarray(zp))
    rc = H.mehrotra(A, b, c)
    ref = _highs(A, b, c)
    assert rw["status"] == "optimal" and rc["status"] == "optimal"
    assert rw["bumps"] == 0 and rw["first_step"] >= 1e-6
    assert abs(float(c @ rw["x"]) - ref) <= 1e-7 * (1 + abs(ref))
    assert H._converged(A, b, c, rw["x"], rw["y"], rw["z"], 1e-8)
    assert rw["iters"] < rc["iters"], (rw["iters"], rc["iters"])


def test_degenerate_gpu_start_drives_the_bump_loop():
    """Algorithm 1 on the GPU with delta_max = 0 (no centering move) and
    alpha_min = 1e-12, with the complementary pairs reversed (x' and z'
    swapped: every entry the PDHG point puts at zero is large and vice
    versa): the first interior-point step from it is far below 1e-6, so the
    bump loop multiplies alpha_min by 10 until the first step reaches 1e-6,
    and the method then reaches the HiGHS optimum."""
    lp = lpgen.planted_lp(200, 500, seed=0)
    with pdhg.Solver.from_lp(lp) as s:
        assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
        xp, y, zp, _ = s.warmstart_point(mu_min=1e-12, delta_max=0.0, alpha_min=1e-12)
        sc = s.scaling()
    A, b, c = _scaled_lp(lp, sc)
    xp, y, zp = np.asarray(xp), np.asarray(y), np.asarray(zp)
    # delta_max = 0: each entry is only lifted to alpha_min
    assert np.all(xp >= 1e-12) and np.all(zp >= 1e-12)
    a = 1e-12
    r0 = H.mehrotra(A, b, c, start=(np.maximum(zp, a), y, np.maximum(xp, a)), max_iter=1)
    assert r0["first_step"] < 1e-6
    r = H.warm_start(A, b, c, zp, y, xp, alpha_min=a, min_step=1e-6)
    assert r["bumps"] >= 1 and r["alpha_min"] == pytest.approx(a * 10.0 ** r["bumps"])
    assert r["status"] == "optimal" and r["first_step"] >= 1e-6
    ref = _highs(A, b, c)
    assert abs(float(c @ r["x"]) - ref) <= 1e-7 * (1 + abs(ref))
