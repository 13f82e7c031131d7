"""pdhg_centered_point_noalloc: the start point of Algorithm 1 on
caller-provided device vectors, with its scratch in a static device array,
for callers that cannot allocate device memory (an interior-point solver
that owns a fixed memory pool, a thread that must not take the allocator's
locks).

It must give what pdhg_warmstart_point gives for the same scaled (x, z), on
two calls in a row (the shared scratch keeps the previous call's contents);
it must agree with the oracle's Algorithm 1 and the hand-worked cases; and
it must accept n up to its scratch limit, 8,388,608 entries (all 4096
partial-sum slots).  Kept in a file of its own that pytest collects last."""
import json
import os

import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2603_03150_gb300 import build as B
from paper_2603_03150_gb300 import lpgen
from paper_2603_03150_gb300 import pdhg

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rel_inf(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def _noalloc(x, z, mu_min=1e-6, delta_max=1e-4, alpha_min=1e-6):
    import torch
    x_t = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")
    z_t = torch.as_tensor(np.ascontiguousarray(z, dtype=np.float64), device="cuda")
    xo = torch.full_like(x_t, np.nan)
    zo = torch.full_like(z_t, np.nan)
    mo = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    pdhg.centered_point_noalloc(x_t, z_t, xo, zo, mo, mu_min=mu_min, delta_max=delta_max,
                                alpha_min=alpha_min)
    torch.cuda.synchronize()
    return xo.cpu().numpy(), zo.cpu().numpy(), mo.item()


@pytest.mark.parametrize("m,n", [(200, 500), (4000, 10000)])
def test_noalloc_matches_warmstart_point_on_two_calls(m, n):
    B.build()
    lp = lpgen.planted_lp(m, n, seed=1)
    with pdhg.Solver.from_lp(lp) as s:
        s.solve(1e-4, 200_000)
        info = s.info(violation=False)
        st = s.state()
        g = s.get()
        sc = s.scaling()
        xw, yw, zw, mu = s.warmstart_point()
    # the scaled iterate Algorithm 1 starts from: x~ and z~ = D_c z
    xs = st["x_avg"] if info["chosen_average"] else st["x"]
    zs = g["z"] * sc["D_c"]
    for _ in range(2):
        xo, zo, mo = _noalloc(xs, zs)
        assert abs(mo - mu) <= 1e-12 * mu
        assert rel_inf(xo, xw) < 1e-9
        assert rel_inf(zo, zw) < 1e-9


def test_noalloc_hand_cases_and_oracle():
    """Each hand-worked Algorithm 1 case (both branches, both clamps, the
    tie, the mu_min floor, the unclamped mu) on device, then the oracle on a
    random vector."""
    B.build()
    with open(os.path.join(GOLD, "alg1_cases.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        xo, zo, mo = _noalloc(c["x"], c["z"], c["mu_min"], c["delta_max"], c["alpha_min"])
        # the oracle pins' tolerances on the same cases
        assert abs(mo - c["mu"]) <= 1e-15 * max(1.0, c["mu"]), c["name"]
        np.testing.assert_allclose(xo, c["x_out"], rtol=1e-12, err_msg=c["name"])
        np.testing.assert_allclose(zo, c["z_out"], rtol=1e-12, err_msg=c["name"])
    rng = np.random.default_rng(7)
    x = np.where(rng.random(5000) < 0.3, rng.uniform(0, 2, 5000), 0.0)
    z = np.where(x > 0, 0.0, rng.uniform(0, 2, 5000)) + rng.uniform(0, 1e-4, 5000)
    ox, oz, omu = O.centered_start_point(x, z, 1e-6, 1e-2, 1e-6)
    xo, zo, mo = _noalloc(x, z, 1e-6, 1e-2, 1e-6)
    assert abs(mo - omu) <= 1e-12 * omu
    assert rel_inf(xo, ox) < 1e-13 and rel_inf(zo, oz) < 1e-13


def test_noalloc_at_its_scratch_limit_then_smaller():
    """n = 8,388,608 fills all 4096 partial-sum slots; a smaller call after
    it reads only the slots it writes (two calls of each size)."""
    B.build()
    rng = np.random.default_rng(11)
    for n in (8_388_608, 8_388_608, 3_000_001, 3_000_001):
        x = np.where(rng.random(n) < 0.3, rng.uniform(0, 2, n), 0.0)
        z = rng.uniform(0, 1e-3, n)
        ox, oz, omu = O.centered_start_point(x, z)
        xo, zo, mo = _noalloc(x, z)
        # mu sums 8M products in another order than numpy's pairwise sum
        assert abs(mo - omu) <= 1e-11 * omu, n
        assert rel_inf(xo, ox) < 1e-9 and rel_inf(zo, oz) < 1e-9, n


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    B.build()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pdhg.PDHGError) as e:
        pdhg._check(pdhg.lib().pdhg_centered_point_noalloc(
            8_388_609, pdhg._ptr(x), pdhg._ptr(x), 1e-6, 1e-4, 1e-6, pdhg._ptr(x), pdhg._ptr(x),
            None, None))
    assert e.value.status == pdhg.PDHG_INVALID_ARG
    assert "outside" in str(e.value)
