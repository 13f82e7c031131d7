"""pdhg_centered_point_noalloc: Algorithm 1 on caller-provided device vectors
with its scratch in a static device array (for callers that cannot allocate
device memory, e.g. during stream capture or inside a fixed memory pool).

It must give what pdhg_warmstart_point gives for the same scaled (x, z), on
two calls in a row (the shared scratch keeps the previous call's contents).
Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

from paper_2603_03150_gb300 import build as B
from paper_2603_03150_gb300 import lpgen
from paper_2603_03150_gb300 import pdhg

pytestmark = pytest.mark.gpu


def rel_inf(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


@pytest.mark.parametrize("m,n", [(200, 500), (4000, 10000)])
def test_noalloc_matches_warmstart_point_on_two_calls(m, n):
    import torch
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
    x_t = torch.tensor(xs, dtype=torch.float64, device="cuda")
    z_t = torch.tensor(zs, dtype=torch.float64, device="cuda")
    for _ in range(2):
        xo = torch.full_like(x_t, np.nan)
        zo = torch.full_like(z_t, np.nan)
        mo = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        pdhg.centered_point_noalloc(x_t, z_t, xo, zo, mo)
        torch.cuda.synchronize()
        assert abs(mo.item() - mu) <= 1e-12 * mu
        assert rel_inf(xo.cpu().numpy(), xw) < 1e-9
        assert rel_inf(zo.cpu().numpy(), zw) < 1e-9


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
