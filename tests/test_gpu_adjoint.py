"""Differentiation through x*(b, c): the GPU active-set polish and adjoint
against a dense least-squares reference, central finite differences with
independent HiGHS re-solves, and the autograd Function.  Tolerance: 1e-4
relative (the gradient target), 1e-6 against the dense reference."""
import dataclasses

import numpy as np
import pytest

from oracle import adjoint_ref as R
from oracle import pdhg_oracle as O
from paper_2603_03150_gb300 import build as B
from paper_2603_03150_gb300 import lpgen
from paper_2603_03150_gb300 import pdhg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(1e-300, np.linalg.norm(b)))


def highs_x(lp, b, c):
    from scipy.optimize import linprog
    A = O.as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    r = linprog(c, A_eq=A, b_eq=b, bounds=(0, None), method="highs-ds",
                options={"primal_feasibility_tolerance": 1e-10,
                         "dual_feasibility_tolerance": 1e-10})
    assert r.status == 0
    return r.x


def solve_batch(lps, **kw):
    s = pdhg.BatchSolver(lps, **kw)
    assert s.solve(1e-4, 200_000) == pdhg.PDHG_CONVERGED
    return s


def test_polish_recovers_planted_optimum_and_support():
    lps = [lpgen.planted_lp(200, 500, 5, seed=s) for s in range(4)]
    with solve_batch(lps) as s:
        p = s.polish()
    xs = s.split(p["x"], "n")
    for i, lp in enumerate(lps):
        assert p["active"][i] == np.count_nonzero(lp.x_star)
        assert np.array_equal(xs[i] > 0, lp.x_star > 0)
        assert rel(xs[i], lp.x_star) < 1e-10


def test_adjoint_matches_dense_reference_and_zero_grad_c():
    lps = [lpgen.planted_lp(200, 500, 5, seed=s) for s in range(3)]
    tg = [np.random.default_rng(100 + i).uniform(0, 1, lp.n) for i, lp in enumerate(lps)]
    with solve_batch(lps) as s:
        p = s.polish()
        g = 2.0 * (p["x"] - np.concatenate(tg))
        a = s.adjoint(g)
    gbs = s.split(a["grad_b"], "m")
    assert np.all(a["grad_c"] == 0.0)
    for i, lp in enumerate(lps):
        r = O.solve(lp, 1e-4, 200_000)
        Bset = R.active_set(r)
        assert np.array_equal(Bset, s.split(p["x"], "n")[i] > 0)
        A = lp.dense()
        xr = R.polish(A, lp.b, Bset)
        gr = R.grad_b(A, Bset, 2.0 * (xr - tg[i]))
        assert rel(gbs[i], gr) < 1e-6, i


def _loss(lp, b, c, t):
    x = highs_x(lp, b, c)
    return float(np.sum((x - t) ** 2))


def test_adjoint_matches_central_fd_along_range_directions():
    """db = A_B v keeps the LP feasible on B, so x*(b) is linear along db and L
    quadratic: the central difference is exact up to the re-solve accuracy."""
    lp = lpgen.planted_lp(200, 500, 5, seed=7)
    t = np.random.default_rng(5).uniform(0, 1, lp.n)
    with solve_batch([lp]) as s:
        p = s.polish()
        a = s.adjoint(2.0 * (p["x"] - t))
    Bset = p["x"] > 0
    A = lp.dense()
    rng = np.random.default_rng(11)
    h = 1e-3
    for _ in range(2):
        v = np.zeros(lp.n)
        v[Bset] = rng.standard_normal(int(Bset.sum()))
        db = A @ v
        db /= np.linalg.norm(db)
        fd = (_loss(lp, lp.b + h * db, lp.c, t) - _loss(lp, lp.b - h * db, lp.c, t)) / (2 * h)
        an = float(a["grad_b"] @ db)
        assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-3 * np.linalg.norm(a["grad_b"]))


def test_grad_c_zero_by_fd():
    lp = lpgen.planted_lp(200, 500, 5, seed=8)
    t = np.random.default_rng(6).uniform(0, 1, lp.n)
    h = 1e-3
    for j in [0, 7, 123]:
        e = np.zeros(lp.n)
        e[j] = 1.0
        fd = (_loss(lp, lp.b, lp.c + h * e, t) - _loss(lp, lp.b, lp.c - h * e, t)) / (2 * h)
        assert abs(fd) < 1e-6


def test_vertex_variant_per_coordinate_fd():
    """Exactly m positive entries: A_B is square and every coordinate of b
    has a two-sided derivative."""
    lp = lpgen.planted_lp(60, 150, 5, seed=3, n_pos=60)
    t = np.random.default_rng(9).uniform(0, 1, lp.n)
    with solve_batch([lp]) as s:
        p = s.polish()
        a = s.adjoint(2.0 * (p["x"] - t))
    assert p["active"][0] == 60
    h = 1e-4
    gb = a["grad_b"]
    for i in range(0, 60, 7):
        e = np.zeros(lp.m)
        e[i] = 1.0
        fd = (_loss(lp, lp.b + h * e, lp.c, t) - _loss(lp, lp.b - h * e, lp.c, t)) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-4 * max(abs(gb[i]), 1e-3 * np.linalg.norm(gb)), i


def test_autograd_function_backward():
    import torch
    from paper_2603_03150_gb300.autograd import lp_solution
    lps = [lpgen.planted_lp(200, 500, 5, seed=s) for s in range(2)]
    st = dict(m=np.array([lp.m for lp in lps], np.int32), n=np.array([lp.n for lp in lps], np.int32),
              row_ptr=np.concatenate([lp.row_ptr for lp in lps]),
              col=np.concatenate([lp.col for lp in lps]), val=np.concatenate([lp.val for lp in lps]))
    b = torch.tensor(np.concatenate([lp.b for lp in lps]), requires_grad=True)
    c = torch.tensor(np.concatenate([lp.c for lp in lps]), requires_grad=True)
    t = torch.tensor(np.random.default_rng(1).uniform(0, 1, sum(lp.n for lp in lps)))
    x = lp_solution(b, c, st)
    loss = ((x - t) ** 2).sum()
    loss.backward()
    assert torch.all(c.grad == 0)
    off = 0
    for i, lp in enumerate(lps):
        xi = x.detach().numpy()[off:off + lp.n]
        Bset = xi > 0
        A = lp.dense()
        gr = R.grad_b(A, Bset, 2.0 * (xi - t.numpy()[off:off + lp.n]))
        mo = sum(l.m for l in lps[:i])
        assert rel(b.grad.numpy()[mo:mo + lp.m], gr) < 1e-6
        off += lp.n


def test_adjoint_full_size_batch_sampled():
    """64 LPs of 2000 x 5000 (5 nnz per column); sampled LPs against the dense
    reference."""
    lps, targets = lpgen.adjoint_batch(64, 2000, 5000)
    with solve_batch(lps, precision="fp64") as s:
        p = s.polish()
        g = 2.0 * (p["x"] - np.concatenate(targets))
        a = s.adjoint(g)
    gbs, xs = s.split(a["grad_b"], "m"), s.split(p["x"], "n")
    assert np.all(p["active"] == 1500)
    for i in [0, 17, 63]:
        lp = lps[i]
        Bset = lp.x_star > 0
        assert np.array_equal(xs[i] > 0, Bset)
        A = lp.dense()
        gr = R.grad_b(A, Bset, 2.0 * (R.polish(A, lp.b, Bset) - targets[i]))
        assert rel(gbs[i], gr) < 1e-4, i


def test_autograd_on_device_reuses_one_context():
    """A BatchLP keeps A's context across calls: each forward sends new b, c
    (pdhg_batch_set_rhs) and everything stays on the GPU.  Two calls with
    different b give the solutions and gradients of fresh contexts (and of
    the dense reference); a backward after the BatchLP solved another b is
    refused."""
    import torch
    from paper_2603_03150_gb300.autograd import BatchLP, lp_solution
    lps = [lpgen.planted_lp(200, 500, 5, seed=s) for s in range(3)]
    st = dict(m=np.array([lp.m for lp in lps], np.int32), n=np.array([lp.n for lp in lps], np.int32),
              row_ptr=np.concatenate([lp.row_ptr for lp in lps]),
              col=np.concatenate([lp.col for lp in lps]), val=np.concatenate([lp.val for lp in lps]))
    rng = np.random.default_rng(4)
    b0 = np.concatenate([lp.b for lp in lps])
    c0 = np.concatenate([lp.c for lp in lps])
    # a second b inside range(A_B) of each LP: b + A_B v keeps the active set
    b1 = np.concatenate([lp.b + lp.dense()[:, lp.x_star > 0] @ rng.uniform(-0.1, 0.1, int((lp.x_star > 0).sum()))
                         for lp in lps])
    t = torch.tensor(rng.uniform(0, 1, c0.size), device="cuda")
    blp = BatchLP(st, device="cuda")
    for bv in (b0, b1):
        b = torch.tensor(bv, device="cuda", requires_grad=True)
        c = torch.tensor(c0, device="cuda", requires_grad=True)
        x = lp_solution(b, c, blp)
        assert x.is_cuda
        ((x - t) ** 2).sum().backward()
        assert b.grad.is_cuda and torch.all(c.grad == 0)
        mo = np.concatenate([[0], np.cumsum([lp.m for lp in lps])])
        with solve_batch([dataclasses.replace(lp, b=bv[mo[i]:mo[i + 1]]) for i, lp in enumerate(lps)],
                         precision="fp64") as s:
            p = s.polish()
        assert rel(x.detach().cpu().numpy(), np.asarray(p["x"])) < 1e-8
        off, mo = 0, 0
        for lp in lps:
            xi = x.detach().cpu().numpy()[off:off + lp.n]
            gr = R.grad_b(lp.dense(), xi > 0, 2.0 * (xi - t.cpu().numpy()[off:off + lp.n]))
            assert rel(b.grad.cpu().numpy()[mo:mo + lp.m], gr) < 1e-6
            off += lp.n
            mo += lp.m
    # two forwards on one BatchLP, then the first one's backward: refused
    b = torch.tensor(b0, device="cuda", requires_grad=True)
    c = torch.tensor(c0, device="cuda")
    x1 = lp_solution(b, c, blp)
    lp_solution(torch.tensor(b1, device="cuda"), c, blp)
    with pytest.raises(RuntimeError):
        x1.sum().backward()
    blp.close()
