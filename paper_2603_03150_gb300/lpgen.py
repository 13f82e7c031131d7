"""Seeded synthetic LP generators in standard form  min c^T x  s.t.  Ax = b, x >= 0.

This module only builds inputs. It holds none of the solver's arithmetic and is
shared, as plain data, by the CPU oracle (``oracle/``) and the CUDA path.

The LP pair and the optimality conditions the planted instances satisfy are
those of Section 2 ("Background"): primal  min c^T x, Ax=b, x>=0;  dual
max b^T y, A^T y + z = c, z >= 0.  A planted instance fixes a complementary
pair (x*, z*) with x*_j z*_j = 0, x*, z* >= 0, and a free y*, then sets
b = A x* and c = A^T y* + z*, so (x*, y*, z*) is optimal by construction and
c^T x* = b^T y* exactly (up to the rounding of the two products).

Workloads (the paper measures on the Mittelmann LP set and a private broad
set, Section 4.2; neither is available, and these synthetic shapes stand in):

* ``planted_lp(200, 500)``  -- small planted LP, 5 nnz per column.
* ``powerlaw_lp()``         -- 200k x 1M, 5M nnz, power-law row lengths
                               (exponent 2.1, 4..20000), 1% rows scaled 1e3.
* ``transportation_lp()``   -- balanced 2000 x 2000 transportation problem,
                               n = 4M arcs, m = 4000 rows.
* ``planted_batch()``       -- 512 planted LPs, m log-uniform in [50, 5000].
* ``adjoint_batch()``       -- 64 planted LPs 2000 x 5000 with targets.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class LP:
    """A standard-form LP in CSR (row-major, columns ascending within a row)."""

    m: int
    n: int
    row_ptr: np.ndarray  # int32 [m+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]
    b: np.ndarray        # float64 [m]
    c: np.ndarray        # float64 [n]
    x_star: Optional[np.ndarray] = None
    y_star: Optional[np.ndarray] = None
    z_star: Optional[np.ndarray] = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        A = np.zeros((self.m, self.n))
        for i in range(self.m):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            A[i, self.col[s:e]] = self.val[s:e]
        return A


def _coo_to_csr(m: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return (row_ptr.astype(np.int32), cols.astype(np.int32),
            np.ascontiguousarray(vals, dtype=np.float64))


def _csr_matvec(m, row_ptr, col, val, v):
    """y = A v for building b (input construction only)."""
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    out = np.zeros(m)
    np.add.at(out, rows, val * v[col])
    return out


def _csr_rmatvec(n, m, row_ptr, col, val, w):
    """A^T w for building c (input construction only)."""
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    out = np.zeros(n)
    np.add.at(out, col, val * w[rows])
    return out


def _plant(rng, m, n, row_ptr, col, val, n_pos):
    """Complementary x*, z* and free y*; b = A x*, c = A^T y* + z*."""
    pos = rng.choice(n, size=n_pos, replace=False)
    x = np.zeros(n)
    x[pos] = rng.uniform(0.5, 2.0, size=n_pos)
    z = rng.uniform(0.5, 2.0, size=n)
    z[pos] = 0.0
    y = rng.standard_normal(m)
    b = _csr_matvec(m, row_ptr, col, val, x)
    c = _csr_rmatvec(n, m, row_ptr, col, val, y) + z
    return x, y, z, b, c


def planted_lp(m: int = 200, n: int = 500, nnz_per_col: int = 5, seed: int = 0,
               frac_pos: float = 0.3, n_pos: Optional[int] = None) -> LP:
    """Planted-optimum LP: each column has ``nnz_per_col`` entries at distinct
    uniformly random rows, values N(0,1); x* > 0 on exactly
    round(frac_pos*n) entries (U[0.5,2]), z* ~ U[0.5,2] on the rest,
    y* ~ N(0,1).  ``n_pos=m`` gives the vertex variant (square basis)."""
    rng = np.random.default_rng(seed)
    k = min(nnz_per_col, m)
    # distinct rows per column: draw, then re-draw repeats until none remain
    R = rng.integers(0, m, size=(n, k))
    for _ in range(1000):
        R.sort(axis=1)
        dup = np.zeros_like(R, dtype=bool)
        dup[:, 1:] = R[:, 1:] == R[:, :-1]
        if not dup.any():
            break
        R[dup] = rng.integers(0, m, size=int(dup.sum()))
    rows = R.reshape(-1)
    cols = np.repeat(np.arange(n), k)
    vals = rng.standard_normal(n * k)
    row_ptr, col, val = _coo_to_csr(m, rows, cols, vals)
    if n_pos is None:
        n_pos = int(round(frac_pos * n))
    x, y, z, b, c = _plant(rng, m, n, row_ptr, col, val, n_pos)
    return LP(m, n, row_ptr, col, val, b, c, x, y, z,
              name=f"planted_m{m}_n{n}_s{seed}", meta={"seed": seed, "n_pos": n_pos})


def powerlaw_lp(m: int = 200_000, n: int = 1_000_000, nnz: int = 5_000_000,
                exponent: float = 2.1, k_min: int = 4, k_max: int = 20_000,
                frac_scaled_rows: float = 0.01, row_scale: float = 1e3,
                seed: int = 0) -> LP:
    """Large planted LP with heavy-tailed row lengths.

    Row lengths follow the discrete power law P(k) ~ k^-exponent on
    [k_min, k_max]; random rows are then adjusted so the total is exactly
    ``nnz`` and the longest row is exactly ``k_max``.  Columns are uniform
    without replacement within a row; every column is given at least one
    entry by reassignment.  Values N(0,1); ``frac_scaled_rows`` of the rows
    are multiplied by ``row_scale`` before the optimum is planted (30%)."""
    rng = np.random.default_rng(seed)
    ks = np.arange(k_min, k_max + 1)
    p = ks.astype(np.float64) ** (-exponent)
    p /= p.sum()
    lens = rng.choice(ks, size=m, p=p).astype(np.int64)
    # force the longest row, then fix the total at random rows
    lens[int(np.argmax(lens))] = k_max
    top = int(np.argmax(lens))
    for _ in range(100):
        d = nnz - int(lens.sum())
        if d == 0:
            break
        idx = rng.integers(0, m, size=abs(d))
        idx = idx[idx != top]
        add = np.bincount(idx, minlength=m)
        lens = lens + add if d > 0 else lens - add
        lens = np.clip(lens, k_min, k_max)
        lens[top] = k_max
    assert int(lens.sum()) == nnz and int(lens.max()) == k_max
    rows = np.repeat(np.arange(m, dtype=np.int64), lens)
    cols = rng.integers(0, n, size=nnz, dtype=np.int64)
    # re-draw duplicates within a row until every row's columns are distinct
    for _ in range(100):
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        sk = key[order]
        dup = np.zeros(nnz, dtype=bool)
        dup[order[1:][sk[1:] == sk[:-1]]] = True
        if not dup.any():
            break
        cols[dup] = rng.integers(0, n, size=int(dup.sum()))
    # every column gets >= 1 entry: move entries out of columns with count >= 2
    for _ in range(1000):
        cnt = np.bincount(cols, minlength=n)
        empty = np.flatnonzero(cnt == 0)
        if empty.size == 0:
            break
        donors = np.flatnonzero(cnt[cols] >= 2)
        donors = rng.permutation(donors)
        _, first = np.unique(cols[donors], return_index=True)
        donors = donors[np.sort(first)][: empty.size]
        cols[donors] = empty[: donors.size]
    assert np.bincount(cols, minlength=n).min() >= 1
    vals = rng.standard_normal(nnz)
    scaled = rng.choice(m, size=int(round(frac_scaled_rows * m)), replace=False)
    row_factor = np.ones(m)
    row_factor[scaled] = row_scale
    vals *= row_factor[rows]
    row_ptr, col, val = _coo_to_csr(m, rows, cols, vals)
    x, y, z, b, c = _plant(rng, m, n, row_ptr, col, val, int(round(0.3 * n)))
    return LP(m, n, row_ptr, col, val, b, c, x, y, z,
              name=f"powerlaw_m{m}_n{n}_nnz{nnz}_s{seed}",
              meta={"seed": seed, "scaled_rows": scaled})


def transportation_lp(n_supply: int = 2000, n_demand: int = 2000, seed: int = 0) -> LP:
    """Balanced transportation problem in equality form.

    Arc (i, j) is column i*n_demand + j with a 1.0 in supply row i and in
    demand row n_supply + j.  Supplies and demands ~U[1,100], demands
    rescaled to the supply total; costs ~U[1,100].  No planted optimum: the
    supply and demand rows sum to the same vector, so A has rank m-1."""
    rng = np.random.default_rng(seed)
    m = n_supply + n_demand
    n = n_supply * n_demand
    s = rng.uniform(1.0, 100.0, size=n_supply)
    d = rng.uniform(1.0, 100.0, size=n_demand)
    d *= s.sum() / d.sum()
    cost = rng.uniform(1.0, 100.0, size=n)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:n_supply + 1] = np.arange(1, n_supply + 1) * n_demand
    row_ptr[n_supply + 1:] = n_supply * n_demand + np.arange(1, n_demand + 1) * n_supply
    sup_cols = np.arange(n, dtype=np.int64)
    dem_cols = (np.arange(n_supply, dtype=np.int64)[None, :] * n_demand
                + np.arange(n_demand, dtype=np.int64)[:, None]).reshape(-1)
    col = np.concatenate([sup_cols, dem_cols]).astype(np.int32)
    val = np.ones(2 * n)
    b = np.concatenate([s, d])
    return LP(m, n, row_ptr.astype(np.int32), col, val, b, cost,
              name=f"transport_{n_supply}x{n_demand}_s{seed}",
              meta={"seed": seed, "n_supply": n_supply, "n_demand": n_demand})


def batch_sizes(count: int = 512, m_lo: int = 50, m_hi: int = 5000, seed: int = 0):
    """m ~ floor(exp(U[ln m_lo, ln m_hi])), n = floor(2.5 m)."""
    rng = np.random.default_rng(seed)
    ms = np.floor(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), size=count))).astype(int)
    ns = np.floor(2.5 * ms).astype(int)
    return ms, ns


def planted_batch(count: int = 512, m_lo: int = 50, m_hi: int = 5000,
                  size_seed: int = 0) -> List[LP]:
    """Batch of uneven planted LPs; LP i is ``planted_lp`` with seed i."""
    ms, ns = batch_sizes(count, m_lo, m_hi, size_seed)
    return [planted_lp(int(ms[i]), int(ns[i]), 5, seed=i) for i in range(count)]


def adjoint_batch(count: int = 64, m: int = 2000, n: int = 5000, vertex: bool = False):
    """LPs with seeds 0..count-1 and targets x_target ~ U[0,1] (seed 1000+i).
    ``vertex=True`` plants exactly m positive entries (square basis)."""
    lps, targets = [], []
    for i in range(count):
        lps.append(planted_lp(m, n, 5, seed=i, n_pos=(m if vertex else None)))
        targets.append(np.random.default_rng(1000 + i).uniform(0.0, 1.0, size=n))
    return lps, targets


def concat_batch(lps: List[LP]):
    """Block-diagonal concatenation of a batch into one CSR with offsets."""
    m_off = np.zeros(len(lps) + 1, dtype=np.int64)
    n_off = np.zeros(len(lps) + 1, dtype=np.int64)
    z_off = np.zeros(len(lps) + 1, dtype=np.int64)
    for i, lp in enumerate(lps):
        m_off[i + 1] = m_off[i] + lp.m
        n_off[i + 1] = n_off[i] + lp.n
        z_off[i + 1] = z_off[i] + lp.nnz
    row_ptr = np.zeros(m_off[-1] + 1, dtype=np.int64)
    col = np.empty(z_off[-1], dtype=np.int32)
    val = np.empty(z_off[-1])
    for i, lp in enumerate(lps):
        row_ptr[m_off[i] + 1:m_off[i + 1] + 1] = lp.row_ptr[1:].astype(np.int64) + z_off[i]
        col[z_off[i]:z_off[i + 1]] = lp.col  # local column ids
        val[z_off[i]:z_off[i + 1]] = lp.val
    b = np.concatenate([lp.b for lp in lps])
    c = np.concatenate([lp.c for lp in lps])
    return dict(m_off=m_off, n_off=n_off, nnz_off=z_off, row_ptr=row_ptr.astype(np.int32),
                col=col, val=val, b=b, c=c)


def tiny_feasible_lp(m: int, n: int, seed: int) -> LP:
    """Small dense random LP with b = A x0 (x0 > 0) and c > 0: feasible and
    bounded below by 0, so its optimum sits at a vertex (for brute force)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    x0 = rng.uniform(0.5, 1.5, size=n)
    b = A @ x0
    c = rng.uniform(0.5, 2.0, size=n)
    rows, cols = np.nonzero(A)
    row_ptr, col, val = _coo_to_csr(m, rows, cols, A[rows, cols])
    return LP(m, n, row_ptr, col, val, b, c, name=f"tiny_m{m}_n{n}_s{seed}")
