"""Host-side consumer of the warm-start point: a minimal primal-dual
interior-point method and the bump loop of Algorithm 1 (Section 3.1).

The paper runs PDHG on the GPU and its interior-point solver on the CPU
(Section 4.1), warm-started from Algorithm 1's point (x', y, z') and raising
alpha_min tenfold for as long as the first interior-point step stays below a
minimum length (1e-6 in its tests).  This module is that CPU stage in its
plainest textbook form - Mehrotra's predictor-corrector on the normal
equations, dense Cholesky - so that the effect of the GPU's start point on
interior-point iteration counts can be measured (Section 4.6 reports the
warm/cold iteration ratio, the success rate and the count solved in <= 10
iterations).  It is not part of the PDHG path and never stands in for it.

LP: min c^T x  s.t.  A x = b, x >= 0  (dual: max b^T y, A^T y + z = c, z >= 0).
Termination: the Section 2 test with tolerance `tol`
    ||b - Ax|| <= tol (1 + ||b||), ||c - A^T y - z|| <= tol (1 + ||c||),
    |c^T x - b^T y| <= tol (1 + |c^T x| + |b^T y|).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def _max_step(v, dv):
    """Largest a in (0, 1] with v + a dv >= 0 (v > 0)."""
    neg = dv < 0
    if not np.any(neg):
        return 1.0
    return float(min(1.0, np.min(-v[neg] / dv[neg])))


def _converged(A, b, c, x, y, z, tol):
    rp = np.linalg.norm(b - A @ x)
    rd = np.linalg.norm(c - A.T @ y - z)
    px, dy = float(c @ x), float(b @ y)
    return (rp <= tol * (1 + np.linalg.norm(b)) and rd <= tol * (1 + np.linalg.norm(c)) and
            abs(px - dy) <= tol * (1 + abs(px) + abs(dy)))


class _Normal:
    """Cholesky of A D A^T (D = diag(d) > 0), with a small diagonal shift when
    A has dependent rows (the system is consistent; the shift only picks one
    solution)."""

    def __init__(self, A, d):
        M = (A.multiply(d) @ A.T) if sp.issparse(A) else (A * d) @ A.T
        M = M.toarray() if sp.issparse(M) else np.asarray(M)
        scale = max(1.0, float(np.max(np.abs(np.diag(M)))))
        for shift in (0.0, 1e-14, 1e-12, 1e-10, 1e-8):
            try:
                self.f = sla.cho_factor(M + shift * scale * np.eye(M.shape[0]), lower=True,
                                        check_finite=False)
                return
            except np.linalg.LinAlgError:
                continue
        raise np.linalg.LinAlgError("normal equations not positive definite")

    def solve(self, r):
        return sla.cho_solve(self.f, r, check_finite=False)


def cold_start(A, b, c):
    """Mehrotra's starting point: least-squares x and (y, z), shifted to be
    positive and balanced in complementarity."""
    M = A @ A.T
    M = M.toarray() if sp.issparse(M) else np.asarray(M)
    Mi = sla.pinvh(M)
    x = A.T @ (Mi @ b)
    y = Mi @ (A @ c)
    z = c - A.T @ y
    x = x + max(-1.5 * float(np.min(x)), 0.0)
    z = z + max(-1.5 * float(np.min(z)), 0.0)
    xz = float(x @ z)
    x = x + 0.5 * xz / max(float(np.sum(z)), 1e-300)
    z = z + 0.5 * xz / max(float(np.sum(x)), 1e-300)
    x = np.maximum(x, 1e-12)
    z = np.maximum(z, 1e-12)
    return x, y, z


def mehrotra(A, b, c, start=None, tol=1e-8, max_iter=200, step_frac=0.99,
             first_step_min=0.0):
    """Mehrotra predictor-corrector from `start` = (x, y, z) with x, z > 0 (or
    the cold start).  Returns a dict with status 'optimal', 'max_iter' or
    'stuck' (the first step was shorter than first_step_min; nothing taken),
    the iterations done, the point, and the first iteration's step length."""
    A = sp.csr_matrix(A) if sp.issparse(A) else np.asarray(A, dtype=float)
    b, c = np.asarray(b, float), np.asarray(c, float)
    if start is None:
        x, y, z = cold_start(A, b, c)
    else:
        x, y, z = (np.array(v, dtype=float, copy=True) for v in start)
        if np.any(x <= 0) or np.any(z <= 0):
            raise ValueError("start point must have x > 0 and z > 0")
    n = x.size
    first_step = None
    for k in range(max_iter + 1):
        if _converged(A, b, c, x, y, z, tol):
            return dict(status="optimal", iters=k, x=x, y=y, z=z, first_step=first_step)
        if k == max_iter:
            break
        rp = b - A @ x
        rd = c - A.T @ y - z
        mu = float(x @ z) / n
        d = x / z
        N = _Normal(A, d)

        def direction(rc):
            # A D A^T dy = rp + A(d rd - rc / z);  dx = d (A^T dy - rd) + rc / z;
            # dz = (rc - z dx) / x    (from A dx = rp, A^T dy + dz = rd, Z dx + X dz = rc)
            dy = N.solve(rp + A @ (d * rd - rc / z))
            dx = d * (A.T @ dy - rd) + rc / z
            dz = (rc - z * dx) / x
            return dx, dy, dz

        dxa, dya, dza = direction(-x * z)                      # predictor (affine)
        ap, ad = _max_step(x, dxa), _max_step(z, dza)
        mu_aff = float((x + ap * dxa) @ (z + ad * dza)) / n
        sigma = (mu_aff / mu) ** 3
        dx, dy, dz = direction(-x * z + sigma * mu - dxa * dza)  # corrector
        ap = min(1.0, step_frac * _max_step(x, dx))
        ad = min(1.0, step_frac * _max_step(z, dz))
        if k == 0:
            first_step = min(ap, ad)
            if first_step < first_step_min:
                return dict(status="stuck", iters=0, x=x, y=y, z=z, first_step=first_step)
        x = x + ap * dx
        y = y + ad * dy
        z = z + ad * dz
    return dict(status="max_iter", iters=max_iter, x=x, y=y, z=z, first_step=first_step)


def warm_start(A, b, c, x, y, z, alpha_min=1e-6, min_step=1e-6, max_bumps=12, **kw):
    """Algorithm 1's bump loop: start the interior-point method from
    (x', y, z'); while its first step is shorter than min_step, multiply
    alpha_min by 10 and raise every x'_j, z'_j to at least alpha_min.
    Returns the interior-point result with 'bumps' (how many times alpha_min
    grew) and 'alpha_min' (its final value)."""
    xw = np.maximum(np.asarray(x, float), alpha_min)
    zw = np.maximum(np.asarray(z, float), alpha_min)
    bumps = 0
    while True:
        r = mehrotra(A, b, c, start=(xw, y, zw), first_step_min=min_step, **kw)
        if r["status"] != "stuck" or bumps >= max_bumps:
            break
        alpha_min *= 10.0
        xw = np.maximum(xw, alpha_min)
        zw = np.maximum(zw, alpha_min)
        bumps += 1
    r["bumps"] = bumps
    r["alpha_min"] = alpha_min
    return r
