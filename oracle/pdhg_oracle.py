"""Plain FP64 CPU oracle for restarted PDHG and Algorithm 1 (centered start point).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  The CUDA path never
calls it, and it shares no code with that path: its sole common input is the
seeded generator module, which holds no solver arithmetic.

Everything here is deliberately slow and literal: one library sparse
mat-vec per product, no fusion, no cached products, all in float64.

What the paper fixes and what is a reading
------------------------------------------
The paper (Rothberg, "Hybridizing PDHG and Interior-Point Methods") fixes:

* the LP pair  min c^T x, Ax=b, x>=0  /  max b^T y, A^T y + z = c, z>=0
  (Section 2);
* the residuals r_P = b - Ax, r_D = c - A^T y - z and the three optimality
  conditions (Section 2);
* the termination test  ||r_P||_2 <= eps(1+||b||_2),
  ||r_D||_2 <= eps(1+||c||_2),  |c^T x - b^T y| <= eps(1+|c^T x|+|b^T y|)
  with eps = 1e-4 as the usual setting (Section 2);
* that scaling makes row and column norms roughly 1 and is essential for
  PDHG (Sections 2.1 and 3.1);
* the maximum-violation metric (Section 4.3);
* Algorithm 1's centered start point with mu_min = alpha_min = 1e-6, delta_max = 1e-4
  (Section 3.1).

It does NOT give the PDHG update, scaling method, step size, restart rule or
the definition of z for a PDHG iterate (it says only that its PDHG follows
cuPDLP+, Section 4.1).  This oracle takes the following readings, which the
CUDA path implements independently:

* z = max(0, c - A^T y), so r_D = min(0, c - A^T y).
* Scaling: 10 rounds of Ruiz (infinity norm), then one Pock-Chambolle step
  with alpha = 1; A~ = D_r A D_c, b~ = D_r b, c~ = D_c c.
* Step: eta = 0.95 / sigma_max(A~) by power iteration on A~^T A~;
  tau = eta / omega, sigma = eta * omega, omega_0 = ||c~|| / ||b~||.
* Iteration (scaled space, from x=0, y=0):
      x+ = max(0, x - tau (c~ - A~^T y))
      y+ = y + sigma (b~ - A~ (2 x+ - x))
  with uniform running averages since the last restart.
* Every F = 64 iterations: termination test (unscaled; current iterate
  first), then the KKT restart rule with beta = 0.2 / 0.8 / 0.36 and the
  primal-weight update with theta = 0.5.
These constants are a convention shared with the CUDA path: parity unpinned
against the paper for the restart constants, the omega rule and eta.
Optional primal-weight rule (``Options.omega_rule = "pid"``): PID control of
log omega at each restart, the reading of cuPDLP+'s primal-weight control
(``omega_update_pid``; gains kp = 0.99, ki = 0.01, kd = 0 by default).

Optional iteration (``Options.method = "halpern"``): the reflected Halpern
scheme of cuPDLP+, the solver Section 4.1 says its PDHG follows (the paper
prints none of its formulas; this is the reading).  With T the PDHG map
above, z = (x, y), anchor z0 = the last restart point and t the iterations
since it,
      z_{t+1} = lam_t ((1 + rho) T(z_t) - rho z_t) + (1 - lam_t) z0,
      lam_t = (t + 1) / (t + 2),  rho = Options.reflection in [0, 1];
the second candidate of the evaluation (where the averaged method uses the
running average) is T(z_t), the last PDHG output; evaluation, termination,
restart rule and omega update are unchanged.  Pinned by the Halpern bound
||z_t - T z_t||_M <= 2 ||z_0 - z*||_M / ((1 + rho)(t + 1)) for the PDHG
metric M (T is firmly nonexpansive in M, so (1+rho)T - rho I is
nonexpansive for rho <= 1), and by the rho = 1 first step being one plain
PDHG step.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

STATUS_CONVERGED = 0
STATUS_MAX_ITER = 1


@dataclass
class Options:
    eval_freq: int = 64
    ruiz_iters: int = 10
    pock_chambolle: bool = True
    eta_safety: float = 0.95
    power_max_iter: int = 200
    power_rel_tol: float = 1e-10
    beta_sufficient: float = 0.2
    beta_necessary: float = 0.8
    beta_artificial: float = 0.36
    theta: float = 0.5
    omega_update_min: float = 1e-10
    method: str = "averaged"   # or "halpern" (reflected Halpern, see the header)
    reflection: float = 1.0    # rho of the Halpern method, in [0, 1]
    omega_rule: str = "smooth"  # or "pid" (PID control of log omega, see omega_update_pid)
    pid_kp: float = 0.99
    pid_ki: float = 0.01
    pid_kd: float = 0.0
    step_rule: str = "constant"  # or "adaptive" (PDLP's adaptive step, see adaptive_step)


# ---------------------------------------------------------------------------
# a1: transpose
# ---------------------------------------------------------------------------
def transpose_csr(m: int, n: int, row_ptr, col, val):
    """CSR of A^T by a stable counting sort on the column index: row j of A^T
    lists the entries of column j of A in increasing row order."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))
    counts = np.bincount(col, minlength=n)
    row_ptr_t = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr_t[1:])
    order = np.argsort(col, kind="stable")
    return row_ptr_t, rows[order], val[order]


def as_csr(m: int, n: int, row_ptr, col, val) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(val, dtype=np.float64),
                          np.asarray(col, dtype=np.int64),
                          np.asarray(row_ptr, dtype=np.int64)), shape=(m, n))


# ---------------------------------------------------------------------------
# a2: diagonal preconditioning (Sections 2.1 and 3.1: row/column norms ~ 1)
# ---------------------------------------------------------------------------
def _row_absmax(M: sp.csr_matrix) -> np.ndarray:
    return np.asarray(abs(M).max(axis=1).todense()).ravel()


def _col_absmax(M: sp.csr_matrix) -> np.ndarray:
    return np.asarray(abs(M).max(axis=0).todense()).ravel()


def _row_abssum(M: sp.csr_matrix) -> np.ndarray:
    return np.asarray(abs(M).sum(axis=1)).ravel()


def _col_abssum(M: sp.csr_matrix) -> np.ndarray:
    return np.asarray(abs(M).sum(axis=0)).ravel()


def scale(A: sp.csr_matrix, ruiz_iters: int = 10, pock_chambolle: bool = True):
    """Ruiz equilibration in the infinity norm, then one Pock-Chambolle step
    (alpha = 1).  Returns D_r, D_c and A~ = D_r A D_c.  An empty row or
    column gets factor 1."""
    m, n = A.shape
    D_r = np.ones(m)
    D_c = np.ones(n)
    At = A.copy().astype(np.float64)
    for _ in range(ruiz_iters):
        r = np.sqrt(_row_absmax(At))
        s = np.sqrt(_col_absmax(At))
        r[r == 0.0] = 1.0
        s[s == 0.0] = 1.0
        D_r = D_r / r
        D_c = D_c / s
        At = sp.diags(1.0 / r) @ At @ sp.diags(1.0 / s)
    if pock_chambolle:
        r = np.sqrt(_row_abssum(At))
        s = np.sqrt(_col_abssum(At))
        r[r == 0.0] = 1.0
        s[s == 0.0] = 1.0
        D_r = D_r / r
        D_c = D_c / s
        At = sp.diags(1.0 / r) @ At @ sp.diags(1.0 / s)
    return D_r, D_c, sp.csr_matrix(At)


# ---------------------------------------------------------------------------
# a3: step size from the largest singular value
# ---------------------------------------------------------------------------
def power_iteration(At: sp.csr_matrix, max_iter: int = 200, rel_tol: float = 1e-10):
    """Power iteration on A~^T A~ from v = 1/sqrt(n).  After iteration k,
    lambda_k = v^T A~^T A~ v (v of unit norm) and v <- w/||w||; stop once
    |lambda_k - lambda_{k-1}| <= rel_tol * lambda_k or k = max_iter.
    Returns (sqrt(lambda), iterations)."""
    m, n = At.shape
    if At.nnz == 0 or n == 0:
        return 0.0, 0
    v = np.full(n, 1.0 / np.sqrt(n))
    lam_prev = None
    lam = 0.0
    k = 0
    for k in range(1, max_iter + 1):
        w = At.T @ (At @ v)
        lam = float(v @ w)
        nw = float(np.linalg.norm(w))
        if nw == 0.0:
            break
        v = w / nw
        if lam_prev is not None and abs(lam - lam_prev) <= rel_tol * lam:
            break
        lam_prev = lam
    return float(np.sqrt(max(lam, 0.0))), k


def initial_omega(b_t: np.ndarray, c_t: np.ndarray) -> float:
    nb, nc = float(np.linalg.norm(b_t)), float(np.linalg.norm(c_t))
    return nc / nb if (nb > 0.0 and nc > 0.0) else 1.0


# ---------------------------------------------------------------------------
# a4 + a5: one PDHG iteration
# ---------------------------------------------------------------------------
def pdhg_step(At: sp.csr_matrix, b_t, c_t, x, y, tau: float, sigma: float):
    """x+ = max(0, x - tau (c - A^T y));  y+ = y + sigma (b - A (2 x+ - x))."""
    x_new = np.maximum(0.0, x - tau * (c_t - At.T @ y))
    y_new = y + sigma * (b_t - At @ (2.0 * x_new - x))
    return x_new, y_new


# ---------------------------------------------------------------------------
# a7: residuals, gap, KKT error, termination (Section 2)
# ---------------------------------------------------------------------------
def residuals(A: sp.csr_matrix, b, c, x, y):
    """Section 2 residuals for (x, y, z) with z = max(0, c - A^T y)."""
    ATy = A.T @ y
    z = np.maximum(0.0, c - ATy)
    r_P = b - A @ x
    r_D = c - ATy - z
    return r_P, r_D, z


def termination_test(A, b, c, x, y, eps_rel: float):
    """The three Section 2 inequalities on the original (unscaled) model."""
    r_P, r_D, _ = residuals(A, b, c, x, y)
    pobj, dobj = float(c @ x), float(b @ y)
    nrp, nrd = float(np.linalg.norm(r_P)), float(np.linalg.norm(r_D))
    gap = abs(pobj - dobj)
    ok = (nrp <= eps_rel * (1.0 + np.linalg.norm(b))
          and nrd <= eps_rel * (1.0 + np.linalg.norm(c))
          and gap <= eps_rel * (1.0 + abs(pobj) + abs(dobj)))
    return bool(ok), nrp, nrd, gap


def kkt_error(At, b_t, c_t, x, y, omega: float) -> float:
    """Weighted KKT error in the scaled space used by the restart rule:
    sqrt(omega^2 ||b~ - A~x||^2 + ||min(0, c~ - A~^T y)||^2 / omega^2 + gap^2)."""
    rp = b_t - At @ x
    rd = np.minimum(0.0, c_t - At.T @ y)
    gap = float(c_t @ x) - float(b_t @ y)
    return float(np.sqrt(omega ** 2 * (rp @ rp) + (rd @ rd) / omega ** 2 + gap ** 2))


def max_violation(A, b, c, x, y) -> float:
    """Section 4.3: max(||r_P||_inf, ||r_D||_inf, x^T z / (1 + |c^T x|))."""
    r_P, r_D, z = residuals(A, b, c, x, y)
    ni = lambda v: float(np.max(np.abs(v))) if v.size else 0.0
    return max(ni(r_P), ni(r_D), float(x @ z) / (1.0 + abs(float(c @ x))))


# ---------------------------------------------------------------------------
# a8: the restart rule and the primal-weight update, as pure functions of the
# scalars of one evaluation (the loop below calls them; tests pin them by hand)
# ---------------------------------------------------------------------------
def restart_decision(kkt_cur: float, kkt_avg: float, kkt_last: float, kkt_prev: float,
                     t: int, k: int, opts: Optional["Options"] = None) -> dict:
    """One evaluation of the KKT restart rule (the cuPDLP reading of the
    paper's "PDHG following cuPDLP+", Section 4.1).

    The candidate is the lower of KKT(current) and KKT(average); a tie keeps
    the current iterate.  Three criteria, any of which restarts:
      r1 (sufficient):  KKT(cand) <= beta_suff * KKT(last restart point)
      r2 (necessary):   KKT(cand) <= beta_nec * KKT(last restart point) and
                        KKT(cand) >  KKT(candidate of the previous evaluation)
      r3 (artificial):  t >= beta_art * k  (t: iterations since the last
                        restart, k: iterations in all)
    Returns use_avg, k_cand, r1, r2, r3 and restart."""
    opts = opts or Options()
    use_avg = kkt_avg < kkt_cur
    k_cand = kkt_avg if use_avg else kkt_cur
    r1 = k_cand <= opts.beta_sufficient * kkt_last
    r2 = (k_cand <= opts.beta_necessary * kkt_last) and (k_cand > kkt_prev)
    r3 = t >= opts.beta_artificial * k
    return dict(use_avg=bool(use_avg), k_cand=float(k_cand), r1=bool(r1), r2=bool(r2),
                r3=bool(r3), restart=bool(r1 or r2 or r3))


def advance_restart_kkts(kkt_last: float, k_cand: float, restart: bool):
    """The two KKT references after an evaluation: the previous-candidate
    value always becomes this evaluation's candidate; the last-restart value
    becomes it only on a restart.  Returns (kkt_last, kkt_prev)."""
    return (k_cand if restart else kkt_last), k_cand


def omega_update(dx: float, dy: float, omega: float, theta: float = 0.5,
                 min_dist: float = 1e-10) -> float:
    """Primal weight at a restart: the geometric blend
    exp(theta log(dy / dx) + (1 - theta) log omega) of the new ratio of the
    dual to the primal distance moved since the last restart point and the
    old weight; unchanged unless both distances exceed min_dist."""
    if dx > min_dist and dy > min_dist:
        return float(np.exp(theta * np.log(dy / dx) + (1.0 - theta) * np.log(omega)))
    return float(omega)


def omega_update_pid(dx: float, dy: float, omega: float, integral: float, prev_error: float,
                     kp: float = 0.99, ki: float = 0.01, kd: float = 0.0,
                     min_dist: float = 1e-10):
    """Primal weight at a restart under PID control of log omega (the
    reading of cuPDLP+'s primal-weight control, the solver Section 4.1 says
    the paper's PDHG follows).  The error is the log of the ratio of the
    dual to the primal distance moved since the last restart point, against
    the current weight:
        e = log(dy / dx) - log(omega),   I <- I + e,
        log omega <- log omega + kp e + ki I + kd (e - e_prev).
    With ki = kd = 0 this is the smoothing of omega_update with theta = kp.
    Unchanged (weight, integral and previous error) unless both distances
    exceed min_dist.  Returns (omega, integral, error)."""
    if dx > min_dist and dy > min_dist:
        e = float(np.log(dy / dx) - np.log(omega))
        integral = integral + e
        lw = float(np.log(omega)) + kp * e + ki * integral + kd * (e - prev_error)
        return float(np.exp(lw)), float(integral), e
    return float(omega), float(integral), float(prev_error)


# ---------------------------------------------------------------------------
# the restarted loop (a4-a8)
# ---------------------------------------------------------------------------
@dataclass
class Setup:
    A: sp.csr_matrix
    b: np.ndarray
    c: np.ndarray
    D_r: np.ndarray
    D_c: np.ndarray
    At: sp.csr_matrix
    b_t: np.ndarray
    c_t: np.ndarray
    sigma_max: float
    power_iters: int
    eta: float
    omega0: float


def setup(lp, opts: Optional[Options] = None) -> Setup:
    opts = opts or Options()
    A = as_csr(lp.m, lp.n, lp.row_ptr, lp.col, lp.val)
    D_r, D_c, At = scale(A, opts.ruiz_iters, opts.pock_chambolle)
    b_t = D_r * np.asarray(lp.b, dtype=np.float64)
    c_t = D_c * np.asarray(lp.c, dtype=np.float64)
    smax, pit = power_iteration(At, opts.power_max_iter, opts.power_rel_tol)
    eta = opts.eta_safety / smax if smax > 0.0 else 1.0
    return Setup(A, np.asarray(lp.b, float), np.asarray(lp.c, float), D_r, D_c, At,
                 b_t, c_t, smax, pit, eta, initial_omega(b_t, c_t))


@dataclass
class State:
    """Scaled-space solver state (what a checkpoint holds)."""
    x: np.ndarray
    y: np.ndarray
    x_avg: np.ndarray
    y_avg: np.ndarray
    x_last: np.ndarray
    y_last: np.ndarray
    omega: float
    k: int = 0              # iterations done
    t: int = 0              # iterations since the last restart
    restarts: int = 0
    kkt_last: float = 0.0   # KKT error of the last restart point
    kkt_prev: float = 0.0   # KKT error of the previous evaluation's candidate
    pid_integral: float = 0.0  # omega_rule "pid": sum of the errors so far
    pid_prev: float = 0.0      # omega_rule "pid": the previous restart's error
    eta: float = 0.0           # step_rule "adaptive": the next attempt's step (0: setup's eta)
    eta_sum: float = 0.0       # step_rule "adaptive": accepted steps since the last restart
    step_rejects: int = 0      # step_rule "adaptive": rejected attempts so far


@dataclass
class Result:
    status: int
    iters: int
    restarts: int
    chosen: str             # "current" or "average"
    x: np.ndarray           # unscaled primal
    y: np.ndarray           # unscaled dual
    z: np.ndarray           # unscaled reduced costs
    r_P: float
    r_D: float
    gap: float
    max_violation: float
    x_scaled: np.ndarray
    y_scaled: np.ndarray
    state: State
    setup: Setup
    log: List[dict] = field(default_factory=list)


def initial_state(S: Setup) -> State:
    m, n = S.At.shape
    st = State(np.zeros(n), np.zeros(m), np.zeros(n), np.zeros(m), np.zeros(n),
               np.zeros(m), S.omega0)
    # the first restart point is (0, 0)
    st.kkt_last = kkt_error(S.At, S.b_t, S.c_t, st.x, st.y, st.omega)
    st.kkt_prev = st.kkt_last
    return st


def adaptive_step(dx, dy, A_dx, eta: float, omega: float, j: int) -> dict:
    """PDLP's adaptive step size (Applegate et al. 2021, "Practical large-scale
    linear programming using primal-dual hybrid gradient"), as read here.  An
    attempt with step eta moved the iterate by (dx, dy), and A_dx = A~ dx (A~
    applied to the move itself: a difference of the products A~ x+ and A~ x
    would lose the term's leading digits when the move is small).
    The largest step the move allows is
        eta_max = (omega ||dx||^2 + ||dy||^2 / omega) / (2 |dy^T A_dx|)
    (infinite when dy^T A_dx = 0); the attempt is accepted when eta <= eta_max,
    and the next attempt uses
        min((1 - (j + 1)^-0.3) eta_max, (1 + (j + 1)^-0.6) eta),
    j = step attempts so far including this one (so the first factor is
    positive from the first attempt)."""
    inter = abs(float(np.dot(dy, A_dx)))
    num = omega * float(np.dot(dx, dx)) + float(np.dot(dy, dy)) / omega
    eta_max = num / (2.0 * inter) if inter > 0.0 else float("inf")
    eta_next = min((1.0 - (j + 1.0) ** -0.3) * eta_max, (1.0 + (j + 1.0) ** -0.6) * eta)
    return dict(accept=eta <= eta_max, eta_max=eta_max, eta_next=eta_next)


def step_weighted_average(avg, x, eta: float, eta_sum_before: float):
    """Running average weighted by the accepted steps: after accepting x with
    step eta, avg = (sum of eta_i x_i) / (sum of eta_i) over the accepted
    iterates since the last restart (eta_sum_before = that sum before x)."""
    total = eta_sum_before + eta
    return avg + (x - avg) * (eta / total), total


def _unscale(S: Setup, xs, ys):
    return S.D_c * xs, S.D_r * ys


def solve(lp, eps_rel: float = 1e-4, max_iter: int = 100_000,
          opts: Optional[Options] = None, S: Optional[Setup] = None,
          state: Optional[State] = None) -> Result:
    """Restarted PDHG until the Section 2 test holds or max_iter iterations.

    Evaluation points are k % F == 0 and k == max_iter.  At each: the
    termination test on the current iterate, then on the average (Halpern
    method: on T of the previous iterate); at
    k == max_iter the loop stops; otherwise (k % F == 0) the restart rule:
    candidate = the lower KKT error (tie: current); restart if
      (i)   KKT(cand) <= beta_suff * KKT(last restart), or
      (ii)  KKT(cand) <= beta_nec * KKT(last restart) and
            KKT(cand) >  KKT(candidate at the previous evaluation), or
      (iii) t >= beta_art * k.
    On restart: omega <- exp(theta log(dy/dx) + (1-theta) log omega) when
    both distances to the last restart point exceed 1e-10; the iterate
    becomes the candidate and the averages restart."""
    opts = opts or Options()
    S = S or setup(lp, opts)
    st = state or initial_state(S)
    At, b_t, c_t, F = S.At, S.b_t, S.c_t, opts.eval_freq
    log: List[dict] = []
    status, chosen = STATUS_MAX_ITER, "current"
    xs_out, ys_out = st.x, st.y

    halpern = opts.method == "halpern"
    if opts.method not in ("averaged", "halpern") or not 0.0 <= opts.reflection <= 1.0:
        raise ValueError("method must be 'averaged' or 'halpern', reflection in [0, 1]")
    if opts.omega_rule not in ("smooth", "pid"):
        raise ValueError("omega_rule must be 'smooth' or 'pid'")
    adaptive = opts.step_rule == "adaptive"
    if opts.step_rule not in ("constant", "adaptive") or (adaptive and halpern):
        raise ValueError("step_rule must be 'constant' or 'adaptive' (averaged method only)")
    if adaptive and st.eta <= 0.0:
        st.eta = S.eta  # the first attempt takes the constant step
    while st.k < max_iter:
        eta = st.eta if adaptive else S.eta
        tau, sigma = eta / st.omega, eta * st.omega
        if adaptive:
            # one step attempt: accepted (the iterate and the step-weighted
            # averages move) or rejected (nothing moves); either way the next
            # attempt's step comes from adaptive_step and k, t count it
            xn, yn = pdhg_step(At, b_t, c_t, st.x, st.y, tau, sigma)
            dx = xn - st.x
            a = adaptive_step(dx, yn - st.y, At @ dx, eta, st.omega, st.k + 1)
            if a["accept"]:
                st.x, st.y = xn, yn
                st.x_avg, _ = step_weighted_average(st.x_avg, st.x, eta, st.eta_sum)
                st.y_avg, st.eta_sum = step_weighted_average(st.y_avg, st.y, eta, st.eta_sum)
            else:
                st.step_rejects += 1
            st.eta = a["eta_next"]
            st.k += 1
            st.t += 1
        elif halpern:
            # z <- lam ((1 + rho) T(z) - rho z) + (1 - lam) z0, z0 = last restart point
            xh, yh = pdhg_step(At, b_t, c_t, st.x, st.y, tau, sigma)
            lam, rho = (st.t + 1.0) / (st.t + 2.0), opts.reflection
            st.x = lam * ((1.0 + rho) * xh - rho * st.x) + (1.0 - lam) * st.x_last
            st.y = lam * ((1.0 + rho) * yh - rho * st.y) + (1.0 - lam) * st.y_last
            st.x_avg, st.y_avg = xh, yh  # second candidate: T(z)
            st.k += 1
            st.t += 1
        else:
            st.x, st.y = pdhg_step(At, b_t, c_t, st.x, st.y, tau, sigma)
            st.k += 1
            st.t += 1
            st.x_avg = st.x_avg + (st.x - st.x_avg) / st.t
            st.y_avg = st.y_avg + (st.y - st.y_avg) / st.t
        if st.k % F != 0 and st.k != max_iter:
            continue
        # termination, current iterate first (Section 2 inequalities)
        done = False
        for name, xs, ys in (("current", st.x, st.y), ("average", st.x_avg, st.y_avg)):
            x, y = _unscale(S, xs, ys)
            ok = termination_test(S.A, S.b, S.c, x, y, eps_rel)[0]
            if ok:
                done, chosen, xs_out, ys_out = True, name, xs, ys
                break
        if done:
            status = STATUS_CONVERGED
            break
        if st.k % F != 0 or st.k >= max_iter:
            break  # k == max_iter: stop without applying the restart rule
        k_cur = kkt_error(At, b_t, c_t, st.x, st.y, st.omega)
        k_avg = kkt_error(At, b_t, c_t, st.x_avg, st.y_avg, st.omega)
        d = restart_decision(k_cur, k_avg, st.kkt_last, st.kkt_prev, st.t, st.k, opts)
        use_avg, k_cand, restart = d["use_avg"], d["k_cand"], d["restart"]
        entry = dict(k=st.k, kkt_cur=k_cur, kkt_avg=k_avg, cand="average" if use_avg else "current",
                     restart=restart, r1=d["r1"], r2=d["r2"], r3=d["r3"], kkt_last=st.kkt_last,
                     kkt_prev=st.kkt_prev, omega=st.omega, t=st.t)
        st.kkt_last, st.kkt_prev = advance_restart_kkts(st.kkt_last, k_cand, restart)
        if restart:
            xc = st.x_avg if use_avg else st.x
            yc = st.y_avg if use_avg else st.y
            dx = float(np.linalg.norm(xc - st.x_last))
            dy = float(np.linalg.norm(yc - st.y_last))
            if opts.omega_rule == "pid":
                st.omega, st.pid_integral, st.pid_prev = omega_update_pid(
                    dx, dy, st.omega, st.pid_integral, st.pid_prev, opts.pid_kp, opts.pid_ki,
                    opts.pid_kd, opts.omega_update_min)
            else:
                st.omega = omega_update(dx, dy, st.omega, opts.theta, opts.omega_update_min)
            st.x, st.y = xc.copy(), yc.copy()
            st.x_last, st.y_last = xc.copy(), yc.copy()
            st.x_avg = np.zeros_like(st.x)
            st.y_avg = np.zeros_like(st.y)
            st.t = 0
            st.eta_sum = 0.0
            st.restarts += 1
            entry.update(dx=dx, dy=dy, omega_new=st.omega, pid_integral=st.pid_integral)
        log.append(entry)
        xs_out, ys_out = st.x, st.y

    if status == STATUS_MAX_ITER:
        xs_out, ys_out, chosen = st.x, st.y, "current"
    x, y = _unscale(S, xs_out, ys_out)
    _, nrp, nrd, gap = termination_test(S.A, S.b, S.c, x, y, eps_rel)
    _, _, z = residuals(S.A, S.b, S.c, x, y)
    return Result(status, st.k, st.restarts, chosen, x, y, z, nrp, nrd, gap,
                  max_violation(S.A, S.b, S.c, x, y), xs_out.copy(), ys_out.copy(), st, S, log)


# ---------------------------------------------------------------------------
# a9: Algorithm 1's centered start point (Section 3.1)
# ---------------------------------------------------------------------------
def centered_start_point(x, z, mu_min: float = 1e-6, delta_max: float = 1e-4,
                         alpha_min: float = 1e-6):
    """Algorithm 1 ("Centered start point"): the target mu, then the per-entry update.

    mu_target = max(x^T z / n, mu_min) from the unclamped input; each pair is
    lifted to at least alpha_min, then the smaller of (x'_j, z'_j) is moved
    first toward mu_target / (the other), within +-delta_max of itself, and
    the other is then moved toward mu_target / (the first, updated), also
    within +-delta_max.  A tie x'_j = z'_j takes the else-branch (z' first)."""
    x = np.asarray(x, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    n = x.size
    mu = max(float(x @ z) / n, mu_min) if n else mu_min
    xp = np.maximum(x, alpha_min)
    zp = np.maximum(z, alpha_min)

    def move(target, v):
        return np.minimum(np.maximum(target, v - delta_max), v + delta_max)

    first = xp < zp
    # branch x' < z':  x' then z' (using the new x')
    x1 = move(mu / zp, xp)
    z1 = move(mu / x1, zp)
    # else-branch:      z' then x' (using the new z')
    z2 = move(mu / xp, zp)
    x2 = move(mu / z2, xp)
    return np.where(first, x1, x2), np.where(first, z1, z2), mu


def warmstart_point(res: Result, mu_min=1e-6, delta_max=1e-4, alpha_min=1e-6,
                    unscaled: bool = False):
    """Algorithm 1 on the scaled PDHG solution (x~, y~, z~ = max(0, c~ - A~^T y~)).
    Returns (x', y, z') in the scaled space, or mapped back to the original
    model (x = D_c x', y = D_r y~, z = z' / D_c) when ``unscaled``."""
    S = res.setup
    zs = np.maximum(0.0, S.c_t - S.At.T @ res.y_scaled)
    xp, zp, mu = centered_start_point(res.x_scaled, zs, mu_min, delta_max, alpha_min)
    if unscaled:
        return S.D_c * xp, S.D_r * res.y_scaled, zp / S.D_c, mu
    return xp, res.y_scaled.copy(), zp, mu
