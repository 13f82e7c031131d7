"""Dense CPU reference for differentiating x*(b, c) through the active set.

TEST INFRASTRUCTURE (tests only).  Plain numpy on dense matrices.

At a PDHG fixed point x = max(0, x - tau (c - A^T y)) the positive set B
satisfies A_B x_B = b, x_j = 0 off B.  From an approximate iterate it is
predicted by complementarity in the scaled model: B = {j : x~_j > z~_j} with
z~ = max(0, c~ - A~^T y~).
With B fixed: x_B = least-squares solution of A_B x_B = b (exact, b is in
the range), and for a loss L(x) with g = dL/dx the min-norm active-set
Jacobian gives dL/db = A_B (A_B^T A_B)^{-1} g_B -- the minimum-norm u with
A_B^T u = g_B -- and dL/dc = 0 (x_B does not depend on c while B is fixed).
"""
import numpy as np

from . import pdhg_oracle as O


def active_set(res: "O.Result") -> np.ndarray:
    """B from the oracle's returned iterate in the scaled model."""
    S = res.setup
    zs = np.maximum(0.0, S.c_t - S.At.T @ res.y_scaled)
    return res.x_scaled > zs


def polish(A: np.ndarray, b: np.ndarray, B: np.ndarray) -> np.ndarray:
    x = np.zeros(A.shape[1])
    x[B] = np.linalg.lstsq(A[:, B], b, rcond=None)[0]
    return x


def grad_b(A: np.ndarray, B: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Minimum-norm u with A_B^T u = g_B (= A_B (A_B^T A_B)^{-1} g_B)."""
    return np.linalg.lstsq(A[:, B].T, g[B], rcond=None)[0]
