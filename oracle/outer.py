"""Outer (reweighting) loop of the oracle; test infrastructure only.

Section 2.1-2.2 and the last three steps of the "Shifted Recycling Algorithm"
(Section 5.5): after all shifts of step k are solved, the L-curve
(log ||C x - d||, log ||D_k L x||) picks l_* at its corner (maximum
curvature), and x^(k, l_*) defines the next weights.

Readings: the corner is the interior point of maximum signed Menger curvature
of consecutive points ordered by increasing gamma (ties: smaller l); the next
weights are the IRN/TV weights w = ((L x)^2 + beta^2)^(-1/2) (rule "irn") or
the paper's cumulative weights D_{k+1} = diag(1 - (|D_k L x| / ||D_k L x||_inf)^p) D_k,
w = D_{k+1}^2 (rule "gazzola", Section 2.1), and ||D_k L x|| = ||w_k^(1/2) .* L x||.
The outer stop rule of Section 8.2 (the same l_* three times running) is
``same_lstar_three``.
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np

from .operator import Operator, gazzola_weights, irn_weights
from .recycle import Params, State, outer_step


def lcurve_points(op: Operator, X: np.ndarray, d: np.ndarray, w: np.ndarray):
    """Residual norms ||H x_l - d|| and seminorms ||w^(1/2) .* L x_l||."""
    rho = np.array([np.linalg.norm(op.blur(x) - d) for x in X])
    eta = np.array([np.sqrt(np.sum(w * op.grad(x) ** 2)) for x in X])
    return rho, eta


def lcurve_corner(rho: np.ndarray, eta: np.ndarray) -> int:
    """0-based index of the maximum signed Menger curvature of the log-log points."""
    x = np.log(rho)
    y = np.log(eta)
    M = len(x)
    if M < 3:
        return 0
    best, best_l = -np.inf, 1
    for l in range(1, M - 1):
        ax, ay = x[l] - x[l - 1], y[l] - y[l - 1]
        bx, by = x[l + 1] - x[l], y[l + 1] - y[l]
        cx, cy = x[l + 1] - x[l - 1], y[l + 1] - y[l - 1]
        cross = ax * by - ay * bx
        den = np.sqrt((ax * ax + ay * ay) * (bx * bx + by * by) * (cx * cx + cy * cy))
        kappa = 2.0 * cross / den if den > 0 else 0.0
        if kappa > best:
            best, best_l = kappa, l
    return best_l


def same_lstar_three(history: List[int]) -> bool:
    """Stop rule of Section 8.2: the selected index is the same three times running."""
    return len(history) >= 3 and history[-1] == history[-2] == history[-3]


def run(op: Operator, b: np.ndarray, d: np.ndarray, gammas: np.ndarray, prm: Params,
        K_steps: int, beta: float, weights: Optional[List[np.ndarray]] = None,
        rule: str = "irn", p_gazzola: float = 2.0):
    """Run K_steps outer steps from W_0 = I. ``weights`` (optional) gives the
    weights of every step explicitly instead of the L-curve rule; otherwise
    ``rule`` ("irn" or "gazzola") makes the next weights from x^(k, l_*). The
    weights used at each step are returned in ``steps[k].extra["w"]``."""
    S = State()
    n = b.shape[0]
    w = np.ones(2 * n) if weights is None else weights[0]
    D = np.ones(2 * n)
    steps, lstars = [], []
    for k in range(K_steps):
        res = outer_step(op, b, gammas, w, S, prm)
        rho, eta = lcurve_points(op, res.X, d, w)
        ls = lcurve_corner(rho, eta)
        res.extra["lstar"] = ls
        res.extra["rho"], res.extra["eta"] = rho, eta
        res.extra["w"] = w
        lstars.append(ls)
        steps.append(res)
        if k + 1 < K_steps:
            if weights is not None:
                w = weights[k + 1]
            elif rule == "gazzola":
                D = gazzola_weights(op, res.X[ls], D, p_gazzola)
                w = D * D
            else:
                w = irn_weights(op, res.X[ls], beta)
    return steps, lstars
