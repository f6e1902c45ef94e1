"""Adjoint gradients of the shifted solves (oracle; test infrastructure only).

For solutions x_l of (A + gamma_l E) x_l = b with E = L^T diag(w) L and a loss
whose gradient with respect to x_l is g_l, the operator is symmetric, so one
adjoint solve per shift with the same operator,

    (A + gamma_l E) lambda_l = g_l,

gives (differentiating (A + gamma_l E) x_l = b)

    d loss / d gamma_l = -lambda_l^T E x_l = -(L lambda_l)^T diag(w) (L x_l),
    d loss / d w       = -sum_l gamma_l (L lambda_l) .* (L x_l)     (2n entries).

The adjoint systems are solved here by plain MINRES (Section 2.3 with an empty
recycle space) to a tight tolerance; nothing is recycled in the oracle.
"""
from __future__ import annotations

import numpy as np

from .minres import recycled_minres
from .operator import Operator


def adjoint_solves(op: Operator, gammas: np.ndarray, w: np.ndarray, G: np.ndarray,
                   tol: float = 1e-13, maxit: int = 100000) -> np.ndarray:
    """lambda_l = (A + gamma_l E)^{-1} g_l for every row g_l of G (M x n)."""
    Lam = np.zeros_like(G)
    for l, g in enumerate(gammas):
        gn = np.linalg.norm(G[l])
        if gn == 0.0:
            continue
        res = recycled_minres(lambda v, g=g: op.apply(v, g, w), G[l], None, tol * gn, maxit)
        Lam[l] = res.xm
    return Lam


def shift_and_weight_gradients(op: Operator, gammas: np.ndarray, w: np.ndarray, X: np.ndarray,
                               Lam: np.ndarray):
    """(d loss/d gamma (M), d loss/d w (2n)) from the solutions X and adjoints Lam."""
    dgamma = np.zeros(len(gammas))
    dw = np.zeros_like(w)
    for l, g in enumerate(gammas):
        Ll = op.grad(Lam[l])
        Lx = op.grad(X[l])
        dgamma[l] = -np.sum(Ll * w * Lx)
        dw -= g * Ll * Lx
    return dgamma, dw
