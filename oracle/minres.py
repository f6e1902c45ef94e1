"""Recycled MINRES (oracle; test infrastructure only).

Section 2.3 and Section 4.2 (Eq. minShift, Eq. xFinal): given K with
orthonormal columns, K = Op U, and a right-hand side r, run the Lanczos process
on (I - K K^T) Op from v_1 = (I - K K^T) r / xi, xi = ||(I - K K^T) r||
(Eq. eq01):

    Op v_j = K h_j + beta_j v_{j-1} + alpha_j v_j + beta_{j+1} v_{j+1},
    h_j = K^T Op v_j,  alpha_j = v_j^T Op v_j,

and solve  min || [K^T r; xi e_1] - [I, K^T Op V_m; 0, T_m] [z; y] ||:
y from the MINRES least-squares problem min || T_m y - xi e_1 ||, then
z = K^T r - K^T Op V_m y. The correction is V_m y + U z.

As the paper notes, V_m y follows from the short recurrences of standard
MINRES (Paige and Saunders): Givens rotations reduce T_m to upper triangular
R_m, the search directions D_m = V_m R_m^{-1} obey a three-term recurrence and
V_m y = sum_j tau_j d_j. The same recurrence applied to the coupling vectors
h_j gives K^T Op V_m y = sum_j tau_j hhat_j, so z is updated in step.
The least-squares residual norm is |eta_m| (the last rotated right-hand side).

With K empty this is plain MINRES.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class MinresResult:
    xm: np.ndarray              # V_m y
    z: np.ndarray               # K^T r - K^T Op V_m y   (length s)
    iters: int                  # m, the number of Lanczos steps (= matvecs)
    eta_hist: List[float]       # |eta_j|, j = 0..m (eta_0 = xi)
    alphas: List[float]
    betas: List[float]          # beta_2 .. beta_{m+1}
    V: Optional[np.ndarray]     # kept Lanczos vectors (n, n_kept), or None
    xi: float


def recycled_minres(op_apply: Callable[[np.ndarray], np.ndarray], r: np.ndarray,
                    K: Optional[np.ndarray], tol_abs: float, maxit: int,
                    keep: int = 0, reorth: bool = False) -> MinresResult:
    """Recycled MINRES on Op g = r with recycle space (U, K), K = Op U.

    Stops when the least-squares residual |eta_j| <= tol_abs, after ``maxit``
    steps, or on a Lanczos breakdown (beta_{j+1} = 0: the Krylov space is
    invariant and the least-squares solution is exact).

    ``keep`` Lanczos vectors v_1..v_keep are returned in ``V``; with
    ``reorth`` each new Lanczos vector is re-orthogonalized (twice, classical
    Gram-Schmidt) against the kept ones while j < keep (Section 8.2: the first
    Krylov vectors are reorthogonalized for the Ritz extraction).
    """
    n = r.shape[0]
    s = 0 if K is None else K.shape[1]
    Ktr = K.T @ r if s else np.zeros(0)
    u = r - K @ Ktr if s else r.copy()
    xi = float(np.linalg.norm(u))
    xm = np.zeros(n)
    z = Ktr.copy()
    res = MinresResult(xm, z, 0, [xi], [], [], None, xi)
    kept: List[np.ndarray] = []
    if xi <= tol_abs or xi == 0.0 or maxit <= 0:
        res.V = np.zeros((n, 0))
        return res

    v_prev = np.zeros(n)
    v = u / xi
    beta = 0.0                       # beta_j, the coefficient of v_{j-1}
    cs2, sn2 = 1.0, 0.0              # rotation G_{j-2}
    cs1, sn1 = 1.0, 0.0              # rotation G_{j-1}
    d1 = np.zeros(n)                 # d_{j-1}
    d2 = np.zeros(n)                 # d_{j-2}
    h1 = np.zeros(s)                 # hhat_{j-1}
    h2 = np.zeros(s)                 # hhat_{j-2}
    eta = xi
    for j in range(1, maxit + 1):
        if keep and len(kept) < keep:
            kept.append(v.copy())
        y = op_apply(v)
        h = K.T @ y if s else np.zeros(0)
        alpha = float(v @ y)
        u = y - alpha * v - beta * v_prev
        if s:
            u = u - K @ h
        if reorth and len(kept) < keep and kept:
            Vk = np.stack(kept, axis=1)
            for _ in range(2):
                u = u - Vk @ (Vk.T @ u)
        beta_next = float(np.linalg.norm(u))

        # apply G_{j-2}, G_{j-1} to column j of T, then build G_j
        eps = sn2 * beta
        dbar = cs2 * beta
        delta = cs1 * dbar + sn1 * alpha
        gbar = -sn1 * dbar + cs1 * alpha
        gamma = float(np.hypot(gbar, beta_next))
        cs, sn = gbar / gamma, beta_next / gamma
        tau = cs * eta
        eta = -sn * eta

        d = (v - delta * d1 - eps * d2) / gamma
        xm = xm + tau * d
        if s:
            hh = (h - delta * h1 - eps * h2) / gamma
            z = z - tau * hh
            h2, h1 = h1, hh
        d2, d1 = d1, d

        res.alphas.append(alpha)
        res.betas.append(beta_next)
        res.eta_hist.append(abs(eta))
        res.iters = j
        cs2, sn2, cs1, sn1 = cs1, sn1, cs, sn
        if abs(eta) <= tol_abs or beta_next == 0.0:
            break
        v_prev, v = v, u / beta_next
        beta = beta_next

    res.xm, res.z = xm, z
    res.V = np.stack(kept, axis=1) if kept else np.zeros((n, 0))
    return res


def recycled_cg(op_apply: Callable[[np.ndarray], np.ndarray], r: np.ndarray,
                K: Optional[np.ndarray], tol_abs: float, maxit: int) -> MinresResult:
    """Projected (recycled) CG on Op g = r with recycle space (U, K), K = Op U: the
    same Lanczos process on (I - K K^T) Op from v_1 = (I - K K^T) r / xi as
    ``recycled_minres`` (Op is SPD on the complement of K, where the projected
    operator is self-adjoint), but y_m solves the square system T_m y = xi e_1
    (Galerkin) instead of the least-squares problem. The LDL^T factorisation of
    T_m gives short recurrences (Lanczos form of CG):

        lambda_j = beta_j / eta_{j-1},  zeta_j = -lambda_j zeta_{j-1}  (zeta_1 = xi),
        eta_j = alpha_j - lambda_j beta_j,
        p_j = (v_j - beta_j p_{j-1}) / eta_j,  V_m y = sum_j zeta_j p_j,

    the same recurrence on h_j = K^T Op v_j gives K^T Op V_m y, so
    z = K^T r - K^T Op V_m y as for MINRES. The residual r - Op (V_m y + U z) is
    -beta_{m+1} (zeta_m / eta_m) v_{m+1}: its norm is the stopping test.
    ``eta_hist`` holds these residual norms."""
    n = r.shape[0]
    s = 0 if K is None else K.shape[1]
    Ktr = K.T @ r if s else np.zeros(0)
    u = r - K @ Ktr if s else r.copy()
    xi = float(np.linalg.norm(u))
    xm = np.zeros(n)
    z = Ktr.copy()
    res = MinresResult(xm, z, 0, [xi], [], [], np.zeros((n, 0)), xi)
    if xi <= tol_abs or xi == 0.0 or maxit <= 0:
        return res
    v_prev = np.zeros(n)
    v = u / xi
    beta = 0.0                       # beta_j, the coefficient of v_{j-1}
    eta_prev, zeta = 1.0, xi
    p = np.zeros(n)                  # p_{j-1}
    hp = np.zeros(s)                 # K^T Op p_{j-1}
    for j in range(1, maxit + 1):
        y = op_apply(v)
        h = K.T @ y if s else np.zeros(0)
        alpha = float(v @ y)
        u = y - alpha * v - beta * v_prev
        if s:
            u = u - K @ h
        beta_next = float(np.linalg.norm(u))
        if j > 1:
            lam = beta / eta_prev
            zeta = -lam * zeta
        else:
            lam = 0.0
        eta = alpha - lam * beta
        p = (v - beta * p) / eta
        xm = xm + zeta * p
        if s:
            hp = (h - beta * hp) / eta
            z = z - zeta * hp
        resn = beta_next * abs(zeta / eta)
        res.alphas.append(alpha)
        res.betas.append(beta_next)
        res.eta_hist.append(resn)
        res.iters = j
        eta_prev = eta
        if resn <= tol_abs or beta_next == 0.0:
            break
        v_prev, v = v, u / beta_next
        beta = beta_next
    res.xm, res.z = xm, z
    return res


def lanczos_tridiagonal(alphas: List[float], betas: List[float], m: int) -> np.ndarray:
    """The m x m Lanczos matrix T_m (alpha on the diagonal, beta_2..beta_m off it)."""
    T = np.diag(np.asarray(alphas[:m], dtype=np.float64))
    for j in range(m - 1):
        T[j, j + 1] = T[j + 1, j] = betas[j]
    return T
