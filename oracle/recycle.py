"""Two-level recycling for one outer step (oracle; test infrastructure only).

Follows the paper's Algorithm "Shifted Recycling Algorithm" (Section 5.5) for a
fixed regularisation matrix E_k:

1. principal space U~ (Section 5.1, Eq. widetildeU for k = 0; Section 5.2,
   Eq. delta and Eq. tildeUupdate for k >= 1), made orthonormal and
   rank-revealing by Algorithm "Stabilized U";
2. the images A U~ and E_k U~ (n_c matvecs, Section 6);
3. (A + gamma_* E_k) U~ = K R (Eq. establishU), U = U~ R^{-1} implicit;
   per shift the orthogonal-projection initial guess of Eq. orthupdate;
4. projected matrices A^ = U~^T A U~, E^ = U~^T E_k U~ (Eq. hq) and the Ritz
   vectors of Algorithm "interior" at gamma_{J_L} and gamma_{J_R};
5. for l = 1..M in order, the local space [W, g^(k-1,l), g^(k,l-1)]
   (Algorithms "updatelocal" / "updatelocalV2"), its QR (Eq. localU) and the
   recycled MINRES correction (Eq. corr_g, minShift, xFinal / upest).

Readings where the paper is silent (each also in the design notes):
* stabilize normalises the columns first and caps n_c at ``p`` (largest
  singular values kept);
* the Ritz extraction uses the Lanczos matrix T_a of the first a
  (reorthogonalized) Lanczos vectors;
* V^(new) = [delta x, v_1..v_m] from at most ``vnew_cap`` MINRES steps on
  Eq. delta, written as (A + gamma_lc E_k) delta x = gamma_lc (E_k - E_{k-1}) x;
* a local column is dropped when its component orthogonal to the previous
  columns of (A + gamma_l E_k) U~_l is below 1e-10 of its own norm; of two
  g's at an angle with |cos| > 0.99 only g^(k,l-1) is kept (footnote of
  Section 5.3);
* with ``batched_local`` the chained g^(k,l-1) is replaced by g^(k-1,l-1) so
  that all shifts are independent.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

from .minres import lanczos_tridiagonal, recycled_cg, recycled_minres
from .operator import Operator

STABILIZE_RATIO = 1e10
LOCAL_DROP = 1e-10
ANGLE_COS = 0.99


@dataclasses.dataclass
class Params:
    """Index choices and sizes of the paper's index table (1-based indices)."""

    M: int
    I_split: int
    i1: int
    i2: int
    i_star: int
    l_c: int
    J_L: int
    J_R: int
    p: int
    a_ritz: int
    b_ritz: int
    n_ritz_local: int
    vnew_cap: int
    tol: float
    maxit: int
    batched_local: bool = False
    # initial guesses: "orthogonal" (Eq. orthupdate), "oblique" (Eq. obliqueupdate,
    # anchor gamma_*), "oblique2" (Eq. updates, anchors gamma_{I_L}, gamma_{I_R})
    guess: str = "orthogonal"
    I_L: int = 0
    I_R: int = 0
    # inner solver of the per-shift corrections: "minres" (the paper's, Eq. minShift)
    # or "cg" (projected CG: the Galerkin solution of the same projected Lanczos process)
    inner: str = "minres"

    @staticmethod
    def from_workload(wl, batched_local: bool = False, guess: str = "orthogonal") -> "Params":
        return Params(wl.M, wl.I_split, wl.i1, wl.i2, wl.i_star, wl.l_c, wl.J_L, wl.J_R,
                      wl.p, wl.a_ritz, wl.b_ritz, wl.n_ritz_local, wl.vnew_cap, wl.tol,
                      wl.maxit, batched_local, guess, wl.i_star, wl.l_c)


@dataclasses.dataclass
class State:
    """What one outer step hands to the next."""

    k: int = -1
    w: Optional[np.ndarray] = None
    w_prev: Optional[np.ndarray] = None
    V_i1: Optional[np.ndarray] = None
    X_prev: Optional[np.ndarray] = None   # (M, n) solutions x^(k-1, l)
    G_prev: Optional[np.ndarray] = None   # (M, n) corrections g^(k-1, l)


@dataclasses.dataclass
class StepResult:
    X: np.ndarray                  # (M, n) solutions x^(k, l)
    X0: np.ndarray                 # (M, n) initial guesses
    G: np.ndarray                  # (M, n) corrections
    iters: np.ndarray              # MINRES steps per shift
    matvecs: np.ndarray            # operator applications per shift
    relres0: np.ndarray            # ||r0|| / ||b||
    relres_est: np.ndarray         # MINRES least-squares residual / ||b||
    relres_true: np.ndarray        # ||b - Op x|| / ||b|| (recomputed)
    local_dim: np.ndarray          # columns of K_l
    nc: int
    overhead_matvecs: int          # principal space construction + images
    Ut: np.ndarray = None          # principal basis used in this step
    extra: Dict = dataclasses.field(default_factory=dict)


# ---------------------------------------------------------------------------
# Algorithm "Stabilized U"
# ---------------------------------------------------------------------------
def stabilize(Ut: np.ndarray, p_max: int, ratio: float = STABILIZE_RATIO) -> np.ndarray:
    """Skinny SVD U~ = Q S W^T; keep the n_c leading columns of Q with
    sigma_1 / sigma_i < ratio (at most p_max of them)."""
    norms = np.linalg.norm(Ut, axis=0)
    cols = Ut[:, norms > 0] / norms[norms > 0]
    if cols.shape[1] == 0:
        return np.zeros((Ut.shape[0], 0))
    Q, S, _ = np.linalg.svd(cols, full_matrices=False)
    nc = int(np.sum(S[0] / np.maximum(S, 1e-300) < ratio))
    nc = min(nc, p_max)
    return Q[:, :nc]


# ---------------------------------------------------------------------------
# Principal space: Section 5.1 (k = 0) and Section 5.2 (k >= 1)
# ---------------------------------------------------------------------------
def init_principal(op: Operator, b: np.ndarray, gammas: np.ndarray, w: np.ndarray,
                   prm: Params):
    """Solve the gamma_{i1} and gamma_{i2} systems by MINRES to tolerance, keeping
    the first a (reorthogonalized) Lanczos vectors of each; Ritz vectors give
    V_{i1} (all a) and V_{i2} (the b' with the smallest Ritz values).
    Returns (U~ = [x_i1, x_i2, V_i1, V_i2], V_i1, matvecs)."""
    tol_abs = prm.tol * np.linalg.norm(b)
    out = {}
    mv = 0
    for tag, idx, nkeep in (("i1", prm.i1, prm.a_ritz), ("i2", prm.i2, prm.a_ritz)):
        g = gammas[idx - 1]
        res = recycled_minres(lambda v: op.apply(v, g, w), b, None, tol_abs, prm.maxit,
                              keep=nkeep, reorth=True)
        mv += res.iters
        m = res.V.shape[1]
        T = lanczos_tridiagonal(res.alphas, res.betas, m)
        theta, S = np.linalg.eigh(T)          # ascending Ritz values
        ritz = res.V @ S
        out[tag] = (res.xm, ritz)
    x1, R1 = out["i1"]
    x2, R2 = out["i2"]
    V_i1 = R1
    V_i2 = R2[:, :prm.b_ritz]
    Ut = np.concatenate([x1[:, None], x2[:, None], V_i1, V_i2], axis=1)
    return Ut, V_i1, mv


def update_principal(op: Operator, b: np.ndarray, gammas: np.ndarray, w: np.ndarray,
                     w_prev: np.ndarray, V_i1: np.ndarray, X_prev: np.ndarray, prm: Params):
    """Eq. delta for l = l_c: (A/gamma + E_k) dx = (E_k - E_{k-1}) x^(k-1,l_c), by at
    most vnew_cap MINRES steps; V^(new) = [dx, v_1..v_m];
    U~ = [V_{i1}, V^(new), x^(k-1,1..M)] (Eq. tildeUupdate). Returns (U~, matvecs)."""
    g = gammas[prm.l_c - 1]
    xc = X_prev[prm.l_c - 1]
    rhs = g * op.grad_adjoint((w - w_prev) * op.grad(xc))
    mv = 1
    res = recycled_minres(lambda v: op.apply(v, g, w), rhs, None,
                          prm.tol * np.linalg.norm(rhs), prm.vnew_cap,
                          keep=prm.vnew_cap, reorth=False)
    mv += res.iters
    Vnew = np.concatenate([res.xm[:, None], res.V], axis=1)
    Ut = np.concatenate([V_i1, Vnew, X_prev.T], axis=1)
    return Ut, mv


# ---------------------------------------------------------------------------
# Section 4.1: orthogonal-projection initial guesses
# ---------------------------------------------------------------------------
def principal_guesses(Ut, AU, EU, b, gammas, gamma_star):
    """(A + gamma_* E) U~ = K R; U = U~ R^{-1}. For every shift, solve
    (I + d M + d M^T + d^2 N) q = K^T b + d U^T E b with d = gamma_l - gamma_*,
    M = K^T E U, N = (E U)^T (E U) (Eq. orthupdate), then x0 = U q and
    r0 = b - (K + d E U) q (Eq. res_initGuessPrincRecy).
    Returns (C, X0, R0) with C[:, l] = R^{-1} q_l (so x0 = U~ C[:, l])."""
    nc = Ut.shape[1]
    M_ = len(gammas)
    n = Ut.shape[0]
    if nc == 0:
        return np.zeros((0, M_)), np.zeros((M_, n)), np.tile(b, (M_, 1))
    B = AU + gamma_star * EU
    K, R = np.linalg.qr(B)
    EUi = np.linalg.solve(R.T, EU.T).T          # E U = E U~ R^{-1}
    Mm = K.T @ EUi
    N = EUi.T @ EUi
    Ktb = K.T @ b
    UtEb = EUi.T @ b
    C = np.zeros((nc, M_))
    X0 = np.zeros((M_, n))
    R0 = np.zeros((M_, n))
    for l, gl in enumerate(gammas):
        d = gl - gamma_star
        Sm = np.eye(nc) + d * (Mm + Mm.T) + d * d * N
        L = np.linalg.cholesky(Sm)
        q = np.linalg.solve(L.T, np.linalg.solve(L, Ktb + d * UtEb))
        c = np.linalg.solve(R, q)
        C[:, l] = c
        X0[l] = Ut @ c
        R0[l] = b - (AU @ c + gl * (EU @ c))
    return C, X0, R0


# ---------------------------------------------------------------------------
# Section 7: oblique-projection initial guesses
# ---------------------------------------------------------------------------
def oblique_anchor(Ut, AU, EU, b, gamma_a):
    """(A + gamma_a E) U~ = K R, U = U~ R^{-1}; returns (K^T E U, K^T b, R), the
    quantities Eq. obliqueupdate needs (no (E U)^T (E U))."""
    K, R = np.linalg.qr(AU + gamma_a * EU)
    EUi = np.linalg.solve(R.T, EU.T).T
    return K.T @ EUi, K.T @ b, R


def oblique_guesses(Ut, AU, EU, b, gammas, gamma_left, gamma_right=None, I_split=None):
    """For every shift, q from K^T b = (I + d K^T E U) q with d = gamma_l - gamma_a
    (Eq. obliqueupdate: the residual is made orthogonal to K, not to
    K + d E U), x0 = U q, r0 = b - (A + gamma_l E) x0. With ``gamma_right`` the
    two-anchor form of Eq. updates: shifts l <= I_split (1-based) use the anchor
    gamma_left, the others gamma_right. Returns (C, X0, R0) as principal_guesses."""
    nc = Ut.shape[1]
    M_ = len(gammas)
    n = Ut.shape[0]
    if nc == 0:
        return np.zeros((0, M_)), np.zeros((M_, n)), np.tile(b, (M_, 1))
    anchors = [(gamma_left,) + oblique_anchor(Ut, AU, EU, b, gamma_left)]
    if gamma_right is not None:
        anchors.append((gamma_right,) + oblique_anchor(Ut, AU, EU, b, gamma_right))
    C = np.zeros((nc, M_))
    X0 = np.zeros((M_, n))
    R0 = np.zeros((M_, n))
    for l, gl in enumerate(gammas):
        right = gamma_right is not None and (l + 1) > I_split
        ga, KtEU, Ktb, R = anchors[1 if right else 0]
        q = np.linalg.solve(np.eye(nc) + (gl - ga) * KtEU, Ktb)
        c = np.linalg.solve(R, q)
        C[:, l] = c
        X0[l] = Ut @ c
        R0[l] = b - (AU @ c + gl * (EU @ c))
    return C, X0, R0


def initial_guesses(Ut, AU, EU, b, gammas, prm: "Params"):
    """The initial guesses that ``prm.guess`` selects (Sections 4.1 and 7)."""
    gstar = gammas[prm.i_star - 1]
    if prm.guess == "orthogonal":
        return principal_guesses(Ut, AU, EU, b, gammas, gstar)
    if prm.guess == "oblique":
        return oblique_guesses(Ut, AU, EU, b, gammas, gstar)
    if prm.guess == "oblique2":
        return oblique_guesses(Ut, AU, EU, b, gammas, gammas[prm.I_L - 1], gammas[prm.I_R - 1],
                               prm.I_split)
    raise ValueError(f"unknown initial guess kind {prm.guess!r}")


# ---------------------------------------------------------------------------
# Algorithm "interior"
# ---------------------------------------------------------------------------
def interior_ritz(Ah: np.ndarray, Eh: np.ndarray, gamma: float, nJ: int) -> np.ndarray:
    """Eigenvectors of H = A^ + gamma E^ for the nJ smallest eigenvalues (as
    columns of an n_c x nJ matrix W~_J; W = U~ W~_J). Ties: lower index."""
    H = Ah + gamma * Eh
    H = 0.5 * (H + H.T)
    theta, Wt = np.linalg.eigh(H)
    return Wt[:, :min(nJ, H.shape[0])]


def qr_with_drops(B: np.ndarray, rel: float = LOCAL_DROP):
    """Householder QR of the columns of B, dropping (one at a time, first offender
    first) any column whose part orthogonal to the previous kept columns is
    <= rel times its own norm. Returns (K, R, kept_indices)."""
    keep = [j for j in range(B.shape[1]) if np.linalg.norm(B[:, j]) > 0]
    while keep:
        Q, R = np.linalg.qr(B[:, keep])
        diag = np.abs(np.diag(R))
        colnorm = np.linalg.norm(B[:, keep], axis=0)
        bad = np.nonzero(diag <= rel * colnorm)[0]
        if bad.size == 0:
            return Q, R, keep
        del keep[int(bad[0])]
    return np.zeros((B.shape[0], 0)), np.zeros((0, 0)), []


# ---------------------------------------------------------------------------
# Algorithm "updatelocal": the corrections that join a local space
# ---------------------------------------------------------------------------
def local_corrections(l: int, k: int, G_prev: Optional[np.ndarray], G_cur: np.ndarray,
                      batched: bool):
    """The two correction vectors of shift l (0-based) in step k (Algorithm
    updatelocal, last step; Figure "local"): g^(k-1,l) from the previous outer
    step, and g^(k,l-1) of the previous shift of this step -- or, with
    ``batched``, g^(k-1,l-1) so that the shifts of a step are independent.
    A vector that does not exist (k = 0, l = 0) is None."""
    g_old = G_prev[l] if (k >= 1 and G_prev is not None) else None
    if batched:
        g_new = G_prev[l - 1] if (k >= 1 and l >= 1 and G_prev is not None) else None
    else:
        g_new = G_cur[l - 1] if l >= 1 else None
    return g_old, g_new


def local_columns(g_old: Optional[np.ndarray], g_new: Optional[np.ndarray],
                  cos_max: float = ANGLE_COS) -> List[np.ndarray]:
    """The correction columns appended to W, in the order [g^(k-1,l), g^(k,l-1)]
    (Algorithm updatelocal). Zero or missing vectors are left out; when both
    exist and |cos angle(g_old, g_new)| > cos_max only g_new is kept (footnote of
    Section 5.3)."""
    gcols = [g for g in (g_old, g_new) if g is not None and np.linalg.norm(g) > 0]
    if len(gcols) == 2:
        c = abs(gcols[0] @ gcols[1]) / (np.linalg.norm(gcols[0]) * np.linalg.norm(gcols[1]))
        if c > cos_max:
            gcols = [gcols[1]]
    return gcols


# ---------------------------------------------------------------------------
# One outer step of the "Shifted Recycling Algorithm"
# ---------------------------------------------------------------------------
def outer_step(op: Operator, b: np.ndarray, gammas: np.ndarray, w: np.ndarray,
               S: State, prm: Params, Ut_given: Optional[np.ndarray] = None,
               iters_override: Optional[List[int]] = None,
               record_local: bool = False, shifts: Optional[List[int]] = None) -> StepResult:
    """Solve all M shifted systems for the weights ``w`` (step k = S.k + 1).

    ``Ut_given`` replaces the principal-space construction (the basis is still
    stabilized); ``iters_override`` fixes the MINRES step count per shift
    (tolerance ignored) for parity checks of iterates. With ``record_local``
    the local basis U~_l of every shift (after drops; None where the initial
    guess already met the tolerance) is returned in ``extra["local_cols"]``,
    and the raw principal basis (before stabilize) in ``extra["Ut_raw"]``. With
    ``shifts`` (0-based, batched local spaces only: their shifts are independent)
    only those shifts are solved; the others are left at zero.
    """
    if shifts is not None and not prm.batched_local:
        raise ValueError("a subset of shifts needs batched local spaces")
    k = S.k + 1
    n = b.shape[0]
    M_ = len(gammas)
    bnorm = float(np.linalg.norm(b))
    tol_abs = prm.tol * bnorm
    overhead = 0

    # -- principal space -------------------------------------------------
    if Ut_given is not None:
        Ut_raw = Ut_given
    elif k == 0:
        Ut_raw, S.V_i1, mv = init_principal(op, b, gammas, w, prm)
        overhead += mv
    else:
        Ut_raw, mv = update_principal(op, b, gammas, w, S.w, S.V_i1, S.X_prev, prm)
        overhead += mv
    Ut = stabilize(Ut_raw, prm.p)
    local_cols: List[Optional[np.ndarray]] = [None] * M_
    nc = Ut.shape[1]
    AU = np.stack([op.apply_A(Ut[:, j]) for j in range(nc)], axis=1) if nc else np.zeros((n, 0))
    EU = np.stack([op.apply_E(Ut[:, j], w) for j in range(nc)], axis=1) if nc else np.zeros((n, 0))
    overhead += nc

    # -- initial guesses -------------------------------------------------
    C, X0, R0 = initial_guesses(Ut, AU, EU, b, gammas, prm)

    # -- Ritz vectors of the projected systems ----------------------------
    Ah = Ut.T @ AU
    Eh = Ut.T @ EU
    Ah, Eh = 0.5 * (Ah + Ah.T), 0.5 * (Eh + Eh.T)
    nJ = prm.n_ritz_local
    WtL = interior_ritz(Ah, Eh, gammas[prm.J_L - 1], nJ) if nc else np.zeros((0, 0))
    WtR = interior_ritz(Ah, Eh, gammas[prm.J_R - 1], nJ) if nc else np.zeros((0, 0))

    X = np.zeros((M_, n))
    G = np.zeros((M_, n))
    iters = np.zeros(M_, dtype=int)
    matvecs = np.zeros(M_, dtype=int)
    relres0 = np.zeros(M_)
    relres_est = np.zeros(M_)
    relres_true = np.zeros(M_)
    local_dim = np.zeros(M_, dtype=int)

    for l in range(M_):
        if shifts is not None and l not in shifts:
            continue
        gl = gammas[l]
        apply_l = (lambda v, gl=gl: op.apply(v, gl, w))
        x0, r0 = X0[l], R0[l]
        relres0[l] = np.linalg.norm(r0) / bnorm
        forced = iters_override[l] if iters_override is not None else None
        if forced is None and relres0[l] <= prm.tol:
            X[l] = x0
            relres_est[l] = relres0[l]
            r = b - apply_l(X[l])
            matvecs[l] = 1
            relres_true[l] = np.linalg.norm(r) / bnorm
            continue

        Wt = WtL if (l + 1) <= prm.I_split else WtR
        cols = [Ut @ Wt] if nc else []
        imgs = [AU @ Wt + gl * (EU @ Wt)] if nc else []
        g_old, g_new = local_corrections(l, k, S.G_prev, G, prm.batched_local)
        gcols = local_columns(g_old, g_new)
        for g in gcols:
            cols.append(g[:, None])
            imgs.append((op.apply_A(g) + gl * op.apply_E(g, w))[:, None])
            matvecs[l] += 1
        Ul_t = np.concatenate(cols, axis=1) if cols else np.zeros((n, 0))
        Bl = np.concatenate(imgs, axis=1) if imgs else np.zeros((n, 0))
        Kl, Rl, kept = qr_with_drops(Bl)
        Ul_t = Ul_t[:, kept]
        local_dim[l] = Kl.shape[1]
        if record_local:
            local_cols[l] = Ul_t.copy()

        solver = recycled_cg if prm.inner == "cg" else recycled_minres
        if forced is not None:
            res = solver(apply_l, r0, Kl if Kl.shape[1] else None, 0.0, forced)
        else:
            res = solver(apply_l, r0, Kl if Kl.shape[1] else None, tol_abs, prm.maxit)
        iters[l] = res.iters
        matvecs[l] += res.iters
        g = res.xm.copy()
        if Kl.shape[1]:
            g += Ul_t @ np.linalg.solve(Rl, res.z)
        G[l] = g
        X[l] = x0 + g
        relres_est[l] = res.eta_hist[-1] / bnorm
        r = b - apply_l(X[l])
        matvecs[l] += 1
        relres_true[l] = np.linalg.norm(r) / bnorm

    S.k = k
    S.w_prev, S.w = S.w, w.copy()
    S.X_prev = X.copy()
    S.G_prev = G.copy()
    extra = {"C": C, "AU": AU, "EU": EU, "Ah": Ah, "Eh": Eh, "WtL": WtL, "WtR": WtR}
    if record_local:
        extra["local_cols"] = local_cols
        extra["Ut_raw"] = Ut_raw
    return StepResult(X, X0, G, iters, matvecs, relres0, relres_est, relres_true, local_dim,
                      nc, overhead, Ut, extra)


def naive_minres(op: Operator, b: np.ndarray, gammas: np.ndarray, w: np.ndarray, tol: float,
                 maxit: int):
    """The comparison of Section 8: every shift solved by plain MINRES from zero."""
    tol_abs = tol * np.linalg.norm(b)
    X, its = [], []
    for g in gammas:
        res = recycled_minres(lambda v, g=g: op.apply(v, g, w), b, None, tol_abs, maxit)
        X.append(res.xm)
        its.append(res.iters)
    return np.stack(X), np.array(its)
