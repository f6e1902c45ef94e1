"""Pins of the oracle's (recycled) MINRES: SciPy's MINRES, brute-force least
squares over explicit bases, and the Petrov-Galerkin / Lanczos relations of
Section 2.3 (Eq. eq01, eqrecyc) and Section 4.2 (Eq. minShift, xFinal)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle.minres import lanczos_tridiagonal, recycled_minres
from oracle.operator import Operator
from tests.dense import operator_dense


def _problem(h=9, w=8, gamma=1e-2, seed=0):
    op = Operator(h, w, 1.0, 2)
    wt = synth.random_weights(h * w, seed)
    _, _, Op = operator_dense(h, w, op.taps, wt, gamma)
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(h * w)
    return op, wt, Op, r


def _orth_krylov(apply, v, m):
    """Orthonormal basis of span{v, Op v, ..., Op^{m-1} v}, Arnoldi with full
    re-orthogonalisation (independent of the Lanczos short recurrence)."""
    Q = [v / np.linalg.norm(v)]
    for _ in range(m - 1):
        u = apply(Q[-1])
        for _ in range(2):
            for q in Q:
                u = u - (q @ u) * q
        Q.append(u / np.linalg.norm(u))
    return np.stack(Q, axis=1)


@pytest.mark.parametrize("m", [1, 2, 5, 12, 25])
def test_plain_minres_matches_scipy_iterates(m):
    _, _, Op, r = _problem()
    res = recycled_minres(lambda v: Op @ v, r, None, 0.0, m)
    assert res.iters == m
    x_sp, _ = spla.minres(Op, r, rtol=0.0, maxiter=m)
    np.testing.assert_allclose(res.xm, x_sp, rtol=1e-9, atol=1e-10 * np.linalg.norm(x_sp))


@pytest.mark.parametrize("m", [1, 3, 8])
def test_plain_minres_is_the_krylov_least_squares_minimiser(m):
    _, _, Op, r = _problem(seed=3)
    res = recycled_minres(lambda v: Op @ v, r, None, 0.0, m)
    V = _orth_krylov(lambda v: Op @ v, r, m)
    c, *_ = np.linalg.lstsq(Op @ V, r, rcond=None)
    np.testing.assert_allclose(res.xm, V @ c, rtol=1e-8, atol=1e-10)
    assert abs(res.eta_hist[-1] - np.linalg.norm(r - Op @ res.xm)) < 1e-10 * np.linalg.norm(r)


def test_residual_history_non_increasing_and_converges():
    _, _, Op, r = _problem(seed=4)
    res = recycled_minres(lambda v: Op @ v, r, None, 1e-12 * np.linalg.norm(r), 10000)
    h = np.array(res.eta_hist)
    assert np.all(np.diff(h) <= 1e-14 * h[0])
    x = np.linalg.solve(Op, r)
    kappa = np.linalg.cond(Op)
    assert np.linalg.norm(res.xm - x) / np.linalg.norm(x) < 10 * kappa * 1e-12


@pytest.mark.parametrize("s,m", [(1, 4), (3, 6), (5, 10)])
def test_recycled_minres_is_least_squares_over_U_and_Krylov(s, m):
    """Eq. (minShift): the correction minimises ||r - Op g|| over
    Range[U, V_m], V_m spanning the Krylov space of (I - K K^T) Op from
    (I - K K^T) r; K^T (r - Op g) = 0; ||r - Op g|| = |eta_m|."""
    _, _, Op, r = _problem(seed=7 + s)
    n = r.shape[0]
    rng = np.random.default_rng(s)
    Ut = rng.standard_normal((n, s))
    K, R = np.linalg.qr(Op @ Ut)
    U = np.linalg.solve(R.T, Ut.T).T                 # U = U~ R^{-1}, Op U = K
    res = recycled_minres(lambda v: Op @ v, r, K, 0.0, m)
    g = res.xm + U @ res.z
    P = np.eye(n) - K @ K.T
    V = _orth_krylov(lambda v: P @ (Op @ v), P @ r, m)
    S = np.concatenate([U, V], axis=1)
    c, *_ = np.linalg.lstsq(Op @ S, r, rcond=None)
    g_bf = S @ c
    np.testing.assert_allclose(g, g_bf, rtol=1e-7, atol=1e-9 * np.linalg.norm(g_bf))
    rr = r - Op @ g
    assert np.linalg.norm(K.T @ rr) < 1e-10 * np.linalg.norm(r)
    assert abs(np.linalg.norm(rr) - res.eta_hist[-1]) < 1e-10 * np.linalg.norm(r)
    # x_m = V_m y lies in the Krylov space and is orthogonal to K
    assert np.linalg.norm(K.T @ res.xm) < 1e-10 * (np.linalg.norm(res.xm) + 1)


def test_recycled_minres_exact_when_r_in_range_of_K():
    _, _, Op, _ = _problem(seed=9)
    n = Op.shape[0]
    rng = np.random.default_rng(2)
    Ut = rng.standard_normal((n, 4))
    K, R = np.linalg.qr(Op @ Ut)
    r = K @ rng.standard_normal(4)
    res = recycled_minres(lambda v: Op @ v, r, K, 1e-14, 50)
    assert res.iters == 0
    U = np.linalg.solve(R.T, Ut.T).T
    np.testing.assert_allclose(Op @ (U @ res.z), r, rtol=1e-9, atol=1e-12)


def test_lanczos_relation_with_reorthogonalisation():
    """Eq. (eq01) with K = []: Op V_m = V_{m+1} T_m; with reorthogonalisation the
    kept vectors are orthonormal and V^T Op V = T (the Rayleigh quotient used
    for the Ritz vectors of Section 5.1)."""
    _, _, Op, r = _problem(seed=12)
    m = 15
    res = recycled_minres(lambda v: Op @ v, r, None, 0.0, m, keep=m, reorth=True)
    V = res.V
    assert V.shape[1] == m
    np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-13)
    T = lanczos_tridiagonal(res.alphas, res.betas, m)
    np.testing.assert_allclose(V.T @ Op @ V, T, atol=1e-11 * np.linalg.norm(Op, 2))


def test_zero_rhs_and_zero_iterations():
    _, _, Op, r = _problem()
    res = recycled_minres(lambda v: Op @ v, np.zeros_like(r), None, 0.0, 10)
    assert res.iters == 0 and np.all(res.xm == 0)
    res = recycled_minres(lambda v: Op @ v, r, None, 0.0, 0)
    assert res.iters == 0
