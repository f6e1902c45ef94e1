"""Pins of the oracle's projected (recycled) CG: with no recycle space it is
textbook CG (Hestenes-Stiefel, written out here) step by step; with a recycle
space its residual is orthogonal to K and to the Krylov basis (Galerkin
condition), consecutive residuals are mutually orthogonal, and the correction
equals the dense Galerkin solution over the explicit basis [U, V_m]."""
import numpy as np

from oracle.minres import recycled_cg
from tests.dense import operator_dense


def _spd(n=40, seed=0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.logspace(-2, 1, n)
    return (Q * lam) @ Q.T, rng.standard_normal(n)


def test_without_recycling_it_is_textbook_cg():
    A, b = _spd()
    for m in (1, 3, 7, 15):
        res = recycled_cg(lambda v: A @ v, b, None, 0.0, m)
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        for _ in range(m):
            Ap = A @ p
            a = (r @ r) / (p @ Ap)
            x = x + a * p
            rn = r - a * Ap
            p = rn + ((rn @ rn) / (r @ r)) * p
            r = rn
        # the two forms of CG differ only by rounding (condition number 1e3 here)
        assert np.linalg.norm(res.xm - x) <= 1e-9 * np.linalg.norm(x), m
        assert abs(res.eta_hist[-1] - np.linalg.norm(r)) <= 1e-9 * np.linalg.norm(b)


def _recycled_setup(seed=3):
    from oracle.operator import Operator
    h, w = 7, 6
    op = Operator(h, w, 1.2, 2)
    rng = np.random.default_rng(seed)
    wt = rng.uniform(0.5, 3.0, 2 * op.n)
    _, _, Op = operator_dense(h, w, op.taps, wt, 0.05)
    U = rng.standard_normal((op.n, 3))
    K, R = np.linalg.qr(Op @ U)
    U = U @ np.linalg.inv(R)                  # K = Op U, K^T K = I
    r = rng.standard_normal(op.n)
    return Op, U, K, r


def test_recycled_cg_galerkin_conditions_and_dense_solution():
    Op, U, K, r = _recycled_setup()
    m = 6
    res = recycled_cg(lambda v: Op @ v, r, K, 0.0, m)
    g = res.xm + U @ res.z
    resid = r - Op @ g
    assert np.linalg.norm(K.T @ resid) < 1e-10 * np.linalg.norm(r)
    # the Krylov basis of (I - K K^T) Op from (I - K K^T) r
    P = np.eye(len(r)) - K @ K.T
    vs = [P @ r]
    for _ in range(m - 1):
        vs.append(P @ (Op @ vs[-1]))
    V, _ = np.linalg.qr(np.stack(vs, axis=1))
    assert np.linalg.norm(V.T @ resid) < 1e-9 * np.linalg.norm(r)
    # dense Galerkin solution over [U, V]: find g in span with [K, V]^T (r - Op g) = 0
    B = np.concatenate([U, V], axis=1)
    W = np.concatenate([K, V], axis=1)
    c = np.linalg.solve(W.T @ Op @ B, W.T @ r)
    np.testing.assert_allclose(g, B @ c, rtol=1e-8, atol=1e-10 * np.linalg.norm(B @ c))
    assert abs(res.eta_hist[-1] - np.linalg.norm(resid)) <= 1e-8 * np.linalg.norm(r)


def test_recycled_cg_residuals_are_mutually_orthogonal_and_it_converges():
    Op, U, K, r = _recycled_setup(5)
    resids = []
    for m in range(1, 8):
        res = recycled_cg(lambda v: Op @ v, r, K, 0.0, m)
        resids.append(r - Op @ (res.xm + U @ res.z))
    R = np.stack(resids, axis=1)
    Rn = R / np.linalg.norm(R, axis=0)
    off = Rn.T @ Rn - np.eye(R.shape[1])
    assert np.max(np.abs(off)) < 1e-8
    res = recycled_cg(lambda v: Op @ v, r, K, 1e-12 * np.linalg.norm(r), 500)
    g = res.xm + U @ res.z
    assert np.linalg.norm(r - Op @ g) <= 1e-11 * np.linalg.norm(r)


def test_outer_step_with_projected_cg_solves_every_shift():
    import synth
    from oracle.operator import Operator, make_data
    from oracle.recycle import Params, State, outer_step
    wl = synth.tiny(16, 14, M=6, p=6, n_ritz_local=2, seed=9, tol=1e-10)
    op = Operator(wl.height, wl.width, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(wl.height, wl.width, wl.seed)
    z = synth.noise_direction(wl.height, wl.width, wl.seed)
    d, b = make_data(op, x, z, wl.eta)
    w = np.ones(2 * op.n)
    ref = outer_step(op, b, wl.gammas(), w, State(), Params.from_workload(wl))
    prm = Params.from_workload(wl)
    prm.inner = "cg"
    res = outer_step(op, b, wl.gammas(), w, State(), prm)
    assert np.all(res.relres_true <= wl.tol * (1 + 1e-6))
    for l in range(wl.M):
        assert np.linalg.norm(res.X[l] - ref.X[l]) <= 1e-6 * np.linalg.norm(ref.X[l])
