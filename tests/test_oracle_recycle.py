"""Pins of the oracle's recycle-space machinery (Sections 4, 5) and outer loop."""
import json
import os

import numpy as np
import pytest

import synth
from oracle.operator import Operator, irn_weights, make_data
from oracle.outer import lcurve_corner, lcurve_points, run, same_lstar_three
from oracle.recycle import (Params, State, interior_ritz, naive_minres, outer_step,
                            principal_guesses, qr_with_drops, stabilize)
from tests.dense import operator_dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _orthonormal(n, k, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, k)))
    return q


def _same_span(A, B, tol):
    PA = A @ np.linalg.pinv(A)
    PB = B @ np.linalg.pinv(B)
    return np.linalg.norm(PA - PB, 2) < tol


def test_stabilize_drops_near_dependent_columns_at_ratio_1e10():
    n = 60
    Q = _orthonormal(n, 6, 0)
    q1, q2, q3, q4, q5, q6 = Q.T
    cols = [q1, q2, 3.0 * q3,
            q1 + 1e-12 * q4,            # sigma ~ 7e-13 after normalisation: dropped
            2.0 * q2,                   # exact duplicate direction: dropped
            q3 + 1e-7 * q5,             # sigma ~ 7e-8: kept
            np.zeros(n)]                # zero column: ignored
    Ut = np.stack(cols, axis=1)
    out = stabilize(Ut, p_max=10)
    assert out.shape[1] == 4
    np.testing.assert_allclose(out.T @ out, np.eye(4), atol=1e-14)
    assert _same_span(out, np.stack([q1, q2, q3, q5], axis=1), 1e-6)
    # the cap keeps the largest singular directions
    capped = stabilize(np.stack([q1, q2, q3, q4], axis=1) * np.array([5.0, 1.0, 1.0, 1.0]), p_max=2)
    assert capped.shape[1] == 2


def _tiny_setup(h=10, w=9, seed=4, M=6):
    wl = synth.tiny(h, w, M=M, seed=seed)
    op = Operator(h, w, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(h, w, wl.seed)
    z = synth.noise_direction(h, w, wl.seed)
    d, b = make_data(op, x, z, wl.eta)
    return wl, op, d, b


def test_principal_guess_is_the_least_squares_minimiser_over_the_principal_space():
    """Section 4.1: x0 = argmin_{x in Range U~} ||b - (A + gamma_l E) x||; the
    residual satisfies the Petrov-Galerkin condition ((A+gamma_l E) U~)^T r0 = 0
    (Eq. orthupdate) and equals the true residual b - (A + gamma_l E) x0."""
    wl, op, d, b = _tiny_setup()
    n = op.n
    wt = synth.random_weights(n, 2)
    Ut = _orthonormal(n, 7, 3)
    AU = np.stack([op.apply_A(Ut[:, j]) for j in range(7)], axis=1)
    EU = np.stack([op.apply_E(Ut[:, j], wt) for j in range(7)], axis=1)
    gammas = wl.gammas()
    C, X0, R0 = principal_guesses(Ut, AU, EU, b, gammas, gammas[2])
    for l, g in enumerate(gammas):
        _, _, Op = operator_dense(op.height, op.width, op.taps, wt, g)
        B = Op @ Ut
        c, *_ = np.linalg.lstsq(B, b, rcond=None)
        np.testing.assert_allclose(X0[l], Ut @ c, rtol=1e-7, atol=1e-9 * np.linalg.norm(Ut @ c))
        np.testing.assert_allclose(R0[l], b - Op @ X0[l], atol=1e-11 * np.linalg.norm(b))
        assert np.linalg.norm(B.T @ R0[l]) < 1e-9 * np.linalg.norm(B) * np.linalg.norm(b)


def test_interior_ritz_on_the_full_space_gives_the_smallest_eigenvectors():
    """Algorithm "interior" with U~ = I: the Ritz pairs are the eigenpairs of
    A + gamma E and the smallest ones are returned."""
    h, w = 5, 6
    op = Operator(h, w, 1.0, 2)
    wt = synth.random_weights(h * w, 8)
    A, E, _ = operator_dense(h, w, op.taps, wt, 0.0)
    for gamma, nJ in [(1e-3, 3), (0.7, 5)]:
        Wt = interior_ritz(A, E, gamma, nJ)
        lam, V = np.linalg.eigh(A + gamma * E)
        for j in range(nJ):
            assert abs(abs(Wt[:, j] @ V[:, j]) - 1.0) < 1e-8
        np.testing.assert_allclose(np.diag(Wt.T @ (A + gamma * E) @ Wt), lam[:nJ], rtol=1e-10, atol=1e-14)


def test_qr_with_drops():
    n = 40
    rng = np.random.default_rng(1)
    a, b_, c = rng.standard_normal((3, n))
    B = np.stack([a, b_, a + 2 * b_ + 1e-12 * c, c, np.zeros(n)], axis=1)
    K, R, kept = qr_with_drops(B)
    assert kept == [0, 1, 3]
    np.testing.assert_allclose(K.T @ K, np.eye(3), atol=1e-14)
    np.testing.assert_allclose(K @ R, B[:, kept], atol=1e-13)


def _check_step(op, b, gammas, wt, res, prm, kappa_factor=20.0):
    for l, g in enumerate(gammas):
        _, _, Op = operator_dense(op.height, op.width, op.taps, wt, g)
        x = np.linalg.solve(Op, b)
        r_true = np.linalg.norm(b - Op @ res.X[l]) / np.linalg.norm(b)
        assert r_true <= prm.tol * 1.01, (l, r_true)
        assert abs(r_true - res.relres_true[l]) <= 1e-12
        kappa = np.linalg.cond(Op)
        err = np.linalg.norm(res.X[l] - x) / np.linalg.norm(x)
        assert err <= kappa_factor * kappa * prm.tol, (l, err, kappa)
    np.testing.assert_allclose(res.Ut.T @ res.Ut, np.eye(res.nc), atol=1e-12)


def test_outer_steps_solve_every_shift_to_tolerance():
    wl, op, d, b = _tiny_setup(h=10, w=9)
    prm = Params.from_workload(wl)
    gammas = wl.gammas()
    S = State()
    w0 = np.ones(2 * op.n)
    r0 = outer_step(op, b, gammas, w0, S, prm)
    _check_step(op, b, gammas, w0, r0, prm)
    assert r0.nc <= prm.p
    w1 = irn_weights(op, r0.X[2], wl.beta)
    r1 = outer_step(op, b, gammas, w1, S, prm)
    _check_step(op, b, gammas, w1, r1, prm)
    assert S.k == 1


def test_batched_local_variant_also_solves_to_tolerance():
    wl, op, d, b = _tiny_setup(h=8, w=11, seed=9)
    prm = Params.from_workload(wl, batched_local=True)
    gammas = wl.gammas()
    S = State()
    w0 = np.ones(2 * op.n)
    _check_step(op, b, gammas, w0, outer_step(op, b, gammas, w0, S, prm), prm)
    w1 = synth.random_weights(op.n, 5)
    _check_step(op, b, gammas, w1, outer_step(op, b, gammas, w1, S, prm), prm)


def test_iteration_override_runs_exactly_that_many_steps():
    wl, op, d, b = _tiny_setup()
    prm = Params.from_workload(wl)
    S = State()
    w0 = np.ones(2 * op.n)
    res = outer_step(op, b, wl.gammas(), w0, S, prm, iters_override=[3] * wl.M)
    assert list(res.iters) == [3] * wl.M


def test_naive_minres_matches_dense_solves():
    wl, op, d, b = _tiny_setup(h=7, w=7)
    wt = synth.random_weights(op.n, 1)
    X, its = naive_minres(op, b, wl.gammas(), wt, 1e-11, 10000)
    for l, g in enumerate(wl.gammas()):
        _, _, Op = operator_dense(op.height, op.width, op.taps, wt, g)
        x = np.linalg.solve(Op, b)
        assert np.linalg.norm(X[l] - x) / np.linalg.norm(x) < 10 * np.linalg.cond(Op) * 1e-11


def test_lcurve_corner_on_a_constructed_l_shape():
    # vertical arm, then a corner at index 3, then a horizontal arm
    rho = np.exp([0.0, 0.01, 0.02, 0.05, 1.0, 2.0, 3.0])
    eta = np.exp([3.0, 2.0, 1.0, 0.05, 0.02, 0.01, 0.0])
    assert lcurve_corner(rho, eta) == 3
    # an exactly symmetric pair of corners: the smaller index wins
    rho = np.exp([0.0, 0.0, 1.0, 1.0, 2.0])
    eta = np.exp([2.0, 1.0, 1.0, 0.0, 0.0])
    assert lcurve_corner(rho, eta) == 1
    assert same_lstar_three([4, 2, 2, 2]) and not same_lstar_three([2, 2, 3])


def test_lcurve_points_match_their_definition():
    wl, op, d, b = _tiny_setup(h=6, w=5)
    X = np.random.default_rng(3).standard_normal((3, op.n))
    wt = synth.random_weights(op.n, 4)
    rho, eta = lcurve_points(op, X, d, wt)
    from tests.dense import blur_dense, grad_dense
    H, L = blur_dense(6, 5, op.taps), grad_dense(6, 5)
    for l in range(3):
        assert abs(rho[l] - np.linalg.norm(H @ X[l] - d)) < 1e-12
        assert abs(eta[l] - np.linalg.norm(np.sqrt(wt) * (L @ X[l]))) < 1e-12


def test_full_run_small_workload_converges_every_system():
    wl, op, d, b = _tiny_setup(h=12, w=12, M=6)
    prm = Params.from_workload(wl)
    steps, lstars = run(op, b, d, wl.gammas(), prm, 3, wl.beta)
    assert len(steps) == 3 and len(lstars) == 3
    for s in steps:
        assert np.all(s.relres_true <= prm.tol * 1.01)


def test_paper_index_table_reading():
    """The index reading I = round(0.75 M), i2 = i* = M/2, J_L = I, J_R = M - 1
    reproduces the choices printed for the paper's examples (golden fixture)."""
    with open(os.path.join(GOLDEN, "paper_index_choices.json")) as f:
        gold = json.load(f)
    for ex in gold["examples"]:
        wl = synth.Workload("x", 8, 8, 1.0, 1, 0.01, ex["M"], -4, 0, 1, 10, 4)
        for key in ex["reproduced_by_reading"]:
            assert getattr(wl, key) == ex[key], (ex["name"], key)
