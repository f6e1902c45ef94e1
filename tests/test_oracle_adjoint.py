"""Pins of the oracle's adjoint gradients: central finite differences (FP64,
relative step 1e-6) of the loss sum_l ||x_l - x_true||^2 with x_l from dense
Cholesky solves built from the definitions (tests/dense.py), with respect to
every shift and to a sample of the 2n weights; and the adjoint solutions
against dense solves."""
import numpy as np
import scipy.linalg as sla

import synth
from oracle.adjoint import adjoint_solves, shift_and_weight_gradients
from oracle.operator import Operator, make_data
from tests.dense import operator_dense


def _setup(h=7, w=6, M=4, seed=3):
    wl = synth.tiny(h, w, sigma=1.2, radius=2, M=M, seed=seed)
    op = Operator(h, w, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(h, w, wl.seed).reshape(-1)
    z = synth.noise_direction(h, w, wl.seed)
    d, b = make_data(op, x.reshape(h, w), z, 0.02)
    wt = synth.random_weights(op.n, 5, lo=0.3, hi=30.0)
    return op, x, b, wl.gammas(), wt


def _loss(op, b, gammas, wt, x_true):
    tot = 0.0
    for g in gammas:
        _, _, Op = operator_dense(op.height, op.width, op.taps, wt, g)
        xl = sla.cho_solve(sla.cho_factor(Op), b)
        tot += np.sum((xl - x_true) ** 2)
    return tot


def test_adjoint_solves_match_dense_solves():
    op, x_true, b, gammas, wt = _setup()
    G = np.random.default_rng(1).standard_normal((len(gammas), op.n))
    Lam = adjoint_solves(op, gammas, wt, G)
    for l, g in enumerate(gammas):
        _, _, Op = operator_dense(op.height, op.width, op.taps, wt, g)
        ref = np.linalg.solve(Op, G[l])
        assert np.linalg.norm(Lam[l] - ref) <= 1e-9 * np.linalg.norm(ref)


def test_gradients_match_central_finite_differences():
    op, x_true, b, gammas, wt = _setup()
    X = []
    for g in gammas:
        _, _, Op = operator_dense(op.height, op.width, op.taps, wt, g)
        X.append(np.linalg.solve(Op, b))
    X = np.array(X)
    Lam = adjoint_solves(op, gammas, wt, 2.0 * (X - x_true))
    dgamma, dw = shift_and_weight_gradients(op, gammas, wt, X, Lam)
    for l in range(len(gammas)):
        h = 1e-6 * gammas[l]
        gp, gm = gammas.copy(), gammas.copy()
        gp[l] += h
        gm[l] -= h
        fd = (_loss(op, b, gp, wt, x_true) - _loss(op, b, gm, wt, x_true)) / (2 * h)
        assert abs(fd - dgamma[l]) <= 1e-5 * abs(dgamma[l]) + 1e-12, (l, fd, dgamma[l])
    rng = np.random.default_rng(2)
    n = op.n
    # x- and y-direction weights, including ones on the zero last column / row
    idx = list(rng.choice(2 * n, 8, replace=False)) + [op.width - 1, n + (op.height - 1) * op.width]
    for i in idx:
        h = 1e-6 * wt[i]
        wp, wm = wt.copy(), wt.copy()
        wp[i] += h
        wm[i] -= h
        fd = (_loss(op, b, gammas, wp, x_true) - _loss(op, b, gammas, wm, x_true)) / (2 * h)
        assert abs(fd - dw[i]) <= 1e-5 * max(abs(dw[i]), 1e-3 * np.max(np.abs(dw))), (i, fd, dw[i])


def test_shift_gradient_is_minus_lambda_E_x():
    op, x_true, b, gammas, wt = _setup(h=5, w=8)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((len(gammas), op.n))
    Lam = rng.standard_normal((len(gammas), op.n))
    dgamma, dw = shift_and_weight_gradients(op, gammas, wt, X, Lam)
    A, E, _ = operator_dense(op.height, op.width, op.taps, wt, 0.0)
    for l in range(len(gammas)):
        assert abs(dgamma[l] + Lam[l] @ E @ X[l]) <= 1e-12 * np.linalg.norm(Lam[l]) * np.linalg.norm(E @ X[l])
