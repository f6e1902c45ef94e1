"""Pins of the oracle's oblique-projection initial guesses (Section 7): the
Petrov-Galerkin condition K^T r0 = 0 of Eq. obliqueupdate, the residual identity
||r2||^2 = ||r1||^2 + ||Omega^{-1} Sigma Y_c^T b||^2 of Section 7.1 (built here
from a dense QR and SVD, independently of the oracle's formula), agreement with
the orthogonal projection where the paper says they coincide (at the anchor
shift, and when b lies in Range(Y)), and the two-anchor split of Eq. updates."""
import numpy as np

import synth
from oracle.operator import Operator, make_data
from oracle.recycle import Params, State, oblique_guesses, outer_step, principal_guesses
from tests.dense import operator_dense


def _setup(h=10, w=9, seed=4, M=6, nc=7):
    wl = synth.tiny(h, w, M=M, seed=seed)
    op = Operator(h, w, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(h, w, wl.seed)
    z = synth.noise_direction(h, w, wl.seed)
    d, b = make_data(op, x, z, wl.eta)
    wt = synth.random_weights(op.n, 2)
    Ut, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((op.n, nc)))
    AU = np.stack([op.apply_A(Ut[:, j]) for j in range(nc)], axis=1)
    EU = np.stack([op.apply_E(Ut[:, j], wt) for j in range(nc)], axis=1)
    return wl, op, b, wt, Ut, AU, EU


def test_oblique_residual_is_orthogonal_to_K_and_the_guess_lies_in_range_U():
    wl, op, b, wt, Ut, AU, EU = _setup()
    gammas = wl.gammas()
    ga = gammas[2]
    C, X0, R0 = oblique_guesses(Ut, AU, EU, b, gammas, ga)
    K, _ = np.linalg.qr(AU + ga * EU)
    for l, g in enumerate(gammas):
        _, _, Op = operator_dense(op.height, op.width, op.taps, wt, g)
        np.testing.assert_allclose(R0[l], b - Op @ X0[l], atol=1e-12 * np.linalg.norm(b))
        assert np.linalg.norm(K.T @ R0[l]) < 1e-11 * np.linalg.norm(b), l
        np.testing.assert_allclose(X0[l], Ut @ (Ut.T @ X0[l]), atol=1e-12 * np.linalg.norm(X0[l]))


def test_oblique_and_orthogonal_residuals_obey_the_identity_of_section_7_1():
    """r1 (orthogonal, Eq. orthoP) and r2 (oblique, Eq. oblP): with Y S the QR of
    K + d E U, Y^T K = Phi Omega Psi^T and (I - Y Y^T) K Psi = Y_c Sigma,
    ||r2||^2 = ||r1||^2 + ||Omega^{-1} Sigma Y_c^T b||^2."""
    wl, op, b, wt, Ut, AU, EU = _setup()
    gammas = wl.gammas()
    ga = gammas[2]
    _, _, R1 = principal_guesses(Ut, AU, EU, b, gammas, ga)
    _, _, R2 = oblique_guesses(Ut, AU, EU, b, gammas, ga)
    K, R = np.linalg.qr(AU + ga * EU)
    EUi = EU @ np.linalg.inv(R)
    for l, g in enumerate(gammas):
        Y, _ = np.linalg.qr(K + (g - ga) * EUi)
        Phi, om, PsiT = np.linalg.svd(Y.T @ K)
        YcS = (K - Y @ (Y.T @ K)) @ PsiT.T
        sig = np.linalg.norm(YcS, axis=0)
        Yc = np.where(sig > 1e-14, YcS / np.maximum(sig, 1e-300), 0.0)
        extra = np.linalg.norm((sig / om) * (Yc.T @ b))
        lhs = np.linalg.norm(R2[l]) ** 2
        rhs = np.linalg.norm(R1[l]) ** 2 + extra ** 2
        assert abs(lhs - rhs) <= 1e-9 * lhs, (l, lhs, rhs)
        assert np.linalg.norm(R2[l]) >= np.linalg.norm(R1[l]) * (1 - 1e-12)


def test_oblique_equals_orthogonal_at_the_anchor_and_for_b_in_range():
    wl, op, b, wt, Ut, AU, EU = _setup()
    gammas = wl.gammas()
    for a in (0, 3, 5):
        ga = gammas[a]
        _, X1, R1 = principal_guesses(Ut, AU, EU, b, gammas, ga)
        _, X2, R2 = oblique_guesses(Ut, AU, EU, b, gammas, ga)
        np.testing.assert_allclose(X2[a], X1[a], rtol=1e-9, atol=1e-12 * np.linalg.norm(X1[a]))
    # b = (A + gamma_l E) U~ c lies in Range(Y) for shift l: both residuals vanish
    l = 4
    c = np.arange(1.0, Ut.shape[1] + 1)
    bb = AU @ c + gammas[l] * (EU @ c)
    _, X1, R1 = principal_guesses(Ut, AU, EU, bb, gammas, gammas[1])
    _, X2, R2 = oblique_guesses(Ut, AU, EU, bb, gammas, gammas[1])
    assert np.linalg.norm(R1[l]) < 1e-10 * np.linalg.norm(bb)
    assert np.linalg.norm(R2[l]) < 1e-10 * np.linalg.norm(bb)
    np.testing.assert_allclose(X2[l], Ut @ c, rtol=1e-9)


def test_two_anchor_guesses_split_at_I():
    """Eq. updates: shifts l <= I use the anchor gamma_{I_L}, the others gamma_{I_R};
    at l = I_L and l = I_R the guess is the orthogonal one."""
    wl, op, b, wt, Ut, AU, EU = _setup(M=8)
    gammas = wl.gammas()
    I, IL, IR = 5, 3, 7
    _, X2, R2 = oblique_guesses(Ut, AU, EU, b, gammas, gammas[IL - 1], gammas[IR - 1], I)
    _, XL, _ = oblique_guesses(Ut, AU, EU, b, gammas, gammas[IL - 1])
    _, XR, _ = oblique_guesses(Ut, AU, EU, b, gammas, gammas[IR - 1])
    _, XO, _ = principal_guesses(Ut, AU, EU, b, gammas, gammas[0])
    for l in range(len(gammas)):
        ref = XL[l] if l + 1 <= I else XR[l]
        np.testing.assert_allclose(X2[l], ref, rtol=1e-12, atol=1e-14 * np.linalg.norm(ref))
    for a in (IL, IR):
        np.testing.assert_allclose(X2[a - 1], XO[a - 1], rtol=1e-8, atol=1e-11 * np.linalg.norm(XO[a - 1]))


def test_outer_step_with_oblique_guesses_solves_every_shift():
    wl = synth.tiny(16, 14, M=6, p=6, n_ritz_local=2, seed=9, tol=1e-10)
    op = Operator(wl.height, wl.width, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(wl.height, wl.width, wl.seed)
    z = synth.noise_direction(wl.height, wl.width, wl.seed)
    d, b = make_data(op, x, z, wl.eta)
    w = np.ones(2 * op.n)
    ref = outer_step(op, b, wl.gammas(), w, State(), Params.from_workload(wl))
    for kind in ("oblique", "oblique2"):
        prm = Params.from_workload(wl, guess=kind)
        prm.I_L, prm.I_R = 2, wl.M
        res = outer_step(op, b, wl.gammas(), w, State(), prm)
        assert np.all(res.relres_true <= wl.tol * (1 + 1e-6))
        # the orthogonal guess minimises the residual over Range(U~): never worse
        assert np.all(ref.relres0 <= res.relres0 * (1 + 1e-9))
        for l in range(wl.M):
            assert np.linalg.norm(res.X[l] - ref.X[l]) <= 1e-6 * np.linalg.norm(ref.X[l])
