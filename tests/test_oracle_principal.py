"""Pins of the oracle's principal-space construction and local-space assembly.

Each check is against something the oracle does not compute itself: a Krylov
basis built here from a QR of the normalised power sequence, Rayleigh-Ritz on
that basis, dense solves of the systems the paper writes down, the identity
that defines delta x, and the columns the paper lists for each space.

* Section 5.1, Eq. widetildeU: U~ = [x^(0,i1), x^(0,i2), V_i1, V_i2], with V_i1
  all a Ritz vectors of the gamma_i1 Krylov space and V_i2 the b' Ritz vectors
  of the gamma_i2 Krylov space with the smallest Ritz values.
* Section 5.2, Eqs. delta and tildeUupdate: (A / gamma + E_k) dx =
  (E_k - E_{k-1}) x^(k-1,l_c), dx = x^(k-1,l_c) - x^(k,l_c), and
  U~ = [V_i1, V^(new), x^(k-1,1..M)] with V^(new) = [dx, v_1..v_m].
* Section 5.3, Algorithm updatelocal and its footnote: U~_l = [W, g^(k-1,l),
  g^(k,l-1)], the older g left out when |cos| of the two exceeds 0.99; the
  batched variant takes g^(k-1,l-1) in place of g^(k,l-1).
"""
import numpy as np
import pytest

import synth
from oracle.operator import Operator, make_data
from oracle.recycle import (Params, State, init_principal, local_columns, local_corrections,
                            outer_step, update_principal)
from tests.dense import operator_dense


def _problem(h=7, w=6, seed=11, M=6, p=8, tol=1e-11):
    wl = synth.tiny(h, w, sigma=1.0, radius=2, M=M, p=p, seed=seed, tol=tol)
    op = Operator(h, w, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(h, w, wl.seed)
    z = synth.noise_direction(h, w, wl.seed)
    _, b = make_data(op, x, z, wl.eta)
    return wl, op, b


def _krylov_basis(Op, r, m):
    """Orthonormal basis of span{r, Op r, .., Op^(m-1) r} from a QR of the
    normalised power sequence (independent of any Lanczos recurrence)."""
    cols = [r / np.linalg.norm(r)]
    for _ in range(m - 1):
        v = Op @ cols[-1]
        cols.append(v / np.linalg.norm(v))
    Q, R = np.linalg.qr(np.stack(cols, axis=1))
    assert np.min(np.abs(np.diag(R))) > 1e-8      # the sequence is far from dependent
    return Q


def _projector_distance(A, B):
    PA = A @ np.linalg.pinv(A)
    PB = B @ np.linalg.pinv(B)
    return np.linalg.norm(PA - PB, 2)


def test_init_principal_takes_all_ritz_vectors_of_i1_and_the_smallest_of_i2():
    wl, op, b = _problem()
    prm = Params.from_workload(wl)
    a, bp = prm.a_ritz, prm.b_ritz
    assert a == 4 and bp == 2          # 2 smallest of 4: disjoint from the 2 largest
    gammas = wl.gammas()
    w = synth.random_weights(op.n, 3)
    Ut, V_i1, _ = init_principal(op, b, gammas, w, prm)
    assert Ut.shape[1] == 2 + a + bp
    _, _, Op1 = operator_dense(op.height, op.width, op.taps, w, gammas[prm.i1 - 1])
    _, _, Op2 = operator_dense(op.height, op.width, op.taps, w, gammas[prm.i2 - 1])
    # x^(0,i1), x^(0,i2): the two systems solved to tolerance
    for col, Op in ((0, Op1), (1, Op2)):
        x = np.linalg.solve(Op, b)
        assert np.linalg.norm(Ut[:, col] - x) <= 10 * np.linalg.cond(Op) * prm.tol * np.linalg.norm(x)
    # V_i1: all a Ritz vectors of Op1 on K_a(Op1, b): the whole Krylov space, with
    # V^T Op1 V diagonal and equal to the Ritz values
    np.testing.assert_array_equal(Ut[:, 2:2 + a], V_i1)
    Q1 = _krylov_basis(Op1, b, a)
    assert _projector_distance(V_i1, Q1) < 1e-8
    np.testing.assert_allclose(V_i1.T @ V_i1, np.eye(a), atol=1e-10)
    theta1 = np.linalg.eigvalsh(Q1.T @ Op1 @ Q1)
    H1 = V_i1.T @ Op1 @ V_i1
    np.testing.assert_allclose(np.sort(np.diag(H1)), theta1, rtol=1e-8)
    assert np.linalg.norm(H1 - np.diag(np.diag(H1))) < 1e-8 * np.linalg.norm(H1)
    # V_i2: the b' Ritz vectors of Op2 on K_a(Op2, b) with the smallest Ritz values
    Q2 = _krylov_basis(Op2, b, a)
    theta2, S2 = np.linalg.eigh(Q2.T @ Op2 @ Q2)
    assert theta2[bp] - theta2[bp - 1] > 1e-6 * theta2[-1]     # a clear split
    V_i2 = Ut[:, 2 + a:]
    assert _projector_distance(V_i2, Q2 @ S2[:, :bp]) < 1e-6
    assert _projector_distance(V_i2, Q2 @ S2[:, -bp:]) > 0.5


def _update_case():
    wl, op, b = _problem(seed=13, M=5, p=8, tol=1e-12)
    prm = Params.from_workload(wl)
    prm.vnew_cap = 2 * op.n          # Eq. delta solved to tolerance, not capped
    gammas = wl.gammas()
    w_prev = np.ones(2 * op.n)       # E_{k-1} = L^T L
    w = synth.random_weights(op.n, 6)
    X_prev = np.stack([np.linalg.solve(operator_dense(op.height, op.width, op.taps, w_prev, g)[2], b)
                       for g in gammas])
    V_i1 = np.linalg.qr(np.random.default_rng(2).standard_normal((op.n, 3)))[0]
    return wl, op, b, prm, gammas, w, w_prev, X_prev, V_i1


def test_update_principal_solves_eq_delta_and_orders_the_blocks():
    wl, op, b, prm, gammas, w, w_prev, X_prev, V_i1 = _update_case()
    Ut, _ = update_principal(op, b, gammas, w, w_prev, V_i1, X_prev, prm)
    a, M = V_i1.shape[1], len(gammas)
    np.testing.assert_array_equal(Ut[:, :a], V_i1)
    np.testing.assert_array_equal(Ut[:, Ut.shape[1] - M:], X_prev.T)
    dx = Ut[:, a]
    g = gammas[prm.l_c - 1]
    A, Ek, _ = operator_dense(op.height, op.width, op.taps, w, 0.0)
    _, Ekm1, _ = operator_dense(op.height, op.width, op.taps, w_prev, 0.0)
    xc = X_prev[prm.l_c - 1]
    # Eq. delta as printed
    dx_dense = np.linalg.solve(A / g + Ek, (Ek - Ekm1) @ xc)
    assert np.linalg.norm(dx - dx_dense) <= 1e-6 * np.linalg.norm(dx_dense)
    # the definition dx = x^(k-1,l_c) - x^(k,l_c): x^(k-1,l_c) - dx solves step k
    xk = np.linalg.solve(A + g * Ek, b)
    assert np.linalg.norm((xc - dx) - xk) <= 1e-6 * np.linalg.norm(xk)
    # V^(new)'s Lanczos vectors span the Krylov space of A + gamma E_k from the rhs
    V = Ut[:, a + 1:a + 5]
    Q = _krylov_basis(A + g * Ek, (Ek - Ekm1) @ xc, 4)
    assert _projector_distance(V, Q) < 1e-7


def test_local_columns_angle_rule_just_below_and_just_above():
    rng = np.random.default_rng(5)
    n = 50
    u, v = np.linalg.qr(rng.standard_normal((n, 2)))[0].T
    for cos, both in ((0.9899, True), (0.9901, False)):
        g_old = 3.0 * u
        g_new = -0.5 * (cos * u + np.sqrt(1 - cos * cos) * v)   # |cos angle| = cos
        cols = local_columns(g_old, g_new)
        if both:
            assert len(cols) == 2
            np.testing.assert_array_equal(cols[0], g_old)
            np.testing.assert_array_equal(cols[1], g_new)
        else:
            assert len(cols) == 1
            np.testing.assert_array_equal(cols[0], g_new)    # g^(k,l-1) survives
    np.testing.assert_array_equal(local_columns(None, v)[0], v)
    np.testing.assert_array_equal(local_columns(u, None)[0], u)
    assert len(local_columns(np.zeros(n), v)) == 1
    assert local_columns(None, None) == []


def test_local_corrections_pick_the_paper_vectors():
    M, n = 5, 7
    G_prev = np.arange(M * n, dtype=float).reshape(M, n) + 1.0
    G_cur = -np.arange(M * n, dtype=float).reshape(M, n) - 1.0
    for l in range(M):
        go, gn = local_corrections(l, 2, G_prev, G_cur, False)
        np.testing.assert_array_equal(go, G_prev[l])                   # g^(k-1,l)
        if l == 0:
            assert gn is None
        else:
            np.testing.assert_array_equal(gn, G_cur[l - 1])            # g^(k,l-1)
        go, gn = local_corrections(l, 2, G_prev, G_cur, True)
        np.testing.assert_array_equal(go, G_prev[l])
        if l == 0:
            assert gn is None
        else:
            np.testing.assert_array_equal(gn, G_prev[l - 1])           # g^(k-1,l-1)
        go, gn = local_corrections(l, 0, None, G_cur, False)
        assert go is None and (gn is None if l == 0 else np.array_equal(gn, G_cur[l - 1]))
        assert local_corrections(l, 0, None, G_cur, True) == (None, None)


@pytest.mark.parametrize("batched", [False, True])
def test_outer_step_local_spaces_are_the_listed_columns(batched):
    wl, op, b = _problem(h=9, w=8, seed=21, M=6, p=8, tol=1e-10)
    prm = Params.from_workload(wl, batched_local=batched)
    gammas = wl.gammas()
    S = State()
    r0 = outer_step(op, b, gammas, np.ones(2 * op.n), S, prm)
    G_prev = r0.G.copy()
    w1 = synth.random_weights(op.n, 9)
    r1 = outer_step(op, b, gammas, w1, S, prm, record_local=True)
    checked = 0
    for l in range(wl.M):
        got = r1.extra["local_cols"][l]
        if got is None:
            continue
        Wt = r1.extra["WtL"] if (l + 1) <= prm.I_split else r1.extra["WtR"]
        cols = list((r1.Ut @ Wt).T)
        g_old = G_prev[l]
        g_new = None if l == 0 else (G_prev[l - 1] if batched else r1.G[l - 1])
        gs = [g for g in (g_old, g_new) if g is not None and np.linalg.norm(g) > 0]
        if len(gs) == 2:
            c = abs(gs[0] @ gs[1]) / (np.linalg.norm(gs[0]) * np.linalg.norm(gs[1]))
            if c > 0.99:
                gs = [gs[1]]
        expect = np.stack(cols + gs, axis=1)
        if got.shape[1] != expect.shape[1]:
            continue                  # a column dropped as dependent: compared elsewhere
        np.testing.assert_array_equal(got, expect)
        checked += 1
    assert checked >= wl.M - 2
