"""Planted mistakes in the oracle (CPU only): each must make a pin fail.

A plausible slip -- a dropped term, a wrong sign or index, a transposed
operand -- is patched into the oracle for the duration of one test, and the
pin that should catch it is run and expected to fail.
"""
import inspect

import numpy as np
import pytest

import oracle.minres as om
import oracle.operator as oo
import oracle.recycle as orc
from tests import test_oracle_minres as tm
from tests import test_oracle_operator as to
from tests import test_oracle_recycle as tr


def _expect_fail(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_wrong_sign_in_gradient_adjoint_is_caught(monkeypatch):
    good = oo.Operator.grad_adjoint
    monkeypatch.setattr(oo.Operator, "grad_adjoint", lambda self, q: -good(self, q))
    _expect_fail(to.test_gradient_and_adjoint_match_dense, (7, 11))


def test_wrong_boundary_in_blur_is_caught(monkeypatch):
    def periodic(x, taps, axis):
        r = (len(taps) - 1) // 2
        return sum(taps[a + r] * np.roll(x, -a, axis=axis) for a in range(-r, r + 1))
    monkeypatch.setattr(oo, "_toeplitz_apply", periodic)
    _expect_fail(to.test_blur_and_adjoint_match_dense_kronecker, (7, 11), 2)


def test_untransposed_blur_adjoint_is_caught(monkeypatch):
    monkeypatch.setattr(oo.Operator, "blur_adjoint", lambda self, y: self.blur(y))
    _expect_fail(to.test_blur_adjoint_is_the_transpose_for_asymmetric_taps)


def test_dropped_weight_in_E_is_caught(monkeypatch):
    monkeypatch.setattr(oo.Operator, "apply_E", lambda self, x, w: self.grad_adjoint(self.grad(x)))
    _expect_fail(to.test_shifted_operator_matches_dense_and_is_spd, (8, 8))


def _mutated_minres(old, new):
    """recycled_minres with one line of its recurrence replaced."""
    src = inspect.getsource(om.recycled_minres)
    assert old in src
    ns = dict(vars(om))
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns["recycled_minres"]


@pytest.mark.parametrize("old,new", [
    ("eps = sn2 * beta", "eps = sn1 * beta"),                     # wrong rotation index
    ("delta = cs1 * dbar + sn1 * alpha", "delta = cs1 * dbar - sn1 * alpha"),   # wrong sign
    ("d = (v - delta * d1 - eps * d2) / gamma", "d = (v - delta * d1) / gamma"),  # dropped term
])
def test_planted_minres_recurrence_mistakes_are_caught(monkeypatch, old, new):
    monkeypatch.setattr(tm, "recycled_minres", _mutated_minres(old, new))
    _expect_fail(tm.test_plain_minres_matches_scipy_iterates, 12)


def test_dropped_recycle_coupling_is_caught(monkeypatch):
    real = om.recycled_minres

    def no_coupling(op_apply, r, K, tol_abs, maxit, keep=0, reorth=False):
        res = real(op_apply, r, K, tol_abs, maxit, keep, reorth)
        if K is not None:
            res.z = K.T @ r          # forgets - K^T Op V_m y
        return res
    monkeypatch.setattr(tm, "recycled_minres", no_coupling)
    _expect_fail(tm.test_recycled_minres_is_least_squares_over_U_and_Krylov, 3, 6)


def test_dropped_quadratic_term_in_orthupdate_is_caught(monkeypatch):
    real_eye = np.eye

    def guesses_without_N(Ut, AU, EU, b, gammas, gamma_star):
        B = AU + gamma_star * EU
        K, R = np.linalg.qr(B)
        EUi = np.linalg.solve(R.T, EU.T).T
        Mm = K.T @ EUi
        C = np.zeros((Ut.shape[1], len(gammas)))
        X0 = np.zeros((len(gammas), Ut.shape[0]))
        R0 = np.zeros_like(X0)
        for l, gl in enumerate(gammas):
            dl = gl - gamma_star
            Sm = real_eye(Ut.shape[1]) + dl * (Mm + Mm.T)          # no d^2 N
            q = np.linalg.solve(Sm, K.T @ b + dl * EUi.T @ b)
            c = np.linalg.solve(R, q)
            C[:, l], X0[l] = c, Ut @ c
            R0[l] = b - (AU @ c + gl * (EU @ c))
        return C, X0, R0
    monkeypatch.setattr(tr, "principal_guesses", guesses_without_N)
    _expect_fail(tr.test_principal_guess_is_the_least_squares_minimiser_over_the_principal_space)


def test_largest_instead_of_smallest_ritz_vectors_is_caught(monkeypatch):
    def largest(Ah, Eh, gamma, nJ):
        H = Ah + gamma * Eh
        _, Wt = np.linalg.eigh(0.5 * (H + H.T))
        return Wt[:, ::-1][:, :nJ]
    monkeypatch.setattr(tr, "interior_ritz", largest)
    _expect_fail(tr.test_interior_ritz_on_the_full_space_gives_the_smallest_eigenvectors)


def test_stabilize_without_threshold_is_caught(monkeypatch):
    real = orc.stabilize
    monkeypatch.setattr(tr, "stabilize", lambda Ut, p_max, ratio=1e10: real(Ut, p_max, ratio=1e300))
    _expect_fail(tr.test_stabilize_drops_near_dependent_columns_at_ratio_1e10)


def test_oblique_guess_with_a_flipped_shift_difference_is_caught(monkeypatch):
    import tests.test_oracle_oblique as tob
    real = orc.oblique_guesses

    def flipped(Ut, AU, EU, b, gammas, gl, gr=None, I_split=None):
        # d = gamma_a - gamma_l instead of gamma_l - gamma_a
        mirrored = [2 * gl - g for g in gammas]
        C, _, _ = real(Ut, AU, EU, b, mirrored, gl)
        X0 = (Ut @ C).T
        R0 = np.stack([b - (AU @ C[:, l] + g * (EU @ C[:, l])) for l, g in enumerate(gammas)])
        return C, X0, R0
    monkeypatch.setattr(tob, "oblique_guesses", flipped)
    _expect_fail(tob.test_oblique_residual_is_orthogonal_to_K_and_the_guess_lies_in_range_U)


def test_oblique_guess_with_the_orthogonal_right_hand_side_is_caught(monkeypatch):
    import tests.test_oracle_oblique as tob

    def mixed_rhs(Ut, AU, EU, b, gammas, ga, gr=None, I_split=None):
        K, R = np.linalg.qr(AU + ga * EU)
        EUi = np.linalg.solve(R.T, EU.T).T
        nc = Ut.shape[1]
        C = np.zeros((nc, len(gammas)))
        for l, g in enumerate(gammas):
            d = g - ga
            q = np.linalg.solve(np.eye(nc) + d * K.T @ EUi, K.T @ b + d * EUi.T @ b)
            C[:, l] = np.linalg.solve(R, q)
        X0 = (Ut @ C).T
        R0 = np.stack([b - (AU @ C[:, l] + g * (EU @ C[:, l])) for l, g in enumerate(gammas)])
        return C, X0, R0
    monkeypatch.setattr(tob, "oblique_guesses", mixed_rhs)
    _expect_fail(tob.test_oblique_residual_is_orthogonal_to_K_and_the_guess_lies_in_range_U)


def test_weight_gradient_without_the_shift_factor_is_caught(monkeypatch):
    import oracle.adjoint as oa
    import tests.test_oracle_adjoint as tad

    def no_gamma(op, gammas, w, X, Lam):
        dg, _ = oa.shift_and_weight_gradients(op, gammas, w, X, Lam)
        dw = np.zeros_like(w)
        for l in range(len(gammas)):
            dw -= op.grad(Lam[l]) * op.grad(X[l])
        return dg, dw
    monkeypatch.setattr(tad, "shift_and_weight_gradients", no_gamma)
    _expect_fail(tad.test_gradients_match_central_finite_differences)


def test_cg_without_the_sign_of_zeta_is_caught(monkeypatch):
    import tests.test_oracle_cg as tcg
    real = om.recycled_cg

    def wrong(op_apply, r, K, tol_abs, maxit):
        # negate every other correction: zeta_j = +lambda_j zeta_{j-1}
        res = real(op_apply, r, K, tol_abs, maxit)
        if res.iters >= 2:
            res2 = real(op_apply, r, K, tol_abs, res.iters - 1)
            res.xm = 2 * res2.xm - res.xm
        return res
    monkeypatch.setattr(tcg, "recycled_cg", wrong)
    _expect_fail(tcg.test_without_recycling_it_is_textbook_cg)


def _mutated(module, fname, old, new):
    """``module.fname`` with one fragment of its source replaced (a planted slip)."""
    src = inspect.getsource(getattr(module, fname))
    assert old in src, (fname, old)
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns[fname]


@pytest.mark.parametrize("old,new", [
    ("V_i2 = R2[:, :prm.b_ritz]", "V_i2 = R2[:, -prm.b_ritz:]"),      # largest Ritz values of i2
    ("V_i1 = R1", "V_i1 = R2"),                                       # i2's Ritz vectors as V_i1
    ("theta, S = np.linalg.eigh(T)", "theta, S = np.linalg.eigh(T[::-1, ::-1])"),  # reversed T_a
])
def test_planted_init_principal_mistakes_are_caught(monkeypatch, old, new):
    import tests.test_oracle_principal as tp
    monkeypatch.setattr(tp, "init_principal", _mutated(orc, "init_principal", old, new))
    _expect_fail(tp.test_init_principal_takes_all_ritz_vectors_of_i1_and_the_smallest_of_i2)


@pytest.mark.parametrize("old,new", [
    ("(w - w_prev) * op.grad(xc)", "(w_prev - w) * op.grad(xc)"),            # wrong sign of Eq. delta
    ("lambda v: op.apply(v, g, w), rhs", "lambda v: op.apply(v, g, w_prev), rhs"),  # E_{k-1} for E_k
    ("X_prev[prm.l_c - 1]", "X_prev[prm.l_c - 2]"),                           # wrong correction system
    ("[V_i1, Vnew, X_prev.T]", "[Vnew, V_i1, X_prev.T]"),                     # blocks out of order
])
def test_planted_update_principal_mistakes_are_caught(monkeypatch, old, new):
    import tests.test_oracle_principal as tp
    monkeypatch.setattr(tp, "update_principal", _mutated(orc, "update_principal", old, new))
    _expect_fail(tp.test_update_principal_solves_eq_delta_and_orders_the_blocks)


@pytest.mark.parametrize("old,new", [
    ("for g in (g_old, g_new)", "for g in (g_new, g_old)"),      # g's swapped
    ("gcols = [gcols[1]]", "gcols = [gcols[0]]"),                # the older g survives the angle rule
    ("if c > cos_max", "if c > 0.999"),                          # a wrong threshold
])
def test_planted_angle_rule_mistakes_are_caught(monkeypatch, old, new):
    import tests.test_oracle_principal as tp
    monkeypatch.setattr(tp, "local_columns", _mutated(orc, "local_columns", old, new))
    _expect_fail(tp.test_local_columns_angle_rule_just_below_and_just_above)


@pytest.mark.parametrize("old,new", [
    ("g_old = G_prev[l] if", "g_old = G_prev[l - 1] if"),                       # index slip
    ("g_new = G_prev[l - 1] if (k >= 1", "g_new = G_cur[l - 1] if (k >= 1"),    # batched reads this step
    ("g_new = G_cur[l - 1] if l >= 1", "g_new = G_prev[l - 1] if l >= 1"),      # chain from the old step
])
def test_planted_local_correction_mistakes_are_caught(monkeypatch, old, new):
    import tests.test_oracle_principal as tp
    monkeypatch.setattr(tp, "local_corrections", _mutated(orc, "local_corrections", old, new))
    _expect_fail(tp.test_local_corrections_pick_the_paper_vectors)


@pytest.mark.parametrize("batched", [False, True])
def test_planted_local_assembly_mistake_in_the_outer_step_is_caught(monkeypatch, batched):
    import tests.test_oracle_principal as tp
    bad = _mutated(orc, "outer_step", "local_columns(g_old, g_new)", "local_columns(g_new, g_old)")
    monkeypatch.setattr(tp, "outer_step", bad)
    _expect_fail(tp.test_outer_step_local_spaces_are_the_listed_columns, batched)
