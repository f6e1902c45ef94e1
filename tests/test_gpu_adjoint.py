"""GPU parity of the adjoint solves and the shift / weight gradients (the
autograd backward) against the FP64 oracle, through the C ABI.

The oracle's gradients are pinned by central finite differences of dense
solves (tests/test_oracle_adjoint.py); here the GPU's adjoint solutions must
match the oracle's within kappa * tol (1e-6 relative in FP64, 1e-4 mixed), and
its gradient kernels must reproduce the oracle's formula to rounding."""
import numpy as np
import pytest

import synth
from oracle.adjoint import adjoint_solves, shift_and_weight_gradients
from paper_2306_15049_gb300.recyc import make_desc
from tests.gpu_util import Pair, rel

pytestmark = pytest.mark.gpu


def _forward(pr, w):
    wl = pr.wl
    pr.P.rs_set_weights(pr.t(w))
    pr.P.rs_update_recycle(0)
    X = pr.torch.empty(wl.M, wl.n, dtype=pr.torch.float64, device=pr.dev)
    st = pr.P.rs_solve_shifts(X)
    return X, st


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_solves_and_gradients_match_oracle(precision):
    wl = synth.tiny(40, 36, sigma=1.5, radius=4, M=6, p=8, n_ritz_local=3, seed=31, tol=1e-10)
    pr = Pair(wl, precision=precision)
    w = synth.random_weights(wl.n, 6, lo=1.0, hi=100.0)
    X, _ = _forward(pr, w)
    Xn = pr.n(X)
    G = 2.0 * (Xn - pr.x_true)
    Gt = pr.t(G)
    Lam = pr.torch.empty_like(X)
    stats = pr.P.rs_solve_adjoint(Gt, Lam)
    Lam_o = adjoint_solves(pr.op, pr.gammas, w, G, tol=1e-13)
    tol_l = 1e-6 if precision == 0 else 1e-4
    Ln = pr.n(Lam)
    for l in range(wl.M):
        assert stats[l]["relres_true"] <= wl.tol * (1 + 1e-6), (l, stats[l])
        assert rel(Ln[l], Lam_o[l]) <= tol_l, (l, rel(Ln[l], Lam_o[l]))
    dw = pr.torch.empty(2 * wl.n, dtype=pr.torch.float64, device=pr.dev)
    dg = pr.P.rs_shift_gradients(X, Lam, dw)
    dg_o, dw_o = shift_and_weight_gradients(pr.op, pr.gammas, w, Xn, Lam_o)
    np.testing.assert_allclose(dg, dg_o, rtol=10 * tol_l)
    assert rel(pr.n(dw), dw_o) <= 10 * tol_l


def test_gradient_kernels_reproduce_the_formula_to_rounding():
    wl = synth.tiny(37, 53, M=5, p=4, n_ritz_local=1)
    pr = Pair(wl)
    w = synth.random_weights(wl.n, 2)
    pr.P.rs_set_weights(pr.t(w))
    rng = np.random.default_rng(7)
    X = rng.standard_normal((wl.M, wl.n))
    Lam = rng.standard_normal((wl.M, wl.n))
    dw = pr.torch.empty(2 * wl.n, dtype=pr.torch.float64, device=pr.dev)
    dg = pr.P.rs_shift_gradients(pr.t(X), pr.t(Lam), dw)
    dg_o, dw_o = shift_and_weight_gradients(pr.op, pr.gammas, w, X, Lam)
    np.testing.assert_allclose(dg, dg_o, rtol=1e-12)
    assert rel(pr.n(dw), dw_o) <= 1e-13


def test_zero_right_hand_sides_and_the_forward_state_are_left_alone():
    """g_l = 0 gives lambda_l = 0; an adjoint solve between two outer steps does
    not change the next step's results (deterministic kernels: bit-identical)."""
    wl = synth.C1
    w0 = np.ones(2 * wl.n)
    outs = []
    for with_adjoint in (False, True):
        pr = Pair(wl)
        X, _ = _forward(pr, w0)
        if with_adjoint:
            G = 2.0 * (pr.n(X) - pr.x_true)
            G[3] = 0.0
            Lam = pr.torch.empty_like(X)
            st = pr.P.rs_solve_adjoint(pr.t(G), Lam)
            assert np.all(pr.n(Lam)[3] == 0.0) and st[3]["iters"] == 0
        w1 = synth.random_weights(wl.n, 3, lo=1.0, hi=1000.0)
        pr.P.rs_set_weights(pr.t(w1))
        pr.P.rs_update_recycle(1)
        X1 = pr.torch.empty(wl.M, wl.n, dtype=pr.torch.float64, device=pr.dev)
        pr.P.rs_solve_shifts(X1)
        outs.append(pr.n(X1))
    assert np.array_equal(outs[0], outs[1])


def test_autograd_function_gives_the_oracle_gradient():
    import torch

    from paper_2306_15049_gb300.autograd import solve_shifts
    wl = synth.tiny(32, 30, sigma=1.5, radius=4, M=5, p=8, n_ritz_local=3, seed=41, tol=1e-10)
    pr = Pair(wl)
    w = synth.random_weights(wl.n, 9, lo=1.0, hi=50.0)

    def mk(g):
        return make_desc(wl.height, wl.width, wl.sigma, wl.radius, g, wl.tol, 20000, wl.p, wl.a_ritz,
                         wl.b_ritz, wl.n_ritz_local, wl.vnew_cap, wl.I_split, wl.i1, wl.i2,
                         wl.i_star, wl.l_c, wl.J_L, wl.J_R)
    gam = torch.tensor(pr.gammas, dtype=torch.float64, requires_grad=True)
    wt = pr.t(w).requires_grad_(True)
    xt = pr.t(pr.x_true)
    X = solve_shifts(gam, wt, pr.d_gpu, mk)
    loss = ((X - xt) ** 2).sum()
    loss.backward()
    Xn = X.detach().cpu().numpy()
    Lam_o = adjoint_solves(pr.op, pr.gammas, w, 2.0 * (Xn - pr.x_true), tol=1e-13)
    dg_o, dw_o = shift_and_weight_gradients(pr.op, pr.gammas, w, Xn, Lam_o)
    np.testing.assert_allclose(gam.grad.numpy(), dg_o, rtol=1e-5)
    assert rel(wt.grad.cpu().numpy(), dw_o) <= 1e-5
