"""Pins of the oracle's operator against dense matrices and closed forms.

The shifted operator of Eq. (blkeqn) / Eq. (shift): A = H^T H, E = L^T W L.
"""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle.operator import Operator, gaussian_taps, gazzola_weights, irn_weights, make_data
from tests.dense import blur_dense, grad_dense, operator_dense, toeplitz_dense

SIZES = [(8, 8), (7, 11), (12, 20), (1, 9), (5, 3)]


def test_taps_are_a_normalised_sampled_gaussian():
    for sigma, r in [(1.5, 4), (2.5, 8), (4.0, 12), (1.0, 2)]:
        g = gaussian_taps(sigma, r)
        assert g.shape == (2 * r + 1,)
        assert abs(g.sum() - 1.0) < 1e-15
        np.testing.assert_allclose(g, g[::-1], rtol=0, atol=0)
        # log g is a parabola with second difference -1/sigma^2
        dd = np.diff(np.log(g), 2)
        np.testing.assert_allclose(dd, -1.0 / sigma ** 2, rtol=1e-12)
    # with a wide window the second moment of the sampled Gaussian is sigma^2
    g = gaussian_taps(1.3, 12)
    a = np.arange(-12, 13)
    assert abs(np.sum(a * a * g) - 1.3 ** 2) < 1e-8


@pytest.mark.parametrize("hw", SIZES)
@pytest.mark.parametrize("radius", [1, 2, 5])
def test_blur_and_adjoint_match_dense_kronecker(hw, radius):
    h, w = hw
    rng = np.random.default_rng(h * 100 + w + radius)
    op = Operator(h, w, 1.2, radius)
    # Kronecker form H = T_h (x) T_w (row-major vectorisation)
    Hk = np.kron(toeplitz_dense(h, op.taps), toeplitz_dense(w, op.taps))
    Hd = blur_dense(h, w, op.taps)
    np.testing.assert_allclose(Hk, Hd, rtol=0, atol=1e-15)
    x = rng.standard_normal(h * w)
    np.testing.assert_allclose(op.blur(x), Hd @ x, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(op.blur_adjoint(x), Hd.T @ x, rtol=1e-13, atol=1e-14)


def test_blur_adjoint_is_the_transpose_for_asymmetric_taps():
    # a transposed-operand mistake is invisible with symmetric taps; use random ones
    h, w, r = 6, 9, 3
    rng = np.random.default_rng(5)
    op = Operator(h, w, 1.0, r)
    op.taps = rng.standard_normal(2 * r + 1)
    Hd = blur_dense(h, w, op.taps)
    x = rng.standard_normal(h * w)
    np.testing.assert_allclose(op.blur(x), Hd @ x, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(op.blur_adjoint(x), Hd.T @ x, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("hw", SIZES)
def test_gradient_and_adjoint_match_dense(hw):
    h, w = hw
    rng = np.random.default_rng(h + 31 * w)
    op = Operator(h, w, 1.0, 1)
    L = grad_dense(h, w)
    x = rng.standard_normal(h * w)
    q = rng.standard_normal(2 * h * w)
    np.testing.assert_allclose(op.grad(x), L @ x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(op.grad_adjoint(q), L.T @ q, rtol=0, atol=1e-13)
    # null space of L is exactly the constants (Section 3.1)
    np.testing.assert_allclose(op.grad(np.ones(h * w)), 0.0, atol=0)
    if h * w > 1:
        assert np.linalg.matrix_rank(L) == h * w - 1


@pytest.mark.parametrize("hw", [(8, 8), (7, 11), (12, 20)])
def test_shifted_operator_matches_dense_and_is_spd(hw):
    h, w = hw
    rng = np.random.default_rng(77 + h)
    op = Operator(h, w, 1.0, 2)
    wt = synth.random_weights(h * w, 3)
    for gamma in [1e-6, 1e-3, 0.5, 10.0]:
        A, E, Op = operator_dense(h, w, op.taps, wt, gamma)
        x = rng.standard_normal(h * w)
        np.testing.assert_allclose(op.apply_A(x), A @ x, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(op.apply_E(x, wt), E @ x, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(op.apply(x, gamma, wt), Op @ x, rtol=1e-12, atol=1e-12)
        y = rng.standard_normal(h * w)
        lhs = y @ op.apply(x, gamma, wt)
        rhs = x @ op.apply(y, gamma, wt)
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)
        np.linalg.cholesky(Op)          # SPD for gamma > 0


def test_generalized_eigen_closed_form():
    """Section 3.1, Eq. (x_gamma): E V = A V diag(mu), V^T A V = I,
    x_gamma = sum_j v_j dtilde_j / (1 + gamma mu_j), dtilde = V^T b."""
    h, w = 6, 7
    op = Operator(h, w, 0.9, 2)
    wt = synth.random_weights(h * w, 11)
    A, E, _ = operator_dense(h, w, op.taps, wt, 0.0)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(h * w)
    mu, V = scipy.linalg.eigh(E, A)
    np.testing.assert_allclose(V.T @ A @ V, np.eye(h * w), atol=1e-8)
    assert np.min(np.abs(mu)) < 1e-8 * np.max(mu)      # mu_n = 0: L has a null space
    dt = V.T @ b
    for gamma in [1e-4, 1e-2, 1.0, 30.0]:
        x_closed = V @ (dt / (1.0 + gamma * mu))
        x_dir = np.linalg.solve(A + gamma * E, b)
        np.testing.assert_allclose(x_closed, x_dir, rtol=1e-7, atol=1e-9 * np.linalg.norm(x_dir))
    # Eq. (compare): the difference of two solutions
    ga, gb = 1e-3, 1e-1
    diff = V @ ((gb - ga) * mu / ((1 + gb * mu) * (1 + ga * mu)) * dt)
    np.testing.assert_allclose(diff, np.linalg.solve(A + ga * E, b) - np.linalg.solve(A + gb * E, b),
                               rtol=1e-6, atol=1e-9)


def test_irn_weights_closed_form_on_a_step_edge():
    h, w, beta = 4, 6, 1e-3
    op = Operator(h, w, 1.0, 1)
    X = np.zeros((h, w))
    X[:, 3:] = 1.0                       # vertical edge between columns 2 and 3
    wt = irn_weights(op, X.reshape(-1), beta)
    wx = wt[:h * w].reshape(h, w)
    wy = wt[h * w:].reshape(h, w)
    expect_x = np.full((h, w), 1.0 / beta)
    expect_x[:, 2] = 1.0 / np.sqrt(1.0 + beta ** 2)
    np.testing.assert_allclose(wx, expect_x, rtol=1e-15)
    np.testing.assert_allclose(wy, 1.0 / beta, rtol=1e-15)


def test_gazzola_weights_closed_form():
    h, w = 3, 4
    op = Operator(h, w, 1.0, 1)
    X = np.zeros((h, w))
    X[:, 2:] = 2.0
    d0 = np.ones(2 * h * w)
    dnew = gazzola_weights(op, X.reshape(-1), d0, 2.0)
    # |q| / ||q||_inf is 1 on the edge, 0 elsewhere -> weight 0 on the edge, 1 elsewhere
    qx_edge = np.zeros((h, w))
    qx_edge[:, 1] = 1.0
    expect = 1.0 - np.concatenate([qx_edge.reshape(-1), np.zeros(h * w)])
    np.testing.assert_allclose(dnew, expect)
    # cumulative: D_2 = diag(w) D_1
    d1 = np.full(2 * h * w, 0.5)
    np.testing.assert_allclose(gazzola_weights(op, X.reshape(-1), d1, 2.0), 0.5 * expect)


def test_make_data_noise_level():
    wl = synth.tiny(16, 12)
    op = Operator(wl.height, wl.width, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(wl.height, wl.width, wl.seed)
    z = synth.noise_direction(wl.height, wl.width, wl.seed)
    d, b = make_data(op, x, z, 0.05)
    hx = blur_dense(wl.height, wl.width, op.taps) @ x.reshape(-1)
    assert abs(np.linalg.norm(d - hx) / np.linalg.norm(hx) - 0.05) < 1e-13
    np.testing.assert_allclose(b, blur_dense(wl.height, wl.width, op.taps).T @ d, rtol=1e-12)
