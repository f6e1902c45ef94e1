"""GPU parity of the fused shifted-operator kernel (matvec) against the FP64
oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import synth
from tests.gpu_util import Pair, rel

pytestmark = pytest.mark.gpu

CASES = [
    # (height, width, sigma, radius): one tile, odd sizes, several tiles with a
    # ragged tail, radius >= image/2, radius 0 and the workload radii
    (8, 8, 1.0, 2), (37, 53, 1.5, 4), (64, 64, 1.5, 4), (130, 70, 2.5, 8),
    (9, 7, 3.0, 12), (1, 40, 1.0, 3), (33, 1, 1.0, 3), (50, 45, 1.0, 0), (96, 100, 4.0, 12),
]


@pytest.mark.parametrize("h,w,sigma,r", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_operator_modes_match_oracle(h, w, sigma, r, precision):
    wl = synth.tiny(h, w, sigma=sigma, radius=r, M=4, p=4, n_ritz_local=1, seed=h * 7 + w)
    # a random image: the piecewise-constant generator can be empty on 1-pixel-wide images
    pr = Pair(wl, precision=precision, x_image=synth.random_vectors(h * w, 1, h + w)[:, 0])
    n = h * w
    wts = synth.random_weights(n, 3)
    pr.P.rs_set_weights(pr.t(wts))
    rng = np.random.default_rng(h + w)
    x = rng.standard_normal(n)
    xt = pr.t(x)
    y = pr.torch.empty_like(xt)
    y2 = pr.torch.empty_like(xt)
    for wp in ([False, True] if precision == 1 else [False]):
        tol = 1e-13 if not wp else 2e-6
        for gamma in [1e-5, 0.3, 7.0]:
            pr.P.rs_apply_operator(gamma, xt, y, mode=0, working_precision=wp)
            assert rel(pr.n(y), pr.op.apply(x, gamma, wts)) < tol
        pr.P.rs_apply_operator(0.0, xt, y, y2, mode=1, working_precision=wp)
        assert rel(pr.n(y), pr.op.apply_A(x)) < tol
        assert rel(pr.n(y2), pr.op.apply_E(x, wts)) < tol
        pr.P.rs_apply_operator(0.0, xt, y, mode=2, working_precision=wp)
        assert rel(pr.n(y), pr.op.apply_E(x, wts)) < tol
    pr.P.rs_apply_operator(0.0, xt, y, mode=3)
    assert rel(pr.n(y), pr.op.blur(x)) < 1e-13


def test_synthesized_data_and_rhs_match_oracle():
    wl = synth.tiny(40, 33, sigma=2.0, radius=6, M=4, p=4, n_ritz_local=1)
    pr = Pair(wl)
    assert rel(pr.n(pr.d_gpu), pr.d) < 1e-14


def test_irn_weights_match_oracle():
    from oracle.operator import irn_weights
    wl = synth.tiny(29, 31, M=4, p=4, n_ritz_local=1)
    pr = Pair(wl)
    x = synth.piecewise_constant_image(29, 31, 5).reshape(-1) + 1e-3 * np.arange(29 * 31)
    w = pr.torch.empty(2 * 29 * 31, dtype=pr.torch.float64, device=pr.dev)
    pr.P.rs_irn_weights(pr.t(x), 1e-3, w)
    assert rel(pr.n(w), irn_weights(pr.op, x, 1e-3)) < 1e-14


def test_operator_at_full_workload_size():
    """512 x 512, radius 8: every pixel against the oracle's matvec."""
    wl = synth.C2
    pr = Pair(wl)
    n = wl.n
    wts = synth.random_weights(n, 9, lo=1.0, hi=1000.0)
    pr.P.rs_set_weights(pr.t(wts))
    x = synth.piecewise_constant_image(wl.height, wl.width, 77).reshape(-1)
    xt = pr.t(x)
    y = pr.torch.empty_like(xt)
    pr.P.rs_apply_operator(1e-3, xt, y)
    assert rel(pr.n(y), pr.op.apply(x, 1e-3, wts)) < 1e-13


CASES2 = [
    # even radii of the two-pass form: images smaller than the radius, one row or
    # column, ragged tiles, and the workload radii
    (8, 8, 1.0, 4), (9, 7, 3.0, 12), (1, 40, 1.0, 4), (33, 1, 1.0, 6), (37, 53, 1.5, 4),
    (130, 70, 2.5, 8), (70, 130, 3.0, 10), (96, 100, 4.0, 12),
]


@pytest.mark.parametrize("h,w,sigma,r", CASES2)
@pytest.mark.parametrize("precision", [0, 1])
def test_two_pass_operator_matches_oracle(h, w, sigma, r, precision):
    """RS_STENCIL2=1: A as two autocorrelation passes with edge corrections."""
    import os
    old = os.environ.get("RS_STENCIL2")
    os.environ["RS_STENCIL2"] = "1"
    try:
        wl = synth.tiny(h, w, sigma=sigma, radius=r, M=4, p=4, n_ritz_local=1, seed=h * 5 + w)
        pr = Pair(wl, precision=precision, x_image=synth.random_vectors(h * w, 1, h + 2 * w)[:, 0])
    finally:
        if old is None:
            del os.environ["RS_STENCIL2"]
        else:
            os.environ["RS_STENCIL2"] = old
    n = h * w
    wts = synth.random_weights(n, 4)
    pr.P.rs_set_weights(pr.t(wts))
    x = np.random.default_rng(h * w).standard_normal(n)
    xt = pr.t(x)
    y = pr.torch.empty_like(xt)
    y2 = pr.torch.empty_like(xt)
    for wp in ([False, True] if precision == 1 else [False]):
        tol = 1e-13 if not wp else 2e-6
        pr.P.rs_apply_operator(0.3, xt, y, mode=0, working_precision=wp)
        assert rel(pr.n(y), pr.op.apply(x, 0.3, wts)) < tol
        pr.P.rs_apply_operator(0.0, xt, y, y2, mode=1, working_precision=wp)
        assert rel(pr.n(y), pr.op.apply_A(x)) < tol
        assert rel(pr.n(y2), pr.op.apply_E(x, wts)) < tol


@pytest.mark.parametrize("h,w,sigma,r", CASES2)
@pytest.mark.parametrize("precision", [0, 1])
def test_two_float_operator_matches_oracle(h, w, sigma, r, precision):
    """Mode 5: (A + gamma E) x in two-float arithmetic (the true residuals of mixed
    precision), and mode 6: H x alone (the L-curve misfit), within 1e-12 of the
    FP64 oracle, for every even radius of the two-pass form and images smaller
    than the radius."""
    wl = synth.tiny(h, w, sigma=sigma, radius=r, M=4, p=4, n_ritz_local=1, seed=h * 3 + w)
    pr = Pair(wl, precision=precision, x_image=synth.random_vectors(h * w, 1, 2 * h + w)[:, 0])
    n = h * w
    wts = synth.random_weights(n, 5, lo=1.0, hi=300.0)
    pr.P.rs_set_weights(pr.t(wts))
    x = np.random.default_rng(h * w + 1).standard_normal(n)
    xt = pr.t(x)
    y = pr.torch.empty_like(xt)
    for gamma in [1e-6, 0.3, 7.0]:
        pr.P.rs_apply_operator(gamma, xt, y, mode=5)
        assert rel(pr.n(y), pr.op.apply(x, gamma, wts)) < 1e-12, gamma
    # mode 6: the blur H x alone (the misfit of the L-curve)
    pr.P.rs_apply_operator(0.0, xt, y, mode=6)
    assert rel(pr.n(y), pr.op.blur(x)) < 1e-12


def test_two_float_residual_at_full_workload_size():
    """512 x 512, radius 8: a residual b - (A + gamma E) x a billion times smaller
    than (A + gamma E) x keeps its leading digits when the product is taken in
    two-float arithmetic (what the refinement of mixed precision needs)."""
    wl = synth.C2
    pr = Pair(wl, precision=1)
    n = wl.n
    wts = synth.random_weights(n, 11, lo=1.0, hi=1000.0)
    pr.P.rs_set_weights(pr.t(wts))
    x = synth.piecewise_constant_image(wl.height, wl.width, 78).reshape(-1)
    gamma = 1e-4
    ax = pr.op.apply(x, gamma, wts)
    delta = 1e-9 * np.linalg.norm(ax) / np.sqrt(n) * np.random.default_rng(3).standard_normal(n)
    b = ax + delta
    y = pr.torch.empty(n, dtype=pr.torch.float64, device=pr.dev)
    pr.P.rs_apply_operator(gamma, pr.t(x), y, mode=5)
    r_gpu = b - pr.n(y)
    assert rel(pr.n(y), ax) < 1e-13
    assert rel(r_gpu, delta) < 1e-3


def test_two_float_mode_rejects_the_radon_operator():
    from paper_2306_15049_gb300.recyc import RecycError
    wl = synth.tiny(24, 24, M=4, p=4, n_ritz_local=1, radon_angles=12)
    pr = Pair(wl)
    pr.P.rs_set_weights(pr.t(np.ones(2 * wl.n)))
    xt = pr.t(np.ones(wl.n))
    y = pr.torch.empty_like(xt)
    for mode in (5, 6):
        with pytest.raises(RecycError):
            pr.P.rs_apply_operator(0.1, xt, y, mode=mode)


@pytest.mark.parametrize("precision", [0, 1])
def test_lcurve_points_match_oracle_in_both_precisions(precision):
    """Section 2.2's L-curve of given solutions: rho_l = ||H x_l - d|| (the blur in
    two-float arithmetic under mixed precision, in FP64 otherwise) and eta_l =
    ||w^(1/2) .* L x_l|| match the oracle, and so does the corner. The misfit is
    about 1e-2 of ||H x||, so the two-float product (about 2^-44 of ||H x||)
    leaves it about 1e-11 relative; FP32 would leave 1e-5."""
    from oracle.outer import lcurve_corner, lcurve_points
    wl = synth.tiny(70, 130, sigma=3.0, radius=10, M=6, p=4, n_ritz_local=1, seed=5)
    pr = Pair(wl, precision=precision)
    wts = synth.random_weights(wl.n, 9, lo=0.5, hi=50.0)
    pr.P.rs_set_weights(pr.t(wts))
    # solutions near the data at a range of distances: points along an L-shape
    rng = np.random.default_rng(17)
    X = np.stack([pr.x_true + s * rng.standard_normal(wl.n) for s in np.geomspace(1e-3, 1.0, wl.M)])
    rho, eta, ls = pr.P.rs_lcurve(pr.t(X), wl.M)
    rho_o, eta_o = lcurve_points(pr.op, X, pr.d, wts)
    np.testing.assert_allclose(rho, rho_o, rtol=1e-10)
    np.testing.assert_allclose(eta, eta_o, rtol=1e-12)
    assert ls == lcurve_corner(rho_o, eta_o)
