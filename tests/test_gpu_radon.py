"""GPU parity of the CT forward model (the parallel-beam Radon transform of
Section 8.3, the paper's second example) against the FP64 oracle, through the
C ABI: the operator element by element, the synthesized sinogram data, and the
recycled shifted solves with A = C^T C on a small case and on the 82 x 82,
135-angle stand-in of the paper's example.

Tolerances: operator 1e-13 relative in FP64 (2e-6 in the FP32 working
precision); every GPU solution solves the oracle's system to the tolerance;
solution differences within the bound 2 tol ||b|| / lambda_min that two
solutions at the tolerance can have (dense lambda_min, small images)."""
import numpy as np
import pytest

import synth
from oracle.outer import run as oracle_run
from oracle.recycle import Params, State, outer_step
from tests.gpu_util import Pair, rel

pytestmark = pytest.mark.gpu

CASES = [(13, 11, 17), (40, 36, 60), (1, 9, 5), (82, 82, 135)]


@pytest.mark.parametrize("h,w,na", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_radon_operator_modes_match_oracle(h, w, na, precision):
    wl = synth.tiny(h, w, M=4, p=4, n_ritz_local=1, seed=h + w + na, radon_angles=na)
    pr = Pair(wl, precision=precision, x_image=synth.random_vectors(h * w, 1, h * w)[:, 0])
    n, m = h * w, pr.op.m
    wts = synth.random_weights(n, 4)
    pr.P.rs_set_weights(pr.t(wts))
    rng = np.random.default_rng(na)
    x = rng.standard_normal(n)
    sg = rng.standard_normal(m)
    xt = pr.t(x)
    y = pr.torch.empty_like(xt)
    y2 = pr.torch.empty_like(xt)
    for wp in ([False, True] if precision == 1 else [False]):
        tol = 1e-13 if not wp else 2e-6
        for gamma in [1e-8, 0.3, 70.0]:
            pr.P.rs_apply_operator(gamma, xt, y, mode=0, working_precision=wp)
            assert rel(pr.n(y), pr.op.apply(x, gamma, wts)) < tol, (gamma, wp)
        pr.P.rs_apply_operator(0.0, xt, y, y2, mode=1, working_precision=wp)
        assert rel(pr.n(y), pr.op.apply_A(x)) < tol
        assert rel(pr.n(y2), pr.op.apply_E(x, wts)) < tol
    s = pr.torch.empty(m, dtype=pr.torch.float64, device=pr.dev)
    pr.P.rs_apply_operator(0.0, xt, s, mode=3)
    assert rel(pr.n(s), pr.op.blur(x)) < 1e-13
    pr.P.rs_apply_operator(0.0, pr.t(sg), y, mode=4)
    assert rel(pr.n(y), pr.op.blur_adjoint(sg)) < 1e-13
    # the device C^T is the exact transpose of the device C
    Cx = pr.n(s)
    assert abs(Cx @ sg - x @ pr.n(y)) <= 1e-13 * np.linalg.norm(Cx) * np.linalg.norm(sg) * 10


def test_synthesized_sinogram_matches_oracle():
    wl = synth.tiny(30, 26, M=4, p=4, n_ritz_local=1, radon_angles=45)
    pr = Pair(wl)
    assert pr.d.shape[0] == pr.op.m
    assert rel(pr.n(pr.d_gpu), pr.d) < 1e-13


def _lambda_min(pr, w, gamma):
    """Smallest eigenvalue of the dense A + gamma E (small images only)."""
    from tests.dense import grad_dense
    C = pr.op.C.toarray()
    L = grad_dense(pr.wl.height, pr.wl.width)
    return np.linalg.eigvalsh(C.T @ C + gamma * (L.T @ (w[:, None] * L)))[0]


def _teacher_forced(wl, steps, precision, dense_bound=False):
    """GPU outer steps driven by the oracle's weights. Every GPU solution must
    solve the oracle's own system to the tolerance (residual evaluated by the
    oracle, 1 % margin for the two evaluation orders). CT systems with gamma
    down to 1e-8 are ill-conditioned, so two correct solutions may differ by up
    to 2 tol ||b|| / lambda_min(A + gamma E): checked with the dense lambda_min
    on small images. FP64 step counts must stay within 5 % (+3) of the oracle's."""
    pr = Pair(wl, precision=precision)
    bn = np.linalg.norm(pr.b)
    n_close = n_total = 0
    for k in range(len(steps)):
        w = steps[k].extra["w"]
        pr.P.rs_set_weights(pr.t(w))
        pr.P.rs_update_recycle(0 if k == 0 else 1)
        X = pr.torch.empty(wl.M, wl.n, dtype=pr.torch.float64, device=pr.dev)
        stats = pr.P.rs_solve_shifts(X)
        Xn = pr.n(X)
        for l in range(wl.M):
            st = stats[l]
            g = pr.gammas[l]
            assert st["relres_true"] <= wl.tol * (1 + 1e-6), (k, l, st)
            r_or = np.linalg.norm(pr.b - pr.op.apply(Xn[l], g, w)) / bn
            assert r_or <= 1.01 * wl.tol, (k, l, r_or)
            n_total += 1
            if precision == 0:
                it, it_o = st["iters"], steps[k].iters[l]
                n_close += abs(it - it_o) <= 0.05 * it_o + 3
            if dense_bound:
                bound = 2.0 * wl.tol * (1 + 1e-6) * bn / _lambda_min(pr, w, g)
                assert np.linalg.norm(Xn[l] - steps[k].X[l]) <= bound, (k, l)
    return n_close, n_total


@pytest.mark.parametrize("precision", [0, 1])
def test_small_ct_outer_steps_match_oracle(precision):
    wl = synth.tiny(40, 36, M=8, p=10, n_ritz_local=4, K=2, seed=77, log_lo=-6.0, log_hi=1.0,
                    tol=1e-8, radon_angles=60)
    pr = Pair(wl)
    steps, _ = oracle_run(pr.op, pr.b, pr.d, pr.gammas, pr.prm, wl.K, wl.beta)
    n_close, n_total = _teacher_forced(wl, steps, precision, dense_bound=True)
    if precision == 0:
        assert n_close >= 0.9 * n_total


def test_ct82_first_outer_step_matches_oracle():
    """The 82 x 82, 135-angle stand-in of Section 8.3 (20 shifts over 1e-8..1e2):
    one outer step, FP64."""
    wl = synth.CT82
    pr = Pair(wl)
    ref = outer_step(pr.op, pr.b, pr.gammas, np.ones(2 * wl.n), State(), pr.prm)
    ref.extra["w"] = np.ones(2 * wl.n)
    n_close, n_total = _teacher_forced(wl, [ref], 0)
    assert n_close >= 0.9 * n_total
