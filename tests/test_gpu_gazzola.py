"""GPU parity of the paper's own cumulative reweighting (Section 2.1):
D_{k+1} = diag(1 - (|D_k L x| / ||D_k L x||_inf)^p) D_k, E_{k+1} = L^T D_{k+1}^2 L,
against the FP64 oracle, element by element, and an outer loop driven by it.

Tolerances: the weights within 1e-14 of the entry scale (one pow and one
division per entry in FP64 on each side); solutions as in the other FP64
parity tests (1e-6 relative where both sides run the same step counts)."""
import numpy as np
import pytest

import synth
from oracle.operator import gazzola_weights
from oracle.outer import run as oracle_run
from tests.gpu_util import Pair, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("h,w,p", [(29, 31, 2.0), (64, 64, 1.0), (1, 40, 3.5), (130, 70, 0.5)])
def test_gazzola_weights_match_oracle(h, w, p):
    wl = synth.tiny(h, w, M=4, p=4, n_ritz_local=1)
    pr = Pair(wl, x_image=synth.random_vectors(h * w, 1, h + w)[:, 0])
    n = h * w
    x = synth.piecewise_constant_image(h, w, 5).reshape(-1) + 1e-3 * synth.random_vectors(n, 1, 3)[:, 0]
    dprev = synth.random_weights(n, 4, lo=0.2, hi=1.0)
    ref = gazzola_weights(pr.op, x, dprev, p)
    dnew = pr.torch.empty(2 * n, dtype=pr.torch.float64, device=pr.dev)
    wout = pr.torch.empty_like(dnew)
    pr.P.rs_gazzola_weights(pr.t(x), pr.t(dprev), p, dnew, wout)
    assert np.max(np.abs(pr.n(dnew) - ref)) <= 1e-14
    assert np.max(np.abs(pr.n(wout) - ref * ref)) <= 1e-14
    assert np.min(pr.n(dnew)) == 0.0           # the entry of largest |q| gets weight 0
    # in place: d_new aliases d_prev
    dd = pr.t(dprev)
    pr.P.rs_gazzola_weights(pr.t(x), dd, p, dd, wout)
    assert np.max(np.abs(pr.n(dd) - ref)) <= 1e-14


def test_gazzola_weights_of_a_constant_image_keep_d_prev():
    wl = synth.tiny(20, 24, M=4, p=4, n_ritz_local=1)
    pr = Pair(wl)
    n = wl.n
    dprev = synth.random_weights(n, 8, lo=0.2, hi=1.0)
    dnew = pr.torch.empty(2 * n, dtype=pr.torch.float64, device=pr.dev)
    wout = pr.torch.empty_like(dnew)
    pr.P.rs_gazzola_weights(pr.t(np.full(n, 0.7)), pr.t(dprev), 2.0, dnew, wout)
    assert np.array_equal(pr.n(dnew), dprev)
    assert np.array_equal(pr.n(wout), dprev * dprev)


def test_gazzola_weights_reject_bad_arguments():
    from paper_2306_15049_gb300.recyc import RecycError
    wl = synth.tiny(8, 8, M=4, p=4, n_ritz_local=1)
    pr = Pair(wl)
    v = pr.torch.ones(2 * wl.n, dtype=pr.torch.float64, device=pr.dev)
    for p in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(RecycError):
            pr.P.rs_gazzola_weights(v, v, p, v, v.clone())
    with pytest.raises(RecycError):
        pr.P.rs_gazzola_weights(v, v, 2.0, v, v)      # w aliases d_prev


def test_c1_outer_loop_with_gazzola_weights_matches_oracle():
    """Three outer steps of the 64 x 64 workload with the paper's weights (p = 2):
    the oracle's weights drive the GPU (zero weights on the strongest edges are
    allowed by rs_set_weights); the GPU's own weights from its own x^(k, l_*)
    agree with the oracle's to the accuracy of the solutions."""
    wl = synth.C1
    pr = Pair(wl)
    steps, lstars = oracle_run(pr.op, pr.b, pr.d, pr.gammas, pr.prm, 3, wl.beta, rule="gazzola",
                               p_gazzola=2.0)
    D = pr.torch.ones(2 * wl.n, dtype=pr.torch.float64, device=pr.dev)
    wg = pr.torch.empty_like(D)
    n_equal = n_total = 0
    for k in range(3):
        w = steps[k].extra["w"]
        if k > 0:
            assert np.min(w) == 0.0
        pr.P.rs_set_weights(pr.t(w))
        pr.P.rs_update_recycle(0 if k == 0 else 1)
        X = pr.torch.empty(wl.M, wl.n, dtype=pr.torch.float64, device=pr.dev)
        stats = pr.P.rs_solve_shifts(X)
        Xn = pr.n(X)
        for l in range(wl.M):
            assert stats[l]["relres_true"] <= wl.tol * (1 + 1e-6), (k, l, stats[l])
            e = rel(Xn[l], steps[k].X[l])
            n_total += 1
            if stats[l]["iters"] == steps[k].iters[l]:
                n_equal += 1
                assert e <= 1e-6, (k, l, e)
            else:
                assert e <= 1e-4, (k, l, e)
        rho, eta, ls = pr.P.rs_lcurve(X, wl.M)
        assert ls == lstars[k]
        if k + 1 < 3:
            pr.P.rs_gazzola_weights(X[ls], D, 2.0, D, wg)
            assert np.max(np.abs(pr.n(wg) - steps[k + 1].extra["w"])) < 1e-4
    assert n_equal >= 0.75 * n_total
