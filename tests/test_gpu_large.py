"""Solution parity with the FP64 oracle on the 512 x 512 benchmark workload and
adjoint parity at radius 10, through the C ABI.

* 512 x 512 (sigma 2.5, radius 8, 16 shifts, p = 40), first outer step, FP64,
  batched local spaces (their shifts are independent, so the oracle can solve a
  few of them alone): the oracle takes the GPU's principal basis, solves shifts
  1, 8 and 16; the GPU re-solves those shifts with the oracle's MINRES step
  counts; every solution within 1e-6 of the oracle's, and the free-running
  solutions (the benchmark's) within 1e-4 with their residuals at the tolerance.
* adjoint solves at radius 10 (128 x 124, the 1024 x 1024 workload's blur) in
  FP64 and mixed precision against the oracle's adjoint solutions (plain MINRES
  to 1e-13, the oracle's gradient pinned by central finite differences), and the
  shift and weight gradients against the oracle's formula."""
import numpy as np
import pytest

import synth
from oracle.adjoint import adjoint_solves, shift_and_weight_gradients
from oracle.recycle import State, outer_step
from tests.gpu_util import Pair, rel

pytestmark = pytest.mark.gpu


def test_c2_first_step_solutions_match_the_oracle():
    wl = synth.C2
    pr = Pair(wl, precision=0, batched_local=1)
    w = np.ones(2 * wl.n)
    pr.P.rs_set_weights(pr.t(w))
    pr.P.rs_update_recycle(0)
    X = pr.torch.empty(wl.M, wl.n, dtype=pr.torch.float64, device=pr.dev)
    stats = pr.P.rs_solve_shifts(X)
    U = pr.torch.empty(wl.p, wl.n, dtype=pr.torch.float64, device=pr.dev)
    nc = pr.P.rs_get_principal_basis(U)
    Ut = pr.n(U)[:nc].T.copy()
    shifts = [0, 7, 15]
    o = outer_step(pr.op, pr.b, pr.gammas, w, State(), pr.prm, Ut_given=Ut, shifts=shifts)
    assert o.nc == nc
    Xn = pr.n(X)
    for l in shifts:
        assert stats[l]["relres_true"] <= wl.tol * (1 + 1e-6), (l, stats[l])
        assert rel(Xn[l], o.X[l]) <= 1e-4, (l, rel(Xn[l], o.X[l]))
        assert abs(stats[l]["iters"] - o.iters[l]) <= 2 + 0.02 * o.iters[l], (l, stats[l]["iters"], o.iters[l])
        ov = int(o.iters[l]) if (o.iters[l] > 0 or o.relres0[l] > wl.tol) else -1
        Xf = pr.torch.empty(1, wl.n, dtype=pr.torch.float64, device=pr.dev)
        pr.P.rs_solve_shifts(Xf, l0=l, count=1, iters_override=[ov])
        assert rel(pr.n(Xf)[0], o.X[l]) <= 1e-6, (l, rel(pr.n(Xf)[0], o.X[l]))


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_at_radius_10_matches_the_oracle(precision):
    wl = synth.tiny(128, 124, sigma=3.0, radius=10, M=5, p=10, n_ritz_local=4, seed=33, tol=1e-11,
                    log_lo=-3.0)
    pr = Pair(wl, precision=precision)
    w = synth.random_weights(wl.n, 8, lo=1.0, hi=100.0)
    pr.P.rs_set_weights(pr.t(w))
    pr.P.rs_update_recycle(0)
    X = pr.torch.empty(wl.M, wl.n, dtype=pr.torch.float64, device=pr.dev)
    pr.P.rs_solve_shifts(X)
    Xn = pr.n(X)
    G = 2.0 * (Xn - pr.x_true)
    Lam = pr.torch.empty_like(X)
    stats = pr.P.rs_solve_adjoint(pr.t(G), Lam)
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
