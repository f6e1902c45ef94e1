"""rs_solve_shifts over sub-ranges of the shifts (l0, count), through the C ABI.

Solving the shifts of a step in several calls, in order, is the same
computation as one call over all of them (the chain g^(k,l-1) of Algorithm
updatelocal carries across the calls), so the solutions must agree to the last
bit with a single call on an identical problem; the next outer step (Eq.
tildeUupdate) must then run from them. A step left incomplete must not hand
over to the next one, and ranges outside 0..M-1 are rejected."""
import numpy as np
import pytest

import synth
from oracle.recycle import State, outer_step
from tests.gpu_util import Pair, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,batched", [(0, 0), (1, 0), (0, 1)])
def test_sub_ranges_in_order_equal_one_call(precision, batched):
    wl = synth.tiny(40, 36, sigma=1.5, radius=4, M=7, p=8, n_ritz_local=3, seed=31, tol=1e-9)
    one = Pair(wl, precision=precision, batched_local=batched)
    split = Pair(wl, precision=precision, batched_local=batched)
    S = State()
    weights = [np.ones(2 * wl.n), synth.random_weights(wl.n, 7, lo=1.0, hi=1000.0)]
    for k, w in enumerate(weights):
        o = outer_step(one.op, one.b, one.gammas, w, S, one.prm)
        for pr in (one, split):
            pr.P.rs_set_weights(pr.t(w))
            pr.P.rs_update_recycle(0 if k == 0 else 1)
        X1 = one.torch.empty(wl.M, wl.n, dtype=one.torch.float64, device=one.dev)
        st1 = one.P.rs_solve_shifts(X1)
        parts, st2 = [], []
        for l0, cnt in ((0, 2), (2, 1), (3, 4)):
            Xp = split.torch.empty(cnt, wl.n, dtype=split.torch.float64, device=split.dev)
            st2 += split.P.rs_solve_shifts(Xp, l0=l0, count=cnt)
            parts.append(split.n(Xp))
        X2 = np.concatenate(parts)
        if batched:
            # the full-range call runs every shift in one launch, the sub-ranges shift
            # by shift: the same iteration, different reduction orders
            for l in range(wl.M):
                if st2[l]["iters"] == st1[l]["iters"]:
                    assert rel(X2[l], one.n(X1)[l]) <= (1e-4 if precision else 1e-6)
        else:
            np.testing.assert_array_equal(X2, one.n(X1))
            assert [s["iters"] for s in st2] == [s["iters"] for s in st1]
        for l in range(wl.M):
            assert st2[l]["relres_true"] <= wl.tol * (1 + 1e-6)
            assert rel(X2[l], o.X[l]) <= (1e-4 if precision else 1e-5), (k, l)


def test_incomplete_step_does_not_hand_over_and_bad_ranges_are_rejected():
    from paper_2306_15049_gb300 import recyc
    wl = synth.tiny(24, 22, sigma=1.2, radius=3, M=5, p=6, n_ritz_local=2, seed=32, tol=1e-9)
    pr = Pair(wl)
    pr.P.rs_set_weights(pr.t(np.ones(2 * wl.n)))
    pr.P.rs_update_recycle(0)
    X = pr.torch.empty(wl.M, wl.n, dtype=pr.torch.float64, device=pr.dev)
    for l0, cnt in ((-1, 2), (0, 0), (4, 2), (5, 1)):
        with pytest.raises(recyc.RecycError) as e:
            pr.P.rs_solve_shifts(X, l0=l0, count=cnt)
        assert e.value.status == recyc.RS_EINVAL
    # shifts 2..4 first, then 0..1: every shift solved, the step hands over
    st = pr.P.rs_solve_shifts(X[2:], l0=2, count=3) + pr.P.rs_solve_shifts(X[:2], l0=0, count=2)
    assert all(s["relres_true"] <= wl.tol * (1 + 1e-6) for s in st)
    pr.P.rs_set_weights(pr.t(synth.random_weights(wl.n, 3)))
    pr.P.rs_update_recycle(1)
    st = pr.P.rs_solve_shifts(X[:4], l0=0, count=4)      # shift 4 left out
    assert all(s["relres_true"] <= wl.tol * (1 + 1e-6) for s in st)
    pr.P.rs_set_weights(pr.t(synth.random_weights(wl.n, 4)))
    with pytest.raises(recyc.RecycError) as e:
        pr.P.rs_update_recycle(1)
    assert e.value.status == recyc.RS_ENOTREADY
    pr.P.rs_update_recycle(0)                             # a fresh principal space still works
    st = pr.P.rs_solve_shifts(X)
    assert all(s["relres_true"] <= wl.tol * (1 + 1e-6) for s in st)


@pytest.mark.parametrize("precision,batched,pinned", [(0, 0, True), (1, 0, True), (1, 0, False), (0, 1, True)])
def test_solutions_delivered_to_host_equal_the_device_solve(precision, batched, pinned):
    """rs_solve_shifts_host: the host rows (copied as each shift finishes, or after
    the one batched launch) equal the device rows bit for bit, and both equal an
    rs_solve_shifts call on an identical problem; sub-ranges work the same way."""
    from paper_2306_15049_gb300 import recyc
    wl = synth.tiny(40, 36, sigma=1.5, radius=4, M=7, p=8, n_ritz_local=3, seed=33, tol=1e-9)
    ref = Pair(wl, precision=precision, batched_local=batched)
    hst = Pair(wl, precision=precision, batched_local=batched)
    torch = ref.torch
    for k, w in enumerate([np.ones(2 * wl.n), synth.random_weights(wl.n, 9, lo=1.0, hi=1000.0)]):
        for pr in (ref, hst):
            pr.P.rs_set_weights(pr.t(w))
            pr.P.rs_update_recycle(0 if k == 0 else 1)
        X1 = torch.empty(wl.M, wl.n, dtype=torch.float64, device=ref.dev)
        st1 = ref.P.rs_solve_shifts(X1)
        X2 = torch.empty_like(X1)
        H2 = torch.full((wl.M, wl.n), np.nan, dtype=torch.float64)
        if pinned:
            H2 = H2.pin_memory()
        if k == 0:
            st2 = hst.P.rs_solve_shifts_host(X2, H2)
        else:
            st2 = (hst.P.rs_solve_shifts_host(X2[:3], H2[:3], l0=0, count=3) +
                   hst.P.rs_solve_shifts_host(X2[3:], H2[3:], l0=3, count=4))
        np.testing.assert_array_equal(H2.numpy(), hst.n(X2))
        if not (batched and k == 1):      # batched: the sub-ranges run shift by shift
            np.testing.assert_array_equal(hst.n(X2), ref.n(X1))
            assert [s["iters"] for s in st2] == [s["iters"] for s in st1]
        assert all(s["relres_true"] <= wl.tol * (1 + 1e-6) for s in st2)
    with pytest.raises(recyc.RecycError) as e:
        hst.P.rs_solve_shifts_host(X2, None)
    assert e.value.status == recyc.RS_EINVAL
