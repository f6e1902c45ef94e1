"""GPU parity of the batched solves (batched local spaces [W, g^(k-1,l),
g^(k-1,l-1)]: every shift of a step in one cooperative launch, with per-shift
convergence masks) against the FP64 oracle running the same variant, and
against the same library solving those shifts one after another.

Tolerances as in the other parity tests: FP64 solutions within 1e-6 of the
oracle's where both ran the same step counts (1e-4 otherwise, counts within
2 %+2); mixed precision within 1e-4; every system to its tolerance."""
import os

import numpy as np
import pytest

import synth
from oracle.recycle import State, outer_step
from tests.gpu_util import Pair, rel

pytestmark = pytest.mark.gpu


def _pair(wl, precision, batch):
    old = os.environ.get("RS_BATCH")
    os.environ["RS_BATCH"] = "1" if batch else "0"
    try:
        return Pair(wl, precision=precision, batched_local=1)
    finally:
        if old is None:
            del os.environ["RS_BATCH"]
        else:
            os.environ["RS_BATCH"] = old


def _steps(pr, weights):
    out = []
    for k, w in enumerate(weights):
        pr.P.rs_set_weights(pr.t(w))
        pr.P.rs_update_recycle(0 if k == 0 else 1)
        X = pr.torch.empty(pr.wl.M, pr.wl.n, dtype=pr.torch.float64, device=pr.dev)
        stats = pr.P.rs_solve_shifts(X)
        out.append((pr.n(X), stats))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_launch_matches_the_oracle_batched_variant(precision):
    wl = synth.tiny(64, 56, sigma=1.5, radius=4, M=8, p=10, n_ritz_local=4, seed=12, tol=1e-9)
    pr = _pair(wl, precision, True)
    S = State()
    weights = [np.ones(2 * wl.n), synth.random_weights(wl.n, 5, lo=1.0, hi=300.0),
               synth.random_weights(wl.n, 6, lo=1.0, hi=300.0)]
    gpu = _steps(pr, weights)
    assert pr.P.rs_get_info()["minres_kernel"] == 3      # the batched launch ran
    n_eq = n_tot = 0
    for k, w in enumerate(weights):
        o = outer_step(pr.op, pr.b, pr.gammas, w, S, pr.prm)
        X, stats = gpu[k]
        for l in range(wl.M):
            st = stats[l]
            assert st["relres_true"] <= wl.tol * (1 + 1e-6), (k, l, st)
            e = rel(X[l], o.X[l])
            n_tot += 1
            if precision == 0:
                assert abs(st["iters"] - o.iters[l]) <= max(2, 0.02 * o.iters[l]), (k, l, st["iters"], o.iters[l])
                if st["iters"] == o.iters[l]:
                    n_eq += 1
                    assert e <= 1e-6, (k, l, e)
                else:
                    assert e <= 1e-4, (k, l, e)
            else:
                assert e <= 1e-4, (k, l, e)
    if precision == 0:
        assert n_eq >= 0.6 * n_tot


def test_batched_launch_agrees_with_shift_by_shift_solves_at_512():
    """512 x 512 (radius 8), mixed precision, two outer steps: one launch for all
    16 shifts against the same shifts solved one after another."""
    wl = synth.C2
    w = [np.ones(2 * wl.n), synth.random_weights(wl.n, 7, lo=1.0, hi=1000.0)]
    outs = []
    for batch in (True, False):
        pr = _pair(wl, 1, batch)
        outs.append(_steps(pr, w))
        assert (pr.P.rs_get_info()["minres_kernel"] == 3) == batch
    bnorm = np.linalg.norm(pr.b)
    for k in range(2):
        (Xb, sb), (Xs, ss) = outs[0][k], outs[1][k]
        for l in range(wl.M):
            assert sb[l]["relres_true"] <= wl.tol, (k, l, sb[l])
            assert ss[l]["relres_true"] <= wl.tol, (k, l, ss[l])
            e = rel(Xb[l], Xs[l])
            if e > 1e-4:
                # two solutions to a relative residual of 1e-8 differ by at most 2e-8 |b| in
                # the residual norm; the forward difference of the smallest shifts is that
                # times the condition number of (A + gamma E) (gamma = 1e-5 here)
                dr = pr.op.apply(Xb[l] - Xs[l], pr.gammas[l], w[k])
                assert np.linalg.norm(dr) <= 2 * wl.tol * bnorm * (1 + 1e-6), (k, l, e)
                assert e <= 1e-3, (k, l, e)
            # the FP32 step count of a single ill-conditioned shift moves with the rounding
            # order (gamma = 1e-5: 633 to 800 steps between builds); the step's total does not
            assert sb[l]["iters"] <= 2 * ss[l]["iters"] + 20, (k, l, sb[l]["iters"], ss[l]["iters"])
        tb, ts = sum(x["iters"] for x in sb), sum(x["iters"] for x in ss)
        assert tb <= 1.2 * ts + 10 * wl.M, (k, tb, ts)


@pytest.mark.parametrize("precision", [0, 1])
def test_several_images_of_uneven_size_in_one_launch(precision, monkeypatch):
    monkeypatch.setenv("RS_BATCH_JOINT", "1")       # the joint kernel, not the per-problem choice
    """Three images of different sizes, blurs and shift counts: two outer steps
    solved jointly (rs_solve_shifts_batched: all their shifts in one persistent
    launch) against each image solved on its own, and against the oracle."""
    from paper_2306_15049_gb300 import recyc
    specs = [(96, 80, 1.5, 4, 6), (70, 130, 2.0, 6, 5), (64, 64, 2.5, 8, 7)]
    wls = [synth.tiny(h, w, sigma=sg, radius=r, M=M, p=8, n_ritz_local=3, seed=90 + i, tol=1e-9)
           for i, (h, w, sg, r, M) in enumerate(specs)]
    joint = [_pair(wl, precision, True) for wl in wls]
    alone = [_pair(wl, precision, True) for wl in wls]
    S = [State() for _ in wls]
    for k in range(2):
        ws = [np.ones(2 * wl.n) if k == 0 else synth.random_weights(wl.n, 20 + i, lo=1.0, hi=300.0)
              for i, wl in enumerate(wls)]
        Xj = []
        for pr, w in zip(joint, ws):
            pr.P.rs_set_weights(pr.t(w))
            pr.P.rs_update_recycle(0 if k == 0 else 1)
            Xj.append(pr.torch.empty(pr.wl.M, pr.wl.n, dtype=pr.torch.float64, device=pr.dev))
        stats_j = recyc.rs_solve_shifts_batched([pr.P for pr in joint], Xj)
        for i, (pr, w) in enumerate(zip(alone, ws)):
            pr.P.rs_set_weights(pr.t(w))
            pr.P.rs_update_recycle(0 if k == 0 else 1)
            Xa = pr.torch.empty(pr.wl.M, pr.wl.n, dtype=pr.torch.float64, device=pr.dev)
            stats_a = pr.P.rs_solve_shifts(Xa)
            o = outer_step(pr.op, pr.b, pr.gammas, w, S[i], pr.prm)
            xj, xa = pr.n(Xj[i]), pr.n(Xa)
            for l in range(pr.wl.M):
                sj = stats_j[i][l]
                assert sj["relres_true"] <= pr.wl.tol * (1 + 1e-6), (k, i, l, sj)
                lim = 1e-6 if (precision == 0 and sj["iters"] == stats_a[l]["iters"]) else 1e-4
                assert rel(xj[l], xa[l]) <= lim, (k, i, l)
                lim_o = 1e-6 if (precision == 0 and sj["iters"] == o.iters[l]) else 1e-4
                assert rel(xj[l], o.X[l]) <= lim_o, (k, i, l)
        assert all(pr.P.rs_get_info()["minres_kernel"] == 3 for pr in joint)


def test_joint_solve_rejects_mismatched_problems():
    from paper_2306_15049_gb300 import recyc
    wl = synth.tiny(40, 40, sigma=1.5, radius=4, M=4, p=6, n_ritz_local=2, seed=3)
    a = _pair(wl, 0, True)
    b = Pair(wl, precision=0, batched_local=0)          # not batched_local
    for pr in (a, b):
        pr.P.rs_set_weights(pr.t(np.ones(2 * wl.n)))
        pr.P.rs_update_recycle(0)
    X = [pr.torch.empty(wl.M, wl.n, dtype=pr.torch.float64, device=pr.dev) for pr in (a, b)]
    with pytest.raises(recyc.RecycError):
        recyc.rs_solve_shifts_batched([a.P, b.P], X)
    with pytest.raises(recyc.RecycError):
        recyc.rs_solve_shifts_batched([a.P, a.P], [X[0], X[0]])


def test_joint_call_picks_the_faster_way_and_solves_every_shift():
    """Without RS_BATCH_JOINT the call times the joint launch on its first call
    for a batch shape and the per-problem launches on its second, then keeps the
    faster; every call solves every shift to its tolerance."""
    from paper_2306_15049_gb300 import recyc
    specs = [(96, 80, 1.5, 4, 4), (64, 64, 2.5, 8, 5)]
    wls = [synth.tiny(h, w, sigma=sg, radius=r, M=M, p=6, n_ritz_local=2, seed=95 + i, tol=1e-9)
           for i, (h, w, sg, r, M) in enumerate(specs)]
    prs = [_pair(wl, 1, True) for wl in wls]
    for call in range(3):
        Xs = []
        for pr in prs:
            pr.P.rs_set_weights(pr.t(np.ones(2 * pr.wl.n)))
            pr.P.rs_update_recycle(0)
            Xs.append(pr.torch.empty(pr.wl.M, pr.wl.n, dtype=pr.torch.float64, device=pr.dev))
        stats = recyc.rs_solve_shifts_batched([pr.P for pr in prs], Xs)
        for st, pr in zip(stats, prs):
            assert len(st) == pr.wl.M
            assert all(s_["relres_true"] <= pr.wl.tol * (1 + 1e-6) for s_ in st), (call, st)
