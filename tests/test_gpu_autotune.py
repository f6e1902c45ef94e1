"""The launch-configuration autotuner of the FP32 streaming MINRES solve,
through the C ABI. An image with more 32 x 32 tiles than co-resident CTAs
(640 x 576: 360 tiles) takes the streaming path; the first solve of the shape
times a short trial of each variant and keeps the fastest. Trials must leave
no trace: the tuned run's solutions equal, bit for bit, those of a problem that
pins the same variant with RS_TMA, and every system meets its tolerance."""
import os

import numpy as np
import pytest

import synth
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


def _solve(wl, env):
    old = {k: os.environ.get(k) for k in env}
    for k, v in env.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    try:
        pr = Pair(wl, precision=1)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    pr.P.rs_set_weights(pr.t(np.ones(2 * wl.n)))
    pr.P.rs_update_recycle(0)
    X = pr.torch.empty(wl.M, wl.n, dtype=pr.torch.float64, device=pr.dev)
    stats = pr.P.rs_solve_shifts(X)
    return pr.n(X), stats, pr.P.rs_get_info()


def test_autotuned_variant_runs_and_matches_the_pinned_variant():
    wl = synth.tiny(640, 576, sigma=2.0, radius=6, M=3, p=6, n_ritz_local=2, seed=93, tol=1e-8)
    X1, st1, info1 = _solve(wl, {"RS_TMA": None, "RS_AUTOTUNE": None, "RS_STREAM_CTAS": None})
    v = info1["tuned_variant"]
    assert v in (0, 1, 2), info1
    assert info1["minres_kernel"] == (0 if v == 0 else 2), info1
    assert all(s["relres_true"] <= wl.tol * (1 + 1e-6) for s in st1)
    X2, st2, info2 = _solve(wl, {"RS_TMA": str(v), "RS_AUTOTUNE": None, "RS_STREAM_CTAS": None})
    assert info2["tuned_variant"] == v
    assert [s["iters"] for s in st1] == [s["iters"] for s in st2]
    np.testing.assert_array_equal(X1, X2)
