"""The bounded wait of the grid barrier (every persistent cooperative kernel of
the library) runs out instead of hanging when a CTA never arrives: the
self-test launch's waiting CTA gives up after the barrier's 2 s limit, raises
the error flag and returns; the context then still runs a full solve. No fault
is raised on the device: the missing arrival is a counter nobody increments."""
import ctypes
import time

import numpy as np
import pytest

import synth
from tests.gpu_util import Pair

pytestmark = pytest.mark.gpu


def test_grid_barrier_wait_gives_up_and_the_context_stays_usable():
    from paper_2306_15049_gb300 import recyc
    wl = synth.tiny(40, 36, sigma=1.5, radius=4, M=4, p=6, n_ritz_local=2, seed=91, tol=1e-9)
    pr = Pair(wl)
    lib = recyc.load()
    scratch = pr.torch.zeros(64, dtype=pr.torch.uint8, device=pr.dev)
    err = ctypes.c_int(-1)
    t0 = time.perf_counter()
    st = lib.rs_selftest_grid_barrier(scratch.data_ptr(), 64, None, ctypes.byref(err))
    el = time.perf_counter() - t0
    assert st == recyc.RS_OK, lib.rs_last_error(None)
    assert err.value == 1
    assert 1.5 < el < 30.0           # the 2 s limit, not a hang
    # the same context solves a step afterwards
    pr.P.rs_set_weights(pr.t(np.ones(2 * wl.n)))
    pr.P.rs_update_recycle(0)
    X = pr.torch.empty(wl.M, wl.n, dtype=pr.torch.float64, device=pr.dev)
    stats = pr.P.rs_solve_shifts(X)
    assert all(s["relres_true"] <= wl.tol * (1 + 1e-6) for s in stats)
