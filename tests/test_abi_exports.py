"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/recyc.h declares (no GPU needed: no compute call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2306_15049_gb300 import build, recyc
    try:
        build.build()
    except RuntimeError as e:  # no CUDA toolkit on this machine
        pytest.skip(str(e))
    return recyc.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert {"rs_create_problem", "rs_set_weights", "rs_solve_shifts", "rs_update_recycle"} <= declared
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2306_15049_gb300 import recyc
    assert _declared() == set(recyc.EXPORTS)


def test_workspace_size_and_validation_need_no_gpu(lib):
    import synth
    from paper_2306_15049_gb300 import recyc
    from paper_2306_15049_gb300.workloads import desc_for
    d, keep = desc_for(synth.C1)
    assert recyc.rs_workspace_bytes(d) > 8 * 64 * 64
    bad, keep2 = desc_for(synth.C1)
    bad.radius = 40
    assert recyc.rs_workspace_bytes(bad) == 0
    bad.radius = 4
    bad.i_star = 0
    assert recyc.rs_workspace_bytes(bad) == 0


def test_guess_kind_validation_needs_no_gpu(lib):
    import synth
    from paper_2306_15049_gb300 import recyc
    from paper_2306_15049_gb300.workloads import desc_for
    wl = synth.C1
    base = recyc.rs_workspace_bytes(desc_for(wl)[0])
    assert recyc.rs_workspace_bytes(desc_for(wl, guess=recyc.RS_GUESS_OBLIQUE)[0]) == base
    # two anchors carry one more n x p block and small matrices
    assert recyc.rs_workspace_bytes(desc_for(wl, guess=recyc.RS_GUESS_OBLIQUE2)[0]) > base
    for I_L, I_R in [(0, wl.M), (wl.I_split + 1, wl.M), (1, wl.I_split), (1, wl.M + 1)]:
        d, keep = desc_for(wl, guess=recyc.RS_GUESS_OBLIQUE2, I_L=I_L, I_R=I_R)
        assert recyc.rs_workspace_bytes(d) == 0, (I_L, I_R)
    d, keep = desc_for(wl)
    d.guess = 3
    assert recyc.rs_workspace_bytes(d) == 0


def test_joint_solve_sizes_and_argument_checks_need_no_gpu(lib):
    import ctypes

    from paper_2306_15049_gb300 import recyc
    assert lib.rs_batch_scratch_bytes(0, 10) == 0
    assert lib.rs_batch_scratch_bytes(2, 0) == 0
    assert lib.rs_batch_scratch_bytes(4, 128) > lib.rs_batch_scratch_bytes(1, 16) > 0
    st = lib.rs_solve_shifts_batched(None, 0, None, None, None, 0)
    assert st == recyc.RS_EINVAL
    assert b"need problems" in lib.rs_last_error(None)
    probs = (ctypes.c_void_p * 1)(None)
    xs = (ctypes.c_void_p * 1)(None)
    st = lib.rs_solve_shifts_batched(probs, 1, xs, None, ctypes.c_void_p(256), 1 << 20)
    assert st == recyc.RS_EINVAL


def test_desc_limits_need_no_gpu(lib):
    """Sizes and fields at and beyond their limits are rejected before any work."""
    import synth
    from paper_2306_15049_gb300 import recyc
    from paper_2306_15049_gb300.workloads import desc_for

    def ok(mutate):
        d, keep = desc_for(synth.C1)
        mutate(d)
        return recyc.rs_workspace_bytes(d) > 0

    assert ok(lambda d: None)
    assert not ok(lambda d: setattr(d, "height", 0))
    assert not ok(lambda d: (setattr(d, "height", 1 << 15), setattr(d, "width", (1 << 13) + 1)))   # > 2^28 pixels
    assert ok(lambda d: (setattr(d, "height", 1), setattr(d, "width", 1)))                          # one pixel
    assert not ok(lambda d: setattr(d, "M", 0))
    assert not ok(lambda d: setattr(d, "p_max", 0))
    assert not ok(lambda d: setattr(d, "n_ritz_local", 15))                                         # |J| <= 14
    assert ok(lambda d: setattr(d, "n_ritz_local", 14))
    assert not ok(lambda d: setattr(d, "maxit", 0))
    assert not ok(lambda d: setattr(d, "tol", -1.0))
    assert not ok(lambda d: setattr(d, "inner", 2))
    assert ok(lambda d: setattr(d, "inner", recyc.RS_CG))
    assert not ok(lambda d: setattr(d, "precision", 2))
    assert not ok(lambda d: setattr(d, "radon_angles", 3601))
