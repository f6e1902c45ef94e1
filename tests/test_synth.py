"""The seeded input generators: deterministic, in range, of the stated shapes."""
import numpy as np

import synth


def test_image_is_deterministic_piecewise_constant_in_unit_range():
    a = synth.piecewise_constant_image(64, 64, 123)
    b = synth.piecewise_constant_image(64, 64, 123)
    np.testing.assert_array_equal(a, b)
    assert a.shape == (64, 64) and a.min() >= 0.0 and a.max() <= 1.0
    assert len(np.unique(a)) <= 1 + max(6, 64 // 8)
    assert not np.array_equal(a, synth.piecewise_constant_image(64, 64, 124))


def test_shift_grid_and_workload_indices():
    g = synth.shift_grid(-5, 0, 16)
    assert g.shape == (16,) and abs(g[0] - 1e-5) < 1e-20 and abs(g[-1] - 1.0) < 1e-15
    assert np.all(np.diff(np.log10(g)) > 0)
    wl = synth.C2
    assert (wl.I_split, wl.i1, wl.i2, wl.i_star, wl.J_L, wl.J_R, wl.l_c) == (12, 1, 8, 8, 12, 15, 15)
    assert (wl.a_ritz, wl.b_ritz, wl.vnew_cap) == (25, 13, 38)
    c1 = synth.C1
    assert (c1.I_split, c1.i2, c1.J_L, c1.J_R, c1.l_c, c1.a_ritz, c1.b_ritz) == (6, 4, 6, 7, 7, 5, 3)
    assert c1.a_ritz + c1.b_ritz + 2 == c1.p


def test_noise_and_weights_shapes():
    z = synth.noise_direction(5, 7, 1)
    assert z.shape == (5, 7)
    w = synth.random_weights(35, 2)
    assert w.shape == (70,) and np.all(w > 0)
