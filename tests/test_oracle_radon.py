"""Pins of the oracle's Radon operator (the CT forward model of Section 8.3):
a brute-force matrix from pure-Python loops over (angle, bin, pixel) written
from the definition, unit Frobenius norm, per-pixel interpolation weights that
sum to one at every angle, and the 90-degree projection of an odd-height image
(exact row sums)."""
import numpy as np

from oracle.operator import RadonOperator, radon_bins, radon_matrix


def _brute(h, w, n_angles):
    nb = radon_bins(h, w)
    C = np.zeros((n_angles * nb, h * w))
    for a in range(n_angles):
        th = np.deg2rad(a + 1.0)
        for i in range(h):
            for j in range(w):
                t = (j - (w - 1) / 2.0) * np.cos(th) + ((h - 1) / 2.0 - i) * np.sin(th)
                for k in range(nb):
                    C[a * nb + k, i * w + j] = max(0.0, 1.0 - abs(t + (nb - 1) / 2.0 - k))
    return C / np.linalg.norm(C)


def test_matrix_matches_a_brute_force_construction():
    for h, w, na in [(5, 4, 7), (6, 9, 13), (1, 5, 3)]:
        C = radon_matrix(h, w, na).toarray()
        np.testing.assert_allclose(C, _brute(h, w, na), atol=1e-15)


def test_frobenius_norm_and_weights_summing_to_one():
    h, w, na = 11, 8, 20
    C = radon_matrix(h, w, na)
    assert abs(np.sqrt(np.sum(C.data ** 2)) - 1.0) < 1e-14
    nb = radon_bins(h, w)
    Cd = C.toarray()
    scale = Cd.max() / max(1e-300, np.max(Cd / Cd.max()))   # any nonzero entry fixes the scale
    per_angle = Cd.reshape(na, nb, h * w).sum(axis=1)       # (angle, pixel)
    # every pixel's two interpolation weights sum to 1 before scaling: all equal
    np.testing.assert_allclose(per_angle, per_angle[0, 0], rtol=1e-13)
    assert scale > 0


def test_ninety_degree_projection_of_an_odd_height_image_is_the_row_sums():
    h, w = 7, 6
    op = RadonOperator(h, w, 90)
    nb = op.nb
    x = np.random.default_rng(1).standard_normal(h * w)
    s90 = op.blur(x)[89 * nb:90 * nb]
    X = x.reshape(h, w)
    expect = np.zeros(nb)
    cen = (nb - 1) // 2
    for i in range(h):
        # y_i = (h-1)/2 - i is an integer for odd h: the whole row lands in one bin
        expect[cen + (h - 1) // 2 - i] += X[i].sum()
    c = op.C.data.max()   # weight 1 scaled: the largest entry (a pixel landing on a bin centre)
    np.testing.assert_allclose(s90, c * expect, rtol=1e-12, atol=1e-14)


def test_adjoint_and_operator_symmetry():
    op = RadonOperator(9, 7, 12)
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal((2, op.n))
    s = rng.standard_normal(op.m)
    assert abs(op.blur(x) @ s - x @ op.blur_adjoint(s)) < 1e-13 * np.linalg.norm(x) * np.linalg.norm(s)
    w = rng.uniform(0.5, 2.0, 2 * op.n)
    assert abs(y @ op.apply(x, 0.3, w) - x @ op.apply(y, 0.3, w)) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)
