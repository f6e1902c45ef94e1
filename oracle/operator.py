"""Matrix-free FP64 shifted operator (oracle; test infrastructure only).

The systems are (A + gamma_l E_k) x = b with A = C^T C, E_k = L^T W_k L and
b = C^T d (Section 2.1, Eq. blkeqn; Section 4, Eq. shift). Here:

* C = H is a zero-boundary separable Gaussian blur: H = T_h (x) T_w with
  T[i, i'] = g[i' - i] for |i' - i| <= r, g_a proportional to
  exp(-a^2 / (2 sigma^2)) and normalised to sum 1 (the symmetric Gaussian blur
  with zero boundary conditions of Section 8.2, reduced to one Kronecker term).
* L = [D_x; D_y] are forward differences with a zero last column / last row,
  so that L has the constants as its null space (Section 3.1).
* W_k = diag(w), w of length 2n ordered [w_x; w_y].

Images are (height, width) arrays, vectorised row-major: x[i * width + j].
"""
from __future__ import annotations

import numpy as np


def gaussian_taps(sigma: float, radius: int) -> np.ndarray:
    """Gaussian taps g_{-r..r}, g_a proportional to exp(-a^2/(2 sigma^2)), sum 1."""
    a = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-(a * a) / (2.0 * sigma * sigma))
    return g / g.sum()


def _toeplitz_apply(x: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    """y_i = sum_a taps[a + r] * x_{i+a} along ``axis``, zero outside the image."""
    r = (len(taps) - 1) // 2
    length = x.shape[axis]
    y = np.zeros_like(x)
    for a in range(-r, r + 1):
        lo, hi = max(0, -a), min(length, length - a)
        if hi <= lo:
            continue
        if axis == 0:
            y[lo:hi, :] += taps[a + r] * x[lo + a:hi + a, :]
        else:
            y[:, lo:hi] += taps[a + r] * x[:, lo + a:hi + a]
    return y


class Operator:
    """The pieces H, H^T, L, L^T of the shifted operator for one image."""

    def __init__(self, height: int, width: int, sigma: float, radius: int):
        self.height, self.width = height, width
        self.n = height * width
        self.taps = gaussian_taps(sigma, radius)

    # ---- blur -----------------------------------------------------------
    def blur(self, x: np.ndarray) -> np.ndarray:
        """H x = (T_h (x) T_w) x."""
        X = x.reshape(self.height, self.width)
        Y = _toeplitz_apply(_toeplitz_apply(X, self.taps, axis=1), self.taps, axis=0)
        return Y.reshape(-1)

    def blur_adjoint(self, y: np.ndarray) -> np.ndarray:
        """H^T y: the transpose of T applies the reversed taps."""
        Y = y.reshape(self.height, self.width)
        rev = self.taps[::-1]
        X = _toeplitz_apply(_toeplitz_apply(Y, rev, axis=0), rev, axis=1)
        return X.reshape(-1)

    # ---- gradient -------------------------------------------------------
    def grad(self, x: np.ndarray) -> np.ndarray:
        """L x = [D_x x; D_y x], forward differences, zero last column / row."""
        X = x.reshape(self.height, self.width)
        qx = np.zeros_like(X)
        qy = np.zeros_like(X)
        qx[:, :-1] = X[:, 1:] - X[:, :-1]
        qy[:-1, :] = X[1:, :] - X[:-1, :]
        return np.concatenate([qx.reshape(-1), qy.reshape(-1)])

    def grad_adjoint(self, q: np.ndarray) -> np.ndarray:
        """L^T q: (D_x^T q)(i,j) = q(i,j-1)[j>=1] - q(i,j)[j<w-1], same along y."""
        n = self.n
        Qx = q[:n].reshape(self.height, self.width)
        Qy = q[n:].reshape(self.height, self.width)
        X = np.zeros((self.height, self.width))
        X[:, 1:] += Qx[:, :-1]
        X[:, :-1] -= Qx[:, :-1]
        X[1:, :] += Qy[:-1, :]
        X[:-1, :] -= Qy[:-1, :]
        return X.reshape(-1)

    # ---- the operators of Eq. (shift) -------------------------------------
    def apply_A(self, x: np.ndarray) -> np.ndarray:
        """A x = H^T (H x)."""
        return self.blur_adjoint(self.blur(x))

    def apply_E(self, x: np.ndarray, w: np.ndarray) -> np.ndarray:
        """E x = L^T (w .* (L x))."""
        return self.grad_adjoint(w * self.grad(x))

    def apply(self, x: np.ndarray, gamma: float, w: np.ndarray) -> np.ndarray:
        """(A + gamma E) x."""
        return self.apply_A(x) + gamma * self.apply_E(x, w)


def irn_weights(op: Operator, x: np.ndarray, beta: float) -> np.ndarray:
    """Edge-preserving reweighting w = ((L x)^2 + beta^2)^(-1/2), elementwise over 2n.

    This is the IRN/TV-type rule of the workloads (smoothed TV, Section 2.1,
    Eq. tikhonov); the paper's own Gazzola-type rule is ``gazzola_weights``.
    """
    q = op.grad(x)
    return 1.0 / np.sqrt(q * q + beta * beta)


def gazzola_weights(op: Operator, x: np.ndarray, d_prev: np.ndarray, p: float) -> np.ndarray:
    """Cumulative Gazzola-type weights of Section 2.1 (returns the new D diagonal).

    q = D_prev L x, w = |q| / ||q||_inf, w <- 1 - w^p, D_new = diag(w) D_prev.
    E_k uses D_k^2, i.e. the weight vector of ``apply_E`` is D_new**2.
    """
    q = d_prev * op.grad(x)
    m = np.max(np.abs(q))
    w = np.abs(q) / m if m > 0 else np.zeros_like(q)
    return (1.0 - w ** p) * d_prev


def make_data(op: Operator, x_true: np.ndarray, z: np.ndarray, eta: float):
    """Forward model d = H x_true + e, e = eta ||H x_true|| / ||z|| z (Eq. forward);
    returns (d, b) with b = H^T d."""
    hx = op.blur(x_true.reshape(-1))
    zz = z.reshape(-1)
    d = hx + eta * np.linalg.norm(hx) / np.linalg.norm(zz) * zz
    return d, op.blur_adjoint(d)


# ---------------------------------------------------------------------------
# Second forward operator: parallel-beam Radon transform (Section 8.3)
# ---------------------------------------------------------------------------
def radon_bins(height: int, width: int) -> int:
    """Detector bins: odd, centred, covering the image diagonal with a margin:
    2 ceil(sqrt(((h-1)/2)^2 + ((w-1)/2)^2)) + 3."""
    half = np.sqrt(((height - 1) / 2.0) ** 2 + ((width - 1) / 2.0) ** 2)
    return 2 * int(np.ceil(half)) + 3


def radon_angles(n_angles: int) -> np.ndarray:
    """Projection angles in radians: 1, 2, ..., n_angles degrees (Section 8.3 uses 1..135)."""
    return np.deg2rad(np.arange(1, n_angles + 1, dtype=np.float64))


def radon_matrix(height: int, width: int, n_angles: int):
    """C[(a, k), p] = c max(0, 1 - |f_p(a) - k|), f_p(a) = t_p(a) + (nb - 1)/2,
    t_p(a) = x_j cos(theta_a) + y_i sin(theta_a): pixel p = (i, j) with centre
    x_j = j - (w-1)/2, y_i = (h-1)/2 - i is projected onto the detector and split
    between its two nearest bins by linear interpolation; c makes ||C||_F = 1
    (Section 8.3). Rows ordered a * nb + k. Built pixel by pixel (sparse)."""
    import scipy.sparse as sp
    nb = radon_bins(height, width)
    th = radon_angles(n_angles)
    cen = (nb - 1) / 2.0
    rows, cols, vals = [], [], []
    jj, ii = np.meshgrid(np.arange(width), np.arange(height))
    xj = (jj - (width - 1) / 2.0).reshape(-1)
    yi = ((height - 1) / 2.0 - ii).reshape(-1)
    pix = np.arange(height * width)
    for a, t in enumerate(th):
        f = (xj * np.cos(t) + yi * np.sin(t)) + cen
        k0 = np.floor(f)
        for kk in (k0, k0 + 1.0):
            wgt = np.maximum(0.0, 1.0 - np.abs(f - kk))
            rows.append(a * nb + kk.astype(np.int64))
            cols.append(pix)
            vals.append(wgt)
    C = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n_angles * nb, height * width))
    C.eliminate_zeros()
    return C / np.sqrt(np.sum(C.data ** 2))


class RadonOperator(Operator):
    """The shifted operator with C the Radon transform of ``radon_matrix`` in
    place of the blur: A = C^T C, b = C^T d, d a sinogram of m = n_angles * nb
    entries. L and E are unchanged."""

    def __init__(self, height: int, width: int, n_angles: int):
        self.height, self.width = height, width
        self.n = height * width
        self.n_angles = n_angles
        self.nb = radon_bins(height, width)
        self.m = n_angles * self.nb
        self.C = radon_matrix(height, width, n_angles)
        self.taps = np.ones(1)

    def blur(self, x: np.ndarray) -> np.ndarray:
        """C x (a sinogram, m entries)."""
        return self.C @ x.reshape(-1)

    def blur_adjoint(self, y: np.ndarray) -> np.ndarray:
        """C^T y."""
        return self.C.T @ y.reshape(-1)
