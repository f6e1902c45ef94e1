"""Seeded synthetic workloads for the recycled shifted-system solver.

This module is shared by the FP64 oracle and by the GPU path. It holds no
arithmetic of the method itself (no blur, no gradient, no weights, no solver):
it only draws the seeded random inputs and states the workload parameters.

Every workload follows the structure of the paper's experiments (Section 8):
a piecewise-constant ground-truth image, a zero-boundary Gaussian blur, white
noise of a stated relative level, and shifts gamma_l = lambda_l^2 spread
log-evenly over many decades (Section 2.2). The paper's own test images
(Regtools ``blur.m``, a CT phantom) are not available; the random
rectangles/disks below stand in for them.

Recipe (one image, seed ``s``):

* ``x_true`` starts at zero; ``S = min(64, max(6, width // 8))`` shapes are
  painted in order, alternately an axis-aligned rectangle and a disk; the
  centre is uniform over the image, the half-side / radius uniform in
  ``[width/16, width/4]``, the value uniform in ``[0, 1]``; later shapes
  overwrite earlier ones.
* ``z`` is a standard normal vector of the image size (the noise direction);
  each side forms ``d = H x_true + eta * ||H x_true|| / ||z|| * z`` with its own
  blur. CT workloads draw ``z`` of the sinogram size instead
  (``sinogram_noise``) and use their own Radon transform in place of H.
* shifts ``gamma = logspace(lo, hi, M)``.
* seeds ``20230615 + 10 * config_index + image_index``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np

SEED_BASE = 20230615


@dataclasses.dataclass(frozen=True)
class Workload:
    """Parameters of one shifted-system workload (one image).

    Index fields are 1-based, as in the paper's index table (Section 5.5).
    """

    name: str
    height: int
    width: int
    sigma: float
    radius: int
    eta: float            # relative noise level
    M: int                # number of shifts
    log_lo: float         # gamma_1 = 10**log_lo
    log_hi: float         # gamma_M = 10**log_hi
    K: int                # number of outer (reweighting) steps
    p: int                # principal recycle dimension cap (n_c <= p)
    n_ritz_local: int     # |J|, Ritz vectors per local space
    tol: float = 1e-8
    beta: float = 1e-3    # smoothing of the edge-preserving weights
    seed: int = SEED_BASE
    radon_angles: int = 0  # > 0: CT forward model (angles 1..radon_angles degrees) instead of the blur

    # ---- derived index choices (readings scaled from Ex. 1 / Ex. 2) ----
    @property
    def n(self) -> int:
        return self.height * self.width

    @property
    def I_split(self) -> int:
        return int(round(0.75 * self.M))

    @property
    def i1(self) -> int:
        return 1

    @property
    def i2(self) -> int:
        return max(1, self.M // 2)

    @property
    def i_star(self) -> int:
        return max(1, self.M // 2)

    @property
    def J_L(self) -> int:
        return self.I_split

    @property
    def J_R(self) -> int:
        return max(self.I_split + 1, self.M - 1) if self.I_split < self.M else self.M

    @property
    def l_c(self) -> int:
        return max(1, self.M - 1)

    @property
    def a_ritz(self) -> int:
        """Lanczos vectors kept from the gamma_{i1} solve (all become V_{i1})."""
        return (2 * (self.p - 2)) // 3

    @property
    def b_ritz(self) -> int:
        """Ritz vectors with the smallest Ritz values kept from the gamma_{i2} solve."""
        return self.p - 2 - self.a_ritz

    @property
    def vnew_cap(self) -> int:
        """MINRES steps for V^(new): at most 100, and a pre-stabilize width <= 2p."""
        return max(1, min(100, 2 * self.p - self.a_ritz - 1 - self.M))

    @property
    def maxit(self) -> int:
        return 10 * self.n

    def gammas(self) -> np.ndarray:
        return shift_grid(self.log_lo, self.log_hi, self.M)


def shift_grid(log_lo: float, log_hi: float, M: int) -> np.ndarray:
    """Log-evenly spaced shifts gamma_1 < ... < gamma_M (Section 2.2)."""
    return np.logspace(log_lo, log_hi, M, dtype=np.float64)


def piecewise_constant_image(height: int, width: int, seed: int) -> np.ndarray:
    """Ground-truth image of random rectangles and disks, values in [0, 1].

    Returned as a (height, width) float64 array (row-major vectorisation
    ``x[i * width + j]``).
    """
    rng = np.random.default_rng(seed)
    x = np.zeros((height, width), dtype=np.float64)
    n_shapes = min(64, max(6, width // 8))
    ii, jj = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    lo, hi = width / 16.0, width / 4.0
    for s in range(n_shapes):
        ci = rng.uniform(0, height)
        cj = rng.uniform(0, width)
        size = rng.uniform(lo, hi)
        val = rng.uniform(0.0, 1.0)
        if s % 2 == 0:
            size2 = rng.uniform(lo, hi)
            mask = (np.abs(ii - ci) <= size) & (np.abs(jj - cj) <= size2)
        else:
            mask = (ii - ci) ** 2 + (jj - cj) ** 2 <= size * size
        x[mask] = val
    return x


def noise_direction(height: int, width: int, seed: int) -> np.ndarray:
    """Standard normal noise direction z (scaled by each side to the level eta)."""
    rng = np.random.default_rng(seed + 7919)
    return rng.standard_normal((height, width))


def sinogram_noise(m: int, seed: int) -> np.ndarray:
    """Standard normal noise direction of the m sinogram entries (CT workloads)."""
    rng = np.random.default_rng(seed + 7919)
    return rng.standard_normal(m)


def random_weights(n: int, seed: int, lo: float = 0.5, hi: float = 50.0) -> np.ndarray:
    """Positive test weights of length 2n spread log-uniformly in [lo, hi]."""
    rng = np.random.default_rng(seed + 104729)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=2 * n))


def random_vectors(n: int, k: int, seed: int) -> np.ndarray:
    """k standard normal vectors of length n, as an (n, k) array."""
    rng = np.random.default_rng(seed + 1299709)
    return rng.standard_normal((n, k))


# ---------------------------------------------------------------------------
# The five workloads. C1 is small enough for the oracle in seconds; C2 is the
# single-image GPU workload; C3-C5 are the batched, differentiated and
# large mixed-precision workloads.
# ---------------------------------------------------------------------------

C1 = Workload("C1-64x64-fp64", 64, 64, 1.5, 4, 0.01, 8, -4.0, 0.0, 3, 10, 4,
              seed=SEED_BASE + 10)
C2 = Workload("C2-512x512", 512, 512, 2.5, 8, 0.02, 16, -5.0, 0.0, 5, 40, 8,
              seed=SEED_BASE + 20)
C3_IMAGES: List[Tuple[int, float, int]] = [(256, 1.5, 4), (384, 2.0, 6), (512, 2.5, 8), (1024, 3.0, 10)]
C3 = [Workload(f"C3-{s}x{s}", s, s, sig, r, 0.02, 32, -5.0, 0.0, 1, 40, 8,
               seed=SEED_BASE + 30 + i) for i, (s, sig, r) in enumerate(C3_IMAGES)]
C4 = Workload("C4-1024x1024", 1024, 1024, 3.0, 10, 0.02, 16, -5.0, 0.0, 1, 40, 8,
              seed=SEED_BASE + 40)
C5 = Workload("C5-2048x2048", 2048, 2048, 4.0, 12, 0.03, 64, -6.0, 0.0, 8, 100, 8,
              seed=SEED_BASE + 50)

# Stand-in for the CT example of Section 8.3: an 82 x 82 piecewise-constant image,
# parallel-beam projections at 1..135 degrees, 1 % noise, 20 shifts
# gamma = lambda^2 with lambda log-spaced over 1e-4..1e1; principal dimension 30
# and 8 local Ritz vectors (not stated for this example).
CT82 = Workload("CT82-135deg", 82, 82, 1.0, 0, 0.01, 20, -8.0, 2.0, 3, 30, 8,
                seed=SEED_BASE + 60, radon_angles=135)

WORKLOADS = {"C1": C1, "C2": C2, "C4": C4, "C5": C5, "CT82": CT82}


def tiny(height: int, width: int, sigma: float = 1.0, radius: int = 2, M: int = 6,
         p: int = 8, n_ritz_local: int = 3, K: int = 2, seed: int = SEED_BASE + 1,
         log_lo: float = -3.0, log_hi: float = 0.0, eta: float = 0.01,
         tol: float = 1e-10, radon_angles: int = 0) -> Workload:
    """A small workload for dense-matrix checks (any image size, odd sizes allowed)."""
    return Workload(f"tiny-{height}x{width}", height, width, sigma, radius, eta, M,
                    log_lo, log_hi, K, p, n_ritz_local, tol=tol, seed=seed,
                    radon_angles=radon_angles)
