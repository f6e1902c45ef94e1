"""Map a synthetic workload (``synth.Workload``) to a library problem description."""
from __future__ import annotations

from .recyc import RS_FP64, RS_GUESS_ORTHOGONAL, make_desc


def desc_for(wl, precision: int = RS_FP64, batched_local: int = 0, maxit=None,
             guess: int = RS_GUESS_ORTHOGONAL, I_L=None, I_R=None, inner: int = 0):
    """rs_problem_desc (plus the shift array it points to) for a workload."""
    return make_desc(wl.height, wl.width, wl.sigma, wl.radius, list(wl.gammas()), wl.tol,
                     int(maxit if maxit is not None else min(wl.maxit, 100_000)), wl.p,
                     wl.a_ritz, wl.b_ritz, wl.n_ritz_local, wl.vnew_cap, wl.I_split, wl.i1,
                     wl.i2, wl.i_star, wl.l_c, wl.J_L, wl.J_R, precision, batched_local,
                     guess, I_L, I_R, getattr(wl, "radon_angles", 0), inner)
