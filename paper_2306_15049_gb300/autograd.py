"""torch.autograd.Function over the recycled shifted solves.

Forward: x_l = (A + gamma_l E(w))^{-1} b for all shifts of one outer step
(k = 0: the principal space of Section 5.1) through librecyc. Backward: one
adjoint solve per shift with the same symmetric operator, reusing the
forward's recycle space (rs_solve_adjoint), then d loss / d gamma and
d loss / d w from rs_shift_gradients. No Krylov basis is stored: the saved
state is the solutions X and the problem's recycle space. Argument marshalling
only; every step runs in the library's kernels.
"""
from __future__ import annotations

from typing import Callable

import torch

from . import recyc


class RecycledShiftedSolve(torch.autograd.Function):
    """X = RecycledShiftedSolve.apply(gammas, w, d, make_desc).

    gammas: (M,) float64 tensor, strictly increasing, > 0; w: (2n,) float64 CUDA
    tensor of weights; d: (n,) float64 CUDA data image; make_desc: callable
    gammas (list of floats) -> (rs_problem_desc, keep) as returned by
    ``recyc.make_desc``. Returns X (M x n float64, CUDA).
    """

    @staticmethod
    def forward(ctx, gammas: torch.Tensor, w: torch.Tensor, d: torch.Tensor,
                make_desc: Callable):
        g = [float(v) for v in gammas.detach().cpu().tolist()]
        P = recyc.Problem(make_desc(g), d.detach().contiguous())
        P.rs_set_weights(w.detach().contiguous())
        P.rs_update_recycle(recyc.RS_INIT)
        X = torch.empty(P.M, P.n, dtype=torch.float64, device=d.device)
        ctx.stats = P.rs_solve_shifts(X)
        ctx.P = P
        ctx.gdev = gammas.device
        ctx.save_for_backward(X)
        return X

    @staticmethod
    def backward(ctx, gX: torch.Tensor):
        (X,) = ctx.saved_tensors
        P = ctx.P
        Lam = torch.empty_like(X)
        ctx.adjoint_stats = P.rs_solve_adjoint(gX.contiguous().to(torch.float64), Lam)
        dw = torch.empty(2 * P.n, dtype=torch.float64, device=X.device)
        dg = P.rs_shift_gradients(X, Lam, dw)
        dgamma = torch.tensor(dg, dtype=torch.float64, device=ctx.gdev)
        return dgamma, dw, None, None


def solve_shifts(gammas: torch.Tensor, w: torch.Tensor, d: torch.Tensor, make_desc: Callable):
    """Differentiable solutions of all shifted systems (see RecycledShiftedSolve)."""
    return RecycledShiftedSolve.apply(gammas, w, d, make_desc)
