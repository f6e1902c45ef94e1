"""Thin ctypes binding of librecyc (include/recyc.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels. PyTorch supplies device memory (the workspace, inputs and
outputs) and the stream. There is no CPU fallback: loading fails loudly when
the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librecyc.so")

RS_OK, RS_EINVAL, RS_ENOCONV, RS_EBREAKDOWN, RS_ENOTREADY, RS_ECUDA, RS_ENOMEM = range(7)
RS_FP64, RS_MIXED = 0, 1
RS_INIT, RS_UPDATE = 0, 1
RS_GUESS_ORTHOGONAL, RS_GUESS_OBLIQUE, RS_GUESS_OBLIQUE2 = 0, 1, 2
RS_MINRES, RS_CG = 0, 1
STATUS_NAMES = {0: "RS_OK", 1: "RS_EINVAL", 2: "RS_ENOCONV", 3: "RS_EBREAKDOWN",
                4: "RS_ENOTREADY", 5: "RS_ECUDA", 6: "RS_ENOMEM"}


class rs_problem_desc(ctypes.Structure):
    _fields_ = [
        ("height", ctypes.c_int), ("width", ctypes.c_int),
        ("sigma", ctypes.c_double), ("radius", ctypes.c_int),
        ("M", ctypes.c_int), ("gammas_host", ctypes.POINTER(ctypes.c_double)),
        ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
        ("p_max", ctypes.c_int), ("a_ritz", ctypes.c_int), ("b_ritz", ctypes.c_int),
        ("n_ritz_local", ctypes.c_int), ("vnew_cap", ctypes.c_int),
        ("I_split", ctypes.c_int), ("i1", ctypes.c_int), ("i2", ctypes.c_int),
        ("i_star", ctypes.c_int), ("l_c", ctypes.c_int), ("J_L", ctypes.c_int),
        ("J_R", ctypes.c_int), ("precision", ctypes.c_int), ("batched_local", ctypes.c_int),
        ("guess", ctypes.c_int), ("I_L", ctypes.c_int), ("I_R", ctypes.c_int),
        ("inner", ctypes.c_int), ("radon_angles", ctypes.c_int),
    ]


class rs_solve_stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int), ("matvecs", ctypes.c_int), ("local_dim", ctypes.c_int),
        ("sweeps", ctypes.c_int), ("relres0", ctypes.c_double), ("relres_est", ctypes.c_double),
        ("relres_true", ctypes.c_double), ("status", ctypes.c_int),
    ]


class rs_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("k", ctypes.c_int), ("nc", ctypes.c_int),
        ("matvecs_total", ctypes.c_longlong), ("matvecs_overhead", ctypes.c_longlong),
        ("ld", ctypes.c_int), ("kernel_launches", ctypes.c_longlong), ("minres_kernel", ctypes.c_int),
        ("stab_sweeps", ctypes.c_int), ("stab_candidates", ctypes.c_int), ("stab_kept", ctypes.c_int),
        ("tuned_variant", ctypes.c_int),
    ]


class rs_timing(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * 2), ("ms", ctypes.c_double * 2),
                ("pixels", ctypes.c_longlong * 2), ("bytes", ctypes.c_double * 2),
                ("flops", ctypes.c_double * 2), ("phase_ms", ctypes.c_double * 6)]

PHASES = ("init_solves", "update_vnew", "principal_setup", "shift_setup", "shift_minres",
          "fp64_residuals")


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_SIGS = {
    "rs_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(rs_problem_desc)]),
    "rs_create_problem": (_I, [ctypes.POINTER(rs_problem_desc), _P, _P, ctypes.c_size_t, _P,
                               ctypes.POINTER(_P)]),
    "rs_set_weights": (_I, [_P, _P]),
    "rs_update_recycle": (_I, [_P, _I]),
    "rs_set_recycle_basis": (_I, [_P, _P, _I]),
    "rs_solve_shifts": (_I, [_P, _I, _I, _P, ctypes.POINTER(rs_solve_stats), ctypes.POINTER(_I)]),
    "rs_solve_shifts_host": (_I, [_P, _I, _I, _P, _P, ctypes.POINTER(rs_solve_stats), ctypes.POINTER(_I)]),
    "rs_initial_guesses": (_I, [_P, _P, _P]),
    "rs_solve_plain": (_I, [_P, _P, ctypes.POINTER(rs_solve_stats)]),
    "rs_solve_adjoint": (_I, [_P, _P, _P, ctypes.POINTER(rs_solve_stats)]),
    "rs_batch_scratch_bytes": (ctypes.c_size_t, [_I, _I]),
    "rs_solve_shifts_batched": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P),
                                     ctypes.POINTER(ctypes.POINTER(rs_solve_stats)), _P, ctypes.c_size_t]),
    "rs_shift_gradients": (_I, [_P, _P, _P, ctypes.POINTER(_D), _P]),
    "rs_get_principal_basis": (_I, [_P, _P, ctypes.POINTER(_I)]),
    "rs_apply_operator": (_I, [_P, _D, _P, _P, _P, _I, _I]),
    "rs_irn_weights": (_I, [_P, _P, _D, _P]),
    "rs_gazzola_weights": (_I, [_P, _P, _P, _D, _P, _P]),
    "rs_lcurve": (_I, [_P, _P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "rs_synthesize_data": (_I, [ctypes.POINTER(rs_problem_desc), _P, _P, _D, _P, _P,
                                ctypes.c_size_t, _P]),
    "rs_synthesize_data_noalloc": (_I, [ctypes.POINTER(rs_problem_desc), _P, _P, _D, _P, _P]),
    "rs_selftest_grid_barrier": (_I, [_P, ctypes.c_size_t, _P, ctypes.POINTER(_I)]),
    "rs_measure_fp64_fma": (_I, [_P, ctypes.c_size_t, _P, ctypes.POINTER(_D)]),
    "rs_get_info": (_I, [_P, ctypes.POINTER(rs_info)]),
    "rs_set_timing": (_I, [_P, _I]),
    "rs_get_timing": (_I, [_P, ctypes.POINTER(rs_timing)]),
    "rs_last_error": (ctypes.c_char_p, [_P]),
    "rs_destroy": (None, [_P]),
}
EXPORTS = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librecyc.so (built by ``paper_2306_15049_gb300.build``); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librecyc.so not found at {path}: build it with "
                           "`python -m paper_2306_15049_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RecycError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def make_desc(height: int, width: int, sigma: float, radius: int, gammas: Sequence[float],
              tol: float, maxit: int, p_max: int, a_ritz: int, b_ritz: int, n_ritz_local: int,
              vnew_cap: int, I_split: int, i1: int, i2: int, i_star: int, l_c: int, J_L: int,
              J_R: int, precision: int = RS_FP64, batched_local: int = 0,
              guess: int = RS_GUESS_ORTHOGONAL, I_L: Optional[int] = None,
              I_R: Optional[int] = None, radon_angles: int = 0, inner: int = RS_MINRES):
    """An rs_problem_desc; the returned tuple keeps the shift array alive.
    I_L / I_R (two-anchor oblique guesses) default to i_star and l_c."""
    garr = (ctypes.c_double * len(gammas))(*[float(g) for g in gammas])
    d = rs_problem_desc(height, width, float(sigma), radius, len(gammas),
                        ctypes.cast(garr, ctypes.POINTER(ctypes.c_double)), float(tol), maxit,
                        p_max, a_ritz, b_ritz, n_ritz_local, vnew_cap, I_split, i1, i2, i_star,
                        l_c, J_L, J_R, precision, batched_local, guess,
                        i_star if I_L is None else I_L, l_c if I_R is None else I_R, inner,
                        radon_angles)
    return d, garr


def rs_workspace_bytes(desc) -> int:
    return int(load().rs_workspace_bytes(ctypes.byref(desc)))


def rs_synthesize_data(desc, x_dev, z_dev, eta: float, d_out_dev, workspace, stream=None) -> None:
    lib = load()
    st = lib.rs_synthesize_data(ctypes.byref(desc), _ptr(x_dev), _ptr(z_dev), float(eta),
                                _ptr(d_out_dev), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                stream)
    if st != RS_OK:
        raise RecycError(st, lib.rs_last_error(None).decode())


def rs_synthesize_data_noalloc(desc, x_dev, z_dev, eta: float, d_out_dev, stream=None) -> None:
    """rs_synthesize_data for callers that cannot allocate: no workspace argument."""
    lib = load()
    st = lib.rs_synthesize_data_noalloc(ctypes.byref(desc), _ptr(x_dev), _ptr(z_dev), float(eta),
                                        _ptr(d_out_dev), stream)
    if st != RS_OK:
        raise RecycError(st, lib.rs_last_error(None).decode())


def rs_solve_shifts_batched(problems, X_list, scratch=None):
    """Solve the current step of several batched_local problems together (one
    cooperative launch for all their shifts). Returns one stats list per problem."""
    import torch
    lib = load()
    count = len(problems)
    total = sum(p.M for p in problems)
    nbytes = int(lib.rs_batch_scratch_bytes(count, total))
    if nbytes == 0:
        raise RecycError(RS_EINVAL, "invalid batch")
    if scratch is None or scratch.numel() * scratch.element_size() < nbytes:
        scratch = torch.empty(nbytes, dtype=torch.uint8, device=X_list[0].device)
    probs = (ctypes.c_void_p * count)(*[p.h for p in problems])
    xs = (ctypes.c_void_p * count)(*[_ptr(x) for x in X_list])
    stats = [(rs_solve_stats * p.M)() for p in problems]
    sp = (ctypes.POINTER(rs_solve_stats) * count)(*[ctypes.cast(st, ctypes.POINTER(rs_solve_stats)) for st in stats])
    st = lib.rs_solve_shifts_batched(probs, count, xs, sp, _ptr(scratch), nbytes)
    if st not in (RS_OK, RS_ENOCONV):
        raise RecycError(st, lib.rs_last_error(None).decode())
    return [[dict((f, getattr(s_, f)) for f, _ in rs_solve_stats._fields_) for s_ in stl] for stl in stats]


class Problem:
    """One shifted-system problem: owns the library handle and a torch workspace.

    Methods mirror the C entry points (rs_set_weights, rs_update_recycle,
    rs_solve_shifts, ...); device tensors must be contiguous float64 CUDA
    tensors on the current device.
    """

    def __init__(self, desc_and_keep, d_dev, stream=None, workspace=None):
        import torch
        lib = load()
        self.desc, self._keep = desc_and_keep
        self.n = self.desc.height * self.desc.width
        self.M = self.desc.M
        nbytes = rs_workspace_bytes(self.desc)
        if nbytes == 0:
            raise RecycError(RS_EINVAL, "invalid problem description")
        if workspace is not None and workspace.numel() * workspace.element_size() >= nbytes:
            self.workspace = workspace
        else:
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=d_dev.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(d_dev.device).cuda_stream
        h = ctypes.c_void_p()
        st = lib.rs_create_problem(ctypes.byref(self.desc), _ptr(d_dev), _ptr(self.workspace), nbytes,
                                   self.stream, ctypes.byref(h))
        if st != RS_OK:
            raise RecycError(st, lib.rs_last_error(None).decode())
        self.h = h
        self.lib = lib

    def _check(self, st, allow=(RS_OK,)):
        if st not in allow:
            raise RecycError(st, self.lib.rs_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.rs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rs_set_weights(self, w_dev):
        return self._check(self.lib.rs_set_weights(self.h, _ptr(w_dev)))

    def rs_update_recycle(self, mode: int):
        return self._check(self.lib.rs_update_recycle(self.h, int(mode)))

    def rs_set_recycle_basis(self, U_dev, ncols: int):
        return self._check(self.lib.rs_set_recycle_basis(self.h, _ptr(U_dev), int(ncols)))

    def rs_solve_shifts(self, X_dev, iters_override: Optional[List[int]] = None, allow_noconv=False,
                        l0: int = 0, count: Optional[int] = None):
        """Shifts l0 .. l0 + count - 1 (default: all M); X_dev holds count rows."""
        count = self.M - l0 if count is None else int(count)
        stats = (rs_solve_stats * max(count, 1))()
        ov = None
        if iters_override is not None:
            ov = (ctypes.c_int * len(iters_override))(*[int(v) for v in iters_override])
        st = self.lib.rs_solve_shifts(self.h, int(l0), count, _ptr(X_dev), stats, ov)
        self._check(st, (RS_OK, RS_ENOCONV) if allow_noconv else (RS_OK,))
        return [dict((f, getattr(s, f)) for f, _ in rs_solve_stats._fields_) for s in stats[:count]]

    def rs_solve_shifts_host(self, X_dev, X_host, iters_override: Optional[List[int]] = None,
                             allow_noconv=False, l0: int = 0, count: Optional[int] = None):
        """rs_solve_shifts, each solution also copied into the host tensor X_host
        (count rows; page-locked for overlap) as soon as it is final."""
        count = self.M - l0 if count is None else int(count)
        stats = (rs_solve_stats * max(count, 1))()
        ov = None
        if iters_override is not None:
            ov = (ctypes.c_int * len(iters_override))(*[int(v) for v in iters_override])
        st = self.lib.rs_solve_shifts_host(self.h, int(l0), count, _ptr(X_dev), _ptr(X_host), stats, ov)
        self._check(st, (RS_OK, RS_ENOCONV) if allow_noconv else (RS_OK,))
        return [dict((f, getattr(s, f)) for f, _ in rs_solve_stats._fields_) for s in stats[:count]]

    def rs_solve_plain(self, X_dev, allow_noconv=False):
        stats = (rs_solve_stats * self.M)()
        st = self.lib.rs_solve_plain(self.h, _ptr(X_dev), stats)
        self._check(st, (RS_OK, RS_ENOCONV) if allow_noconv else (RS_OK,))
        return [dict((f, getattr(s, f)) for f, _ in rs_solve_stats._fields_) for s in stats]

    def rs_solve_adjoint(self, G_dev, Lam_dev, allow_noconv=False):
        stats = (rs_solve_stats * self.M)()
        st = self.lib.rs_solve_adjoint(self.h, _ptr(G_dev), _ptr(Lam_dev), stats)
        self._check(st, (RS_OK, RS_ENOCONV) if allow_noconv else (RS_OK,))
        return [dict((f, getattr(s, f)) for f, _ in rs_solve_stats._fields_) for s in stats]

    def rs_shift_gradients(self, X_dev, Lam_dev, dw_dev) -> List[float]:
        dg = (ctypes.c_double * self.M)()
        self._check(self.lib.rs_shift_gradients(self.h, _ptr(X_dev), _ptr(Lam_dev), dg, _ptr(dw_dev)))
        return list(dg)

    def rs_initial_guesses(self, X0_dev, R0_dev):
        return self._check(self.lib.rs_initial_guesses(self.h, _ptr(X0_dev), _ptr(R0_dev)))

    def rs_get_principal_basis(self, U_dev) -> int:
        nc = ctypes.c_int()
        self._check(self.lib.rs_get_principal_basis(self.h, _ptr(U_dev), ctypes.byref(nc)))
        return nc.value

    def rs_apply_operator(self, gamma: float, x_dev, y_dev, y2_dev=None, mode: int = 0,
                          working_precision: bool = False):
        return self._check(self.lib.rs_apply_operator(self.h, float(gamma), _ptr(x_dev), _ptr(y_dev),
                                                      _ptr(y2_dev), int(mode), int(working_precision)))

    def rs_irn_weights(self, x_dev, beta: float, w_dev):
        return self._check(self.lib.rs_irn_weights(self.h, _ptr(x_dev), float(beta), _ptr(w_dev)))

    def rs_gazzola_weights(self, x_dev, d_prev_dev, p: float, d_new_dev, w_dev):
        return self._check(self.lib.rs_gazzola_weights(self.h, _ptr(x_dev), _ptr(d_prev_dev), float(p),
                                                       _ptr(d_new_dev), _ptr(w_dev)))

    def rs_lcurve(self, X_dev, count: int):
        rho = (ctypes.c_double * count)()
        eta = (ctypes.c_double * count)()
        ls = ctypes.c_int()
        self._check(self.lib.rs_lcurve(self.h, _ptr(X_dev), int(count), rho, eta, ctypes.byref(ls)))
        return list(rho), list(eta), ls.value

    def rs_set_timing(self, on: bool):
        return self._check(self.lib.rs_set_timing(self.h, int(bool(on))))

    def rs_get_timing(self) -> dict:
        t = rs_timing()
        self._check(self.lib.rs_get_timing(self.h, ctypes.byref(t)))
        return {"launches": list(t.launches), "ms": list(t.ms), "pixels": list(t.pixels),
                "bytes": list(t.bytes), "flops": list(t.flops),
                "phase_ms": dict(zip(PHASES, list(t.phase_ms)))}

    def rs_get_info(self) -> dict:
        info = rs_info()
        self._check(self.lib.rs_get_info(self.h, ctypes.byref(info)))
        return dict((f, getattr(info, f)) for f, _ in rs_info._fields_)
