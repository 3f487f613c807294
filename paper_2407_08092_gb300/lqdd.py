"""Python binding of the C ABI in ``include/lqdd.h`` (argument marshalling only).

Every function has the name of its C entry point and forwards to it through
ctypes; all arithmetic runs in the CUDA library ``liblqdd.so``.  Field
arguments are CUDA tensors (complex128, contiguous) or raw device pointers.
There is no fallback: if the library is missing, importing this module fails.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# LQ_LIBRARY may name another build of the same library (the index-checked
# liblqdd_checked.so that the bounds tests load in a child process)
LIB_PATH = os.environ.get("LQ_LIBRARY") or os.path.join(_HERE, "liblqdd.so")

(LQ_OK, LQ_ERR_ARG, LQ_ERR_CUDA, LQ_ERR_OOM, LQ_ERR_NOT_CONVERGED, LQ_ERR_BREAKDOWN, LQ_ERR_NAN, LQ_ERR_STATE,
 LQ_ERR_BOUNDS) = range(9)
LQ_F64, LQ_F32, LQ_DF64, LQ_BF16 = 0, 1, 2, 3
LQ_OP_FULL, LQ_OP_SCHUR, LQ_OP_SCHUR_DAG, LQ_OP_EE, LQ_OP_OO_INV = range(5)
LQ_SOLVER_GMRES, LQ_SOLVER_FGMRES = 0, 1
LQ_SMOOTH_NONE, LQ_SMOOTH_RICHARDSON, LQ_SMOOTH_GMRES, LQ_SMOOTH_SAP = 0, 1, 2, 3


class lq_lattice(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("t_bc", ctypes.c_int), ("m0", ctypes.c_double),
                ("csw", ctypes.c_double)]


class lq_solver_params(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("prec", ctypes.c_int), ("tol", ctypes.c_double),
                ("restart", ctypes.c_int), ("max_restarts", ctypes.c_int), ("smoother", ctypes.c_int),
                ("smooth_n", ctypes.c_int), ("smooth_m", ctypes.c_int), ("omega", ctypes.c_double),
                ("smooth_tol", ctypes.c_double), ("inner_prec", ctypes.c_int), ("sap_block", ctypes.c_int * 4)]


class lq_stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("iters", ctypes.c_int), ("inner_iters", ctypes.c_longlong),
                ("rel_resid", ctypes.c_double), ("rel_resid_true", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("bytes", ctypes.c_double), ("launches", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LqError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_2407_08092_gb300.build` (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)
_P = ctypes.c_void_p
_lib.lq_create.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(lq_lattice), _P]
_lib.lq_destroy.argtypes = [_P]
_lib.lq_set_gauge.argtypes = [_P, _P]
_lib.lq_apply.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P]
_lib.lq_prepare.argtypes = [_P, _P, _P]
_lib.lq_reconstruct.argtypes = [_P, _P, _P, _P]
_lib.lq_estimate_norm.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]
_lib.lq_norm2.argtypes = [_P, _P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double)]
_lib.lq_smooth.argtypes = [_P, ctypes.POINTER(lq_solver_params), _P, _P]
_lib.lq_solve.argtypes = [_P, ctypes.POINTER(lq_solver_params), _P, _P, ctypes.POINTER(lq_stats)]
_lib.lq_export_clover.argtypes = [_P, ctypes.c_int, _P]
_lib.lq_counters.argtypes = [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]
_lib.lq_profile.argtypes = [_P, ctypes.c_int]
_lib.lq_profile_read.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)]
_lib.lq_norm2_noalloc.argtypes = [_P, ctypes.c_longlong, _P, _P]
_lib.lq_norm2_noalloc.restype = ctypes.c_int
_lib.lq_bounds_check.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_ulonglong),
                                 ctypes.POINTER(ctypes.c_int)]
_lib.lq_bounds_check.restype = ctypes.c_int
_lib.lq_kernel_class_name.argtypes = [ctypes.c_int]
_lib.lq_kernel_class_name.restype = ctypes.c_char_p
_lib.lq_last_error.argtypes = [_P]
_lib.lq_last_error.restype = ctypes.c_char_p
_lib.lq_status_string.argtypes = [ctypes.c_int]
_lib.lq_status_string.restype = ctypes.c_char_p
for _name in ("lq_create", "lq_destroy", "lq_set_gauge", "lq_apply", "lq_prepare", "lq_reconstruct",
              "lq_estimate_norm", "lq_norm2", "lq_smooth", "lq_solve", "lq_export_clover", "lq_counters",
              "lq_profile", "lq_profile_read"):
    getattr(_lib, _name).restype = ctypes.c_int


def library():
    """The loaded ctypes library (for callers that need a raw symbol)."""
    return _lib


def _status_name(s: int) -> str:
    return _lib.lq_status_string(int(s)).decode()


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        import torch
        if not x.is_cuda:
            raise ValueError("field must be a CUDA tensor")
        if x.dtype != torch.complex128:
            raise ValueError("field must be complex128")
        if not x.is_contiguous():
            raise ValueError("field must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _check(ctx, status: int):
    if status != LQ_OK:
        msg = _lib.lq_last_error(ctx).decode() if ctx else ""
        raise LqError(status, msg)


def lq_status_string(s: int) -> str:
    return _status_name(s)


def lq_last_error(ctx) -> str:
    return _lib.lq_last_error(ctx).decode()


def lq_create(lat: lq_lattice, stream: int | None = None):
    ctx = _P()
    _check(None, _lib.lq_create(ctypes.byref(ctx), ctypes.byref(lat), _P(stream or 0)))
    return ctx


def lq_destroy(ctx) -> None:
    _check(None, _lib.lq_destroy(ctx))


def lq_set_gauge(ctx, U) -> None:
    _check(ctx, _lib.lq_set_gauge(ctx, _ptr(U)))


def lq_apply(ctx, op: int, prec: int, inp, out) -> None:
    _check(ctx, _lib.lq_apply(ctx, int(op), int(prec), _ptr(inp), _ptr(out)))


def lq_prepare(ctx, b, bhat_e) -> None:
    _check(ctx, _lib.lq_prepare(ctx, _ptr(b), _ptr(bhat_e)))


def lq_reconstruct(ctx, b, x_e, x) -> None:
    _check(ctx, _lib.lq_reconstruct(ctx, _ptr(b), _ptr(x_e), _ptr(x)))


def lq_estimate_norm(ctx, prec: int, iters: int, v0) -> float:
    out = ctypes.c_double()
    _check(ctx, _lib.lq_estimate_norm(ctx, int(prec), int(iters), _ptr(v0), ctypes.byref(out)))
    return out.value


def lq_norm2(ctx, v, n_sites: int) -> float:
    out = ctypes.c_double()
    _check(ctx, _lib.lq_norm2(ctx, _ptr(v), int(n_sites), ctypes.byref(out)))
    return out.value


LQ_NORM2_NOALLOC_MAX_SITES = 2796202


def lq_bounds_check():
    """(status, checked, violations, first_code) of the checked build's index
    checks since the last call (synchronises the device); status is LQ_OK or
    LQ_ERR_BOUNDS and is returned, not raised."""
    c, n, f = ctypes.c_int(), ctypes.c_ulonglong(), ctypes.c_int()
    st = _lib.lq_bounds_check(ctypes.byref(c), ctypes.byref(n), ctypes.byref(f))
    if st not in (LQ_OK, LQ_ERR_BOUNDS):
        raise LqError(st, "lq_bounds_check")
    return st, c.value, n.value, f.value


def lq_norm2_noalloc(v, n_sites: int, out, stream: int | None = None) -> None:
    """||v||^2 into the device double `out`, without any device allocation and
    without a context (for callers that cannot allocate device memory).  `out`
    is a CUDA float64 tensor of one element or a raw device pointer; the call
    only enqueues work on `stream`."""
    if hasattr(out, "data_ptr"):
        import torch
        if not out.is_cuda or out.dtype != torch.float64 or out.numel() < 1:
            raise ValueError("out must be a CUDA float64 tensor with at least one element")
        out_p = out.data_ptr()
    else:
        out_p = int(out)
    s = _lib.lq_norm2_noalloc(_P(_ptr(v) if int(n_sites) > 0 else 0), int(n_sites), _P(out_p), _P(stream or 0))
    if s != LQ_OK:
        raise LqError(s, "lq_norm2_noalloc")


def lq_smooth(ctx, params: lq_solver_params, r, e) -> None:
    _check(ctx, _lib.lq_smooth(ctx, ctypes.byref(params), _ptr(r), _ptr(e)))


def lq_solve(ctx, params: lq_solver_params, b, x):
    """Returns (status, stats); raises on every status but OK and NOT_CONVERGED."""
    st = lq_stats()
    s = _lib.lq_solve(ctx, ctypes.byref(params), _ptr(b), _ptr(x), ctypes.byref(st))
    if s not in (LQ_OK, LQ_ERR_NOT_CONVERGED):
        _check(ctx, s)
    return s, st


_lib.lq_solve_batch.argtypes = [_P, ctypes.POINTER(lq_solver_params), ctypes.c_int, _P, _P,
                                ctypes.POINTER(lq_stats)]
_lib.lq_solve_batch.restype = ctypes.c_int


def lq_solve_batch(ctx, params: lq_solver_params, n_rhs: int, b, x):
    """Batched solve of n_rhs systems; b, x are [n_rhs, V, 4, 3] complex128 CUDA
    tensors.  Returns (status, [stats per right-hand side]); raises on every
    status but OK and NOT_CONVERGED."""
    st = (lq_stats * int(n_rhs))()
    s = _lib.lq_solve_batch(ctx, ctypes.byref(params), int(n_rhs), _ptr(b), _ptr(x), st)
    if s not in (LQ_OK, LQ_ERR_NOT_CONVERGED):
        _check(ctx, s)
    return s, list(st)


_lib.lq_force.argtypes = [_P, _P, _P, ctypes.c_double, _P]
_lib.lq_force.restype = ctypes.c_int
_lib.lq_fermion_force.argtypes = [_P, ctypes.POINTER(lq_solver_params), _P, ctypes.POINTER(ctypes.c_double), _P,
                                  ctypes.POINTER(lq_stats)]
_lib.lq_fermion_force.restype = ctypes.c_int


def lq_force(ctx, X, Y, G, coef: float = 1.0):
    """G = coef * grad_U Re(Y^+ D X) for full spinors X, Y ([V, 4, 3] complex128
    CUDA tensors); G is a [V, 4, 3, 3] complex128 CUDA tensor."""
    _check(ctx, _lib.lq_force(ctx, _ptr(X), _ptr(Y), float(coef), _ptr(G)))


_lib.lq_fermion_action.argtypes = [_P, ctypes.POINTER(lq_solver_params), _P, _P, _P, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(lq_stats)]
_lib.lq_fermion_action.restype = ctypes.c_int


def lq_fermion_action(ctx, params: lq_solver_params, phi, X, Y):
    """S = phi^+ (D^+ D)^{-1} phi; writes X = (D^+ D)^{-1} phi and Y = D X.
    Returns (status, S, [stats of the two solves]); raises on every status but
    OK and NOT_CONVERGED."""
    S = ctypes.c_double()
    st = (lq_stats * 2)()
    s = _lib.lq_fermion_action(ctx, ctypes.byref(params), _ptr(phi), _ptr(X), _ptr(Y), ctypes.byref(S), st)
    if s not in (LQ_OK, LQ_ERR_NOT_CONVERGED):
        _check(ctx, s)
    return s, S.value, list(st)


def lq_fermion_force(ctx, params: lq_solver_params, phi, G):
    """S = phi^+ (D^+ D)^{-1} phi and G = dS/dU.  Returns (status, S, [stats of
    the two solves]); raises on every status but OK and NOT_CONVERGED."""
    S = ctypes.c_double()
    st = (lq_stats * 2)()
    s = _lib.lq_fermion_force(ctx, ctypes.byref(params), _ptr(phi), ctypes.byref(S), _ptr(G), st)
    if s not in (LQ_OK, LQ_ERR_NOT_CONVERGED):
        _check(ctx, s)
    return s, S.value, list(st)


_lib.lq_group_create.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int, _P]
_lib.lq_group_create.restype = ctypes.c_int
_lib.lq_group_destroy.argtypes = [_P]
_lib.lq_group_destroy.restype = ctypes.c_int
_lib.lq_solve_group.argtypes = [_P, ctypes.POINTER(lq_solver_params), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(lq_stats)]
_lib.lq_solve_group.restype = ctypes.c_int
_lib.lq_group_set_autotune.argtypes = [_P, ctypes.c_int]
_lib.lq_group_set_autotune.restype = ctypes.c_int
_lib.lq_group_tuning.argtypes = [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
_lib.lq_group_tuning.restype = ctypes.c_int


def lq_group_create(members, stream: int | None = None):
    """A group of contexts solved together; errors are reported through the
    first member's lq_last_error."""
    arr = (_P * len(members))(*[m.value if isinstance(m, _P) else m for m in members])
    grp = _P()
    _check(members[0], _lib.lq_group_create(ctypes.byref(grp), arr, len(members), _P(stream or 0)))
    return grp


def lq_group_destroy(grp) -> None:
    _check(None, _lib.lq_group_destroy(grp))


def lq_solve_group(grp, first_member, params: lq_solver_params, b_list, x_list):
    """Solve every member's right-hand sides together.  b_list[l], x_list[l]:
    [n_rhs_l, V_l, 4, 3] complex128 CUDA tensors.  Returns (status, [stats per
    system, member by member]); raises on every status but OK and NOT_CONVERGED
    (the message comes from `first_member`, the group's first context)."""
    M = len(b_list)
    n = (ctypes.c_int * M)(*[int(b.shape[0]) for b in b_list])
    bp = (_P * M)(*[_ptr(b) for b in b_list])
    xp = (_P * M)(*[_ptr(x) for x in x_list])
    st = (lq_stats * sum(n))()
    s = _lib.lq_solve_group(grp, ctypes.byref(params), n, bp, xp, st)
    if s not in (LQ_OK, LQ_ERR_NOT_CONVERGED):
        _check(first_member, s)
    return s, list(st)


def lq_group_set_autotune(grp, on: bool) -> None:
    _check(None, _lib.lq_group_set_autotune(grp, int(bool(on))))


_lib.lq_group_set_shape.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
_lib.lq_group_set_shape.restype = ctypes.c_int


def lq_group_set_shape(grp, sites_per_tile: int, rhs_per_thread: int, grid_factor: int) -> None:
    _check(None, _lib.lq_group_set_shape(grp, int(sites_per_tile), int(rhs_per_thread), int(grid_factor)))


def lq_group_tuning(grp):
    """(sites per tile, right-hand sides per thread, grid, BLAS blocks per
    system, hop ms, BLAS ms) in use."""
    a, r, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    d, e = ctypes.c_double(), ctypes.c_double()
    _check(None, _lib.lq_group_tuning(grp, ctypes.byref(a), ctypes.byref(r), ctypes.byref(b), ctypes.byref(c),
                                      ctypes.byref(d), ctypes.byref(e)))
    return a.value, r.value, b.value, c.value, d.value, e.value


def make_batch_params(tol=1e-10, restart=8, max_restarts=10, smooth_n=16, smooth_tol=1e-5) -> lq_solver_params:
    """Parameters of lq_solve_batch: df64 defect correction around batched FP32 GMRES(restart)."""
    return make_params(solver=LQ_SOLVER_GMRES, prec=LQ_DF64, tol=tol, restart=restart, max_restarts=max_restarts,
                       smoother=LQ_SMOOTH_GMRES, smooth_n=smooth_n, smooth_m=restart, smooth_tol=smooth_tol,
                       inner_prec=LQ_F32)


def lq_export_clover(ctx, which: int, out) -> None:
    _check(ctx, _lib.lq_export_clover(ctx, int(which), _ptr(out)))


def lq_counters(ctx):
    n = ctypes.c_longlong()
    b = ctypes.c_double()
    _check(ctx, _lib.lq_counters(ctx, ctypes.byref(n), ctypes.byref(b)))
    return n.value, b.value


LQ_K_COUNT = 23


def lq_profile(ctx, on: bool) -> None:
    _check(ctx, _lib.lq_profile(ctx, 1 if on else 0))


def lq_profile_read(ctx, cls: int):
    """(launches, milliseconds, algorithmic bytes, algorithmic flops) of one kernel class."""
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    b = ctypes.c_double()
    f = ctypes.c_double()
    _check(ctx, _lib.lq_profile_read(ctx, int(cls), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b),
                                     ctypes.byref(f)))
    return n.value, ms.value, b.value, f.value


def lq_kernel_class_name(cls: int) -> str:
    return _lib.lq_kernel_class_name(int(cls)).decode()


# ---- small conveniences (no arithmetic) ----------------------------------------------

def make_lattice(L, t_bc: int = -1, m0: float = 0.0, csw: float = 1.0) -> lq_lattice:
    lat = lq_lattice()
    for i in range(4):
        lat.L[i] = int(L[i])
    lat.t_bc, lat.m0, lat.csw = int(t_bc), float(m0), float(csw)
    return lat


def make_params(solver=LQ_SOLVER_GMRES, prec=LQ_F64, tol=1e-10, restart=30, max_restarts=1000,
                smoother=LQ_SMOOTH_NONE, smooth_n=0, smooth_m=1, omega=0.0, smooth_tol=0.0,
                inner_prec=LQ_F64, sap_block=(0, 0, 0, 0)) -> lq_solver_params:
    return lq_solver_params(solver, prec, tol, restart, max_restarts, smoother, smooth_n, smooth_m,
                            omega, smooth_tol, inner_prec, (ctypes.c_int * 4)(*sap_block))
