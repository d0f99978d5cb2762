"""Python binding of the C ABI in include/nswe.h (libnswe_gb300.so).

Argument marshalling only: every step of the method runs in the CUDA
library. Device arrays are torch tensors (float64, CUDA, contiguous) whose
pointers are passed through; PyTorch supplies device memory and the stream.
There is no CPU fallback: if the library is missing or no GPU is present,
loading raises.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

MAX_LEVELS = 16
JAC_SIMPLIFIED, JAC_FULL = 3, 5
JAC_FROZEN = 0x100
FLUX_HLL, FLUX_LLF = 0, 1  # 2D: OR'd into the Jacobian choice, the frozen linearisation
PREC_FP64, PREC_MIXED = 0, 1
BC_DISCHARGE, BC_DEPTH, BC_STATE, BC_EXTRAP = 1, 2, 3, 4
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ENAN", 6: "ENEGDEPTH",
          7: "ESINGULAR"}


class BC1D(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("h", ctypes.c_double), ("q", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("tau", ctypes.c_double), ("omega", ctypes.c_double),
                ("tol", ctypes.c_double), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("nu3", ctypes.c_int),
                ("n_max", ctypes.c_int), ("jacobian", ctypes.c_int), ("nest_start", ctypes.c_int),
                ("precision", ctypes.c_int), ("colours2d", ctypes.c_int), ("eps", ctypes.c_double * MAX_LEVELS)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int * MAX_LEVELS),
                ("res", ctypes.c_double * MAX_LEVELS), ("level_status", ctypes.c_int * MAX_LEVELS),
                ("total_iters", ctypes.c_int), ("vcycles", ctypes.c_int),
                ("t_start_ns", ctypes.c_ulonglong), ("t_end_ns", ctypes.c_ulonglong)]

    def as_dict(self, levels=MAX_LEVELS):
        return {"status": self.status, "iters": list(self.iters)[:levels], "res": list(self.res)[:levels],
                "level_status": list(self.level_status)[:levels], "total_iters": self.total_iters,
                "vcycles": self.vcycles, "t_start_ns": self.t_start_ns, "t_end_ns": self.t_end_ns}


class NsweError(RuntimeError):
    def __init__(self, call, status):
        super().__init__(f"{call} failed: {STATUS.get(status, status)} ({lib().nswe_status_str(status).decode()})")
        self.status = status


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_size_t), ("host_bytes", ctypes.c_size_t), ("streams", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("batch_window_s", ctypes.c_double), ("device_bytes_2d", ctypes.c_size_t)]


class ServerTimes(ctypes.Structure):
    _fields_ = [("t_submit_ns", ctypes.c_ulonglong), ("t_admit_ns", ctypes.c_ulonglong),
                ("t_launch_ns", ctypes.c_ulonglong), ("t_done_ns", ctypes.c_ulonglong)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("launches", ctypes.c_longlong),
                ("waiting", ctypes.c_int), ("running", ctypes.c_int), ("device_bytes_used", ctypes.c_size_t),
                ("device_bytes_peak", ctypes.c_size_t)]


_lib = None

# Live handles, closed at interpreter exit in dependency order (servers and
# problems before the contexts they use), before CUDA is torn down.
_live = {"server": weakref.WeakSet(), "prob": weakref.WeakSet(), "ctx": weakref.WeakSet()}


@atexit.register
def _close_all():
    for kind in ("server", "prob", "ctx"):
        for obj in list(_live[kind]):
            try:
                obj.close()
            except Exception:
                pass
_vp, _dp, _i, _d = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double

EXPORTS = {
    "nswe_status_str": (ctypes.c_char_p, [_i]),
    "nswe_params_default": (_i, [ctypes.POINTER(Params), _i, _i]),
    "nswe_ctx_create": (_i, [ctypes.POINTER(_vp), _i, _vp]),
    "nswe_ctx_set_stream": (_i, [_vp, _vp]),
    "nswe_ctx_destroy": (_i, [_vp]),
    "nswe_prob_create_1d": (_i, [_vp, ctypes.POINTER(_vp), _i, _i, _d, _d, _d, _dp, _dp,
                                 ctypes.POINTER(BC1D), ctypes.POINTER(BC1D)]),
    "nswe_prob_set_geometry_1d": (_i, [_vp, _vp, _dp, _dp, ctypes.POINTER(BC1D), ctypes.POINTER(BC1D)]),
    "nswe_prob_create_2d": (_i, [_vp, ctypes.POINTER(_vp), _i, _i, _i, _d, _d, _d, _d, _d, _dp, _dp, _dp]),
    "nswe_prob_destroy": (_i, [_vp]),
    "nswe_prob_cells": (_i, [_vp, _i]),
    "nswe_prob_dim": (_i, [_vp]),
    "nswe_residual": (_i, [_vp, _vp, _i, _dp, _dp, _dp]),
    "nswe_jacobian_simplified": (_i, [_vp, _vp, _i, _dp, _d, _d, _dp, _dp, _dp]),
    "nswe_jacobian_full": (_i, [_vp, _vp, _i, _dp, _d, _d, _dp, _dp, _dp]),
    "nswe_mg_vcycle": (_i, [_vp, _vp, _i, _i, _dp, _dp, _dp, ctypes.POINTER(Params)]),
    "nswe_jacobian_f32": (_i, [_vp, _vp, _i, _i, _dp, _d, _d, _dp, _dp, _dp]),
    "nswe_jacobian_frozen": (_i, [_vp, _vp, _i, _i, _dp, _d, _d, _dp, _dp, _dp]),
    "nswe_ctx_set_colour_major_2d": (_i, [_vp, _i]),
    "nswe_ctx_set_jacobian_cells_2d": (_i, [_vp, _i]),
    "nswe_ctx_set_batch_2d": (_i, [_vp, _i]),
    "nswe_ctx_set_tail_2d": (_i, [_vp, _i, _i]),
    "nswe_set_launch_overlap_2d": (_i, [_i]),
    "nswe_autotune_2d": (_i, [_vp, _vp, _dp, ctypes.POINTER(Params), ctypes.POINTER(_i), _i, ctypes.POINTER(_i), _i,
                              _i, ctypes.POINTER(_d), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "nswe_ctx_get_tuned_2d": (_i, [_vp, _i, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "nswe_prob_set_flux_1d": (_i, [_vp, _vp, _i]),
    "nswe_prob_set_geometry_batch_1d": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_dp), ctypes.POINTER(_dp),
                                             ctypes.POINTER(BC1D), ctypes.POINTER(BC1D)]),
    "nswe_mg_vcycle_f32": (_i, [_vp, _vp, _i, _i, _dp, _dp, _dp, ctypes.POINTER(Params)]),
    "nswe_mg_smooth": (_i, [_vp, _vp, _i, _i, _dp, _dp, _dp, ctypes.POINTER(Params), _i, ctypes.POINTER(_i)]),
    "nswe_newton_solve": (_i, [_vp, _vp, _dp, _dp, ctypes.POINTER(Params), ctypes.POINTER(Info)]),
    "nswe_newton_solve_batch": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_dp), ctypes.POINTER(_dp),
                                     ctypes.POINTER(Params), ctypes.POINTER(Info)]),
    "nswe_newton_solve_batch_each": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_dp), ctypes.POINTER(_dp),
                                     ctypes.POINTER(Params), ctypes.POINTER(Info)]),
    "nswe_newton_solve_noalloc": (_i, [_i, _vp, _i, _i, _d, _d, _d, _dp, _dp, ctypes.POINTER(BC1D),
                                       ctypes.POINTER(BC1D), _dp, _dp, ctypes.POINTER(Params), _vp]),
    "nswe_probe_fma": (_i, [_vp, _i, _i, _i, _i, _vp, ctypes.POINTER(_d)]),
    "nswe_solve_shape_count": (_i, []),
    "nswe_solve_shape_info": (_i, [_i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "nswe_ctx_set_solve_shape": (_i, [_vp, _i, _i]),
    "nswe_ctx_get_solve_shape": (_i, [_vp, _i, ctypes.POINTER(_i)]),
    "nswe_ctx_set_solve_cluster": (_i, [_vp, _i, _i]),
    "nswe_server_set_cluster": (_i, [_vp, _i, _i, _i]),
    "nswe_ctx_get_solve_cluster": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "nswe_autotune_solve_batch": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_dp), ctypes.POINTER(_dp),
                                       ctypes.POINTER(Params), _i, ctypes.POINTER(_d), ctypes.POINTER(_i)]),
    "nswe_server_footprint_1d": (ctypes.c_size_t, [_i, _i, _i]),
    "nswe_server_footprint_2d": (ctypes.c_size_t, [_i, _i, _i, _i]),
    "nswe_server_submit_2d": (_i, [_vp, _i, _i, _i, _d, _d, _d, _d, _d, _dp, ctypes.POINTER(ctypes.c_int), _dp, _dp,
                                   ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_ulonglong)]),
    "nswe_server_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(ServerConfig)]),
    "nswe_server_submit_1d": (_i, [_vp, _i, _i, _d, _d, _d, _dp, _dp, ctypes.POINTER(BC1D), ctypes.POINTER(BC1D),
                                   _dp, ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_ulonglong)]),
    "nswe_server_poll": (_i, [_vp, ctypes.POINTER(ctypes.c_ulonglong), _i, ctypes.POINTER(_i)]),
    "nswe_server_wait": (_i, [_vp, _i, _d]),
    "nswe_server_take": (_i, [_vp, ctypes.c_ulonglong, _dp, ctypes.POINTER(Info), ctypes.POINTER(ServerTimes)]),
    "nswe_server_query": (_i, [_vp, ctypes.POINTER(ServerStats)]),
    "nswe_server_destroy": (_i, [_vp]),
    "nswe_arena_create": (_i, [ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.c_size_t]),
    "nswe_arena_alloc": (_i, [_vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "nswe_arena_free": (_i, [_vp, ctypes.c_size_t]),
    "nswe_arena_query": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                              ctypes.POINTER(ctypes.c_size_t)]),
    "nswe_arena_destroy": (_i, [_vp]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Loads libnswe_gb300.so (building it with nvcc if absent)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing; run paper_2505_10857_gb300.build.build()")
            _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(call, rc):
    if rc != 0:
        raise NsweError(call, rc)


def _ptr(t, f32=False) -> Optional[int]:
    """Device pointer of a contiguous CUDA float64 (float32 with f32) tensor,
    or None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    import torch
    dt = torch.float32 if f32 else torch.float64
    if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
        raise ValueError(f"expected a contiguous {dt} CUDA tensor")
    return t.data_ptr()


def params(N, levels, **kw) -> Params:
    """Paper defaults (nswe_params_default) with keyword overrides; eps may be
    a sequence (per nested level) or a scalar."""
    p = Params()
    _check("nswe_params_default", lib().nswe_params_default(ctypes.byref(p), int(N), int(levels)))
    for k, v in kw.items():
        if k == "eps":
            vals = list(v) if hasattr(v, "__len__") else [v] * MAX_LEVELS
            for i in range(MAX_LEVELS):
                p.eps[i] = float(vals[min(i, len(vals) - 1)])
        elif k == "nb":
            p.jacobian = int(v)
        elif k == "lex":
            if v:
                raise ValueError("the CUDA path implements the multicolour smoother only")
        elif k == "levels":
            pass
        else:
            setattr(p, k, v)
    return p


def params_from(prm) -> Params:
    """From an inputs.Params1D (whose eps list is filled per nested level)."""
    if not prm.eps:
        raise ValueError("eps per level must be given")
    return params(96, prm.levels, alpha=prm.alpha, tau=prm.tau, omega=prm.omega, tol=prm.tol, nu1=prm.nu1,
                  nu2=prm.nu2, nu3=prm.nu3, n_max=prm.n_max, nb=prm.nb, nest_start=prm.nest_start, eps=prm.eps,
                  lex=prm.lex)


class Context:
    """nswe_ctx bound to a device and (by default) torch's current stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the NMGM library runs on the GPU only")
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.device = device
        self.h = _vp()
        _check("nswe_ctx_create", lib().nswe_ctx_create(ctypes.byref(self.h), int(device), _vp(stream)))
        _live["ctx"].add(self)

    def set_stream(self, stream):
        _check("nswe_ctx_set_stream", lib().nswe_ctx_set_stream(self.h, _vp(stream)))

    def close(self):
        if self.h:
            lib().nswe_ctx_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bc(b) -> BC1D:
    return BC1D(int(b[0]), float(b[1]), float(b[2]))


class Problem1D:
    """nswe_prob of a 1D problem (host arrays copied to device)."""

    def __init__(self, ctx: Context, N, levels, x0, x1, g, sigma_face, gauss_geom_all, bcl, bcr):
        self.ctx = ctx
        self.N, self.levels = int(N), int(levels)
        sf = np.ascontiguousarray(sigma_face, dtype=np.float64)
        gq = np.ascontiguousarray(gauss_geom_all, dtype=np.float64)
        self.h = _vp()
        _check("nswe_prob_create_1d", lib().nswe_prob_create_1d(
            ctx.h, ctypes.byref(self.h), self.N, self.levels, float(x0), float(x1), float(g),
            sf.ctypes.data, gq.ctypes.data, ctypes.byref(_bc(bcl)), ctypes.byref(_bc(bcr))))
        _live["prob"].add(self)

    @staticmethod
    def from_inputs(ctx: Context, inp) -> "Problem1D":
        p = Problem1D(ctx, inp.N, inp.levels, inp.x0, inp.x1, inp.g, inp.sig_face, inp.gq_all(), inp.bcl, inp.bcr)
        if getattr(inp, "flux", 0):
            p.set_flux(inp.flux)
        return p

    def set_flux(self, flux):
        """FLUX_HLL (the default) or FLUX_LLF."""
        _check("nswe_prob_set_flux_1d", lib().nswe_prob_set_flux_1d(self.ctx.h, self.h, int(flux)))

    def set_geometry(self, sigma_face, gauss_geom_all, bcl, bcr):
        """Arrays must stay alive until the stream has consumed them."""
        _check("nswe_prob_set_geometry_1d", lib().nswe_prob_set_geometry_1d(
            self.ctx.h, self.h, _host_ptr(sigma_face), _host_ptr(gauss_geom_all),
            ctypes.byref(_bc(bcl)), ctypes.byref(_bc(bcr))))

    def cells(self, level=0):
        return lib().nswe_prob_cells(self.h, int(level))

    def close(self):
        if self.h:
            lib().nswe_prob_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem2D:
    """nswe_prob of a 2D problem (host arrays copied to device)."""

    def __init__(self, ctx: Context, Nx, Ny, levels, x0, x1, y0, y1, g, gauss_geom_all, bc_kind_all, bc_state):
        self.ctx = ctx
        self.Nx, self.Ny, self.levels = int(Nx), int(Ny), int(levels)
        gq = np.ascontiguousarray(gauss_geom_all, dtype=np.float64)
        kinds = np.ascontiguousarray(bc_kind_all, dtype=np.int32)
        st = np.ascontiguousarray(bc_state, dtype=np.float64).reshape(-1)
        self.h = _vp()
        _check("nswe_prob_create_2d", lib().nswe_prob_create_2d(
            ctx.h, ctypes.byref(self.h), self.Nx, self.Ny, self.levels, float(x0), float(x1), float(y0), float(y1),
            float(g), gq.ctypes.data, kinds.ctypes.data, st.ctypes.data))
        _live["prob"].add(self)

    @staticmethod
    def from_inputs(ctx: Context, inp) -> "Problem2D":
        return Problem2D(ctx, inp.Nx, inp.Ny, inp.levels, inp.x0, inp.x1, inp.y0, inp.y1, inp.g, inp.gq_all(),
                         inp.bc_kind_all(), inp.bc_state)

    def cells(self, level=0):
        return lib().nswe_prob_cells(self.h, int(level))

    def close(self):
        if self.h:
            lib().nswe_prob_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def params2d_from(prm, levels=None) -> Params:
    """From an inputs.Params2D (one eps for every level, scalar smoothing counts)."""
    nu1 = prm.nu1[0] if hasattr(prm.nu1, "__len__") else prm.nu1
    nu2 = prm.nu2[0] if hasattr(prm.nu2, "__len__") else prm.nu2
    return params(96, levels or prm.levels, alpha=prm.alpha, tau=prm.tau, omega=prm.omega, tol=prm.tol, nu1=nu1,
                  nu2=nu2, nu3=prm.nu3, n_max=prm.n_max,
                  nb=(JAC_FULL if prm.st == 1 else JAC_SIMPLIFIED) | (JAC_FROZEN if getattr(prm, "frozen", False) else 0),
                  nest_start=prm.nest_start, eps=prm.eps, colours2d=getattr(prm, "colours", 0))


def _host_ptr(a) -> int:
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()  # pinned CPU torch tensor


# ---------------------------------------------------------------- calls (same names as the C ABI)

def _check_level_sizes(call, prob, level, nb=None, **arrays):
    """The arrays of a call on one nested level must hold that level: U, R,
    dU [comps][n_l] and J [nb][comps^2][n_l] (comps = 2 in 1D, 3 in 2D);
    the C entry points take bare pointers and cannot check this. A level or
    nb the call does not accept is left to the C entry point to refuse."""
    if not 0 <= int(level) < prob.levels:
        return
    two_d = isinstance(prob, Problem2D)
    comps = 3 if two_d else 2
    n = prob.cells(int(level))
    for name, t in arrays.items():
        if t is None or isinstance(t, int):
            continue
        if name == "J" and int(nb) not in ((9, 21) if two_d else (3, 5)):
            continue
        need = (int(nb) * comps * comps if name == "J" else comps) * n
        if t.numel() < need:
            raise ValueError(f"{call}: {name} holds {t.numel()} values; level {level} needs {need}")


def _nb_default(prob, full):
    if isinstance(prob, Problem2D):
        return 21 if full else 9
    return 5 if full else 3


def nswe_residual(ctx: Context, prob: Problem1D, level, U, R, res=None):
    _check_level_sizes("nswe_residual", prob, level, U=U, R=R)
    _check("nswe_residual", lib().nswe_residual(ctx.h, prob.h, int(level), _ptr(U), _ptr(R), _ptr(res)))


def nswe_jacobian_simplified(ctx, prob, level, U, eps, alpha, R, J, res=None):
    _check_level_sizes("nswe_jacobian_simplified", prob, level, _nb_default(prob, False), U=U, R=R, J=J)
    _check("nswe_jacobian_simplified", lib().nswe_jacobian_simplified(
        ctx.h, prob.h, int(level), _ptr(U), float(eps), float(alpha), _ptr(R), _ptr(J), _ptr(res)))


def nswe_jacobian_full(ctx, prob, level, U, eps, alpha, R, J, res=None):
    _check_level_sizes("nswe_jacobian_full", prob, level, _nb_default(prob, True), U=U, R=R, J=J)
    _check("nswe_jacobian_full", lib().nswe_jacobian_full(
        ctx.h, prob.h, int(level), _ptr(U), float(eps), float(alpha), _ptr(R), _ptr(J), _ptr(res)))


def nswe_prob_set_geometry_batch_1d(ctx, probs, sigma_faces, gauss_geoms, lefts, rights):
    """Geometry re-upload of several 1D problems (host float64 arrays)."""
    n = len(probs)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in list(sigma_faces) + list(gauss_geoms)]
    ph = (_vp * n)(*[p.h.value for p in probs])
    sf = (_dp * n)(*[a.ctypes.data for a in arrs[:n]])
    gq = (_dp * n)(*[a.ctypes.data for a in arrs[n:]])
    bl = (BC1D * n)(*[_bc(b) for b in lefts])
    br = (BC1D * n)(*[_bc(b) for b in rights])
    _check("nswe_prob_set_geometry_batch_1d", lib().nswe_prob_set_geometry_batch_1d(ctx.h, n, ph, sf, gq, bl, br))


def nswe_ctx_set_colour_major_2d(ctx, min_cells):
    """2D Newton levels of at least min_cells cells keep J9 colour-major (<0: never)."""
    _check("nswe_ctx_set_colour_major_2d", lib().nswe_ctx_set_colour_major_2d(ctx.h, int(min_cells)))


BATCH2D_CONCURRENT, BATCH2D_LOCKSTEP = 0, 1


def nswe_ctx_set_batch_2d(ctx, mode):
    """How batches of 2D problems run: BATCH2D_CONCURRENT (per-problem
    streams) or BATCH2D_LOCKSTEP (shared launches); see include/nswe.h."""
    _check("nswe_ctx_set_batch_2d", lib().nswe_ctx_set_batch_2d(ctx.h, int(mode)))


COLOURS2D_AUTO = -1


def nswe_set_launch_overlap_2d(enable):
    """Programmatic dependent launch of the 2D kernels (process-wide, on by default)."""
    _check("nswe_set_launch_overlap_2d", lib().nswe_set_launch_overlap_2d(int(bool(enable))))


def nswe_ctx_set_tail_2d(ctx, precision, max_cells):
    _check("nswe_ctx_set_tail_2d", lib().nswe_ctx_set_tail_2d(ctx.h, int(precision), int(max_cells)))


def nswe_autotune_2d(ctx, prob, U, prm: Params, schedules, tails, reps=3):
    """Times V-cycles of the 2D problem for every (schedule, tail) pair (see
    include/nswe.h); returns (ms[len(schedules)][len(tails)], best schedule,
    best tail) and records the choice in the context."""
    if U.numel() < 3 * prob.Nx * prob.Ny:
        raise ValueError("nswe_autotune_2d: U must hold the finest level")
    ns, nt = len(schedules), len(tails)
    sc = (_i * ns)(*[int(v) for v in schedules])
    tl = (_i * nt)(*[int(v) for v in tails])
    ms = (_d * (ns * nt))()
    bs, bt = _i(), _i()
    _check("nswe_autotune_2d", lib().nswe_autotune_2d(ctx.h, prob.h, _ptr(U), ctypes.byref(prm), sc, ns, tl, nt,
                                                      int(reps), ms, ctypes.byref(bs), ctypes.byref(bt)))
    return [[ms[a * nt + b] for b in range(nt)] for a in range(ns)], bs.value, bt.value


def nswe_ctx_get_tuned_2d(ctx, Nx, Ny, precision):
    """(schedule, tail) recorded by the autotuner, or None."""
    s_, t_ = _i(), _i()
    rc = lib().nswe_ctx_get_tuned_2d(ctx.h, int(Nx), int(Ny), int(precision), ctypes.byref(s_), ctypes.byref(t_))
    return (s_.value, t_.value) if rc == 0 else None


def nswe_ctx_set_jacobian_cells_2d(ctx, min_cells):
    """2D levels of at least min_cells cells take the per-cell Jacobian kernel (<0: never)."""
    _check("nswe_ctx_set_jacobian_cells_2d", lib().nswe_ctx_set_jacobian_cells_2d(ctx.h, int(min_cells)))


def nswe_jacobian_frozen(ctx, prob, level, nb, U, eps, alpha, R, J, res=None):
    """2D Jacobian (nb 9 or 21) under the frozen linearisation."""
    _check_level_sizes("nswe_jacobian_frozen", prob, level, nb, U=U, R=R, J=J)
    _check("nswe_jacobian_frozen", lib().nswe_jacobian_frozen(
        ctx.h, prob.h, int(level), int(nb), _ptr(U), float(eps), float(alpha), _ptr(R), _ptr(J), _ptr(res)))


def nswe_mg_vcycle(ctx, prob, level, nb, J, R, dU, prm: Params):
    _check_level_sizes("nswe_mg_vcycle", prob, level, nb, J=J, R=R, dU=dU)
    _check("nswe_mg_vcycle", lib().nswe_mg_vcycle(ctx.h, prob.h, int(level), int(nb), _ptr(J), _ptr(R), _ptr(dU),
                                                  ctypes.byref(prm)))


def colour_major_size(Nx, Ny):
    """Cells' slots of the colour-major block layout (see nswe_mg_smooth)."""
    return 3 * Ny * ((Nx + 2) // 3)


def nswe_mg_smooth(ctx, prob, level, nb, J, R, dU, prm: Params, colour_major=False):
    """prm.nu1 steps of the 2D multicolour block SOR on one level (see
    include/nswe.h); returns the number of colour-pass launches."""
    _check_level_sizes("nswe_mg_smooth", prob, level, None, R=R, dU=dU)
    if isinstance(prob, Problem2D) and 0 <= int(level) < prob.levels:
        nx, ny = prob.Nx >> int(level), prob.Ny >> int(level)
        slots = colour_major_size(nx, ny) if colour_major else nx * ny
        if J.numel() < int(nb) * 9 * slots:
            raise ValueError(f"nswe_mg_smooth: J holds {J.numel()} values; level {level} needs {int(nb) * 9 * slots}")
    n = ctypes.c_int(0)
    _check("nswe_mg_smooth", lib().nswe_mg_smooth(ctx.h, prob.h, int(level), int(nb), _ptr(J), _ptr(R), _ptr(dU),
                                                  ctypes.byref(prm), int(bool(colour_major)), ctypes.byref(n)))
    return n.value


def nswe_jacobian_f32(ctx, prob, level, nb, U, eps, alpha, R, J, res=None):
    """R (float64) and the FP32 Jacobian J (float32) of a mixed-precision step."""
    _check_level_sizes("nswe_jacobian_f32", prob, level, nb, U=U, R=R, J=J)
    _check("nswe_jacobian_f32", lib().nswe_jacobian_f32(
        ctx.h, prob.h, int(level), int(nb), _ptr(U), float(eps), float(alpha), _ptr(R), _ptr(J, True), _ptr(res)))


def nswe_mg_vcycle_f32(ctx, prob, level, nb, J, R, dU, prm: Params):
    _check_level_sizes("nswe_mg_vcycle_f32", prob, level, nb, J=J, R=R, dU=dU)
    _check("nswe_mg_vcycle_f32", lib().nswe_mg_vcycle_f32(ctx.h, prob.h, int(level), int(nb), _ptr(J, True),
                                                          _ptr(R, True), _ptr(dU, True), ctypes.byref(prm)))


def _check_solve_sizes(prob, U0, U, prm: Params):
    """The guess must hold the start level's state and U the finest level's
    (the C entry points take bare pointers and cannot check this)."""
    s = prm.nest_start if 0 <= prm.nest_start < prob.levels else prob.levels - 1
    comps = 3 if isinstance(prob, Problem2D) else 2
    for name, t, lev in (("U0", U0, s), ("U", U, 0)):
        if t is None or isinstance(t, int):
            continue
        need = comps * prob.cells(lev)
        if t.numel() < need:
            raise ValueError(f"{name} holds {t.numel()} values; level {lev} needs {comps} x {need // comps}")


def nswe_newton_solve(ctx, prob, U0, U, prm: Params, want_info=True, raise_on_status=False):
    _check_solve_sizes(prob, U0, U, prm)
    info = Info() if want_info else None
    rc = lib().nswe_newton_solve(ctx.h, prob.h, _ptr(U0), _ptr(U), ctypes.byref(prm),
                                 ctypes.byref(info) if info is not None else None)
    if rc in (1, 2, 3) or (raise_on_status and rc):
        raise NsweError("nswe_newton_solve", rc)
    return info.as_dict(prob.levels) if info is not None else None


def nswe_newton_solve_batch(ctx, probs: Sequence[Problem1D], U0s, Us, prm: Params, want_info=True):
    n = len(probs)
    for p, u0, u in zip(probs, U0s, Us):
        _check_solve_sizes(p, u0, u, prm)
    ph = (_vp * n)(*[p.h.value for p in probs])
    u0 = (_dp * n)(*[_ptr(u) for u in U0s])
    uu = (_dp * n)(*[_ptr(u) for u in Us])
    infos = (Info * n)() if want_info else None
    rc = lib().nswe_newton_solve_batch(ctx.h, n, ph, u0, uu, ctypes.byref(prm), infos)
    if rc in (1, 2, 3):
        raise NsweError("nswe_newton_solve_batch", rc)
    return [infos[i].as_dict(probs[i].levels) for i in range(n)] if infos is not None else None


def nswe_newton_solve_batch_each(ctx, probs, U0s, Us, prms: Sequence[Params], want_info=True):
    """Batched solve with one parameter record per problem."""
    n = len(probs)
    if len(prms) != n:
        raise ValueError("one parameter record per problem")
    for p, u0, u, q in zip(probs, U0s, Us, prms):
        _check_solve_sizes(p, u0, u, q)
    ph = (_vp * n)(*[p.h.value for p in probs])
    u0 = (_dp * n)(*[_ptr(u) for u in U0s])
    uu = (_dp * n)(*[_ptr(u) for u in Us])
    pa = (Params * n)(*prms)
    infos = (Info * n)() if want_info else None
    rc = lib().nswe_newton_solve_batch_each(ctx.h, n, ph, u0, uu, pa, infos)
    if rc in (1, 2, 3):
        raise NsweError("nswe_newton_solve_batch_each", rc)
    return [infos[i].as_dict(probs[i].levels) for i in range(n)] if infos is not None else None


def solve_shapes():
    """[(threads per block, blocks per SM)] of the batched 1D solve kernel."""
    out = []
    for i in range(lib().nswe_solve_shape_count()):
        t, b = _i(), _i()
        _check("nswe_solve_shape_info", lib().nswe_solve_shape_info(i, ctypes.byref(t), ctypes.byref(b)))
        out.append((t.value, b.value))
    return out


def nswe_ctx_set_solve_shape(ctx, precision, shape):
    _check("nswe_ctx_set_solve_shape", lib().nswe_ctx_set_solve_shape(ctx.h, int(precision), int(shape)))


def nswe_ctx_set_solve_cluster(ctx, ctas, team_cells=1024):
    """1D solves on a cluster of `ctas` CTAs per problem (1: a block per problem)."""
    _check("nswe_ctx_set_solve_cluster", lib().nswe_ctx_set_solve_cluster(ctx.h, int(ctas), int(team_cells)))


def nswe_ctx_get_solve_cluster(ctx):
    """(ctas, team_cells) of the context."""
    a, b = _i(), _i()
    _check("nswe_ctx_get_solve_cluster", lib().nswe_ctx_get_solve_cluster(ctx.h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def nswe_ctx_get_solve_shape(ctx, precision):
    v = _i()
    _check("nswe_ctx_get_solve_shape", lib().nswe_ctx_get_solve_shape(ctx.h, int(precision), ctypes.byref(v)))
    return v.value


def nswe_autotune_solve_batch(ctx, probs, U0s, Us, prm: Params, reps=2):
    """Times every launch shape on the batch; returns (ms per shape, chosen shape)."""
    n = len(probs)
    ph = (_vp * n)(*[p.h.value for p in probs])
    u0 = (_dp * n)(*[_ptr(u) for u in U0s])
    uu = (_dp * n)(*[_ptr(u) for u in Us])
    k = lib().nswe_solve_shape_count()
    ms = (_d * k)()
    best = _i()
    _check("nswe_autotune_solve_batch", lib().nswe_autotune_solve_batch(ctx.h, n, ph, u0, uu, ctypes.byref(prm),
                                                                        int(reps), ms, ctypes.byref(best)))
    return [ms[i] for i in range(k)], best.value


def nswe_newton_solve_noalloc(device, stream, N, levels, x0, x1, g, sigma_face, gauss_geom, bcl, bcr, U0, U,
                              prm: Params, info=None):
    """Allocation-free solve of one problem (see include/nswe.h): every array
    is a device tensor; `info` is a device buffer of sizeof(Info) bytes (a
    uint8 CUDA tensor) or None. Returns the status code of the call."""
    rc = lib().nswe_newton_solve_noalloc(
        int(device), _vp(stream), int(N), int(levels), float(x0), float(x1), float(g), _ptr(sigma_face),
        _ptr(gauss_geom), ctypes.byref(_bc(bcl)), ctypes.byref(_bc(bcr)), _ptr(U0), _ptr(U), ctypes.byref(prm),
        _vp(info.data_ptr()) if info is not None else None)
    if rc:
        raise NsweError("nswe_newton_solve_noalloc", rc)
    return rc


def nswe_probe_fma(stream, precision, blocks, threads, iters, sink) -> float:
    """FMA throughput probe (see include/nswe.h): launches on `stream`
    (a cudaStream_t handle) and returns the flops the launch performs; the
    caller times it with CUDA events. `sink` is a device tensor of
    blocks*threads float64 (FP64) or float32 (FP32) values."""
    if sink.numel() < blocks * threads:
        raise ValueError("sink holds fewer values than blocks * threads")
    fl = ctypes.c_double()
    _check("nswe_probe_fma", lib().nswe_probe_fma(_vp(stream), int(precision), int(blocks), int(threads), int(iters),
                                                  _vp(sink.data_ptr()), ctypes.byref(fl)))
    return fl.value


def info_from_bytes(raw: bytes, levels=MAX_LEVELS) -> dict:
    """Decodes an nswe_info copied back from the device."""
    inf = Info.from_buffer_copy(raw)
    return inf.as_dict(levels)


# ---------------------------------------------------------------- continuous-batching server (1D)

class Server:
    """nswe_server: 1D requests are Problem1DInputs-like objects (N, levels,
    x0, x1, g, sig_face, gq_all(), bcl, bcr, U0_start), 2D requests
    Problem2DInputs-like ones (submit2d), each with its Params."""

    def __init__(self, device=0, device_bytes=1 << 30, host_bytes=256 << 20, streams=4, max_batch=1024,
                 batch_window_s=0.0, device_bytes_2d=0):
        cfg = ServerConfig(int(device_bytes), int(host_bytes), int(streams), int(max_batch), float(batch_window_s),
                           int(device_bytes_2d))
        self.h = _vp()
        _check("nswe_server_create", lib().nswe_server_create(ctypes.byref(self.h), int(device), ctypes.byref(cfg)))
        self.N = {}
        _live["server"].add(self)

    def set_cluster(self, ctas, max_in_flight, team_cells=1024):
        """Light-load latency form: launches with at most max_in_flight 1D solves in
        flight run each problem on a cluster of `ctas` CTAs (ctas 1: off)."""
        _check("nswe_server_set_cluster",
               lib().nswe_server_set_cluster(self.h, int(ctas), int(max_in_flight), int(team_cells)))

    @staticmethod
    def footprint(N, levels, nest_start=-1) -> int:
        return int(lib().nswe_server_footprint_1d(int(N), int(levels), int(nest_start)))

    def submit(self, inp, prm: Params) -> int:
        sf = np.ascontiguousarray(inp.sig_face, dtype=np.float64)
        gq = np.ascontiguousarray(inp.gq_all(), dtype=np.float64)
        u0 = np.ascontiguousarray(inp.U0_start, dtype=np.float64)
        t = ctypes.c_ulonglong()
        _check("nswe_server_submit_1d", lib().nswe_server_submit_1d(
            self.h, int(inp.N), int(inp.levels), float(inp.x0), float(inp.x1), float(inp.g), sf.ctypes.data,
            gq.ctypes.data, ctypes.byref(_bc(inp.bcl)), ctypes.byref(_bc(inp.bcr)), u0.ctypes.data,
            ctypes.byref(prm), ctypes.byref(t)))
        self.N[t.value] = int(inp.N)
        return t.value

    @staticmethod
    def footprint2d(Nx, Ny, levels, nest_start=-1) -> int:
        return int(lib().nswe_server_footprint_2d(int(Nx), int(Ny), int(levels), int(nest_start)))

    def submit2d(self, inp, prm: Params) -> int:
        gq = np.ascontiguousarray(inp.gq_all(), dtype=np.float64)
        kinds = np.ascontiguousarray(inp.bc_kind_all(), dtype=np.int32)
        st = np.ascontiguousarray(inp.bc_state, dtype=np.float64).reshape(-1)
        u0 = np.ascontiguousarray(inp.U0_start, dtype=np.float64)
        t = ctypes.c_ulonglong()
        _check("nswe_server_submit_2d", lib().nswe_server_submit_2d(
            self.h, int(inp.Nx), int(inp.Ny), int(inp.levels), float(inp.x0), float(inp.x1), float(inp.y0),
            float(inp.y1), float(inp.g), gq.ctypes.data, kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            st.ctypes.data, u0.ctypes.data, ctypes.byref(prm), ctypes.byref(t)))
        self.N[t.value] = (3, int(inp.Nx) * int(inp.Ny))
        return t.value

    def poll(self, max_n=4096):
        buf = (ctypes.c_ulonglong * max_n)()
        n = _i()
        _check("nswe_server_poll", lib().nswe_server_poll(self.h, buf, max_n, ctypes.byref(n)))
        return [buf[i] for i in range(n.value)]

    def wait(self, min_completed=1, timeout_s=60.0) -> bool:
        rc = lib().nswe_server_wait(self.h, int(min_completed), float(timeout_s))
        if rc == 8:
            return False
        _check("nswe_server_wait", rc)
        return True

    def take(self, ticket):
        shape = self.N.pop(ticket)
        U = np.empty(shape if isinstance(shape, tuple) else (2, shape), dtype=np.float64)
        info, times = Info(), ServerTimes()
        _check("nswe_server_take", lib().nswe_server_take(self.h, ctypes.c_ulonglong(ticket), U.ctypes.data,
                                                          ctypes.byref(info), ctypes.byref(times)))
        return U, info.as_dict(MAX_LEVELS), {f: getattr(times, f) for f, _ in ServerTimes._fields_}

    def stats(self) -> dict:
        st = ServerStats()
        _check("nswe_server_query", lib().nswe_server_query(self.h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            lib().nswe_server_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Arena:
    """nswe_arena: the server's first-fit allocator (host logic only)."""

    def __init__(self, nbytes, align=256):
        self.h = _vp()
        _check("nswe_arena_create", lib().nswe_arena_create(ctypes.byref(self.h), int(nbytes), int(align)))

    def alloc(self, nbytes):
        off = ctypes.c_size_t()
        rc = lib().nswe_arena_alloc(self.h, int(nbytes), ctypes.byref(off))
        return off.value if rc == 0 else None

    def free(self, off) -> bool:
        return lib().nswe_arena_free(self.h, int(off)) == 0

    def query(self):
        u, p, l = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
        _check("nswe_arena_query", lib().nswe_arena_query(self.h, ctypes.byref(u), ctypes.byref(p), ctypes.byref(l)))
        return u.value, p.value, l.value

    def close(self):
        if self.h:
            lib().nswe_arena_destroy(self.h)
            self.h = _vp()
