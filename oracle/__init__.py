"""CPU oracle for the NMGM of arXiv 2505.10857 (test infrastructure only).

A plain, slow, single-threaded FP64 C restatement of the paper's equations
and algorithms (Sections 3-4, Algorithms 1-3, Appendix A), loaded through
ctypes. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package. It shares no code with the CUDA
library in ``paper_2505_10857_gb300`` and never stands in for it.

Parity status per function is recorded in the module docstrings of the C
sources; every function here is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_nswe.so")
_SOURCES = ["nswe_oracle_1d.c", "nswe_oracle_2d.c"]
_lock = threading.Lock()
_lib = None

BC_DISCHARGE, BC_DEPTH, BC_STATE, BC_EXTRAP = 1, 2, 3, 4
BC_REFLECT, BC_INFLOW, BC_OUTFLOW, BC2_DISCHARGE, BC2_DEPTH = 5, 6, 7, 8, 9
ST_J9, ST_J21, ST_P5, ST_P9 = 0, 1, 2, 3


CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off"]


def compiler_info() -> dict:
    """The compiler and flags the oracle is built with (for reports that time it)."""
    try:
        ver = subprocess.run(["gcc", "--version"], capture_output=True, text=True).stdout.splitlines()[0]
    except (OSError, IndexError):
        ver = "gcc (version unknown)"
    return {"compiler": ver, "flags": " ".join(CFLAGS), "threads_per_solve": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C11, -O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "nswe_oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc"] + CFLAGS + ["-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Grid1D(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("dx", ctypes.c_double), ("g", ctypes.c_double),
        ("sig_face", ctypes.POINTER(ctypes.c_double)),
        ("gq", ctypes.POINTER(ctypes.c_double)),
        ("bcl_kind", ctypes.c_int), ("bcr_kind", ctypes.c_int),
        ("bcl_h", ctypes.c_double), ("bcl_q", ctypes.c_double),
        ("bcr_h", ctypes.c_double), ("bcr_q", ctypes.c_double), ("flux", ctypes.c_int),
    ]


class Params1D(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("tau", ctypes.c_double), ("omega", ctypes.c_double), ("tol", ctypes.c_double),
        ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("nu3", ctypes.c_int), ("levels", ctypes.c_int),
        ("n_max", ctypes.c_int), ("nb", ctypes.c_int), ("lex", ctypes.c_int),
        ("nest_start", ctypes.c_int),
        ("eps", ctypes.c_double * 32),
    ]


class Info1D(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("iters", ctypes.c_int * 32), ("res", ctypes.c_double * 32),
        ("total_iters", ctypes.c_int), ("vcycles", ctypes.c_int),
    ]


class Grid2D(ctypes.Structure):
    _fields_ = [
        ("Nx", ctypes.c_int), ("Ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("g", ctypes.c_double),
        ("gq", ctypes.POINTER(ctypes.c_double)),
        ("bc_kind", ctypes.POINTER(ctypes.c_int)),
        ("bc_state", ctypes.POINTER(ctypes.c_double)),
    ]


class Params2D(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("tau", ctypes.c_double), ("omega", ctypes.c_double), ("tol", ctypes.c_double),
        ("nu1", ctypes.c_int * 16), ("nu2", ctypes.c_int * 16),
        ("nu3", ctypes.c_int), ("levels", ctypes.c_int), ("n_max", ctypes.c_int), ("st", ctypes.c_int),
        ("nest_start", ctypes.c_int), ("eps", ctypes.c_double), ("colours", ctypes.c_int),
        ("frozen", ctypes.c_int),
    ]


class Info2D(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int * 16), ("res", ctypes.c_double * 16),
                ("total_iters", ctypes.c_int), ("vcycles", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dbl, i32, P = ctypes.c_double, ctypes.c_int, ctypes.POINTER
            sig = {
                "or_weno3": (None, [dbl, dbl, dbl, _D, _D]),
                "or_set_weno_zeta": (None, [dbl]),
                "or_get_weno_zeta": (dbl, []),
                "or_flux1d": (None, [dbl, dbl, dbl, dbl, _D]),
                "or_hll1d": (None, [dbl, dbl, dbl, dbl, dbl, dbl, _D]),
                "or_llf1d": (None, [dbl, dbl, dbl, dbl, dbl, dbl, _D]),
                "or_cubic4": (dbl, [_D, dbl]),
                "or_residual_cell1d": (None, [P(Grid1D), _D, _D, i32, _D]),
                "or_residual1d": (dbl, [P(Grid1D), _D, _D, _D]),
                "or_jacobian1d": (dbl, [P(Grid1D), _D, _D, dbl, dbl, i32, _D, _D]),
                "or_coarse_count": (i32, [i32]),
                "or_coarse_operator1d": (None, [i32, i32, _D, _D]),
                "or_block_inverse1d": (None, [i32, i32, _D, _D]),
                "or_sor_step1d": (None, [i32, i32, _D, _D, _D, _D, dbl]),
                "or_sor_step_lex1d": (None, [i32, i32, _D, _D, _D, _D, dbl]),
                "or_restrict1d": (None, [i32, i32, _D, _D, _D, _D]),
                "or_prolong1d": (None, [i32, _D, _D]),
                "or_dense_solve": (i32, [i32, _D, _D]),
                "or_direct_solve1d": (i32, [i32, i32, _D, _D, _D]),
                "or_vcycle1d": (i32, [i32, i32, i32, _D, _D, _D, dbl, i32, i32, i32]),
                "or_interp1d": (None, [P(Grid1D), _D, _D, _D, _D]),
                "or_nmgm1d": (i32, [P(Grid1D), _D, _D, P(Params1D), P(Info1D)]),
                "or_newton1d": (i32, [P(Grid1D), _D, i32, dbl, P(Params1D), P(Info1D)]),
            }
            G2 = P(Grid2D)
            sig.update({
                "or_llf2d": (None, [i32, _D, _D, dbl, _D]),
                "or_residual_cell2d": (None, [G2, _D, i32, i32, _D]),
                "or_face_gauss2d": (None, [G2, _D, i32, i32, i32, i32, _D]),
                "or_residual2d": (dbl, [G2, _D, _D]),
                "or_jacobian2d": (dbl, [G2, _D, dbl, dbl, i32, _D, _D]),
                "or_jacobian2d_frozen": (dbl, [G2, _D, dbl, dbl, i32, _D, _D]),
                "or_stencil_size": (i32, [i32]),
                "or_stencil_offset": (i32, [i32, i32, i32]),
                "or_coarse_operator2d": (None, [i32, i32, i32, _D, _D]),
                "or_block_inverse2d": (None, [i32, i32, _D, _D]),
                "or_colours2d": (i32, [i32]),
                "or_colour_of": (i32, [i32, i32, i32]),
                "or_sor_step2d": (None, [i32, i32, i32, _D, _D, _D, _D, dbl, i32]),
                "or_diag_colour": (i32, [i32, i32, i32, i32, i32]),
                "or_restrict2d": (None, [i32, i32, i32, _D, _D, _D, _D]),
                "or_prolong2d": (None, [i32, i32, _D, _D]),
                "or_direct_solve2d": (i32, [i32, i32, i32, _D, _D, _D]),
                "or_vcycle2d": (i32, [i32, i32, i32, i32, _D, _D, _D, dbl, i32, i32, i32]),
                "or_interp2d": (None, [G2, _D, _D]),
                "or_nmgm2d": (i32, [G2, _D, _D, P(Params2D), P(Info2D)]),
                "or_newton2d": (i32, [G2, _D, i32, P(Params2D), P(Info2D)]),
            })
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
        return _lib


def lib():
    return _lib_handle()


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


class Problem1D:
    """Holds one nested level of a 1D problem as an oracle grid struct.

    sig_face: [N+1] width at faces; gq: [3,2,N] (sigma, sigma_x, b_x at the
    two Gauss points x_j -+ dx/(2 sqrt 3)); bc = (kind, h, q) per side.
    """

    def __init__(self, N, x0, x1, g, sig_face, gq, bcl, bcr, flux=0):
        self.sig_face = _f64(sig_face).reshape(-1)
        self.gq = _f64(gq).reshape(-1)
        assert self.sig_face.size == N + 1 and self.gq.size == 6 * N
        self.N = int(N)
        self.s = Grid1D(int(N), float(x0), float(x1), (float(x1) - float(x0)) / N, float(g),
                        ptr(self.sig_face), ptr(self.gq),
                        int(bcl[0]), int(bcr[0]), float(bcl[1]), float(bcl[2]), float(bcr[1]), float(bcr[2]),
                        int(flux))

    def ref(self):
        return ctypes.byref(self.s)


def weno3(a, b, c):
    up, um = ctypes.c_double(), ctypes.c_double()
    lib().or_weno3(a, b, c, ctypes.byref(up), ctypes.byref(um))
    return up.value, um.value


class weno_zeta:
    """Context manager that sets the zeta of Eq. 8 (1e-6 in the paper) for the
    oracle's reconstructions and restores it on exit."""

    def __init__(self, zeta):
        self.zeta = float(zeta)

    def __enter__(self):
        self.old = lib().or_get_weno_zeta()
        lib().or_set_weno_zeta(self.zeta)
        return self

    def __exit__(self, *exc):
        lib().or_set_weno_zeta(self.old)
        return False


def hll1d(HL, QL, HR, QR, sig, g):
    F = np.zeros(2)
    lib().or_hll1d(HL, QL, HR, QR, sig, g, ptr(F))
    return F


def llf1d(HL, QL, HR, QR, sig, g):
    F = np.zeros(2)
    lib().or_llf1d(HL, QL, HR, QR, sig, g, ptr(F))
    return F


def flux1d(H, Q, sig, g):
    F = np.zeros(2)
    lib().or_flux1d(H, Q, sig, g, ptr(F))
    return F


def cubic4(p, t):
    p = _f64(p)
    return lib().or_cubic4(ptr(p), t)


def residual1d(prob: Problem1D, U):
    """Global residual R [2,N] and res = mean_j ||R_j||_1 (Eq. 10, Alg. 1)."""
    U = _f64(U).reshape(2, prob.N).copy()
    R = np.zeros((2, prob.N))
    res = lib().or_residual1d(prob.ref(), ptr(U[0]), ptr(U[1]), ptr(R))
    return R, res


def residual_cell1d(prob: Problem1D, U, j):
    U = _f64(U).reshape(2, prob.N).copy()
    R = np.zeros(2)
    lib().or_residual_cell1d(prob.ref(), ptr(U[0]), ptr(U[1]), int(j), ptr(R))
    return R


def jacobian1d(prob: Problem1D, U, eps, alpha, nb):
    """FD Jacobian J [nb,4,N] (Eq. 12-13), residual R [2,N], res."""
    U = _f64(U).reshape(2, prob.N).copy()
    R = np.zeros((2, prob.N))
    J = np.zeros((nb, 4, prob.N))
    res = lib().or_jacobian1d(prob.ref(), ptr(U[0]), ptr(U[1]), float(eps), float(alpha), int(nb), ptr(R), ptr(J))
    return J, R, res


def coarse_count(N):
    return lib().or_coarse_count(int(N))


def coarse_operator1d(Jf, nbf):
    Jf = _f64(Jf)
    Nf = Jf.shape[-1]
    Jc = np.zeros((3, 4, coarse_count(Nf)))
    lib().or_coarse_operator1d(Nf, nbf, ptr(Jf), ptr(Jc))
    return Jc


def block_inverse1d(J, nb):
    J = _f64(J)
    N = J.shape[-1]
    D = np.zeros((4, N))
    lib().or_block_inverse1d(N, nb, ptr(J), ptr(D))
    return D


def sor_step1d(J, Dinv, R, dU, omega, nb, lex=False):
    J, Dinv, R = _f64(J), _f64(Dinv), _f64(R)
    dU = _f64(dU).copy()
    N = R.shape[-1]
    f = lib().or_sor_step_lex1d if lex else lib().or_sor_step1d
    f(N, nb, ptr(J), ptr(Dinv), ptr(R), ptr(dU), float(omega))
    return dU


def restrict1d(J, R, dU, nb):
    J, R, dU = _f64(J), _f64(R), _f64(dU)
    Nf = R.shape[-1]
    Rc = np.zeros((2, coarse_count(Nf)))
    lib().or_restrict1d(Nf, nb, ptr(J), ptr(R), ptr(dU), ptr(Rc))
    return Rc


def prolong1d(dU, dUc):
    dU = _f64(dU).copy()
    dUc = _f64(dUc)
    lib().or_prolong1d(dU.shape[-1], ptr(dU), ptr(dUc))
    return dU


def dense_solve(A, b):
    A = _f64(A).copy()
    b = _f64(b).copy()
    rc = lib().or_dense_solve(A.shape[0], ptr(A), ptr(b))
    if rc:
        raise ZeroDivisionError("zero pivot")
    return b


def direct_solve1d(J, R, nb):
    J, R = _f64(J), _f64(R)
    N = R.shape[-1]
    dU = np.zeros((2, N))
    rc = lib().or_direct_solve1d(N, nb, ptr(J), ptr(R), ptr(dU))
    if rc:
        raise ZeroDivisionError("zero pivot")
    return dU


def vcycle1d(J, R, dU, nb, nlev, omega, nu1, nu2, lex=False):
    """One V-cycle (Algorithm 2) on J dU = -R; returns the new dU."""
    J, R = _f64(J), _f64(R)
    dU = _f64(dU).copy()
    N = R.shape[-1]
    rc = lib().or_vcycle1d(N, nb, nlev, ptr(J), ptr(R), ptr(dU), float(omega), int(nu1), int(nu2), int(lex))
    if rc:
        raise ZeroDivisionError("zero pivot")
    return dU


def interp1d(prob_coarse: Problem1D, Uc):
    Uc = _f64(Uc).reshape(2, prob_coarse.N)
    Uf = np.zeros((2, 2 * prob_coarse.N))
    lib().or_interp1d(prob_coarse.ref(), ptr(Uc[0]), ptr(Uc[1]), ptr(Uf[0]), ptr(Uf[1]))
    return Uf


def make_params1d(alpha, tau, omega, tol, nu1, nu2, nu3, levels, n_max, nb, eps, lex=False, nest_start=-1):
    p = Params1D()
    p.alpha, p.tau, p.omega, p.tol = alpha, tau, omega, tol
    p.nu1, p.nu2, p.nu3, p.levels, p.n_max, p.nb, p.lex = nu1, nu2, nu3, levels, n_max, nb, int(lex)
    p.nest_start = int(nest_start)
    eps = list(eps)
    for i in range(32):
        p.eps[i] = float(eps[min(i, len(eps) - 1)])
    return p


def nmgm1d(probs, U0_start, params: Params1D):
    """Algorithm 3: nested NMGM. probs[l] = nested level l (0 finest);
    U0_start = initial guess on the start level (params.nest_start, or the
    coarsest when negative). Returns (U [2,N0], info dict)."""
    arr = (Grid1D * len(probs))(*[p.s for p in probs])
    U0 = _f64(U0_start).reshape(-1)
    U = np.zeros(2 * probs[0].N)
    info = Info1D()
    lib().or_nmgm1d(arr, ptr(U0), ptr(U), ctypes.byref(params), ctypes.byref(info))
    L = params.levels
    return U.reshape(2, -1), {
        "status": info.status,
        "iters": [info.iters[l] for l in range(L)],
        "res": [info.res[l] for l in range(L)],
        "total_iters": info.total_iters,
        "vcycles": info.vcycles,
    }


def newton1d(prob: Problem1D, U_init, nlev, eps, params: Params1D):
    """Algorithm 1 on a single grid from U_init; linear solves by nu3 V-cycles."""
    U = _f64(U_init).reshape(-1).copy()
    info = Info1D()
    lib().or_newton1d(prob.ref(), ptr(U), int(nlev), float(eps), ctypes.byref(params), ctypes.byref(info))
    return U.reshape(2, -1), {"status": info.status, "iters": info.iters[0], "res": info.res[0],
                              "vcycles": info.vcycles}


def problem_levels(inp):
    """Oracle grids for every nested level of an inputs.Problem1DInputs."""
    return [Problem1D(inp.N_level(l), inp.x0, inp.x1, inp.g, inp.sig_face_level(l), inp.gq[l], inp.bcl, inp.bcr,
                      getattr(inp, "flux", 0)) for l in range(inp.levels)]


def params_from(prm):
    """Oracle parameter struct from an inputs.Params1D."""
    return make_params1d(prm.alpha, prm.tau, prm.omega, prm.tol, prm.nu1, prm.nu2, prm.nu3, prm.levels,
                         prm.n_max, prm.nb, prm.eps, lex=getattr(prm, "lex", False),
                         nest_start=getattr(prm, "nest_start", -1))


def solve_problem(inp, prm):
    """Nested NMGM of an inputs.Problem1DInputs with inputs.Params1D."""
    return nmgm1d(problem_levels(inp), inp.U0_start, params_from(prm))


def newton_sor1d(inp, prm, max_sweeps=10, var_tol=1e-7):
    """The Newton-SOR reference solver of Section 5.1.1 (Table 2): the nested
    iteration of Algorithm 3 in which each regularized linear system (Eq. 13)
    is solved on its own grid by symmetric block SOR steps (Eq. 19) from
    dU = 0, without coarse grids; the steps stop once the l1 norm of the change
    between two successive iterates (mean over cells, the convention of res)
    falls below var_tol, or after max_sweeps. Returns (U, info) like
    solve_problem."""
    probs = problem_levels(inp)
    L = inp.levels - 1
    s0 = L if prm.nest_start < 0 or prm.nest_start > L else prm.nest_start
    U = _f64(inp.U0_start).reshape(2, -1).copy()
    info = {"status": 0, "iters": [0] * inp.levels, "res": [0.0] * inp.levels, "sweeps": 0}
    for l in range(s0, -1, -1):
        pr = probs[l]
        if l < s0:
            U = interp1d(probs[l + 1], U)
        n, res = 0, 0.0
        while True:
            J, R, _ = jacobian1d(pr, U, prm.eps[l], prm.alpha, prm.nb)
            D = block_inverse1d(J, prm.nb)
            dU = np.zeros_like(R)
            for _ in range(max_sweeps):
                new = sor_step1d(J, D, R, dU, prm.omega, prm.nb, lex=getattr(prm, "lex", False))
                var = np.abs(new - dU).sum() / pr.N
                dU = new
                info["sweeps"] += 1
                if var < var_tol:
                    break
            U = U + prm.tau * dU
            n += 1
            _, res = residual1d(pr, U)
            if not np.isfinite(res) or not (U[0] > 0).all():
                info["status"] = 2
                break
            if res < prm.tol:
                break
            if n >= prm.n_max:
                info["status"] = 1
                break
        info["iters"][l], info["res"][l] = n, res
        if info["status"] == 2:
            break
    return U, info


# ------------------------------------------------------------------------------------------------
# Two-dimensional oracle (Section 4).

class Problem2D:
    """One nested level of a 2D problem: gq [2,4,Ny*Nx] (b_x, b_y at the Gauss
    points q = 2*beta + gamma), bc_kind [2*Ny + 2*Nx] (left, right, bottom,
    top), bc_state [4,3] (per side (h, hu, hv) data)."""

    def __init__(self, Nx, Ny, x0, x1, y0, y1, g, gq, bc_kind, bc_state):
        self.Nx, self.Ny = int(Nx), int(Ny)
        self.gq = _f64(gq).reshape(-1)
        self.kind = np.ascontiguousarray(bc_kind, dtype=np.int32).reshape(-1)
        self.state = _f64(bc_state).reshape(-1)
        assert self.gq.size == 8 * Nx * Ny and self.kind.size == 2 * (Nx + Ny) and self.state.size == 12
        self.s = Grid2D(self.Nx, self.Ny, float(x0), float(x1), float(y0), float(y1), (x1 - x0) / Nx,
                        (y1 - y0) / Ny, float(g), ptr(self.gq),
                        self.kind.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ptr(self.state))

    @property
    def n(self):
        return self.Nx * self.Ny

    def ref(self):
        return ctypes.byref(self.s)


def residual2d(prob: Problem2D, U):
    U = _f64(U).reshape(3, prob.n).copy()
    R = np.zeros((3, prob.n))
    res = lib().or_residual2d(prob.ref(), ptr(U), ptr(R))
    return R, res


def residual_cell2d(prob: Problem2D, U, i, j):
    U = _f64(U).reshape(3, prob.n).copy()
    R = np.zeros(3)
    lib().or_residual_cell2d(prob.ref(), ptr(U), int(i), int(j), ptr(R))
    return R


def face_gauss2d(prob: Problem2D, U, direction, line, k, side):
    """States at the two Gauss points of the face between cells k and k+1 of a
    row (direction 0) or column (direction 1); side 0 = U^-, 1 = U^+.
    Returns [2, 3]: lower then upper transverse Gauss point."""
    U = _f64(U).reshape(3, prob.n).copy()
    out = np.zeros(6)
    lib().or_face_gauss2d(prob.ref(), ptr(U), int(direction), int(line), int(k), int(side), ptr(out))
    return out.reshape(2, 3)


def llf2d(direction, UL, UR, g):
    UL, UR, F = _f64(UL).copy(), _f64(UR).copy(), np.zeros(3)
    lib().or_llf2d(int(direction), ptr(UL), ptr(UR), float(g), ptr(F))
    return F


def stencil2d(st):
    K = lib().or_stencil_size(st)
    return [(lib().or_stencil_offset(st, k, 0), lib().or_stencil_offset(st, k, 1)) for k in range(K)]


def jacobian2d(prob: Problem2D, U, eps, alpha, st, frozen=False):
    """Eq. 12-13; frozen=True: the frozen linearisation (WENO weights and
    characteristic eigenvectors from U, an option beside the paper)."""
    U = _f64(U).reshape(3, prob.n).copy()
    K = lib().or_stencil_size(st)
    R = np.zeros((3, prob.n))
    J = np.zeros((K, 9, prob.n))
    f = lib().or_jacobian2d_frozen if frozen else lib().or_jacobian2d
    res = f(prob.ref(), ptr(U), float(eps), float(alpha), int(st), ptr(R), ptr(J))
    return J, R, res


def coarse_stencil(st):
    return ST_P5 if st in (ST_J9, ST_P5) else ST_P9


def coarse_operator2d(Jf, Nx, Ny, st):
    Jf = _f64(Jf)
    cs = coarse_stencil(st)
    Jc = np.zeros((lib().or_stencil_size(cs), 9, (Nx // 2) * (Ny // 2)))
    lib().or_coarse_operator2d(Nx, Ny, st, ptr(Jf), ptr(Jc))
    return Jc


def block_inverse2d(J, st):
    J = _f64(J)
    n = J.shape[-1]
    D = np.zeros((9, n))
    lib().or_block_inverse2d(n, st, ptr(J), ptr(D))
    return D


def sor_step2d(J, Dinv, R, dU, Nx, Ny, st, omega, colours=0):
    J, Dinv, R = _f64(J), _f64(Dinv), _f64(R)
    dU = _f64(dU).copy()
    lib().or_sor_step2d(Nx, Ny, st, ptr(J), ptr(Dinv), ptr(R), ptr(dU), float(omega), int(colours))
    return dU


def restrict2d(J, R, dU, Nx, Ny, st):
    J, R, dU = _f64(J), _f64(R), _f64(dU)
    Rc = np.zeros((3, (Nx // 2) * (Ny // 2)))
    lib().or_restrict2d(Nx, Ny, st, ptr(J), ptr(R), ptr(dU), ptr(Rc))
    return Rc


def prolong2d(dU, dUc, Nx, Ny):
    dU = _f64(dU).copy()
    lib().or_prolong2d(Nx, Ny, ptr(dU), ptr(_f64(dUc)))
    return dU


def direct_solve2d(J, R, Nx, Ny, st):
    J, R = _f64(J), _f64(R)
    dU = np.zeros((3, Nx * Ny))
    if lib().or_direct_solve2d(Nx, Ny, st, ptr(J), ptr(R), ptr(dU)):
        raise ZeroDivisionError("zero pivot")
    return dU


def vcycle2d(J, R, dU, Nx, Ny, st, nlev, omega, nu1, nu2, colours=0):
    J, R = _f64(J), _f64(R)
    dU = _f64(dU).copy()
    if lib().or_vcycle2d(Nx, Ny, st, nlev, ptr(J), ptr(R), ptr(dU), float(omega), int(nu1), int(nu2),
                         int(colours)):
        raise ZeroDivisionError("zero pivot")
    return dU


def interp2d(prob_coarse: Problem2D, Uc):
    Uc = _f64(Uc).reshape(3, prob_coarse.n)
    Uf = np.zeros((3, 4 * prob_coarse.n))
    lib().or_interp2d(prob_coarse.ref(), ptr(Uc), ptr(Uf))
    return Uf


def make_params2d(alpha, tau, omega, tol, nu1, nu2, nu3, levels, n_max, st, eps, nest_start=-1, colours=0,
                  frozen=False):
    p = Params2D()
    p.alpha, p.tau, p.omega, p.tol = alpha, tau, omega, tol
    nu1 = list(nu1) if hasattr(nu1, "__len__") else [nu1] * 16
    nu2 = list(nu2) if hasattr(nu2, "__len__") else [nu2] * 16
    for i in range(16):
        p.nu1[i] = int(nu1[min(i, len(nu1) - 1)])
        p.nu2[i] = int(nu2[min(i, len(nu2) - 1)])
    p.nu3, p.levels, p.n_max, p.st, p.nest_start, p.eps = nu3, levels, n_max, st, nest_start, eps
    p.colours = colours
    p.frozen = int(bool(frozen))
    return p


def problem_levels2d(inp):
    return [Problem2D(inp.Nx >> l, inp.Ny >> l, inp.x0, inp.x1, inp.y0, inp.y1, inp.g, inp.gq[l], inp.bc_kind[l],
                      inp.bc_state) for l in range(inp.levels)]


def solve_problem2d(inp, prm):
    """Nested NMGM (Algorithm 3) of an inputs.Problem2DInputs."""
    probs = problem_levels2d(inp)
    arr = (Grid2D * len(probs))(*[p.s for p in probs])
    p = make_params2d(prm.alpha, prm.tau, prm.omega, prm.tol, prm.nu1, prm.nu2, prm.nu3, prm.levels, prm.n_max,
                      prm.st, prm.eps, prm.nest_start, getattr(prm, "colours", 0), getattr(prm, "frozen", False))
    U0 = _f64(inp.U0_start).reshape(-1)
    U = np.zeros(3 * inp.Nx * inp.Ny)
    info = Info2D()
    lib().or_nmgm2d(arr, ptr(U0), ptr(U), ctypes.byref(p), ctypes.byref(info))
    L = prm.levels
    return U.reshape(3, -1), {"status": info.status, "iters": [info.iters[l] for l in range(L)],
                              "res": [info.res[l] for l in range(L)], "total_iters": info.total_iters,
                              "vcycles": info.vcycles}


def newton2d(prob: Problem2D, U_init, nlev, prm):
    p = make_params2d(prm.alpha, prm.tau, prm.omega, prm.tol, prm.nu1, prm.nu2, prm.nu3, nlev, prm.n_max,
                      prm.st, prm.eps, colours=getattr(prm, "colours", 0), frozen=getattr(prm, "frozen", False))
    U = _f64(U_init).reshape(-1).copy()
    info = Info2D()
    lib().or_newton2d(prob.ref(), ptr(U), int(nlev), ctypes.byref(p), ctypes.byref(info))
    return U.reshape(3, -1), {"status": info.status, "iters": info.iters[0], "res": info.res[0],
                              "vcycles": info.vcycles}
