"""Seeded synthetic workloads for the steady shallow-water NMGM.

This module builds problem *inputs* only: bottom and width profiles, their
samples at the points the library's interface asks for, boundary data, the
coarse initial guess and the solver parameters. It holds none of the
method's arithmetic (no reconstruction, flux, source, Jacobian or solver
step), so it can feed both the CUDA library and the CPU oracle.

Sampling contract (shared by both sides, 1D): on a grid of N cells over
[x0, x1] with dx = (x1-x0)/N, cell j (0-based) has centre x_j = x0+(j+1/2)dx
and the two Gauss points of Eq. 9, x_j -+ dx/(2 sqrt 3). The library takes
  sigma_face[N+1]      width at the faces x0 + f dx,
  gq[3][2][N]          (sigma, d sigma/dx, db/dx) at the two Gauss points,
for every nested level l (N_l = N / 2^l).

Workload families follow the paper's tests: Eq. 26 (smooth subcritical flow,
Section 5.1.1), Eq. 28 with the contractions of Section 5.1.2, and the
seeded channels of the benchmark (Gaussian hump, sinusoidal width).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Tuple

import numpy as np

BC_DISCHARGE, BC_DEPTH, BC_STATE, BC_EXTRAP = 1, 2, 3, 4

G_PAPER = 9.812  # Section 2
G_CONFIG = 9.81


# --------------------------------------------------------------------------
# Geometry families: each returns (f(x), f'(x)) as numpy functions.

def bottom_eq26():
    """b(x) of Eq. 26 on [-10, 10]."""
    def b(x):
        return 0.2 * np.exp(-0.5 * (x + 1.0) ** 2) + 0.3 * np.exp(-(x - 1.5) ** 2)

    def bx(x):
        return -0.2 * (x + 1.0) * np.exp(-0.5 * (x + 1.0) ** 2) - 0.6 * (x - 1.5) * np.exp(-(x - 1.5) ** 2)
    return b, bx


def bottom_eq28():
    """b(x) of Eq. 28 on [0, 25] (parabolic bump on [8, 12])."""
    def b(x):
        x = np.asarray(x, dtype=np.float64)
        return np.where((x >= 8.0) & (x <= 12.0), 0.2 - 0.05 * (x - 10.0) ** 2, 0.0)

    def bx(x):
        x = np.asarray(x, dtype=np.float64)
        return np.where((x > 8.0) & (x < 12.0), -0.1 * (x - 10.0), 0.0)
    return b, bx


def bottom_gaussian(A, xc, w):
    """b(x) = A exp(-((x-xc)/w)^2), the benchmark hump."""
    def b(x):
        return A * np.exp(-(((x - xc) / w) ** 2))

    def bx(x):
        return -2.0 * A * (x - xc) / (w * w) * np.exp(-(((x - xc) / w) ** 2))
    return b, bx


def bottom_linear(b0, slope):
    def b(x):
        return b0 + slope * np.asarray(x, dtype=np.float64)

    def bx(x):
        return np.full_like(np.asarray(x, dtype=np.float64), slope)
    return b, bx


def width_constant(s=1.0):
    def s_(x):
        return np.full_like(np.asarray(x, dtype=np.float64), s)

    def sx(x):
        return np.zeros_like(np.asarray(x, dtype=np.float64))
    return s_, sx


def width_sine(B0, k, Lc):
    """sigma(x) = B0 (1 + 0.2 sin(2 pi k x / Lc)), the benchmark channel."""
    def s_(x):
        return B0 * (1.0 + 0.2 * np.sin(2.0 * np.pi * k * x / Lc))

    def sx(x):
        return B0 * 0.2 * (2.0 * np.pi * k / Lc) * np.cos(2.0 * np.pi * k * x / Lc)
    return s_, sx


def width_contraction(sigma0, xl, xr):
    """Smooth contraction of Section 5.1.2 on [xl, xr], 1 elsewhere."""
    xm, span = 0.5 * (xl + xr), xr - xl

    def s_(x):
        x = np.asarray(x, dtype=np.float64)
        inside = (x >= xl) & (x <= xr)
        return np.where(inside, 1.0 - sigma0 * (1.0 + np.cos(2.0 * np.pi * (x - xm) / span)), 1.0)

    def sx(x):
        x = np.asarray(x, dtype=np.float64)
        inside = (x > xl) & (x < xr)
        return np.where(inside, sigma0 * np.sin(2.0 * np.pi * (x - xm) / span) * 2.0 * np.pi / span, 0.0)
    return s_, sx


# --------------------------------------------------------------------------

@dataclass
class Problem1DInputs:
    """All arrays a 1D nested solve needs (host, float64)."""
    N: int
    levels: int
    x0: float
    x1: float
    g: float
    sig_face: np.ndarray            # [N+1]
    gq: List[np.ndarray]            # per level [3,2,N_l]
    bcl: Tuple[int, float, float]   # (kind, h, q)
    bcr: Tuple[int, float, float]
    U0_start: np.ndarray            # [2, N_s] guess on the start level s
    start_level: int = -1           # nested start level s (-1: coarsest)
    omega: float = 1.0              # SOR relaxation suited to the family
    eps_levels: List[float] = field(default_factory=list)  # FD eps per nested level (empty: eps_for_n)
    b_fn: Callable = field(repr=False, default=None)
    sig_fn: Callable = field(repr=False, default=None)
    meta: dict = field(default_factory=dict)
    flux: int = 0                   # numerical flux: 0 HLL (the paper's 1D choice), 1 LLF

    def N_level(self, l):
        return self.N >> l

    def sig_face_level(self, l):
        return np.ascontiguousarray(self.sig_face[:: 1 << l])

    def centres(self, l=0):
        n = self.N_level(l)
        dx = (self.x1 - self.x0) / n
        return self.x0 + (np.arange(n) + 0.5) * dx

    def gq_all(self):
        """Concatenation over levels of gq[l] (the library's layout)."""
        return np.ascontiguousarray(np.concatenate([a.reshape(-1) for a in self.gq]))


def gauss_points(x0, x1, n):
    dx = (x1 - x0) / n
    xc = x0 + (np.arange(n) + 0.5) * dx
    d = dx / (2.0 * math.sqrt(3.0))
    return xc - d, xc + d


def sample_geometry(x0, x1, n, b_fn, sig_fn):
    """gq[3,2,n] = (sigma, sigma_x, b_x) at the two Gauss points of each cell."""
    (s, sx), (_, bx) = sig_fn, b_fn
    out = np.empty((3, 2, n))
    for q, xg in enumerate(gauss_points(x0, x1, n)):
        out[0, q] = s(xg)
        out[1, q] = sx(xg)
        out[2, q] = bx(xg)
    return out


def make_problem_1d(N, levels, x0, x1, g, b_fns, sig_fns, bcl, bcr, init="lake", h_init=None, q_init=None,
                    meta=None, start_level=-1, omega=1.0, eps_levels=None) -> Problem1DInputs:
    """Samples geometry for every nested level and builds the start guess.

    init = "lake": guess on the start level h = h_init - b(x_c), Q = q_init
    (Section 5.1.2 uses h = 0.5 - b, u = 0; the benchmark uses h = h_out - b,
    Q = q).
    """
    if N % (1 << (levels - 1)):
        raise ValueError("N must be divisible by 2^(levels-1) for the nested solve")
    b, _ = b_fns
    s, _ = sig_fns
    faces = x0 + np.arange(N + 1) * (x1 - x0) / N
    sig_face = s(faces).astype(np.float64)
    gq = [sample_geometry(x0, x1, N >> l, b_fns, sig_fns) for l in range(levels)]
    sl = levels - 1 if start_level < 0 else start_level
    NL = N >> sl
    xc = x0 + (np.arange(NL) + 0.5) * (x1 - x0) / NL
    if init == "lake":
        h = h_init - b(xc)
        U0 = np.stack([s(xc) * h, np.full(NL, q_init)])
    else:
        raise ValueError(init)
    return Problem1DInputs(N, levels, x0, x1, g, sig_face, gq, tuple(bcl), tuple(bcr),
                           np.ascontiguousarray(U0, dtype=np.float64), sl, omega, list(eps_levels or []), b, s,
                           meta or {})


# --------------------------------------------------------------------------
# Solver parameters (Section 5).

def eps_for_n(n, floor=0.05):
    """FD perturbation: 0.2/0.15/0.1/0.05 at N=96/192/384/768 (Section 5.1);
    in between, the same log2 progression, clipped to [floor, 0.2]. The paper
    suggests 0.01 on finer grids; with the multicolour smoother that value
    makes the FD Jacobian lose block-diagonal dominance on the N >= 2048
    channels (the smoother diverges), so the default floor is 0.05, the value
    the paper uses at N = 768."""
    e = 0.2 - 0.05 * math.log2(n / 96.0)
    return float(min(0.2, max(floor, e)))


def eps_channel(n):
    """FD perturbation for the sinusoidal-width channels: 0.2 up to 512 cells,
    0.1 below 2048, 0.05 from 2048 cells."""
    return 0.2 if n <= 512 else (0.1 if n < 2048 else 0.05)


@dataclass
class Params1D:
    alpha: float = 3.0
    tau: float = 0.6
    omega: float = 1.0
    tol: float = 1e-11
    nu1: int = 2
    nu2: int = 2
    nu3: int = 2
    levels: int = 4
    n_max: int = 2000
    nb: int = 3
    eps: List[float] = field(default_factory=list)
    nest_start: int = -1
    lex: bool = False

    @staticmethod
    def for_problem(p: Problem1DInputs, **kw):
        kw.setdefault("omega", p.omega)
        kw.setdefault("nest_start", p.start_level)
        prm = Params1D(levels=p.levels, **kw)
        if not prm.eps:
            prm.eps = list(p.eps_levels) or [eps_for_n(p.N_level(l)) for l in range(p.levels)]
        return prm


# --------------------------------------------------------------------------
# Paper workloads.

def paper_smooth_subcritical(N, levels=4):
    """Section 5.1.1: Eq. 26 on [-10, 10], sigma = 1, h = 1 and hu = 1 at both
    ends, g = 9.812."""
    return make_problem_1d(N, levels, -10.0, 10.0, G_PAPER, bottom_eq26(), width_constant(1.0),
                           (BC_STATE, 1.0, 1.0), (BC_STATE, 1.0, 1.0), h_init=1.0, q_init=1.0,
                           meta={"case": "eq26"})


def paper_bump(N, levels=4, regime="sub", width="const"):
    """Section 5.1.2 on [0, 25] (Eq. 28). regime sub: q=4.42, h_out=2,
    sigma0=0.05; trans: q=1.53, h_out=0.66, sigma0=0.15. Coarsest guess
    h = 0.5 - b, u = 0 as in the paper."""
    q, hout, s0 = (4.42, 2.0, 0.05) if regime == "sub" else (1.53, 0.66, 0.15)
    sig = {"const": width_constant(1.0), "left": width_contraction(s0, 3.75, 16.25),
           "right": width_contraction(s0, 8.75, 21.25)}[width]
    p = make_problem_1d(N, levels, 0.0, 25.0, G_PAPER, bottom_eq28(), sig,
                        (BC_DISCHARGE, 0.0, q), (BC_DEPTH, hout, 0.0), h_init=0.5, q_init=0.0,
                        meta={"case": f"eq28-{regime}-{width}"})
    return p


def _seeded_hump(rng):
    A = float(rng.uniform(0.05, 0.2))
    xc = float(rng.uniform(8.0, 12.0))
    w = float(rng.uniform(1.0, 2.0))
    return A, xc, w


def channel_small(k, N=200, levels=4):
    """Seeded 1D smooth subcritical channel, N=200 cells on [0, 25]: constant
    width, Gaussian hump with A~U[0.05,0.2], xc~U[8,12], w~U[1,2], upstream
    discharge 4.42, downstream depth 2.0, g=9.81. Seed 1000 + k."""
    rng = np.random.default_rng(1000 + k)
    A, xc, w = _seeded_hump(rng)
    return make_problem_1d(N, levels, 0.0, 25.0, G_CONFIG, bottom_gaussian(A, xc, w), width_constant(1.0),
                           (BC_DISCHARGE, 0.0, 4.42), (BC_DEPTH, 2.0, 0.0), h_init=2.0, q_init=4.42,
                           meta={"A": A, "xc": xc, "w": w, "seed": 1000 + k}, omega=1.2)


def critical_margin(q, hout, b_fn, sig_fn, g=G_CONFIG, x0=0.0, x1=25.0, n=4001):
    """E - max_x E_c(x) for the downstream energy E (a positive margin means
    the smooth subcritical steady state exists). Problem classification only."""
    b, _ = b_fn
    s, _ = sig_fn
    x = np.linspace(x0, x1, n)
    E = q * q / (2.0 * s(x1) ** 2 * hout * hout) + g * (hout + b(x1))
    qx = q / s(x)
    hc = (qx * qx / g) ** (1.0 / 3.0)
    Ec = 1.5 * g * hc + g * b(x)
    return float(E - Ec.max())


def channel_irregular(k, N=4096, levels=8, regime="sub", min_margin=0.5, start_level=4, q_sub=4.42):
    """Seeded 1D channel with sinusoidal width B(x)=B0(1+0.2 sin(2 pi k' x/25)),
    B0 = 1, k' ~ U{1..4}, Gaussian hump as in channel_small, N=4096 on [0,25],
    8-level multigrid (4096 -> 32 cells).
    regime "sub": q=4.42, h_out=2.0; seeds whose hump meets a narrow section
    and would choke the subcritical flow are redrawn (deterministically, same
    generator) until the energy margin exceeds min_margin. Seed 2000 + k.
    The nested solve starts on level 4 (256 cells): coarser grids do not
    resolve the width oscillation for k' >= 2. SOR relaxation 0.7. FD eps per
    level (eps_channel): larger than the Section 5.1 progression below 2048
    cells, without which the Newton iteration breaks down on k' = 4."""
    rng = np.random.default_rng(2000 + k)
    q, hout = (q_sub, 2.0) if regime == "sub" else (1.53, 0.66)
    for draw in range(1000):
        A, xc, w = _seeded_hump(rng)
        kk = int(rng.integers(1, 5))
        b_fns, s_fns = bottom_gaussian(A, xc, w), width_sine(1.0, kk, 25.0)
        margin = critical_margin(q, hout, b_fns, s_fns)
        if regime != "sub" or margin > min_margin:
            break
    return make_problem_1d(N, levels, 0.0, 25.0, G_CONFIG, b_fns, s_fns,
                           (BC_DISCHARGE, 0.0, q), (BC_DEPTH, hout, 0.0), h_init=hout, q_init=q,
                           meta={"A": A, "xc": xc, "w": w, "k": kk, "seed": 2000 + k, "draws": draw + 1,
                                 "margin": margin, "regime": regime}, start_level=start_level, omega=0.7,
                           eps_levels=[eps_channel(N >> l) for l in range(levels)])


def serving_instance(k, n_min=256, n_max=16384, min_margin=0.5):
    """Seeded request of the 1D serving workload (seed 4000 + k): N drawn
    log-uniform in [n_min, n_max], then rounded to a multiple of 2^(L-1) with
    L the number of levels that brings the coarsest grid into [32, 64) cells
    (the nested solve needs N divisible by 2^(L-1)); discharge q ~ U[1, 6];
    width B(x) = 1 + 0.2 sin(2 pi k' x/25), k' ~ U{1..4};
    Gaussian hump as in channel_small; downstream depth 2.0, raised in steps
    of 0.25 until the subcritical energy margin exceeds min_margin (q up to 6
    chokes at depth 2 where the width narrows). The nested solve starts on the
    level of [256, 512) cells (level 0 for N < 512); SOR relaxation 0.7; eps
    per level as for the sinusoidal channels."""
    rng = np.random.default_rng(4000 + k)
    n_raw = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
    levels = max(1, int(math.floor(math.log2(n_raw / 32.0))) + 1)
    m = 1 << (levels - 1)
    N = max(m * 32, int(round(n_raw / m)) * m)
    q = float(rng.uniform(1.0, 6.0))
    A, xc, w = _seeded_hump(rng)
    kk = int(rng.integers(1, 5))
    b_fns, s_fns = bottom_gaussian(A, xc, w), width_sine(1.0, kk, 25.0)
    hout = 2.0
    while critical_margin(q, hout, b_fns, s_fns) <= min_margin:
        hout += 0.25
    margin = critical_margin(q, hout, b_fns, s_fns)
    start = max(0, levels - 4)
    return make_problem_1d(N, levels, 0.0, 25.0, G_CONFIG, b_fns, s_fns,
                           (BC_DISCHARGE, 0.0, q), (BC_DEPTH, hout, 0.0), h_init=hout, q_init=q,
                           meta={"A": A, "xc": xc, "w": w, "k": kk, "q": q, "h_out": hout, "seed": 4000 + k,
                                 "margin": margin, "N_raw": n_raw}, start_level=start, omega=0.7,
                           eps_levels=[eps_channel(N >> l) for l in range(levels)])


def uniform_flow(N, levels, h, q, sigma=1.0, x0=0.0, x1=10.0, g=G_CONFIG, bc=BC_STATE):
    """Flat bottom, constant width, uniform state (the residual is zero)."""
    return make_problem_1d(N, levels, x0, x1, g, bottom_linear(0.0, 0.0), width_constant(sigma),
                           (bc, h, q), (bc, h, q), h_init=h, q_init=q, meta={"case": "uniform"})


def random_state(rng, N, H_range=(1.5, 2.5), Q_range=(3.5, 5.0)):
    """A smooth-ish random state for operator tests (positive depth)."""
    x = np.linspace(0, 1, N)
    H = rng.uniform(*H_range) + 0.2 * np.sin(2 * np.pi * rng.uniform(1, 3) * x) + 0.02 * rng.standard_normal(N)
    Q = rng.uniform(*Q_range) + 0.1 * np.cos(2 * np.pi * rng.uniform(1, 3) * x) + 0.02 * rng.standard_normal(N)
    return np.ascontiguousarray(np.stack([H, Q]))


# ==========================================================================
# Two-dimensional problems (Section 4; Section 5.2 workloads).
#
# Sampling contract (2D): cell (i, j) of an Nx x Ny grid over [x0,x1]x[y0,y1]
# has centre (x_i, y_j) and Gauss points x_i^g = x_i -+ dx/(2 sqrt 3) (g = 0, 1),
# y_j^b = y_j -+ dy/(2 sqrt 3) (b = 0, 1); gq[2][4][Ny*Nx] holds b_x and b_y at
# point q = 2 b + g, cell index j*Nx + i. Boundary kinds per boundary cell:
# [Ny left | Ny right | Nx bottom | Nx top]; bc_state[4][3] gives the (h, hu,
# hv) data per side (left, right, bottom, top).

BC2_REFLECT, BC2_INFLOW, BC2_OUTFLOW, BC2_DISCHARGE, BC2_DEPTH = 5, 6, 7, 8, 9
ST_J9, ST_J21, ST_P5, ST_P9 = 0, 1, 2, 3


def bottom2d_flat():
    z = lambda x, y: np.zeros(np.broadcast(x, y).shape)
    return z, z, z


def bottom2d_linear(b0, sx, sy):
    def b(x, y):
        return b0 + sx * np.asarray(x, dtype=np.float64) + sy * np.asarray(y, dtype=np.float64)
    return (b, lambda x, y: np.full(np.broadcast(x, y).shape, float(sx)),
            lambda x, y: np.full(np.broadcast(x, y).shape, float(sy)))


def bottom2d_eq29():
    """Parabolic bump of Eq. 29 on [-4, 4] x [0, 4]."""
    def r2(x, y):
        return np.asarray(x, dtype=np.float64) ** 2 + (np.asarray(y, dtype=np.float64) - 2.0) ** 2

    def b(x, y):
        return np.where(r2(x, y) < 1.0, 0.4 - 0.4 * r2(x, y), 0.0)

    def bx(x, y):
        return np.where(r2(x, y) < 1.0, -0.8 * np.asarray(x, dtype=np.float64), 0.0)

    def by(x, y):
        return np.where(r2(x, y) < 1.0, -0.8 * (np.asarray(y, dtype=np.float64) - 2.0), 0.0)
    return b, bx, by


def bottom2d_parabolic(A, R, xc, yc):
    """Parabolic bump of height A and radius R centred at (xc, yc): the
    shape of Eq. 29 (A = 0.4, R = 1, centre (0, 2)) moved and scaled."""
    c = A / (R * R)

    def r2(x, y):
        return (np.asarray(x, dtype=np.float64) - xc) ** 2 + (np.asarray(y, dtype=np.float64) - yc) ** 2

    def b(x, y):
        return np.where(r2(x, y) < R * R, A - c * r2(x, y), 0.0)

    def bx(x, y):
        return np.where(r2(x, y) < R * R, -2.0 * c * (np.asarray(x, dtype=np.float64) - xc), 0.0)

    def by(x, y):
        return np.where(r2(x, y) < R * R, -2.0 * c * (np.asarray(y, dtype=np.float64) - yc), 0.0)
    return b, bx, by


def bottom2d_gaussians(bumps):
    """Sum of Gaussian bumps A exp(-((x-xc)^2 + (y-yc)^2)/w^2)."""
    def b(x, y):
        return sum(A * np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (w * w)) for A, xc, yc, w in bumps) + 0 * x

    def bx(x, y):
        return sum(-2 * A * (x - xc) / (w * w) * np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (w * w))
                   for A, xc, yc, w in bumps) + 0 * x

    def by(x, y):
        return sum(-2 * A * (y - yc) / (w * w) * np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (w * w))
                   for A, xc, yc, w in bumps) + 0 * y
    return b, bx, by


@dataclass
class Problem2DInputs:
    Nx: int
    Ny: int
    levels: int
    x0: float
    x1: float
    y0: float
    y1: float
    g: float
    gq: List[np.ndarray]          # per level [2,4,Ny_l*Nx_l]
    bc_kind: List[np.ndarray]     # per level int32 [2*Ny_l + 2*Nx_l]
    bc_state: np.ndarray          # [4,3]
    U0_start: np.ndarray          # [3, n_s]
    start_level: int = -1
    b_fns: tuple = field(repr=False, default=None)
    meta: dict = field(default_factory=dict)

    def dims(self, l=0):
        return self.Nx >> l, self.Ny >> l

    def centres(self, l=0):
        nx, ny = self.dims(l)
        xc = self.x0 + (np.arange(nx) + 0.5) * (self.x1 - self.x0) / nx
        yc = self.y0 + (np.arange(ny) + 0.5) * (self.y1 - self.y0) / ny
        return np.meshgrid(xc, yc)  # [ny, nx] arrays

    def gq_all(self):
        return np.ascontiguousarray(np.concatenate([a.reshape(-1) for a in self.gq]))

    def bc_kind_all(self):
        return np.ascontiguousarray(np.concatenate([a.reshape(-1) for a in self.bc_kind]).astype(np.int32))


def sample_geometry_2d(x0, x1, y0, y1, nx, ny, b_fns):
    _, bx, by = b_fns
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    xc = x0 + (np.arange(nx) + 0.5) * dx
    yc = y0 + (np.arange(ny) + 0.5) * dy
    ox, oy = dx / (2.0 * math.sqrt(3.0)), dy / (2.0 * math.sqrt(3.0))
    out = np.empty((2, 4, ny * nx))
    for b in range(2):
        for gm in range(2):
            X, Y = np.meshgrid(xc + (2 * gm - 1) * ox, yc + (2 * b - 1) * oy)
            out[0, 2 * b + gm] = bx(X, Y).reshape(-1)
            out[1, 2 * b + gm] = by(X, Y).reshape(-1)
    return out


def _kinds(spec, coords):
    """spec: an int kind, or a callable coordinate -> kind."""
    if callable(spec):
        return np.array([spec(c) for c in coords], dtype=np.int32)
    return np.full(len(coords), int(spec), dtype=np.int32)


def make_problem_2d(Nx, Ny, levels, x0, x1, y0, y1, g, b_fns, sides, bc_state, U0_fn, start_level=-1, meta=None):
    """sides = (left, right, bottom, top) kind specs; U0_fn(x, y) -> (h, hu, hv)
    arrays evaluated at the start level's cell centres."""
    if Nx % (1 << (levels - 1)) or Ny % (1 << (levels - 1)):
        raise ValueError("grid sizes must be divisible by 2^(levels-1)")
    gq, kinds = [], []
    for l in range(levels):
        nx, ny = Nx >> l, Ny >> l
        gq.append(sample_geometry_2d(x0, x1, y0, y1, nx, ny, b_fns))
        xc = x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx
        yc = y0 + (np.arange(ny) + 0.5) * (y1 - y0) / ny
        kinds.append(np.concatenate([_kinds(sides[0], yc), _kinds(sides[1], yc), _kinds(sides[2], xc),
                                     _kinds(sides[3], xc)]))
    sl = levels - 1 if start_level < 0 else start_level
    nx, ny = Nx >> sl, Ny >> sl
    X, Y = np.meshgrid(x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx, y0 + (np.arange(ny) + 0.5) * (y1 - y0) / ny)
    h, hu, hv = U0_fn(X, Y)
    U0 = np.stack([np.broadcast_to(h, X.shape).reshape(-1), np.broadcast_to(hu, X.shape).reshape(-1),
                   np.broadcast_to(hv, X.shape).reshape(-1)]).astype(np.float64)
    return Problem2DInputs(Nx, Ny, levels, x0, x1, y0, y1, g, gq, kinds, np.asarray(bc_state, dtype=np.float64),
                           np.ascontiguousarray(U0), sl, b_fns, meta or {})


def paper_parabolic_bump(Nx=16, Ny=8, levels=2):
    """Section 5.2.1: Eq. 29 on [-4, 4] x [0, 4]; discharge hu = 1 at x = -4,
    depth h = 1 at x = 4, reflective side walls; guess h = 1, hu = 1, hv = 0
    (Eq. 30) on the start level; g = 9.812."""
    st = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0, 0, 0], [0, 0, 0]])
    return make_problem_2d(Nx, Ny, levels, -4.0, 4.0, 0.0, 4.0, G_PAPER, bottom2d_eq29(),
                           (BC2_DISCHARGE, BC2_DEPTH, BC2_REFLECT, BC2_REFLECT), st,
                           lambda X, Y: (1.0, 1.0, 0.0), meta={"case": "eq29"})


def bump_channel_2d(k, Nx=64, Ny=32, levels=4, start_level=-1):
    """Seeded subcritical 2D channel around Section 5.2.1 (seed 5000 + k):
    [-4, 4] x [0, 4] with one parabolic bump shaped as Eq. 29, height
    ~U[0.2, 0.4], radius ~U[0.75, 1.25], centre ~U([-1.5, 1.5] x [1.5, 2.5]);
    inflow discharge hu ~U[0.75, 1.25] at x = -4, depth 1 at x = 4,
    reflective side walls; guess h = 1, hu = the inflow discharge, hv = 0
    (as Eq. 30) on start_level (the coarsest for -1); g = 9.812."""
    rng = np.random.default_rng(5000 + k)
    A, R = float(rng.uniform(0.2, 0.4)), float(rng.uniform(0.75, 1.25))
    xc, yc = float(rng.uniform(-1.5, 1.5)), float(rng.uniform(1.5, 2.5))
    q = float(rng.uniform(0.75, 1.25))
    st = np.array([[0.0, q, 0.0], [1.0, 0.0, 0.0], [0, 0, 0], [0, 0, 0]])
    return make_problem_2d(Nx, Ny, levels, -4.0, 4.0, 0.0, 4.0, G_PAPER, bottom2d_parabolic(A, R, xc, yc),
                           (BC2_DISCHARGE, BC2_DEPTH, BC2_REFLECT, BC2_REFLECT), st,
                           lambda X, Y: (1.0, q, 0.0), start_level=start_level,
                           meta={"case": "bump-channel", "seed": 5000 + k, "bump": (A, R, xc, yc), "q": q})


def gauss_bump_channel_2d(k, Nx=128, Ny=64, levels=5, start_level=-1):
    """Seeded subcritical 2D channel with a Gaussian bottom bump (seed
    6000 + k), the bump family of the batched 2D serving workload: the
    channel of Section 5.2.1, [-4, 4] x [0, 4], discharge hu ~U[0.75, 1.25]
    at x = -4, depth 1 at x = 4, reflective side walls, with
    b = A exp(-((x - xc)^2 + (y - yc)^2) / w^2), A ~U[0.1, 0.3],
    w ~U[0.5, 1.0], centre ~U([-1.5, 1.5] x [1.5, 2.5]); guess h = 1,
    hu = the discharge, hv = 0 (as Eq. 30) on start_level; g = 9.812."""
    rng = np.random.default_rng(6000 + k)
    A, w = float(rng.uniform(0.1, 0.3)), float(rng.uniform(0.5, 1.0))
    xc, yc = float(rng.uniform(-1.5, 1.5)), float(rng.uniform(1.5, 2.5))
    q = float(rng.uniform(0.75, 1.25))
    st = np.array([[0.0, q, 0.0], [1.0, 0.0, 0.0], [0, 0, 0], [0, 0, 0]])
    return make_problem_2d(Nx, Ny, levels, -4.0, 4.0, 0.0, 4.0, G_PAPER, bottom2d_gaussians([(A, xc, yc, w)]),
                           (BC2_DISCHARGE, BC2_DEPTH, BC2_REFLECT, BC2_REFLECT), st,
                           lambda X, Y: (1.0, q, 0.0), start_level=start_level,
                           meta={"case": "gauss-bump-channel", "seed": 6000 + k, "bump": (A, xc, yc, w), "q": q})


def wedge(Nx, Ny, levels, theta_deg=8.95, x1=5.0, y1=2.0, x_wall=1.0, speed=8.57, start_level=-1, meta=None):
    """Hydraulic jump over a wedge in the rotated frame of Section 5.2.2:
    inflow (h, u, v) = (1, speed cos(-theta), speed sin(-theta)) on the left
    and top, extrapolated outflow on the right, bottom outflow for
    x < x_wall / cos(theta) and reflective beyond; flat bottom; guess = the
    inflow state (Eq. 31); g = 9.812."""
    th = math.radians(theta_deg)
    u, v = speed * math.cos(-th), speed * math.sin(-th)
    xw = x_wall / math.cos(th)
    st = np.array([[1.0, u, v], [1.0, u, v], [1.0, u, v], [1.0, u, v]])
    bottom = lambda x: BC2_OUTFLOW if x < xw else BC2_REFLECT
    return make_problem_2d(Nx, Ny, levels, 0.0, x1, 0.0, y1, G_PAPER, bottom2d_flat(),
                           (BC2_INFLOW, BC2_OUTFLOW, bottom, BC2_INFLOW), st, lambda X, Y: (1.0, u, v),
                           start_level=start_level,
                           meta=dict(meta or {}, theta_deg=theta_deg, x_wall=xw, case="wedge"))


def wedge_serving_2d(k, Nx=128, Ny=64, levels=5, start_level=None):
    """Seeded supercritical wedge channel of the batched 2D workload (seed
    7000 + k): the rotated-frame wedge of Section 5.2.2 on [0, 40] x [0, 30]
    with the wall from x = 8 / cos(theta), deflection theta ~ U[5, 15] degrees,
    inflow depth 1 and Froude number F ~ U[2, 4] (speed F sqrt(g)); every draw
    lies below the largest deflection of an attached oblique jump (19.6
    degrees at F = 2). Guess Eq. 31 on start_level (default: the 16 x 8 grid
    of a grid whose coarsest level is 8 x 4, as in Section 5.2.2)."""
    rng = np.random.default_rng(7000 + k)
    th = float(rng.uniform(5.0, 15.0))
    F = float(rng.uniform(2.0, 4.0))
    sl = levels - 2 if start_level is None else start_level
    return wedge(Nx, Ny, levels, theta_deg=th, x1=40.0, y1=30.0, x_wall=8.0, speed=F * math.sqrt(G_PAPER),
                 start_level=sl, meta={"seed": 7000 + k, "froude": F})


def wedge_channel(k, Nx=512, Ny=256, levels=7):
    """Seeded wedge channel: 512 x 256 cells on [0, 40] x [0, 30], deflection
    theta ~ U[8, 15] degrees, inflow depth 1 and speed 8.57 (Froude 2.74), wall
    from x = 8/cos(theta); seed 3000 + k."""
    rng = np.random.default_rng(3000 + k)
    th = float(rng.uniform(8.0, 15.0))
    return wedge(Nx, Ny, levels, theta_deg=th, x1=40.0, y1=30.0, x_wall=8.0, meta={"seed": 3000 + k})


@dataclass
class Params2D:
    alpha: float = 3.0
    tau: float = 0.6
    omega: float = 0.1
    tol: float = 1e-11
    nu1: List[int] = field(default_factory=lambda: [20])
    nu2: List[int] = field(default_factory=lambda: [20])
    nu3: int = 3
    levels: int = 2
    n_max: int = 2000
    st: int = ST_J9
    eps: float = 1e-6
    nest_start: int = -1
    colours: int = 0  # K of the diagonal smoothing schedule for cross stencils (0: stencil colourings)
    frozen: bool = False  # frozen linearisation of the 2D Jacobian (weights and eigenvectors from the iterate)
