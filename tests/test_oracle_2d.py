"""Pins of the 2D CPU oracle (Section 4) against facts fixed by the paper and
by mathematics: exact steady states, symmetries of the equations, brute-force
differentiation, dense linear algebra and convergence to an exact solution.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from paper_2505_10857_gb300 import inputs as I

G = 9.81


def _problem(Nx, Ny, b_fns, sides, state, U0, x1=3.0, y1=2.0, levels=1):
    return I.make_problem_2d(Nx, Ny, levels, 0.0, x1, 0.0, y1, G, b_fns, sides, state, U0)


def _random_state(rng, Nx, Ny):
    X, Y = np.meshgrid(np.linspace(0, 1, Nx), np.linspace(0, 1, Ny))
    h = 1.5 + 0.2 * np.sin(2 * np.pi * X + 1.0) * np.cos(np.pi * Y) + 0.02 * rng.standard_normal(X.shape)
    hu = 2.0 + 0.3 * np.cos(2 * np.pi * Y + X) + 0.05 * rng.standard_normal(X.shape)
    hv = 0.4 * np.sin(np.pi * X) + 0.05 * rng.standard_normal(X.shape)
    return np.stack([h.ravel(), hu.ravel(), hv.ravel()])


BUMPS = I.bottom2d_gaussians([(0.1, 1.2, 0.8, 0.6), (-0.05, 2.0, 1.5, 0.4)])
MIXED_SIDES = (I.BC2_INFLOW, I.BC2_OUTFLOW, lambda x: I.BC2_OUTFLOW if x < 1.5 else I.BC2_REFLECT, I.BC2_DEPTH)
MIXED_STATE = np.array([[1.6, 2.2, 0.3], [0, 0, 0], [0, 0, 0], [1.4, 0.0, 0.0]])


# ---------------------------------------------------------------- exact states

def test_llf_consistency_and_mirror(orc):
    for d in (0, 1):
        U = np.array([1.3, 0.7, -0.4])
        F = orc.llf2d(d, U, U, G)
        h, u, v = U[0], U[1] / U[0], U[2] / U[0]
        ref = [U[1], U[1] * u + 0.5 * G * h * h, U[1] * v] if d == 0 else [U[2], U[2] * u, U[2] * v + 0.5 * G * h * h]
        assert np.allclose(F, ref, rtol=1e-15)
    UL, UR = np.array([1.2, 0.9, 0.3]), np.array([1.5, 0.4, -0.2])
    F = orc.llf2d(0, UL, UR, G)
    Fm = orc.llf2d(0, UR * [1, -1, 1], UL * [1, -1, 1], G)  # x -> -x
    assert np.allclose(Fm, F * [-1, 1, -1], rtol=1e-14)


@pytest.mark.parametrize("sides", [(I.BC2_INFLOW, I.BC2_OUTFLOW, I.BC2_OUTFLOW, I.BC2_INFLOW),
                                   (I.BC2_DISCHARGE, I.BC2_DEPTH, I.BC2_INFLOW, I.BC2_OUTFLOW)])
def test_uniform_state_zero_residual(orc, sides):
    s = np.array([1.3, 2.0, 0.5])
    p = _problem(10, 8, I.bottom2d_flat(), sides, np.tile(s, (4, 1)), lambda X, Y: tuple(s))
    R, _ = orc.residual2d(orc.problem_levels2d(p)[0], p.U0_start)
    assert np.abs(R).max() <= 1e-13 * 0.5 * G * 1.3 ** 2


def test_uniform_flow_along_walls(orc):
    # reflective walls top and bottom, flow along x: the mirror ghosts equal the state
    s = (1.1, 1.7, 0.0)
    p = _problem(10, 6, I.bottom2d_flat(), (I.BC2_INFLOW, I.BC2_OUTFLOW, I.BC2_REFLECT, I.BC2_REFLECT),
                 np.tile(s, (4, 1)), lambda X, Y: s)
    R, _ = orc.residual2d(orc.problem_levels2d(p)[0], p.U0_start)
    assert np.abs(R).max() <= 1e-13


def test_lake_at_rest_linear_bottom(orc):
    # h + b constant, u = v = 0, b linear in x and y: characteristic WENO3 and
    # the transverse quadratic are exact on linear data, LLF is consistent and
    # the Gauss quadratures are exact, so interior R = 0 to rounding.
    b = I.bottom2d_linear(0.1, 0.03, -0.02)
    p = _problem(12, 10, b, (I.BC2_REFLECT,) * 4, np.zeros((4, 3)), lambda X, Y: (2.0 - b[0](X, Y), 0.0, 0.0))
    R, _ = orc.residual2d(orc.problem_levels2d(p)[0], p.U0_start)
    R = R.reshape(3, 10, 12)
    assert np.abs(R[:, 2:-2, 2:-2]).max() <= 1e-12
    assert abs(0.03 * G * 2.0) > 0.1  # the source is exercised


# ---------------------------------------------------------------- transverse Gauss points (Section 4.1)

@pytest.mark.parametrize("direction", [0, 1])
def test_face_gauss_values_exact_for_data_quadratic_across_the_face(orc, direction):
    """Section 4.1 interpolates the three reconstructed edge values of lines
    r-1, r, r+1 to the two Gauss points of the middle edge. The reconstructed
    values are edge averages, so the quadratic through them must keep those
    averages. On a field linear along the line (the WENO reconstruction is
    exact there, whatever its weights, since both candidates coincide) and
    quadratic across it, the Gauss-point states must then be the field's point
    values. Reading the edge averages as point values instead is off by
    (curvature) * d^2 / 12."""
    Nx, Ny, x1, y1 = 12, 10, 1.2, 1.0
    dx, dy = x1 / Nx, y1 / Ny
    coef = np.array([[1.3, 0.4, -0.3, 0.5, 0.2],    # h: a + b s + c t + d t^2 + e s t
                     [0.7, -0.2, 0.3, -0.4, 0.1],
                     [-0.4, 0.3, 0.2, 0.6, -0.2]])  # s along the line, t across it

    def field(x, y):
        s_, t_ = (x, y) if direction == 0 else (y, x)
        return np.stack([a + b * s_ + c * t_ + d * t_ * t_ + e * s_ * t_ for a, b, c, d, e in coef])

    X, Y = np.meshgrid((np.arange(Nx) + 0.5) * dx, (np.arange(Ny) + 0.5) * dy)
    dt = dy if direction == 0 else dx
    T = Y if direction == 0 else X
    S_ = X if direction == 0 else Y
    # exact cell averages: the average of t^2 over a cell is t_c^2 + dt^2/12
    U = np.stack([a + b * S_ + c * T + d * (T * T + dt * dt / 12.0) + e * S_ * T for a, b, c, d, e in coef])
    p = _problem(Nx, Ny, I.bottom2d_flat(), (I.BC2_OUTFLOW,) * 4, np.zeros((4, 3)), lambda X, Y: (1.0, 0, 0),
                 x1=x1, y1=y1)
    pr = orc.problem_levels2d(p)[0]
    U = U.reshape(3, -1)
    g = 1.0 / (2.0 * math.sqrt(3.0))
    nline, nalong = (Ny, Nx) if direction == 0 else (Nx, Ny)
    worst = 0.0
    for r in range(2, nline - 2):
        for k in range(2, nalong - 3):
            for side in (0, 1):
                got = orc.face_gauss2d(pr, U, direction, r, k, side)
                xf, yc = ((k + 1) * dx, (r + 0.5) * dy) if direction == 0 else ((r + 0.5) * dx, (k + 1) * dy)
                for q, sg in enumerate((-1.0, 1.0)):
                    xq, yq = (xf, yc + sg * g * dy) if direction == 0 else (xf + sg * g * dx, yc)
                    worst = max(worst, np.abs(got[q] - field(xq, yq)).max())
    assert worst <= 1e-13, worst
    assert 0.5 * dt * dt / 12.0 > 1e3 * 1e-13  # the point-value reading would fail by far


def test_residual_truncation_error_third_order_for_a_2d_field(orc):
    """The residual of Eq. 20 at the exact cell averages of a smooth field
    that varies in x and y (not a steady state) approximates the cell average
    of F_x + G_y - S with a third-order error (Section 4.1: WENO3, two-point
    Gauss rules on the edges and in the cell). The exact average is computed
    here by 8-point Gauss rules from the field itself. The field's
    cross-stream curvature varies along the stream, so the point-value reading
    of the transverse interpolation, a swapped sign of its slope, or a source
    that pairs each Gauss depth with the wrong Gauss point of b_x, b_y all
    leave an O(d^2) error and fail the order test (checked against planted
    copies while writing this test)."""
    g = 9.812

    def field(x, y):
        return np.stack([1.0 + 0.4 * x - 0.25 * y + 0.1 * np.sin(1.3 * x + 0.7 * y),
                         0.5 + 0.1 * x - 0.1 * y + 0.05 * np.cos(0.9 * x - 1.1 * y),
                         0.2 + 0.08 * x + 0.15 * y + 0.04 * np.sin(1.5 * x + 0.5 * y)])

    b_fns = (lambda x, y: 0.2 * np.sin(1.5 * x) * np.cos(0.5 * y),
             lambda x, y: 0.3 * np.cos(1.5 * x) * np.cos(0.5 * y),
             lambda x, y: -0.1 * np.sin(1.5 * x) * np.sin(0.5 * y))

    def F(U):
        h, hu, hv = U
        return np.stack([hu, hu * hu / h + 0.5 * g * h * h, hu * hv / h])

    def Gf(U):
        h, hu, hv = U
        return np.stack([hv, hu * hv / h, hv * hv / h + 0.5 * g * h * h])

    t, w = np.polynomial.legendre.leggauss(8)
    errs = []
    for n in (16, 32, 64, 128):
        d = 2.0 / n
        X, Y = np.meshgrid((np.arange(n) + 0.5) * d, (np.arange(n) + 0.5) * d)
        Ua = sum(0.25 * wi * wj * field(X + 0.5 * d * ti, Y + 0.5 * d * tj) for ti, wi in zip(t, w) for tj, wj in zip(t, w))
        edge = lambda fl, ox, oy, along_x: sum(0.5 * wk * fl(field(X + ox + (0.5 * d * tk if along_x else 0.0),
                                                                   Y + oy + (0.0 if along_x else 0.5 * d * tk)))
                                               for tk, wk in zip(t, w))
        Rex = (edge(F, 0.5 * d, 0, False) - edge(F, -0.5 * d, 0, False)) / d \
            + (edge(Gf, 0, 0.5 * d, True) - edge(Gf, 0, -0.5 * d, True)) / d
        for ti, wi in zip(t, w):
            for tj, wj in zip(t, w):
                xx, yy = X + 0.5 * d * ti, Y + 0.5 * d * tj
                h = field(xx, yy)[0]
                Rex[1] += 0.25 * wi * wj * g * h * b_fns[1](xx, yy)
                Rex[2] += 0.25 * wi * wj * g * h * b_fns[2](xx, yy)
        p = I.make_problem_2d(n, n, 1, 0.0, 2.0, 0.0, 2.0, g, b_fns, (I.BC2_OUTFLOW,) * 4, np.zeros((4, 3)),
                              lambda X, Y: (1.0, 0.0, 0.0))
        R, _ = orc.residual2d(orc.problem_levels2d(p)[0], Ua.reshape(3, -1))
        e = np.abs(R.reshape(3, n, n) - Rex)[:, 3:-3, 3:-3]  # away from the ghost cells
        errs.append([e[m].mean() for m in range(3)] + [e.max()])
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert (orders[1:] > 2.7).all(), orders
    assert errs[-1, 3] < 2e-6 * np.abs(Rex).max(), errs


# ---------------------------------------------------------------- symmetries of the equations

def test_transpose_symmetry(orc):
    """Swapping x <-> y (and hu <-> hv, b_x <-> b_y, left <-> bottom, right <->
    top) maps the residual onto itself with components 2 and 3 swapped."""
    rng = np.random.default_rng(1)
    Nx, Ny = 8, 6
    b = I.bottom2d_gaussians([(0.1, 1.0, 0.9, 0.5)])
    bt = I.bottom2d_gaussians([(0.1, 0.9, 1.0, 0.5)])
    st = np.array([[1.5, 2.0, 0.2], [0, 0, 0], [1.2, 0.1, 1.0], [1.4, 0, 0]])
    stT = np.array([[1.2, 1.0, 0.1], [1.4, 0, 0], [1.5, 0.2, 2.0], [0, 0, 0]])
    p = I.make_problem_2d(Nx, Ny, 1, 0, 2.0, 0, 1.5, G, b, (I.BC2_INFLOW, I.BC2_OUTFLOW, I.BC2_INFLOW, I.BC2_DEPTH),
                          st, lambda X, Y: (1.0, 0.0, 0.0))
    pT = I.make_problem_2d(Ny, Nx, 1, 0, 1.5, 0, 2.0, G, bt, (I.BC2_INFLOW, I.BC2_DEPTH, I.BC2_INFLOW, I.BC2_OUTFLOW),
                           stT, lambda X, Y: (1.0, 0.0, 0.0))
    U = _random_state(rng, Nx, Ny)
    UT = np.stack([U[m].reshape(Ny, Nx).T.ravel() for m in (0, 2, 1)])
    R, _ = orc.residual2d(orc.problem_levels2d(p)[0], U)
    RT, _ = orc.residual2d(orc.problem_levels2d(pT)[0], UT)
    back = np.stack([RT[m].reshape(Nx, Ny).T.ravel() for m in (0, 2, 1)])
    # corner ghosts apply the x rule before the y rule (a reading), which does
    # not commute with the transposition: compare every cell but the 2x2
    # blocks at the corners
    keep = _off_corners(Nx, Ny)
    assert np.allclose(back[:, keep], R[:, keep], rtol=1e-12, atol=1e-12 * np.abs(R).max())
    assert np.array_equal(back[:, keep] == 0, R[:, keep] == 0)


def _off_corners(Nx, Ny):
    m = np.ones((Ny, Nx), dtype=bool)
    for a in (0, 1, Ny - 2, Ny - 1):
        for b in (0, 1, Nx - 2, Nx - 1):
            if (a < 2 or a >= Ny - 2) and (b < 2 or b >= Nx - 2):
                m[a, b] = False
    return m.ravel()


def test_mirror_symmetry(orc):
    """x -> -x: reverse the cells, negate hu and b_x, swap left and right."""
    rng = np.random.default_rng(2)
    Nx, Ny = 9, 6
    b = I.bottom2d_gaussians([(0.1, 1.1, 0.7, 0.5)])
    bm = I.bottom2d_gaussians([(0.1, 3.0 - 1.1, 0.7, 0.5)])
    st = np.array([[1.5, 2.0, 0.2], [1.3, 0, 0], [1.2, 0.3, 1.0], [0, 0, 0]])
    stm = np.array([[1.3, 0, 0], [1.5, -2.0, 0.2], [1.2, -0.3, 1.0], [0, 0, 0]])
    p = I.make_problem_2d(Nx, Ny, 1, 0, 3.0, 0, 2.0, G, b, (I.BC2_INFLOW, I.BC2_DEPTH, I.BC2_INFLOW, I.BC2_REFLECT),
                          st, lambda X, Y: (1.0, 0, 0))
    pm = I.make_problem_2d(Nx, Ny, 1, 0, 3.0, 0, 2.0, G, bm, (I.BC2_DEPTH, I.BC2_INFLOW, I.BC2_INFLOW, I.BC2_REFLECT),
                           stm, lambda X, Y: (1.0, 0, 0))
    U = _random_state(rng, Nx, Ny)
    Um = np.stack([s * U[m].reshape(Ny, Nx)[:, ::-1].ravel() for m, s in ((0, 1), (1, -1), (2, 1))])
    R, _ = orc.residual2d(orc.problem_levels2d(p)[0], U)
    Rm, _ = orc.residual2d(orc.problem_levels2d(pm)[0], Um)
    back = np.stack([s * Rm[m].reshape(Ny, Nx)[:, ::-1].ravel() for m, s in ((0, 1), (1, -1), (2, 1))])
    assert np.allclose(back, R, rtol=1e-12, atol=1e-12 * np.abs(R).max())  # x rules commute with the mirror


# ---------------------------------------------------------------- Jacobian

def test_jacobian_equals_global_bruteforce_fd(orc):
    rng = np.random.default_rng(3)
    Nx, Ny = 7, 6
    p = _problem(Nx, Ny, BUMPS, MIXED_SIDES, MIXED_STATE, lambda X, Y: (1.0, 0, 0))
    pr = orc.problem_levels2d(p)[0]
    U = _random_state(rng, Nx, Ny)
    eps = 1e-6
    J, R, _ = orc.jacobian2d(pr, U, eps, 0.0, orc.ST_J21)
    off = orc.stencil2d(orc.ST_J21)
    R0, _ = orc.residual2d(pr, U)
    assert np.array_equal(R, R0)
    n = Nx * Ny
    for cp in range(n):
        for m in range(3):
            Up = U.copy()
            Up[m, cp] += eps
            col = (orc.residual2d(pr, Up)[0] - R0) / eps
            pi, pj = cp % Nx, cp // Nx
            for c in range(n):
                i, j = c % Nx, c // Nx
                d = (pi - i, pj - j)
                if d in off:
                    k = off.index(d)
                    for l in range(3):
                        assert J[k, l * 3 + m, c] == col[l, c]
                else:
                    assert np.all(col[:, c] == 0.0), (d, c)


def test_j9_is_j21_restricted_to_the_cross(orc):
    rng = np.random.default_rng(4)
    p = _problem(6, 5, BUMPS, MIXED_SIDES, MIXED_STATE, lambda X, Y: (1.0, 0, 0))
    pr = orc.problem_levels2d(p)[0]
    U = _random_state(rng, 6, 5)
    J21, R21, _ = orc.jacobian2d(pr, U, 1e-6, 3.0, orc.ST_J21)
    J9, R9, _ = orc.jacobian2d(pr, U, 1e-6, 3.0, orc.ST_J9)
    o21, o9 = orc.stencil2d(orc.ST_J21), orc.stencil2d(orc.ST_J9)
    assert len(o21) == 21 and len(o9) == 9 and set(o9) <= set(o21)
    for k, d in enumerate(o9):
        assert np.array_equal(J9[k], J21[o21.index(d)])
    assert np.array_equal(R9, R21)


# ---------------------------------------------------------------- multigrid

def _dense(J, Nx, Ny, st, orc):
    off = orc.stencil2d(st)
    n = Nx * Ny
    A = np.zeros((3 * n, 3 * n))
    for c in range(n):
        i, j = c % Nx, c // Nx
        for k, (dx, dy) in enumerate(off):
            p, q = i + dx, j + dy
            if 0 <= p < Nx and 0 <= q < Ny:
                A[3 * c:3 * c + 3, 3 * (q * Nx + p):3 * (q * Nx + p) + 3] = J[k, :, c].reshape(3, 3)
    return A


def _P(Nx, Ny):
    n, nc = Nx * Ny, (Nx // 2) * (Ny // 2)
    P = np.zeros((3 * n, 3 * nc))
    for c in range(n):
        cc = (c // Nx // 2) * (Nx // 2) + (c % Nx) // 2
        for m in range(3):
            P[3 * c + m, 3 * cc + m] = 1.0
    return P


def _vec(U):
    return np.stack(list(U), 1).reshape(-1)


def _random_op(orc, st, Nx, Ny, rng, dominant=True):
    off = orc.stencil2d(st)
    J = rng.standard_normal((len(off), 9, Nx * Ny))
    for k, (dx, dy) in enumerate(off):
        for c in range(Nx * Ny):
            i, j = c % Nx, c // Nx
            if not (0 <= i + dx < Nx and 0 <= j + dy < Ny):
                J[k, :, c] = 0.0
    if dominant:
        kc = off.index((0, 0))
        for l in range(3):
            J[kc, l * 4] += 5.0 * len(off)
    return J


@pytest.mark.parametrize("st", [0, 1, 2, 3])
def test_coarse_operator_is_galerkin(orc, st):
    rng = np.random.default_rng(10 + st)
    Nx, Ny = 8, 6
    J = _random_op(orc, st, Nx, Ny, rng)
    Jc = orc.coarse_operator2d(J, Nx, Ny, st)
    P = _P(Nx, Ny)
    Ac = _dense(Jc, Nx // 2, Ny // 2, orc.coarse_stencil(st), orc)
    assert np.allclose(Ac, P.T @ _dense(J, Nx, Ny, st, orc) @ P, rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("st", [0, 1, 2, 3])
def test_restriction_prolongation_and_colours(orc, st):
    rng = np.random.default_rng(20 + st)
    Nx, Ny = 8, 6
    J = _random_op(orc, st, Nx, Ny, rng)
    R = rng.standard_normal((3, Nx * Ny))
    dU = rng.standard_normal((3, Nx * Ny))
    P = _P(Nx, Ny)
    Rc = orc.restrict2d(J, R, dU, Nx, Ny, st)
    assert np.allclose(_vec(Rc), P.T @ (_vec(R) + _dense(J, Nx, Ny, st, orc) @ _vec(dU)), rtol=1e-13, atol=1e-12)
    dUc = rng.standard_normal((3, (Nx // 2) * (Ny // 2)))
    assert np.allclose(_vec(orc.prolong2d(dU, dUc, Nx, Ny)), _vec(dU) + P @ _vec(dUc), rtol=1e-15)
    # no two cells of one colour are coupled by the stencil
    for (dx, dy) in orc.stencil2d(st):
        if (dx, dy) == (0, 0):
            continue
        for j in range(6):
            for i in range(6):
                assert orc.lib().or_colour_of(st, i, j) != orc.lib().or_colour_of(st, i + dx + 6, j + dy + 6)


def test_sor_direct_and_two_level_cycle(orc):
    rng = np.random.default_rng(30)
    Nx, Ny = 8, 4
    for st in (0, 2):
        J = _random_op(orc, st, Nx, Ny, rng)
        R = rng.standard_normal((3, Nx * Ny))
        A = _dense(J, Nx, Ny, st, orc)
        x = orc.direct_solve2d(J, R, Nx, Ny, st)
        assert np.abs(A @ _vec(x) + _vec(R)).max() < 1e-11
        D = orc.block_inverse2d(J, st)
        dU = np.zeros_like(R)
        for _ in range(40):
            dU = orc.sor_step2d(J, D, R, dU, Nx, Ny, st, 1.0)
        assert np.abs(dU - x).max() < 1e-10
        # two levels, no smoothing: exactly the coarse correction
        P = _P(Nx, Ny)
        got = orc.vcycle2d(J, R, np.zeros_like(R), Nx, Ny, st, 2, 1.0, 0, 0)
        ref = P @ np.linalg.solve(P.T @ A @ P, -(P.T @ _vec(R)))
        assert np.allclose(_vec(got), ref, rtol=1e-11, atol=1e-12)


def _lexicographic_d1_d4(J, D, R, dU, Nx, Ny, st, omega, orc):
    """The four sweeps D1-D4 of Eq. 22 written out literally: block SOR in
    lexicographic order, i the outer loop, with the directions of the paper."""
    off = orc.stencil2d(st)
    dU = dU.copy()
    order = [(range(Nx), range(Ny)), (range(Nx - 1, -1, -1), range(Ny)),
             (range(Nx - 1, -1, -1), range(Ny - 1, -1, -1)), (range(Nx), range(Ny - 1, -1, -1))]
    for irange, jrange in order:
        for i in irange:
            for j in jrange:
                c = j * Nx + i
                r = R[:, c].copy()
                for k, (dx, dy) in enumerate(off):
                    p, q = i + dx, j + dy
                    if (dx, dy) == (0, 0) or not (0 <= p < Nx and 0 <= q < Ny):
                        continue
                    r += J[k, :, c].reshape(3, 3) @ dU[:, q * Nx + p]
                dU[:, c] = (1.0 - omega) * dU[:, c] - omega * (D[:, c].reshape(3, 3) @ r)
    return dU


@pytest.mark.parametrize("st", [0, 2])
def test_directional_schedule_reduces_to_the_lexicographic_sweeps(orc, st):
    """The multicolour analogue of D1-D4 with K >= Nx + Ny - 1 diagonal colours
    performs exactly the paper's lexicographic sweeps on the cross stencils
    (J9 and the coarse 5-point operator); with fewer colours it still couples
    no two cells of one colour."""
    rng = np.random.default_rng(31 + st)
    Nx, Ny = 7, 5
    J = _random_op(orc, st, Nx, Ny, rng)
    D = orc.block_inverse2d(J, st)
    R = rng.standard_normal((3, Nx * Ny))
    dU0 = rng.standard_normal((3, Nx * Ny))
    ref = _lexicographic_d1_d4(J, D, R, dU0, Nx, Ny, st, 0.7, orc)
    got = orc.sor_step2d(J, D, R, dU0, Nx, Ny, st, 0.7, colours=Nx + Ny - 1)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    few = orc.sor_step2d(J, D, R, dU0, Nx, Ny, st, 0.7, colours=3)
    assert np.abs(few - ref).max() > 1e-8  # a different (multicolour) sequence
    for K in (3, 4, 7):
        for mode in (1, 2):
            for (dx, dy) in orc.stencil2d(st):
                if (dx, dy) == (0, 0):
                    continue
                for j in range(5):
                    for i in range(5):
                        assert orc.lib().or_diag_colour(mode, K, i + 2, j + 2, 9) != \
                            orc.lib().or_diag_colour(mode, K, i + 2 + dx, j + 2 + dy, 9)


def test_interp2d_conservative_and_exact_for_quadratics(orc):
    Ncx, Ncy = 6, 5
    p = I.make_problem_2d(2 * Ncx, 2 * Ncy, 2, 0.0, 1.2, 0.0, 1.0, G, I.bottom2d_flat(), (I.BC2_OUTFLOW,) * 4,
                          np.zeros((4, 3)), lambda X, Y: (1.0, 0, 0))
    pc = orc.problem_levels2d(p)[1]
    # cell averages of q(x, y) = 1 + x + 2y + 3x^2 - xy + 2y^2 by exact integration
    Fx = lambda a, b: (b - a, (b * b - a * a) / 2, (b ** 3 - a ** 3) / 3)

    def avg(nx, ny):
        xs, ys = np.linspace(0, 1.2, nx + 1), np.linspace(0, 1.0, ny + 1)
        out = np.zeros((ny, nx))
        for j in range(ny):
            for i in range(nx):
                X0, X1, X2 = Fx(xs[i], xs[i + 1])
                Y0, Y1, Y2 = Fx(ys[j], ys[j + 1])
                out[j, i] = (X0 * Y0 + X1 * Y0 + 2 * X0 * Y1 + 3 * X2 * Y0 - X1 * Y1 + 2 * X0 * Y2) / (X0 * Y0)
        return out.ravel()
    Uc = np.stack([avg(Ncx, Ncy), 2 * avg(Ncx, Ncy), -avg(Ncx, Ncy)])
    Uf = orc.interp2d(pc, Uc)
    f4 = Uf.reshape(3, 2 * Ncy, 2 * Ncx)
    parent = 0.25 * (f4[:, 0::2, 0::2] + f4[:, 0::2, 1::2] + f4[:, 1::2, 0::2] + f4[:, 1::2, 1::2])
    assert np.allclose(parent.reshape(3, -1), Uc, rtol=1e-14, atol=1e-14)
    ex = avg(2 * Ncx, 2 * Ncy).reshape(2 * Ncy, 2 * Ncx)
    assert np.allclose(f4[0, 2:-2, 2:-2], ex[2:-2, 2:-2], rtol=1e-13)
    assert np.allclose(f4[2, 2:-2, 2:-2], -ex[2:-2, 2:-2], rtol=1e-13)


# ---------------------------------------------------------------- accuracy

def _sparse(J, Nx, Ny, st, orc):
    off = orc.stencil2d(st)
    rows, cols, vals = [], [], []
    for k, (dx, dy) in enumerate(off):
        for c in range(Nx * Ny):
            i, j = c % Nx, c // Nx
            p, q = i + dx, j + dy
            if 0 <= p < Nx and 0 <= q < Ny:
                for l in range(3):
                    for m in range(3):
                        rows.append(3 * c + l)
                        cols.append(3 * (q * Nx + p) + m)
                        vals.append(J[k, l * 3 + m, c])
    n = 3 * Nx * Ny
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n)).tocsc()


@pytest.mark.slow
def test_channel_flow_converges_to_the_1d_exact_solution(orc):
    """The 2D scheme on a narrow channel with reflective side walls over the
    bottom of Eq. 26 has y-invariant discrete steady states that converge to
    the exact solution of Eq. 27 at third order as dx -> 0 (the discrete
    steady state is found with Newton steps and exact sparse solves)."""
    g = I.G_PAPER
    b1, bx1 = I.bottom_eq26()
    b_fns = (lambda x, y: b1(x) + 0 * y, lambda x, y: bx1(x) + 0 * y, lambda x, y: 0 * x + 0 * y)

    def u_exact(x):
        out = np.empty_like(x)
        for i, xx in enumerate(x):
            r = np.roots([1.0, 0.0, 2 * g * b1(xx) - 2 * g - 1.0, 2 * g])
            r = r[np.abs(r.imag) < 1e-10].real
            out[i] = r[np.argmin(np.abs(r - 1.0))]
        return out
    errs, U, ny = [], None, 2
    for nx in (64, 128, 256):
        st = np.array([[1.0, 1.0, 0.0], [1.0, 1.0, 0.0], [0, 0, 0], [0, 0, 0]])
        p = I.make_problem_2d(nx, ny, 1, -10, 10, 0, 20.0 / nx * ny, g, b_fns,
                              (I.BC2_INFLOW, I.BC2_INFLOW, I.BC2_REFLECT, I.BC2_REFLECT), st,
                              lambda X, Y: (1.0 - b1(X), 1.0, 0.0))
        pr = orc.problem_levels2d(p)[0]
        if U is None:
            U = p.U0_start.copy()
        else:
            Uc = orc.interp2d(orc.problem_levels2d(I.make_problem_2d(
                nx // 2, ny // 2, 1, -10, 10, 0, 20.0 / nx * ny, g, b_fns,
                (I.BC2_INFLOW, I.BC2_INFLOW, I.BC2_REFLECT, I.BC2_REFLECT), st, lambda X, Y: (1.0, 1.0, 0.0)))[0],
                U.reshape(3, ny, nx // 2)[:, ::2, :].reshape(3, -1))
            U = Uc
        for _ in range(80):
            J, R, res = orc.jacobian2d(pr, U, 1e-7, 3.0, orc.ST_J21)
            if res < 1e-12:
                break
            x = spl.spsolve(_sparse(J, nx, ny, orc.ST_J21, orc), -_vec(R))
            U = U + 0.6 * np.stack([x[0::3], x[1::3], x[2::3]])
        assert res < 1e-12
        dx = 20.0 / nx
        xc = -10 + (np.arange(nx) + 0.5) * dx
        t, w = np.polynomial.legendre.leggauss(8)
        he = sum(0.5 * wi * (1.0 / u_exact(xc + 0.5 * dx * ti)) for ti, wi in zip(t, w))
        errs.append(np.abs(U[0].reshape(ny, nx) - he[None]).mean())
        assert np.abs(U[2]).max() < 1e-12  # stays y-invariant
    assert math.log2(errs[0] / errs[1]) > 1.5 and math.log2(errs[1] / errs[2]) > 2.5, errs


@pytest.mark.slow
def test_j9_and_j21_reach_the_same_steady_state(orc):
    """NMGM-9 and NMGM-21 solve the same R = 0 (Section 5.2.1): same fixed
    point, nearly the same Newton counts."""
    p = I.paper_parabolic_bump(16, 8, 2)
    out = {}
    for st in (I.ST_J9, I.ST_J21):
        prm = I.Params2D(levels=2, nu1=[15], nu2=[15], tol=1e-11, n_max=400, st=st)
        U, info = orc.solve_problem2d(p, prm)
        out[st] = (U, info)
    (U9, i9), (U21, i21) = out[I.ST_J9], out[I.ST_J21]
    assert i9["res"][0] < 1e-11 and i21["res"][0] < 1e-11
    assert np.abs(U9 - U21).max() <= 1e-9 * np.abs(U9).max()
    assert abs(i9["iters"][0] - i21["iters"][0]) <= max(3, 0.2 * i21["iters"][0])


def test_parabolic_family_contains_eq29():
    """The seeded workload's bump family, at the parameters of Eq. 29
    (height 0.4, radius 1, centre (0, 2)), is Eq. 29 with its gradient."""
    rng = np.random.default_rng(7)
    x, y = rng.uniform(-4, 4, 4000), rng.uniform(0, 4, 4000)
    for f, g in zip(I.bottom2d_parabolic(0.4, 1.0, 0.0, 2.0), I.bottom2d_eq29()):
        assert np.array_equal(f(x, y), g(x, y))
    b, bx, by = I.bottom2d_parabolic(0.3, 0.8, 1.0, 2.5)
    assert b(1.0, 2.5) == 0.3 and b(1.0, 3.31) == 0.0 and b(-2.0, 1.0) == 0.0
    h = 1e-6
    for px, py in ((1.2, 2.3), (0.6, 2.9)):
        assert abs((b(px + h, py) - b(px - h, py)) / (2 * h) - bx(px, py)) < 1e-7
        assert abs((b(px, py + h) - b(px, py - h)) / (2 * h) - by(px, py)) < 1e-7


def test_seeded_bump_channels_converge(orc):
    """The seeded subcritical 2D channels of the batched workload converge to
    res < tol and keep a positive depth (coarse grids, FP64 oracle)."""
    for k in range(3):
        p = I.bump_channel_2d(k, 16, 8, 2)
        U, info = orc.solve_problem2d(p, I.Params2D(levels=2, nu1=[20], nu2=[20], tol=1e-10, n_max=400))
        assert info["status"] == 0 and info["res"][0] < 1e-10, (k, info)
        assert (U[0] > 0).all()


def _oblique_jump(F1, theta):
    """Oblique hydraulic jump of a wedge of deflection theta (radians) in a
    stream of Froude number F1 (the shallow-water analogue of the oblique
    shock relations, weak branch): returns (jump angle beta to the upstream
    flow, depth ratio h2/h1)."""
    from scipy.optimize import brentq

    def f(b):
        s = math.sqrt(1.0 + 8.0 * F1 * F1 * math.sin(b) ** 2)
        return math.tan(b) * (s - 3.0) / (2.0 * math.tan(b) ** 2 + s - 1.0) - math.tan(theta)
    b = brentq(f, math.asin(1.0 / F1) + 1e-9, math.radians(60.0))
    return b, 0.5 * (math.sqrt(1.0 + 8.0 * F1 * F1 * math.sin(b) ** 2) - 1.0)


def test_frozen_linearisation_is_eq12_at_a_uniform_state(orc):
    """With linear WENO weights the characteristic basis cancels, so at a
    uniform state the frozen Jacobian and Eq. 12 differ only by the weights'
    response to the perturbation itself, of relative size about eps/zeta * eps;
    the residuals are the same bits."""
    p = I.make_problem_2d(8, 8, 1, 0, 2.0, 0, 2.0, 9.81, I.bottom2d_flat(),
                          (I.BC2_INFLOW, I.BC2_OUTFLOW, I.BC2_REFLECT, I.BC2_REFLECT),
                          np.array([[1.0, 2.0, 0.1], [0, 0, 0], [0, 0, 0], [0, 0, 0]]), lambda X, Y: (1.0, 2.0, 0.1))
    pr = orc.problem_levels2d(p)[0]
    U = np.array([1.0, 2.0, 0.1])[:, None] * np.ones((3, 64))
    Ja, Ra, _ = orc.jacobian2d(pr, U, 1e-6, 3.0, I.ST_J21)
    Jb, Rb, _ = orc.jacobian2d(pr, U, 1e-6, 3.0, I.ST_J21, frozen=True)
    assert np.array_equal(Ra, Rb)
    assert np.abs(Ja - Jb).max() <= 2e-5 * np.abs(Ja).max()


def test_frozen_linearisation_freezes_the_weights(orc):
    """Near-uniform data whose differences (1e-3) make the smoothness
    indicators comparable to zeta: the Eq. 12 quotient moves by percents
    between eps = 1e-4 and 1e-6 (the weights react to the perturbation), the
    frozen one only by the flux curvature, O(eps)."""
    rng = np.random.default_rng(3)
    p = I.make_problem_2d(8, 8, 1, 0, 2.0, 0, 2.0, 9.81, I.bottom2d_flat(),
                          (I.BC2_INFLOW, I.BC2_OUTFLOW, I.BC2_REFLECT, I.BC2_REFLECT),
                          np.array([[1.0, 2.0, 0.1], [0, 0, 0], [0, 0, 0], [0, 0, 0]]), lambda X, Y: (1.0, 2.0, 0.1))
    pr = orc.problem_levels2d(p)[0]
    U = np.array([1.0, 2.0, 0.1])[:, None] + 1e-3 * rng.standard_normal((3, 64))
    moved = {}
    for frozen in (False, True):
        Ja, _, _ = orc.jacobian2d(pr, U, 1e-4, 3.0, I.ST_J21, frozen=frozen)
        Jb, _, _ = orc.jacobian2d(pr, U, 1e-6, 3.0, I.ST_J21, frozen=frozen)
        moved[frozen] = np.abs(Ja - Jb).max() / np.abs(Jb).max()
    assert moved[True] < 5e-4 and moved[False] > 1e-2, moved


def test_wedge_reaches_the_oblique_jump_with_the_frozen_linearisation(orc):
    """Section 5.2.2 with the paper's parameters (omega = 0.1, nu3 = 3, nested
    from 16 x 8 with nu = 10, 15 on 16 x 8, 32 x 16) and the frozen
    linearisation: the solve converges, and the steady state is the oblique
    jump of the wedge: upstream depth 1, downstream depth h2 and jump angle
    beta - theta to the wall from the oblique jump relations at
    F1 = 8.57 / sqrt(g)."""
    Nx, Ny = 32, 16
    inp = I.wedge(Nx, Ny, 3, start_level=1)
    U, info = orc.solve_problem2d(inp, I.Params2D(levels=3, nu1=[15, 10, 10], nu2=[15, 10, 10], tol=1e-11,
                                                  n_max=400, nest_start=1, omega=0.1, frozen=True))
    assert info["status"] == 0 and info["res"][0] < 1e-11, info
    th = math.radians(8.95)
    beta, ratio = _oblique_jump(8.57 / math.sqrt(I.G_PAPER), th)
    assert abs(ratio - 1.5) < 1e-3  # the wedge of Section 5.2.2 is designed for h2 = 1.5
    h = U[0].reshape(Ny, Nx)
    dx, dy = 5.0 / Nx, 2.0 / Ny
    assert np.abs(h[:, :4] - 1.0).max() < 1e-3          # undisturbed inflow
    assert np.abs(h[:3, -8:] / ratio - 1.0).max() < 2e-3  # behind the jump, along the wall
    mid, pts = 0.5 * (1.0 + ratio), []
    for j in range(Ny):
        k = int(np.argmax(h[j] > mid))
        if k > 0:
            pts.append(((j + 0.5) * dy, (k - 0.5 + (mid - h[j, k - 1]) / (h[j, k] - h[j, k - 1])) * dx))
    pts = np.array(pts)
    slope, icpt = np.polyfit(pts[:, 1], pts[:, 0], 1)
    assert abs(math.degrees(math.atan(slope)) - math.degrees(beta - th)) < 1.0
    assert abs(-icpt / slope - 1.0 / math.cos(th)) < dx  # the jump starts where the wall does


@pytest.mark.parametrize("k", [0, 2, 4])
def test_seeded_wedges_reach_their_oblique_jump(orc, k):
    """The seeded wedges of the batched 2D workload (Froude ~U[2, 4],
    deflection ~U[5, 15] degrees, [0, 40] x [0, 30]) converge under the frozen
    linearisation with the paper's omega = 0.1, and the depth along the wall
    behind the jump is the oblique-jump value h2 / h1 for that seed's Froude
    number and deflection."""
    inp = I.wedge_serving_2d(k, 32, 16, 3)
    U, info = orc.solve_problem2d(inp, I.Params2D(levels=3, nu1=[20], nu2=[20], tol=1e-10, n_max=400, nest_start=1,
                                                  omega=0.1, frozen=True))
    assert info["status"] == 0 and info["res"][0] < 1e-10, info
    _, ratio = _oblique_jump(inp.meta["froude"], math.radians(inp.meta["theta_deg"]))
    h = U[0].reshape(16, 32)
    assert abs(h[0, -3:].mean() / ratio - 1.0) < 2e-3, (h[0, -3:], ratio)
    assert np.abs(h[-4:, :3] - 1.0).max() < 1e-3  # the inflow corner is undisturbed


def _block_split(orc, inp, U):
    """Entrywise l1 norms of the J21 blocks of in-grid neighbours, split into
    the nine kept by J9 (the cross) and the twelve it drops."""
    pr = orc.problem_levels2d(inp)[0]
    J, _, _ = orc.jacobian2d(pr, U, 1e-6, 3.0, orc.ST_J21)
    cross = {(0, -2), (0, -1), (-2, 0), (-1, 0), (0, 0), (1, 0), (2, 0), (0, 1), (0, 2)}
    kept, dropped = [], []
    for c in range(inp.Nx * inp.Ny):
        i, j = c % inp.Nx, c // inp.Nx
        for k, (dx, dy) in enumerate(orc.stencil2d(orc.ST_J21)):
            if 0 <= i + dx < inp.Nx and 0 <= j + dy < inp.Ny:
                (kept if (dx, dy) in cross else dropped).append(np.abs(J[k, :, c]).sum())
    return np.array(kept), np.array(dropped)


def test_j9_keeps_the_large_blocks(orc):
    """Section 4.1: on the 16 x 8 grid of Section 5.2.1, at its initial state
    (Eq. 30), every block J9 keeps has l1-norm above 0.5, every block it drops
    is below 0.5, and most dropped blocks are below 1e-6 (the paper reports
    83 %); for the wedge of Section 5.2.2 at Eq. 31 every kept block exceeds 1
    (the paper: 100 %)."""
    b = I.paper_parabolic_bump(16, 8, 2)
    kept, dropped = _block_split(orc, b, np.stack([np.ones(128), np.ones(128), np.zeros(128)]))
    assert kept.min() > 0.5 and dropped.max() < 0.5, (kept.min(), dropped.max())
    assert (dropped < 1e-6).mean() > 0.8
    w = I.wedge(16, 8, 1)
    s = w.bc_state[0]
    kept, _ = _block_split(orc, w, np.stack([np.full(128, s[0]), np.full(128, s[1]), np.full(128, s[2])]))
    assert kept.min() > 1.0
