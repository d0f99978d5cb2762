"""GPU parity of the mixed-precision 1D path (NSWE_PREC_MIXED) against the
FP64 oracle.

The FP32 parts are compared with the oracle's FP64 arithmetic on the same
inputs, with bounds derived from FP32 rounding (u = 2^-24):
  Jacobian  the perturbed and base residuals each carry a few u of the flux
            scale, and rounding the state to FP32 moves the perturbation by
            u|U|; their difference over eps gives 8u (scale + |U| |J|)/eps,
            plus 4u |J| for the regularisation rounded to FP32 (the cases
            here reach a third of it).
  V-cycle   the same system in FP32 and FP64 (J and R exactly representable
            in both): the result agrees to the stated 1e-5 relative bound for
            the FP32 parts (the cases here reach 3.5e-6).
The mixed Newton solve must reach the same FP64 stopping test (res < tol,
checked again by the oracle's residual of the returned state) and land on
the FP64 discrete solution to 1e-10 relative. That solution is the oracle's
solve converged to res < 1e-13. A solve stopped at res < 1e-10 is only
within a few 1e-9 of it (Newton damped by tau = 0.6 contracts the error by
0.4 per step, so the last step leaves it at about the size of the previous
correction), whichever precision takes the steps; at res < 1e-12 the 1D
channels here sit within 7.4e-11 of it (48 seeds of the 4096-cell channel on
the oracle). The 1D mixed solves therefore stop at res < 1e-12; the 2D one,
whose residual is divided by the cell area, stops at res < 1e-11 (8e-12 from
the converged solution on the oracle).
"""
import numpy as np
import pytest

from paper_2505_10857_gb300 import inputs as I
from gpu_util import flux_scale

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS32 = 2.0 ** -24
MIXED_BOUND = 1e-10
TOL_CONVERGED = 1e-13
VCYCLE_F32_BOUND = 1e-5


@pytest.fixture(scope="module")
def nswe():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_10857_gb300 import nswe as N
    N.lib()
    return N


@pytest.fixture(scope="module")
def ctx(nswe):
    return nswe.Context(0)


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


def problems():
    return {
        "small": I.channel_small(0),
        "irregular": I.channel_irregular(3),
        "eq26": I.paper_smooth_subcritical(192, levels=2),
        "eq28_right": I.paper_bump(96, levels=2, regime="sub", width="right"),
    }


def state_for(inp, level, seed):
    rng = np.random.default_rng(seed)
    n = inp.N_level(level)
    xc = inp.centres(level)
    H = inp.sig_fn(xc) * (inp.bcr[1] if inp.bcr[1] > 0 else 1.5) * (1 + 0.05 * np.sin(3 * xc)) \
        + 0.01 * rng.standard_normal(n)
    Q = np.full(n, inp.bcl[2] if inp.bcl[2] != 0 else 1.0) + 0.05 * rng.standard_normal(n)
    return np.ascontiguousarray(np.stack([np.abs(H) + 0.5, Q]))


@pytest.mark.parametrize("name", list(problems()))
@pytest.mark.parametrize("nb", [3, 5])
def test_jacobian_f32_parity(nswe, ctx, orc, name, nb):
    inp = problems()[name]
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    for level in sorted({0, inp.levels - 1}):
        pr = orc.problem_levels(inp)[level]
        U = state_for(inp, level, 20 + level)
        eps = I.eps_for_n(pr.N)
        Jref, Rref, resref = orc.jacobian1d(pr, U, eps, 3.0, nb)
        dR = torch.zeros((2, pr.N), dtype=torch.float64, device="cuda")
        dres = torch.zeros(1, dtype=torch.float64, device="cuda")
        dJ = torch.full((nb, 4, pr.N), float("nan"), dtype=torch.float32, device="cuda")
        nswe.nswe_jacobian_f32(ctx, prob, level, nb, dev(U), eps, 3.0, dR, dJ, dres)
        J, R = host(dJ), host(dR)
        sc = flux_scale(U, inp.g)
        # the residual of a mixed step is the FP64 one
        assert np.abs(R - Rref).max() <= 1e-12 * sc
        assert abs(host(dres)[0] - resref) <= 1e-12 * max(resref, sc * 1e-3)
        jmax = np.abs(Jref).max()
        tol = 8 * EPS32 * (sc + np.abs(U).max() * jmax) / eps + 4 * EPS32 * jmax
        assert np.isfinite(J).all()
        err = np.abs(J - Jref).max()
        assert err <= tol, (level, err, tol)
        # blocks outside the grid are exactly zero
        assert np.abs(J[Jref == 0.0]).max(initial=0.0) == 0.0


@pytest.mark.parametrize("name,level,nb", [("small", 0, 3), ("small", 0, 5), ("small", 3, 3), ("small", 3, 5),
                                           ("irregular", 0, 3), ("irregular", 4, 3), ("irregular", 0, 5),
                                           ("eq26", 0, 3)])
def test_vcycle_f32_parity(nswe, ctx, orc, name, level, nb):
    inp = problems()[name]
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    pr = orc.problem_levels(inp)[level]
    U = state_for(inp, level, 30 + level)
    J, R, _ = orc.jacobian1d(pr, U, I.eps_for_n(pr.N), 3.0, nb)
    # FP32-representable inputs, so that both sides solve the same system
    J = J.astype(np.float32).astype(np.float64)
    R = R.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(31)
    dU0 = (1e-3 * rng.standard_normal((2, pr.N))).astype(np.float32).astype(np.float64)
    nlev = inp.levels - level
    ref = orc.vcycle1d(J, R, dU0, nb, nlev, inp.omega, 2, 2)
    prm = nswe.params(inp.N, inp.levels, omega=inp.omega, nu1=2, nu2=2)
    ddU = dev(dU0, torch.float32)
    nswe.nswe_mg_vcycle_f32(ctx, prob, level, nb, dev(J, torch.float32), dev(R, torch.float32), ddU, prm)
    got = host(ddU)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= VCYCLE_F32_BOUND, err


CASES = {"small0": lambda: I.channel_small(0), "small1": lambda: I.channel_small(1),
         "irregular3": lambda: I.channel_irregular(3), "eq26": lambda: I.paper_smooth_subcritical(384, 3),
         "small0_j5": lambda: I.channel_small(0)}


@pytest.mark.parametrize("case", list(CASES))
def test_mixed_newton_solve(nswe, ctx, orc, case):
    inp = CASES[case]()
    nb = 5 if case.endswith("j5") else 3
    prm = I.Params1D.for_problem(inp, tol=1e-12, n_max=500, nb=nb)
    _, iref = orc.solve_problem(inp, prm)
    assert iref["status"] == 0
    Uref, iconv = orc.solve_problem(inp, I.Params1D.for_problem(inp, tol=TOL_CONVERGED, n_max=800, nb=nb))
    assert iconv["status"] == 0
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    p = nswe.params_from(prm)
    p.precision = nswe.PREC_MIXED
    dU = torch.zeros((2, inp.N), dtype=torch.float64, device="cuda")
    info = nswe.nswe_newton_solve(ctx, prob, dev(inp.U0_start), dU, p)
    U = host(dU)
    assert info["status"] == 0, info
    assert info["res"][0] < prm.tol
    # the oracle's own residual of the returned state passes the same test
    _, res = orc.residual1d(orc.problem_levels(inp)[0], U)
    assert res < prm.tol, res
    err = np.abs(U - Uref).max() / np.abs(Uref).max()
    assert err <= MIXED_BOUND, err
    # the FP32 Jacobian error (~1e-5 relative) is far below that of the FD
    # Jacobian itself, so the Newton counts stay those of the FP64 solve
    start = inp.start_level if inp.start_level >= 0 else inp.levels - 1
    for l in range(start + 1):
        assert abs(info["iters"][l] - iref["iters"][l]) <= 2 + iref["iters"][l] // 10, (info["iters"], iref["iters"])


def test_mixed_batch_equals_single(nswe, ctx):
    inps = [I.channel_small(k) for k in range(3)]
    prm = nswe.params_from(I.Params1D.for_problem(inps[0], tol=1e-10, n_max=500))
    prm.precision = nswe.PREC_MIXED
    probs = [nswe.Problem1D.from_inputs(ctx, p) for p in inps]
    U0s = [dev(p.U0_start) for p in inps]
    singles = []
    for k in range(3):
        u = torch.zeros((2, inps[k].N), dtype=torch.float64, device="cuda")
        nswe.nswe_newton_solve(ctx, probs[k], U0s[k], u, prm)
        singles.append(host(u))
    Us = [torch.zeros((2, p.N), dtype=torch.float64, device="cuda") for p in inps]
    infos = nswe.nswe_newton_solve_batch(ctx, probs, U0s, Us, prm)
    for k in range(3):
        assert infos[k]["status"] == 0
        assert np.array_equal(host(Us[k]), singles[k])


# ---------------------------------------------------------------- 2D

def _state2d(inp, level, seed):
    rng = np.random.default_rng(seed)
    X, Y = inp.centres(level)
    s0 = inp.bc_state[0]
    h = 1.2 + 0.2 * np.sin(X) * np.cos(Y) + 0.01 * rng.standard_normal(X.shape)
    hu = (s0[1] if s0[1] else 1.0) * (1 + 0.05 * np.cos(Y + X)) + 0.02 * rng.standard_normal(X.shape)
    hv = 0.1 * np.sin(X) + 0.02 * rng.standard_normal(X.shape)
    return np.ascontiguousarray(np.stack([h.ravel(), hu.ravel(), hv.ravel()]))


def _flux_scale2(U, g, d):
    h, m = np.abs(U[0]).max(), np.abs(U[1:]).max()
    return (m * m / np.abs(U[0]).min() + 0.5 * g * h * h + m) / d


@pytest.mark.parametrize("nb", [9, 21])
def test_jacobian_f32_parity_2d(nswe, ctx, orc, nb):
    """2D: the FD Jacobian is evaluated in FP64 (eps = 1e-6 leaves nothing to
    difference in FP32) and rounded to FP32: the FP64 bound plus one FP32
    rounding (2^-24 relative) per entry."""
    inp = I.wedge(32, 16, 2)
    prob = nswe.Problem2D.from_inputs(ctx, inp)
    pr = orc.problem_levels2d(inp)[0]
    U = _state2d(inp, 0, 20)
    Jref, Rref, _ = orc.jacobian2d(pr, U, 1e-6, 3.0, orc.ST_J21 if nb == 21 else orc.ST_J9)
    dR = torch.zeros((3, pr.n), dtype=torch.float64, device="cuda")
    dJ = torch.full((nb, 9, pr.n), float("nan"), dtype=torch.float32, device="cuda")
    nswe.nswe_jacobian_f32(ctx, prob, 0, nb, dev(U), 1e-6, 3.0, dR, dJ)
    J = host(dJ)
    sc = _flux_scale2(U, inp.g, min(pr.s.dx, pr.s.dy))
    assert np.abs(host(dR) - Rref).max() <= 1e-12 * sc
    tol = 1e-12 * np.abs(Jref).max() + 8.0 * 2.0 ** -52 * sc / 1e-6 + EPS32 * np.abs(Jref)
    assert np.isfinite(J).all()
    assert (np.abs(J - Jref) <= tol).all(), np.abs(J - Jref).max()


@pytest.mark.parametrize("name,colours", [("bump", 0), ("wedge", 0), ("bump", 3)])
def test_vcycle_f32_parity_2d(nswe, ctx, orc, name, colours):
    inp = {"bump": I.paper_parabolic_bump(32, 16, 3), "wedge": I.wedge(32, 16, 2)}[name]
    prob = nswe.Problem2D.from_inputs(ctx, inp)
    pr = orc.problem_levels2d(inp)[0]
    J, R, _ = orc.jacobian2d(pr, _state2d(inp, 0, 30), 1e-6, 3.0, orc.ST_J9)
    J = J.astype(np.float32).astype(np.float64)
    R = R.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(31)
    dU0 = (1e-3 * rng.standard_normal((3, pr.n))).astype(np.float32).astype(np.float64)
    nx, ny = inp.dims(0)
    ref = orc.vcycle2d(J, R, dU0, nx, ny, orc.ST_J9, inp.levels, 0.1, 3, 3, colours)
    prm = nswe.params(96, inp.levels, omega=0.1, nu1=3, nu2=3, colours2d=colours)
    ddU = dev(dU0, torch.float32)
    nswe.nswe_mg_vcycle_f32(ctx, prob, 0, 9, dev(J, torch.float32), dev(R, torch.float32), ddU, prm)
    err = np.abs(host(ddU) - ref).max() / np.abs(ref).max()
    assert err <= VCYCLE_F32_BOUND, err


def test_mixed_newton_solve_2d(nswe, ctx, orc):
    inp = I.paper_parabolic_bump(32, 16, 3)
    prm = I.Params2D(levels=3, nu1=[15], nu2=[15], tol=1e-11, n_max=400)
    _, iref = orc.solve_problem2d(inp, prm)
    assert iref["status"] == 0
    Uref, iconv = orc.solve_problem2d(inp, I.Params2D(levels=3, nu1=[15], nu2=[15], tol=TOL_CONVERGED, n_max=400))
    assert iconv["status"] == 0
    prob = nswe.Problem2D.from_inputs(ctx, inp)
    p = nswe.params2d_from(prm)
    p.precision = nswe.PREC_MIXED
    dU = torch.zeros((3, inp.Nx * inp.Ny), dtype=torch.float64, device="cuda")
    info = nswe.nswe_newton_solve(ctx, prob, dev(inp.U0_start), dU, p)
    U = host(dU)
    assert info["status"] == 0, info
    _, res = orc.residual2d(orc.problem_levels2d(inp)[0], U)
    assert res < prm.tol, res
    assert np.abs(U - Uref).max() / np.abs(Uref).max() <= MIXED_BOUND
    for l in range(inp.levels):
        assert abs(info["iters"][l] - iref["iters"][l]) <= 2 + iref["iters"][l] // 10, (info["iters"], iref["iters"])
