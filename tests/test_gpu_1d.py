"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: residual 1e-12 relative to the flux scale; Jacobian 1e-12
relative to the block scale plus 8u*scale/eps for FD cancellation; one
V-cycle 1e-12 relative; converged Newton solutions 1e-10 relative.
"""
import numpy as np
import pytest

from paper_2505_10857_gb300 import inputs as I
from gpu_util import flux_scale, jac_tol

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def problems():
    return {
        "small": I.channel_small(0),
        "small512": I.channel_small(0, N=512, levels=3),  # coarsest level of 128 cells
        "irregular": I.channel_irregular(3),
        "eq26": I.paper_smooth_subcritical(192, levels=2),
        "eq28_right": I.paper_bump(96, levels=2, regime="sub", width="right"),
        "tiny_state_bc": I.make_problem_1d(8, 1, 0.0, 1.0, 9.81, I.bottom_gaussian(0.1, 0.5, 0.2),
                                           I.width_sine(1.0, 1, 1.0), (I.BC_STATE, 2.0, 4.0),
                                           (I.BC_EXTRAP, 0.0, 0.0), h_init=2.0, q_init=4.0),
        "min4": I.make_problem_1d(4, 1, 0.0, 1.0, 9.81, I.bottom_linear(0.0, 0.01), I.width_constant(1.3),
                                  (I.BC_DISCHARGE, 0.0, 1.0), (I.BC_DEPTH, 1.5, 0.0), h_init=1.5, q_init=1.0),
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
def test_residual_parity(nswe, ctx, orc, name):
    inp = problems()[name]
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    for level in range(inp.levels):
        pr = orc.problem_levels(inp)[level]
        U = state_for(inp, level, 10 + level)
        Rref, resref = orc.residual1d(pr, U)
        dU_, dR, dres = dev(U), torch.zeros((2, pr.N), dtype=torch.float64, device="cuda"), \
            torch.zeros(1, dtype=torch.float64, device="cuda")
        nswe.nswe_residual(ctx, prob, level, dU_, dR, dres)
        R, res = host(dR), host(dres)[0]
        sc = flux_scale(U, inp.g)
        assert np.abs(R - Rref).max() <= 1e-12 * sc, (level, np.abs(R - Rref).max())
        assert abs(res - resref) <= 1e-12 * max(resref, sc * 1e-3)


@pytest.mark.parametrize("name", list(problems()))
@pytest.mark.parametrize("nb", [3, 5])
def test_jacobian_parity(nswe, ctx, orc, name, nb):
    inp = problems()[name]
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    for level in sorted({0, inp.levels - 1}):
        pr = orc.problem_levels(inp)[level]
        U = state_for(inp, level, 20 + level)
        eps = I.eps_for_n(pr.N)
        Jref, Rref, resref = orc.jacobian1d(pr, U, eps, 3.0, nb)
        dR = torch.zeros((2, pr.N), dtype=torch.float64, device="cuda")
        dJ = torch.full((nb, 4, pr.N), float("nan"), dtype=torch.float64, device="cuda")
        f = nswe.nswe_jacobian_simplified if nb == 3 else nswe.nswe_jacobian_full
        f(ctx, prob, level, dev(U), eps, 3.0, dR, dJ)
        J, R = host(dJ), host(dR)
        sc = flux_scale(U, inp.g)
        assert np.abs(R - Rref).max() <= 1e-12 * sc
        tol = jac_tol(Jref, sc, eps)
        assert np.isfinite(J).all()
        assert np.abs(J - Jref).max() <= tol, (level, np.abs(J - Jref).max(), tol)
        # blocks outside the grid are exactly zero, as in the oracle
        assert np.array_equal(J == 0.0, Jref == 0.0) or np.abs(J[Jref == 0.0]).max() == 0.0


def _random_system(orc, inp, level, nb, seed):
    pr = orc.problem_levels(inp)[level]
    U = state_for(inp, level, seed)
    J, R, _ = orc.jacobian1d(pr, U, I.eps_for_n(pr.N), 3.0, nb)
    return J, R


@pytest.mark.parametrize("name,level,nb", [("small", 0, 3), ("small", 0, 5), ("small", 2, 3), ("small", 3, 3),
                                           ("small", 3, 5), ("irregular", 0, 3), ("irregular", 4, 3),
                                           ("irregular", 0, 5), ("eq26", 0, 3), ("small512", 0, 3),
                                           ("small512", 2, 5)])
def test_vcycle_parity(nswe, ctx, orc, name, level, nb):
    inp = problems()[name]
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    J, R = _random_system(orc, inp, level, nb, 30 + level)
    N = R.shape[1]
    rng = np.random.default_rng(31)
    dU0 = 1e-3 * rng.standard_normal((2, N))
    prm_o = dict(omega=inp.omega, nu1=2, nu2=2)
    nlev = inp.levels - level
    ref = orc.vcycle1d(J, R, dU0, nb, nlev, prm_o["omega"], 2, 2)
    ref2 = orc.vcycle1d(J, R, ref, nb, nlev, prm_o["omega"], 2, 2)
    prm = nswe.params(inp.N, inp.levels, omega=inp.omega, nu1=2, nu2=2)
    ddU = dev(dU0)
    dJ, dR = dev(J), dev(R)
    nswe.nswe_mg_vcycle(ctx, prob, level, nb, dJ, dR, ddU, prm)
    got = host(ddU)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()
    nswe.nswe_mg_vcycle(ctx, prob, level, nb, dJ, dR, ddU, prm)
    got2 = host(ddU)
    assert np.abs(got2 - ref2).max() <= 1e-12 * np.abs(ref2).max()


def _solve_gpu(nswe, ctx, inp, prm_inputs):
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    prm = nswe.params_from(prm_inputs)
    U = torch.zeros((2, inp.N), dtype=torch.float64, device="cuda")
    info = nswe.nswe_newton_solve(ctx, prob, dev(inp.U0_start), U, prm)
    return host(U), info


@pytest.mark.parametrize("case", ["small0", "small1", "irregular3", "eq26", "small0_j5", "eq28_trans_const",
                                  "eq28_trans_left", "eq28_trans_right", "max_coarse_j3", "direct128_j3",
                                  "direct128_j5"])
def test_newton_solve_parity(nswe, ctx, orc, case):
    inp = {"small0": lambda: I.channel_small(0), "small1": lambda: I.channel_small(1),
           "irregular3": lambda: I.channel_irregular(3), "eq26": lambda: I.paper_smooth_subcritical(384, 3),
           "small0_j5": lambda: I.channel_small(0),
           "eq28_trans_const": lambda: I.paper_bump(192, levels=2, regime="trans", width="const"),
           "eq28_trans_left": lambda: I.paper_bump(192, levels=2, regime="trans", width="left"),
           "eq28_trans_right": lambda: I.paper_bump(192, levels=2, regime="trans", width="right"),
           # the largest coarsest level the library takes (128 cells): band LU of 256 unknowns
           "max_coarse_j3": lambda: I.channel_small(0, N=512, levels=3),
           "direct128_j3": lambda: I.channel_small(0, N=128, levels=1),
           "direct128_j5": lambda: I.channel_small(0, N=128, levels=1)}[case]()
    prm = I.Params1D.for_problem(inp, tol=1e-10 if case != "eq26" else 1e-11, n_max=500,
                                 nb=5 if case.endswith("j5") else 3)
    Uref, iref = orc.solve_problem(inp, prm)
    U, info = _solve_gpu(nswe, ctx, inp, prm)
    assert iref["status"] == 0
    assert info["status"] == 0, info
    assert info["res"][0] < prm.tol
    assert np.abs(U - Uref).max() <= 1e-10 * np.abs(Uref).max(), np.abs(U - Uref).max()
    # same iterates up to rounding: the Newton counts agree per level (near
    # critical flow the contraction per step is close to 1, so rounding moves
    # the step at which res first falls below tol by a few percent)
    start = inp.start_level if inp.start_level >= 0 else inp.levels - 1
    for l in range(start + 1):
        assert abs(info["iters"][l] - iref["iters"][l]) <= 2 + iref["iters"][l] // 20, (l, info["iters"],
                                                                                        iref["iters"])


def test_batch_equals_single(nswe, ctx):
    inps = [I.channel_small(k) for k in range(3)] + [I.channel_small(5, N=400, levels=5)]
    prms = [I.Params1D.for_problem(p, tol=1e-10, n_max=500) for p in inps]
    singles = [_solve_gpu(nswe, ctx, p, q)[0] for p, q in zip(inps, prms)]
    # one launch for all (same parameters: omega / eps per level identical for the N=200 family)
    probs = [nswe.Problem1D.from_inputs(ctx, p) for p in inps[:3]]
    U0s = [dev(p.U0_start) for p in inps[:3]]
    Us = [torch.zeros((2, p.N), dtype=torch.float64, device="cuda") for p in inps[:3]]
    infos = nswe.nswe_newton_solve_batch(ctx, probs, U0s, Us, nswe.params_from(prms[0]))
    for k in range(3):
        assert infos[k]["status"] == 0
        assert np.array_equal(host(Us[k]), singles[k])


def test_batch_with_parameters_per_problem(nswe, ctx):
    """Uneven 1D instances in one launch, each with its own parameters (J3 and
    J5, relaxation, smoothing, sizes and nested starts): every result equals,
    bit for bit, the same problem solved alone with its parameters; a batch
    that mixes arithmetic types is refused."""
    inps = [I.channel_small(0), I.channel_small(1), I.channel_small(5, N=400, levels=5), I.paper_smooth_subcritical(384, 3)]
    prms = [I.Params1D.for_problem(inps[0], tol=1e-10, n_max=500),
            I.Params1D.for_problem(inps[1], tol=1e-10, n_max=500, nb=5),
            I.Params1D.for_problem(inps[2], tol=1e-10, n_max=500, omega=1.0, nu1=3, nu2=3),
            I.Params1D.for_problem(inps[3], tol=1e-11, n_max=500)]
    singles = [_solve_gpu(nswe, ctx, p, q) for p, q in zip(inps, prms)]
    probs = [nswe.Problem1D.from_inputs(ctx, p) for p in inps]
    U0s = [dev(p.U0_start) for p in inps]
    Us = [torch.zeros((2, p.N), dtype=torch.float64, device="cuda") for p in inps]
    cp = [nswe.params_from(q) for q in prms]
    infos = nswe.nswe_newton_solve_batch_each(ctx, probs, U0s, Us, cp)
    for k in range(len(inps)):
        assert infos[k]["status"] == 0 == singles[k][1]["status"], (k, infos[k])
        assert infos[k]["iters"] == singles[k][1]["iters"]
        assert np.array_equal(host(Us[k]), singles[k][0])
    cp[1].precision = nswe.PREC_MIXED
    with pytest.raises(nswe.NsweError):
        nswe.nswe_newton_solve_batch_each(ctx, probs, U0s, Us, cp)


def test_invalid_arguments_rejected(nswe, ctx):
    inp = I.channel_small(0)
    with pytest.raises(nswe.NsweError):
        nswe.Problem1D(ctx, 200, 5, 0.0, 25.0, 9.81, inp.sig_face, inp.gq_all(), inp.bcl, inp.bcr)  # 200 % 16
    with pytest.raises(nswe.NsweError):
        nswe.Problem1D(ctx, 200, 4, 25.0, 0.0, 9.81, inp.sig_face, inp.gq_all(), inp.bcl, inp.bcr)
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    U = torch.zeros((2, 200), dtype=torch.float64, device="cuda")
    with pytest.raises(nswe.NsweError):
        nswe.nswe_residual(ctx, prob, 4, U, U)
    prm = nswe.params(200, 4, tau=1.5)
    with pytest.raises(nswe.NsweError):
        nswe.nswe_newton_solve(ctx, prob, dev(inp.U0_start), U, prm)


def test_negative_depth_reported_not_faulted(nswe, ctx):
    inp = I.channel_small(0)
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    U0 = inp.U0_start.copy()
    U0[0, 3] = -1.0
    U = torch.zeros((2, 200), dtype=torch.float64, device="cuda")
    info = nswe.nswe_newton_solve(ctx, prob, dev(U0), U, nswe.params_from(I.Params1D.for_problem(inp, n_max=50)))
    assert info["status"] in (5, 6)  # ENAN or ENEGDEPTH
    # the context still works afterwards
    R = torch.zeros((2, 200), dtype=torch.float64, device="cuda")
    nswe.nswe_residual(ctx, prob, 0, dev(np.stack([np.full(200, 2.0), np.full(200, 4.42)])), R)
    assert np.isfinite(host(R)).all()


def test_batched_geometry_upload_equals_single(nswe, ctx):
    """nswe_prob_set_geometry_batch_1d leaves every problem as the single
    upload does (the same solve, bit for bit); invalid data in one problem
    refuses the whole batch before any upload."""
    inps = [I.channel_small(k) for k in range(4)]
    prm = nswe.params_from(I.Params1D.for_problem(inps[0], tol=1e-10, n_max=500))
    probs = [nswe.Problem1D.from_inputs(ctx, I.channel_small(9)) for _ in inps]  # other geometry first
    nswe.nswe_prob_set_geometry_batch_1d(ctx, probs, [p.sig_face for p in inps], [p.gq_all() for p in inps],
                                         [p.bcl for p in inps], [p.bcr for p in inps])
    for p, pr in zip(inps, probs):
        U = torch.zeros((2, p.N), dtype=torch.float64, device="cuda")
        info = nswe.nswe_newton_solve(ctx, pr, dev(p.U0_start), U, prm)
        Uref, iref = _solve_gpu(nswe, ctx, p, I.Params1D.for_problem(inps[0], tol=1e-10, n_max=500))
        assert info["status"] == 0 and np.array_equal(host(U), Uref)
    bad = [p.gq_all().copy() for p in inps]
    bad[2][5] = float("nan")
    with pytest.raises(nswe.NsweError):
        nswe.nswe_prob_set_geometry_batch_1d(ctx, probs, [p.sig_face for p in inps], bad,
                                             [p.bcl for p in inps], [p.bcr for p in inps])


@pytest.mark.parametrize("name", ["small", "irregular"])
def test_llf_residual_and_jacobian_parity(nswe, ctx, orc, name):
    """The LLF flux (nswe_prob_set_flux_1d) against the oracle's: residual,
    J3 and J5, on every level of two problems."""
    inp = problems()[name]
    inp.flux = 1  # LLF
    try:
        prob = nswe.Problem1D.from_inputs(ctx, inp)
        for level in sorted({0, inp.levels - 1}):
            pr = orc.problem_levels(inp)[level]
            U = state_for(inp, level, 40 + level)
            sc = flux_scale(U, inp.g)
            Rref, _ = orc.residual1d(pr, U)
            dR = torch.zeros((2, pr.N), dtype=torch.float64, device="cuda")
            nswe.nswe_residual(ctx, prob, level, dev(U), dR)
            assert np.abs(host(dR) - Rref).max() <= 1e-12 * sc
            for nb in (3, 5):
                eps = I.eps_for_n(pr.N)
                Jref, _, _ = orc.jacobian1d(pr, U, eps, 3.0, nb)
                dJ = torch.full((nb, 4, pr.N), float("nan"), dtype=torch.float64, device="cuda")
                f = nswe.nswe_jacobian_simplified if nb == 3 else nswe.nswe_jacobian_full
                f(ctx, prob, level, dev(U), eps, 3.0, dR, dJ)
                assert np.abs(host(dJ) - Jref).max() <= jac_tol(Jref, sc, eps)
        # HLL differs from LLF on these states
        Rllf = host(dR)
        prob.set_flux(nswe.FLUX_HLL)
        nswe.nswe_residual(ctx, prob, inp.levels - 1, dev(U), dR)
        assert not np.allclose(host(dR), Rllf)
    finally:
        inp.flux = 0


@pytest.mark.parametrize("precision", [0, 1])
def test_llf_solve_parity(nswe, ctx, orc, precision):
    """Nested solve of Eq. 26 (192 cells) with the LLF flux against the
    oracle's: FP64 to 1e-10, mixed precision within its bound."""
    inp = I.paper_smooth_subcritical(192, 2)
    inp.flux = 1
    prm = I.Params1D.for_problem(inp, tol=1e-11, n_max=500)
    Uref, iref = orc.solve_problem(inp, prm)
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    p = nswe.params_from(prm)
    p.precision = precision
    U = torch.zeros((2, inp.N), dtype=torch.float64, device="cuda")
    info = nswe.nswe_newton_solve(ctx, prob, dev(inp.U0_start), U, p)
    assert info["status"] == 0 == iref["status"], (info, iref)
    err = np.abs(host(U) - Uref).max() / np.abs(Uref).max()
    assert err <= (1e-10 if precision == 0 else 1e-8), err
    if precision == 0:
        assert abs(info["iters"][0] - iref["iters"][0]) <= 2
