"""The latency form of the 1D solve: one problem per thread-block cluster
(nswe_ctx_set_solve_cluster). Every cell sees the same arithmetic as in the
block form; only the order of the sum that forms res differs, which can move
the Newton step at which res crosses tol. The cluster kernel is a separate
instantiation, so, as between launch shapes, the compiler's fused
multiply-adds may differ: FP64 solutions agree with the block form to a few
ulps, mixed-precision ones within the mixed bound, and both match the
oracle."""
import numpy as np
import pytest

import oracle as orc
from paper_2505_10857_gb300 import inputs as I

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


class Batch:
    def __init__(self, nswe, ctx, inps):
        self.probs = [nswe.Problem1D.from_inputs(ctx, p) for p in inps]
        self.U0s = [torch.from_numpy(p.U0_start).cuda() for p in inps]
        self.Us = [torch.zeros((2, p.N), dtype=torch.float64, device="cuda") for p in inps]

    def solve(self, nswe, ctx, prm):
        infos = nswe.nswe_newton_solve_batch(ctx, self.probs, self.U0s, self.Us, prm)
        return [u.cpu().numpy() for u in self.Us], infos

    def close(self):
        torch.cuda.synchronize()
        for p in self.probs:
            p.close()


def _agree(U, infos, U_ref, infos_ref, precision):
    bound, slack = (1e-13, 1) if precision == 0 else (1e-8, 2)
    for k in range(len(U)):
        assert infos[k]["status"] == 0, (k, infos[k]["status"])
        assert all(abs(x - y) <= slack for x, y in zip(infos[k]["iters"], infos_ref[k]["iters"])), \
            (k, infos[k]["iters"], infos_ref[k]["iters"])
        same_steps = list(infos[k]["iters"]) == list(infos_ref[k]["iters"])
        err = np.abs(U[k] - U_ref[k]).max() / np.abs(U_ref[k]).max()
        # a solve stopped one Newton step later differs by that step (res < 1e-10)
        assert err <= (bound if same_steps else 1e-9), (k, err, infos[k]["iters"], infos_ref[k]["iters"])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("ctas,team_cells", [(2, 256), (8, 1), (8, 1024), (16, 512), (16, 1 << 30)])
def test_cluster_solve_agrees_with_block_solve(nswe, ctx, precision, ctas, team_cells):
    """Three 1024-cell channels nested from 256 cells, every split of the
    multigrid levels between the cluster and its leader CTA (team_cells 1:
    all levels on the cluster; 2^30: all on the leader)."""
    inps = [I.channel_irregular(k, N=1024, levels=6, start_level=2) for k in range(3)]
    prm = nswe.params_from(I.Params1D.for_problem(inps[0], tol=1e-10, n_max=500))
    prm.precision = precision
    b = Batch(nswe, ctx, inps)
    try:
        U_ref, infos_ref = b.solve(nswe, ctx, prm)
        nswe.nswe_ctx_set_solve_cluster(ctx, ctas, team_cells)
        U, infos = b.solve(nswe, ctx, prm)
    finally:
        nswe.nswe_ctx_set_solve_cluster(ctx, 1, 1024)
        b.close()
    _agree(U, infos, U_ref, infos_ref, precision)


def test_cluster_single_solve_of_the_default_channel_matches_the_oracle(nswe, ctx):
    """One N = 4096 channel (8 levels, nested from 256 cells, J3, FP64) on a
    16-CTA cluster, against the oracle's solve with the same stopping test."""
    inp = I.channel_irregular(0)
    p1 = I.Params1D.for_problem(inp, tol=1e-10, n_max=800)
    prm = nswe.params_from(p1)
    b = Batch(nswe, ctx, [inp])
    try:
        nswe.nswe_ctx_set_solve_cluster(ctx, 16, 1024)
        U, infos = b.solve(nswe, ctx, prm)
    finally:
        nswe.nswe_ctx_set_solve_cluster(ctx, 1, 1024)
        b.close()
    assert infos[0]["status"] == 0
    Uo, info_o = orc.solve_problem(inp, p1)
    assert info_o["status"] == 0
    err = np.abs(U[0] - Uo).max() / np.abs(Uo).max()
    assert err <= 1e-10, err


def test_cluster_settings(nswe, ctx):
    assert nswe.nswe_ctx_get_solve_cluster(ctx) == (1, 1024)
    nswe.nswe_ctx_set_solve_cluster(ctx, 4, 2048)
    assert nswe.nswe_ctx_get_solve_cluster(ctx) == (4, 2048)
    for ctas, cells in [(0, 1024), (17, 1024), (4, 0)]:
        with pytest.raises(nswe.NsweError):
            nswe.nswe_ctx_set_solve_cluster(ctx, ctas, cells)
    assert nswe.nswe_ctx_get_solve_cluster(ctx) == (4, 2048)
    nswe.nswe_ctx_set_solve_cluster(ctx, 1, 1024)


@pytest.mark.parametrize("precision", [0, 1])
def test_cluster_solve_with_the_full_jacobian_agrees(nswe, ctx, precision):
    """J5 (nb = 5, Section 3.3's full Jacobian): the coarsest nested level is
    solved directly with the five-block band, on the leader CTA."""
    inps = [I.channel_irregular(k, N=1024, levels=6, start_level=2) for k in range(2)]
    prm = nswe.params_from(I.Params1D.for_problem(inps[0], tol=1e-10, n_max=500, nb=5))
    prm.precision = precision
    b = Batch(nswe, ctx, inps)
    try:
        U_ref, infos_ref = b.solve(nswe, ctx, prm)
        nswe.nswe_ctx_set_solve_cluster(ctx, 8, 512)
        U, infos = b.solve(nswe, ctx, prm)
    finally:
        nswe.nswe_ctx_set_solve_cluster(ctx, 1, 1024)
        b.close()
    _agree(U, infos, U_ref, infos_ref, precision)


def test_llf_problems_keep_the_block_form_under_the_cluster_setting(nswe, ctx):
    """The cluster form is built for the HLL flux; LLF problems (Section 3.1's
    alternative) run in the block form whatever the setting: the same bits as
    with the setting off."""
    inps = [I.channel_irregular(k, N=1024, levels=6, start_level=2) for k in range(2)]
    for p in inps:
        p.flux = nswe.FLUX_LLF
    prm = nswe.params_from(I.Params1D.for_problem(inps[0], tol=1e-10, n_max=500))
    b = Batch(nswe, ctx, inps)
    try:
        U_ref, infos_ref = b.solve(nswe, ctx, prm)
        nswe.nswe_ctx_set_solve_cluster(ctx, 8, 512)
        U, infos = b.solve(nswe, ctx, prm)
    finally:
        nswe.nswe_ctx_set_solve_cluster(ctx, 1, 1024)
        b.close()
    for k in range(len(inps)):
        assert infos[k]["status"] == 0 and np.array_equal(U[k], U_ref[k]), k
