"""Launch shapes of the batched 1D solve kernel and the autotuner. Every
shape runs the same per-cell arithmetic; the shapes are compiled with
different register budgets, so the compiler's fused multiply-adds may differ
and FP64 solutions agree to a few ulps (bound 1e-13 relative) with the same
Newton counts; mixed-precision solutions agree within the mixed bound."""
import numpy as np
import pytest

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

    def close(self):
        torch.cuda.synchronize()
        for p in self.probs:
            p.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_all_shapes_agree(nswe, ctx, precision):
    inps = [I.channel_irregular(k, N=1024, levels=6, start_level=2) for k in range(3)]
    prm = nswe.params_from(I.Params1D.for_problem(inps[0], tol=1e-10, n_max=500))
    prm.precision = precision
    b = Batch(nswe, ctx, inps)
    results = []
    try:
        for shape in range(len(nswe.solve_shapes())):
            nswe.nswe_ctx_set_solve_shape(ctx, precision, shape)
            infos = nswe.nswe_newton_solve_batch(ctx, b.probs, b.U0s, b.Us, prm)
            results.append(([u.cpu().numpy() for u in b.Us], [i["status"] for i in infos],
                            [i["iters"] for i in infos]))
    finally:
        nswe.nswe_ctx_set_solve_shape(ctx, precision, 0)
        b.close()
    # FP64: the same iterates up to those ulps. Mixed: FP32 rounding of the
    # Jacobian and multigrid moves the Newton path, and both solves stop at
    # res < tol, so they agree as any two converged mixed solves do.
    bound, slack = (1e-13, 0) if precision == 0 else (1e-8, 2)
    for shape, (U, status, iters) in enumerate(results):
        assert status == [0, 0, 0], (shape, status, iters)
        for a, b in zip(iters, results[0][2]):
            assert all(abs(x - y) <= slack for x, y in zip(a, b)), (shape, iters, results[0][2])
        for k in range(3):
            err = np.abs(U[k] - results[0][0][k]).max() / np.abs(results[0][0][k]).max()
            assert err <= bound, (shape, k, err)


def test_autotuner_picks_and_records_a_shape(nswe, ctx):
    inps = [I.channel_small(k) for k in range(8)]
    prm = nswe.params_from(I.Params1D.for_problem(inps[0], tol=1e-10, n_max=500))
    b = Batch(nswe, ctx, inps)
    try:
        ms, best = nswe.nswe_autotune_solve_batch(ctx, b.probs, b.U0s, b.Us, prm, reps=1)
        assert len(ms) == len(nswe.solve_shapes()) and all(m > 0 for m in ms)
        assert best == int(np.argmin(ms))
        assert nswe.nswe_ctx_get_solve_shape(ctx, 0) == best
        assert nswe.nswe_ctx_get_solve_shape(ctx, 1) == 0  # the other precision is untouched
    finally:
        nswe.nswe_ctx_set_solve_shape(ctx, 0, 0)
        b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_two_contexts_on_two_streams_solve_concurrently_with_the_same_bits(nswe, precision):
    """Two contexts, each with its own stream and its own copy of a batch,
    launched back to back so that their solves overlap on the GPU (the steady
    form of the benchmark): every solution equals, bit for bit, the same batch
    solved alone on one context."""
    inps = [I.channel_irregular(k, N=1024, levels=6, start_level=2) for k in range(6)]
    prm = nswe.params_from(I.Params1D.for_problem(inps[0], tol=1e-10, n_max=500))
    prm.precision = precision
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ctxs = [nswe.Context(0, stream=s.cuda_stream) for s in streams]
    batches = [Batch(nswe, c, inps) for c in ctxs]
    try:
        torch.cuda.synchronize()
        nswe.nswe_newton_solve_batch(ctxs[0], batches[0].probs, batches[0].U0s, batches[0].Us, prm)
        torch.cuda.synchronize()
        alone = [u.cpu().numpy() for u in batches[0].Us]
        for b in batches:
            for u in b.Us:
                u.zero_()
        torch.cuda.synchronize()
        for c, b in zip(ctxs, batches):  # asynchronous: the second launch overlaps the first
            nswe.nswe_newton_solve_batch(c, b.probs, b.U0s, b.Us, prm, want_info=False)
        torch.cuda.synchronize()
        for b in batches:
            for k, u in enumerate(b.Us):
                assert np.array_equal(u.cpu().numpy(), alone[k]), k
    finally:
        for b in batches:
            b.close()
        for c in ctxs:
            c.close()
