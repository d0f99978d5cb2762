"""The allocation-free solve entry point gives the same results as
nswe_newton_solve.

nswe_newton_solve_noalloc is for callers that cannot call cudaMalloc, for
example code that runs after a framework's caching allocator has reserved the
device memory it may use, or real-time loops that must not block on the
device synchronisation that cudaMalloc/cudaFree imply. It keeps its problem
description and workspace in a fixed device array of the library and runs
the same solve kernel, in the same launch shape, as the allocating entry
point, so its output must be the same bits. This test calls it through the C
ABI several times in a row, on problems of different sizes (large, small,
large again: the array keeps the previous call's contents, which must not
leak into the next result), in FP64 and in mixed precision, with and without
an info record, and compares each output bit for bit with the allocating
entry point's output. It also checks that a problem larger than the array is
rejected before any GPU work.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _reference(nswe, ctx, inp, prm):
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    U = torch.zeros((2, inp.N), dtype=torch.float64, device="cuda")
    info = nswe.nswe_newton_solve(ctx, prob, torch.from_numpy(inp.U0_start).cuda(), U, prm)
    torch.cuda.synchronize()
    assert info["status"] == 0
    return U.cpu().numpy(), info


def _noalloc(nswe, inp, prm, with_info=True):
    stream = torch.cuda.current_stream().cuda_stream
    sf = torch.from_numpy(inp.sig_face).cuda()
    gq = torch.from_numpy(inp.gq_all()).cuda()
    U0 = torch.from_numpy(inp.U0_start).cuda()
    U = torch.full((2, inp.N), float("nan"), dtype=torch.float64, device="cuda")
    info = torch.zeros(ctypes.sizeof(nswe.Info), dtype=torch.uint8, device="cuda") if with_info else None
    nswe.nswe_newton_solve_noalloc(0, stream, inp.N, inp.levels, inp.x0, inp.x1, inp.g, sf, gq, inp.bcl,
                                   inp.bcr, U0, U, prm, info)
    torch.cuda.synchronize()
    rec = nswe.info_from_bytes(bytes(info.cpu().numpy()), inp.levels) if with_info else None
    return U.cpu().numpy(), rec


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_allocating_solve_on_consecutive_calls(precision):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_10857_gb300 import inputs as I
    from paper_2505_10857_gb300 import nswe

    ctx = nswe.Context(0)
    big = I.channel_irregular(5)   # N = 4096, the largest size the fixed array takes
    small = I.channel_small(2)     # N = 200
    refs = {}
    for inp in (big, small):
        prm = nswe.params_from(I.Params1D.for_problem(inp, tol=1e-10, n_max=500))
        if precision == "mixed":
            prm.precision = nswe.PREC_MIXED
        refs[id(inp)] = _reference(nswe, ctx, inp, prm) + (prm,)
    # big -> small -> big with an info record, then big again without one
    for inp, with_info in ((big, True), (small, True), (big, True), (big, False)):
        Uref, iref, prm = refs[id(inp)]
        U, info = _noalloc(nswe, inp, prm, with_info)
        assert np.array_equal(U, Uref), np.abs(U - Uref).max()
        if with_info:
            assert info["status"] == 0, info
            assert info["res"][0] < 1e-10
            assert info["iters"][:inp.levels] == iref["iters"][:inp.levels]


def test_noalloc_rejects_problems_larger_than_its_array():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_10857_gb300 import inputs as I
    from paper_2505_10857_gb300 import nswe

    inp = I.channel_irregular(0, N=8192, levels=8)
    prm = nswe.params_from(I.Params1D.for_problem(inp))
    with pytest.raises(nswe.NsweError) as e:
        _noalloc(nswe, inp, prm)
    assert e.value.status == 1  # NSWE_EINVAL
