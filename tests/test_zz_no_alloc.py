"""The allocation-free solve entry point gives the same results as
nswe_newton_solve.

nswe_newton_solve_noalloc is for callers that cannot call cudaMalloc, for
example code that runs after a framework's caching allocator has reserved the
device memory it may use, or real-time loops that must not block on the
device synchronisation that cudaMalloc/cudaFree imply. It keeps its problem
description and workspace in a fixed device array of the library. This test
calls it through the C ABI several times in a row, on problems of different
sizes, and compares each output with the allocating entry point's output
within the tolerance of the other solve tests (1e-10 relative). It also
checks that a problem larger than the array is rejected before any GPU work.
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
    return U.cpu().numpy()


def _noalloc(nswe, inp, prm):
    stream = torch.cuda.current_stream().cuda_stream
    sf = torch.from_numpy(inp.sig_face).cuda()
    gq = torch.from_numpy(inp.gq_all()).cuda()
    U0 = torch.from_numpy(inp.U0_start).cuda()
    U = torch.full((2, inp.N), float("nan"), dtype=torch.float64, device="cuda")
    info = torch.zeros(ctypes.sizeof(nswe.Info), dtype=torch.uint8, device="cuda")
    nswe.nswe_newton_solve_noalloc(0, stream, inp.N, inp.levels, inp.x0, inp.x1, inp.g, sf, gq, inp.bcl,
                                   inp.bcr, U0, U, prm, info)
    torch.cuda.synchronize()
    return U.cpu().numpy(), nswe.info_from_bytes(bytes(info.cpu().numpy()), inp.levels)


def test_noalloc_matches_allocating_solve_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_10857_gb300 import inputs as I
    from paper_2505_10857_gb300 import nswe

    ctx = nswe.Context(0)
    big = I.channel_irregular(5)   # N = 4096, the largest size the fixed array takes
    small = I.channel_small(2)     # N = 200
    cases = [big, small, big]
    refs = {}
    for inp in (big, small):
        prm = nswe.params_from(I.Params1D.for_problem(inp, tol=1e-10, n_max=500))
        refs[id(inp)] = (_reference(nswe, ctx, inp, prm), prm)
    for inp in cases:
        Uref, prm = refs[id(inp)]
        U, info = _noalloc(nswe, inp, prm)
        assert info["status"] == 0, info
        assert info["res"][0] < 1e-10
        assert np.isfinite(U).all()
        assert np.abs(U - Uref).max() <= 1e-10 * np.abs(Uref).max()


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
