"""GPU tests of the continuous-batching server: every result in a mix of
requests of different sizes, arriving at different times, equals (bitwise)
the same solve run alone through nswe_newton_solve; admission respects the
device budget; a request that can never fit is refused at submission."""
import time

import numpy as np
import pytest

from paper_2505_10857_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KS = [1, 3, 9, 10, 11, 0, 6, 8]  # serving instances of 280..1696 cells


@pytest.fixture(scope="module")
def nswe():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_10857_gb300 import nswe as N
    N.lib()
    return N


def alone(nswe, ctx, inp, prm):
    prob = nswe.Problem1D.from_inputs(ctx, inp)
    U = torch.zeros((2, inp.N), dtype=torch.float64, device="cuda")
    info = nswe.nswe_newton_solve(ctx, prob, torch.from_numpy(inp.U0_start).cuda(), U, prm)
    torch.cuda.synchronize()
    return U.cpu().numpy(), info


def server_ctx(nswe):
    """A context whose 1D launch shapes are the server's (128 x 4 threads x
    blocks in FP64, 256 x 4 in mixed precision), so that a solve alone runs the
    kernel instantiation of the server's launches: the same bits."""
    ctx = nswe.Context(0)
    nswe.nswe_ctx_set_solve_shape(ctx, 0, nswe.solve_shapes().index((128, 4)))
    nswe.nswe_ctx_set_solve_shape(ctx, 1, nswe.solve_shapes().index((256, 4)))
    return ctx


def params(nswe, inp, precision):
    p = nswe.params_from(I.Params1D.for_problem(inp, tol=1e-10, n_max=500))
    p.precision = precision
    return p


def collect(sv, n, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < n:
        assert time.time() - t0 < timeout, "server did not complete"
        sv.wait(1, 1.0)
        for t in sv.poll():
            out[t] = sv.take(t)
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_mix_equals_alone(nswe, precision):
    ctx = server_ctx(nswe)
    inps = [I.serving_instance(k) for k in KS]
    prms = [params(nswe, p, precision) for p in inps]
    ref = [alone(nswe, ctx, p, q) for p, q in zip(inps, prms)]
    sv = nswe.Server(0, device_bytes=256 << 20, host_bytes=64 << 20, streams=3, max_batch=4)
    rng = np.random.default_rng(5)
    tickets = []
    for p, q in zip(inps, prms):
        tickets.append(sv.submit(p, q))
        time.sleep(float(rng.exponential(0.01)))  # Poisson arrivals
    res = collect(sv, len(inps))
    st = sv.stats()
    sv.close()
    levels = dict(zip(tickets, [p.levels for p in inps]))

    def inp_levels(t):
        return levels[t]

    assert st["completed"] == len(inps) and st["launches"] >= 2
    for t, (Uref, iref) in zip(tickets, ref):
        U, info, times = res[t]
        assert info["status"] == 0 and iref["status"] == 0
        assert np.array_equal(U, Uref)
        assert info["iters"][:inp_levels(t)] == iref["iters"][:inp_levels(t)]
        assert times["t_submit_ns"] <= times["t_admit_ns"] <= times["t_launch_ns"] <= times["t_done_ns"]


def test_admission_by_footprint(nswe):
    inps = [I.serving_instance(k) for k in KS]
    prms = [params(nswe, p, 1) for p in inps]
    biggest = max(nswe.Server.footprint(p.N, p.levels, p.start_level) for p in inps)
    budget = int(2.2 * biggest)  # at most two of the largest at a time
    sv = nswe.Server(0, device_bytes=budget, host_bytes=32 << 20, streams=4, max_batch=8)
    tickets = [sv.submit(p, q) for p, q in zip(inps, prms)]
    res = collect(sv, len(inps))
    st = sv.stats()
    sv.close()
    assert st["device_bytes_peak"] <= budget
    assert st["completed"] == len(inps)
    assert all(res[t][1]["status"] == 0 for t in tickets)


def test_oversized_request_refused(nswe):
    inp = I.serving_instance(4)  # 7168 cells, about 6.8 MB resident
    assert nswe.Server.footprint(inp.N, inp.levels, inp.start_level) > 2 << 20
    sv = nswe.Server(0, device_bytes=2 << 20, host_bytes=8 << 20, streams=1, max_batch=4)
    with pytest.raises(nswe.NsweError):
        sv.submit(inp, params(nswe, inp, 1))
    sv.close()


def test_requests_complete_individually(nswe):
    """A small solve launched together with a large one completes (and is
    taken) before the large one ends: completion is per request."""
    small, big = I.serving_instance(11), I.serving_instance(5)  # 280 and 12032 cells
    sv = nswe.Server(0, device_bytes=256 << 20, host_bytes=64 << 20, streams=1, max_batch=8,
                     batch_window_s=0.5)
    tb = sv.submit(big, params(nswe, big, 0))
    ts = sv.submit(small, params(nswe, small, 0))
    res = collect(sv, 2)
    st = sv.stats()
    sv.close()
    assert st["launches"] == 1
    assert res[ts][2]["t_launch_ns"] == res[tb][2]["t_launch_ns"]
    assert res[ts][2]["t_done_ns"] < res[tb][2]["t_done_ns"]
    assert res[ts][1]["status"] == 0 and res[tb][1]["status"] == 0


def alone2d(nswe, ctx, inp, prm):
    prob = nswe.Problem2D.from_inputs(ctx, inp)
    U = torch.zeros((3, inp.Nx * inp.Ny), dtype=torch.float64, device="cuda")
    info = nswe.nswe_newton_solve(ctx, prob, torch.from_numpy(inp.U0_start).cuda(), U, prm)
    torch.cuda.synchronize()
    return U.cpu().numpy(), info


def requests2d(nswe):
    """Seeded wedges (frozen linearisation, omega 0.1, nested from 16 x 8) and
    bump channels (Eq. 12, nested from 8 x 4), two sizes, both precisions."""
    out = []
    for k, (Nx, Ny, lev) in enumerate([(32, 16, 3), (64, 32, 4), (32, 16, 3), (64, 32, 4)]):
        if k % 2 == 0:
            inp = I.wedge_serving_2d(k, Nx, Ny, lev)
            q = I.Params2D(levels=lev, nu1=[20], nu2=[20], tol=1e-10, n_max=400, nest_start=lev - 2, omega=0.1,
                           frozen=True)
        else:
            inp = I.bump_channel_2d(k, Nx, Ny, lev)
            q = I.Params2D(levels=lev, nu1=[20], nu2=[20], tol=1e-10, n_max=400)
        p = nswe.params2d_from(q)
        p.precision = k // 2  # FP64 for the first pair, mixed for the second
        out.append((inp, p))
    return out


def test_2d_requests_equal_alone_beside_1d(nswe):
    """2D requests served by the worker pool, interleaved with 1D requests on
    the same server: every result equals, bit for bit, its solve alone."""
    ctx = server_ctx(nswe)
    reqs = requests2d(nswe)
    ref2 = [alone2d(nswe, ctx, inp, p) for inp, p in reqs]
    one = [I.serving_instance(k) for k in (11, 9)]
    p1 = [params(nswe, p, 0) for p in one]
    ref1 = [alone(nswe, ctx, p, q) for p, q in zip(one, p1)]
    sv = nswe.Server(0, device_bytes=64 << 20, host_bytes=16 << 20, streams=3, max_batch=4, device_bytes_2d=1 << 30)
    t2, t1 = [], []
    for k, (inp, p) in enumerate(reqs):
        t2.append(sv.submit2d(inp, p))
        if k < len(one):
            t1.append(sv.submit(one[k], p1[k]))
    res = collect(sv, len(reqs) + len(one))
    st = sv.stats()
    sv.close()
    assert st["completed"] == len(reqs) + len(one)
    for t, (Uref, iref), (inp, _) in zip(t2, ref2, reqs):
        U, info, times = res[t]
        assert info["status"] == 0 == iref["status"], (info, iref)
        assert np.array_equal(U, Uref)
        assert info["iters"][:inp.levels] == iref["iters"][:inp.levels]
        assert times["t_submit_ns"] <= times["t_admit_ns"] <= times["t_launch_ns"] <= times["t_done_ns"]
    for t, (Uref, iref) in zip(t1, ref1):
        assert res[t][1]["status"] == 0 and np.array_equal(res[t][0], Uref)


def test_2d_admission_by_footprint(nswe):
    """With a 2D budget of the largest footprint, the footprints of the 2D
    solves in flight never add up beyond it; all complete."""
    reqs = requests2d(nswe)
    foot = [nswe.Server.footprint2d(inp.Nx, inp.Ny, inp.levels, p.nest_start) for inp, p in reqs]
    budget = max(foot)
    sv = nswe.Server(0, device_bytes=8 << 20, host_bytes=8 << 20, streams=4, max_batch=4, device_bytes_2d=budget)
    tickets = [sv.submit2d(inp, p) for inp, p in reqs]
    res = collect(sv, len(reqs))
    sv.close()
    assert all(res[t][1]["status"] == 0 for t in tickets)
    spans = [(res[t][2]["t_admit_ns"], res[t][2]["t_done_ns"], f) for t, f in zip(tickets, foot)]
    for a, _, _ in spans:  # footprints in flight at every admission
        assert sum(f for s, e, f in spans if s <= a < e) <= budget


def test_2d_requests_refused(nswe):
    inp, p = requests2d(nswe)[1]
    sv = nswe.Server(0, device_bytes=8 << 20, host_bytes=8 << 20, streams=1, max_batch=4)  # no 2D budget
    with pytest.raises(nswe.NsweError):
        sv.submit2d(inp, p)
    sv.close()
    sv = nswe.Server(0, device_bytes=8 << 20, host_bytes=8 << 20, streams=1, max_batch=4, device_bytes_2d=1 << 20)
    assert nswe.Server.footprint2d(inp.Nx, inp.Ny, inp.levels, p.nest_start) > 1 << 20
    with pytest.raises(nswe.NsweError):  # can never fit
        sv.submit2d(inp, p)
    sv.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_light_load_cluster_form_matches_the_solve_alone(nswe, precision):
    """nswe_server_set_cluster: requests submitted one at a time (one solve
    in flight) run on 8-CTA clusters, the same requests submitted together
    (the form then depends on how many are in flight); every result agrees with
    the block-form solve alone: FP64 to a few ulps with the same Newton
    counts (or within the Newton step that res crossing tol may move),
    mixed within its bound."""
    ctx = server_ctx(nswe)
    inps = [I.serving_instance(k) for k in KS[:5]]
    prms = [params(nswe, p, precision) for p in inps]
    ref = [alone(nswe, ctx, p, q) for p, q in zip(inps, prms)]
    sv = nswe.Server(0, device_bytes=256 << 20, host_bytes=64 << 20, streams=2, max_batch=8)
    try:
        sv.set_cluster(8, 2)
        got = []
        for p, q in zip(inps, prms):  # light load: one in flight
            t = sv.submit(p, q)
            got.append(collect(sv, 1)[t])
        tickets = [sv.submit(p, q) for p, q in zip(inps, prms)]  # five at once: the block form
        together = collect(sv, len(tickets))
        got += [together[t] for t in tickets]
        with pytest.raises(nswe.NsweError):
            sv.set_cluster(17, 2)
        sv.set_cluster(1, 0)
    finally:
        sv.close()
    bound = 1e-13 if precision == 0 else 1e-8
    for k, (U, info, _) in enumerate(got):
        Ur, infr = ref[k % len(inps)]
        assert info["status"] == 0, (k, info["status"])
        same = list(info["iters"]) == list(infr["iters"])
        err = np.abs(U - Ur).max() / np.abs(Ur).max()
        assert err <= (bound if same else 1e-9), (k, err, info["iters"], infr["iters"])
