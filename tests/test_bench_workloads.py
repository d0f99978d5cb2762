"""The seeded workloads bench.py measures (host side, no GPU): the batched 2D
serving sizes, the two 1D configurations and the equal-accuracy settings."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2505_10857_gb300 import inputs as I  # noqa: E402


def test_config5_instances_cover_the_stated_sizes_in_equal_numbers():
    inps, prms = bench.config5_instances(16)
    sizes = [(p.Nx, p.Ny) for p in inps]
    for nx, ny, lev in bench.CONFIG5_SIZES:
        assert sizes.count((nx, ny)) == 4
    for k, (p, q) in enumerate(zip(inps, prms)):
        assert q.levels == p.levels and (p.Nx >> (p.levels - 1), p.Ny >> (p.levels - 1)) == (8, 4)
        if k % 2 == 0:  # wedges: nested from 16 x 8 under the frozen linearisation
            assert "froude" in p.meta and 2.0 <= p.meta["froude"] <= 4.0 and q.frozen
            assert 5.0 <= p.meta["theta_deg"] <= 15.0
            assert q.nest_start == p.levels - 2
        else:  # Gaussian-bump channels: Eq. 12 from the coarsest grid
            assert p.meta["case"] == "gauss-bump-channel" and not q.frozen and q.nest_start == -1
            A, xc, yc, w = p.meta["bump"]
            assert 0.1 <= A <= 0.3 and 0.5 <= w <= 1.0
    # seeded: the same draw twice
    again, _ = bench.config5_instances(16)
    assert all(np.array_equal(a.gq_all(), b.gq_all()) for a, b in zip(inps, again))


def test_gauss_bump_channel_bottom_slopes_match_its_bottom():
    p = I.gauss_bump_channel_2d(3, 32, 16, 3)
    b, bx, by = p.b_fns
    x, y, h = 0.37, 2.11, 1e-6
    assert abs(bx(x, y) - (b(x + h, y) - b(x - h, y)) / (2 * h)) < 1e-8
    assert abs(by(x, y) - (b(x, y + h) - b(x, y - h)) / (2 * h)) < 1e-8


def test_1d_configurations():
    small, _ = bench.make_instances(0, 3, 3, kind="small")
    irr, prm = bench.make_instances(0, 2, 3, kind="irregular")
    assert [p.N for p in small] == [200] * 3 and [p.N for p in irr] == [4096] * 2
    assert bench.CONFIG1D["small"][:3] == (200, 4, 25) and bench.CONFIG1D["irregular"][:3] == (4096, 8, 256)
    assert small[0].N_level(small[0].start_level) == 25 and irr[0].N_level(irr[0].start_level) == 256
    cfg = bench.workload_config(256, 3, kind="small")
    assert cfg["N"] == 200 and "fit in L2" in cfg["l2"]
    assert "exceed" in bench.workload_config(608, 3)["l2"]
    assert prm[0].tol == bench.TOL


def test_equal_accuracy_settings():
    # the equal-accuracy lines stop well below the metric's threshold, and the parity reference is
    # converged further still
    assert bench.TOL_CONVERGED < bench.TOL_SOLUTION < bench.TOL
    assert bench.MIXED_BOUND == 1e-10
