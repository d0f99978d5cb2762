"""Host logic of the serving layer, without a GPU: the arena allocator that
admits solves by footprint, and the footprint function."""
import random

import pytest

from paper_2505_10857_gb300 import nswe


class FirstFit:
    """Reference model: first fit over [0, size) in units of `align`."""

    def __init__(self, size, align):
        self.align = align
        self.free = [(0, size // align * align)]
        self.live = {}

    def alloc(self, n):
        need = max(1, -(-n // self.align)) * self.align
        for i, (o, l) in enumerate(self.free):
            if l >= need:
                self.free[i:i + 1] = [(o + need, l - need)] if l > need else []
                self.live[o] = need
                return o
        return None

    def release(self, o):
        l = self.live.pop(o)
        self.free.append((o, l))
        self.free.sort()
        merged = []
        for fo, fl in self.free:
            if merged and merged[-1][0] + merged[-1][1] == fo:
                merged[-1] = (merged[-1][0], merged[-1][1] + fl)
            else:
                merged.append((fo, fl))
        self.free = merged


def test_arena_basic():
    a = nswe.Arena(4096, 256)
    x = a.alloc(1)
    y = a.alloc(300)
    assert (x, y) == (0, 256)
    assert a.query()[0] == 256 + 512
    assert a.alloc(4096) is None
    assert a.free(x)
    assert not a.free(x)          # double free is rejected
    assert not a.free(12345)      # unknown offset is rejected
    z = a.alloc(200)              # first fit reuses the freed head
    assert z == 0
    a.free(y)
    a.free(z)
    used, peak, largest = a.query()
    assert used == 0 and largest == 4096 and peak == 768
    a.close()


def test_arena_rejects_bad_config():
    with pytest.raises(nswe.NsweError):
        nswe.Arena(4096, 100)  # alignment not a power of two


def test_arena_matches_first_fit_model():
    rng = random.Random(7)
    a, m = nswe.Arena(1 << 20, 256), FirstFit(1 << 20, 256)
    live = []
    for step in range(3000):
        if live and rng.random() < 0.45:
            o = live.pop(rng.randrange(len(live)))
            assert a.free(o)
            m.release(o)
        else:
            n = rng.choice([1, 255, 256, 257, 1000, 5000, 40000, 150000])
            got, exp = a.alloc(n), m.alloc(n)
            assert got == exp, (step, n, got, exp)
            if got is not None:
                live.append(got)
        used, _, largest = a.query()
        assert used == sum(m.live.values())
        assert largest == max((l for _, l in m.free), default=0)
    a.close()


def test_footprint():
    f = nswe.Server.footprint
    assert f(4096, 8, 4) > f(2048, 7, 3) > f(256, 4, 0) > 0
    assert f(4096, 8, 4) >= f(4096, 8, -1)  # a finer start level holds a larger U0
    assert f(2, 1, -1) == 0 and f(4096, 0, -1) == 0
    # about 0.95 KB per finest cell: 34 doubles per cell and level of FP64
    # workspace (x2 over the levels), the Jacobian workspace (34 doubles),
    # geometry and the result
    assert 800 * 4096 < f(4096, 8, 4) < 1100 * 4096


def test_footprint_2d():
    f = nswe.Server.footprint2d
    assert f(512, 256, 7, -1) > f(256, 128, 6, -1) > f(64, 32, 4, -1) > 0
    assert f(512, 256, 7, 5) > f(512, 256, 7, -1)  # a finer start level holds a larger guess
    # invalid: too small, not divisible, coarsest grid below 4 x 4 or above 512 cells
    assert f(2, 2, 1, -1) == 0 and f(100, 64, 4, -1) == 0 and f(64, 32, 5, -1) == 0 and f(512, 256, 2, -1) == 0
    # about 2.3 KB per finest cell: 215 doubles per cell and level (state, residual, update, Gauss-point
    # geometry, 21 Jacobian blocks and the diagonal inverses), x 4/3 over the levels, and the result
    n = 512 * 256
    assert 2200 * n < f(512, 256, 7, -1) < 2400 * n
