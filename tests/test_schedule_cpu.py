"""The work schedule of the row-tiled kernels, on the host (no GPU): every plane of
every column is taken by exactly one CTA, runs are contiguous in the run order,
chunks are zc planes long, and with equal runs the CTAs on y-neighbouring columns
pass each plane at the same point of their sequence (so they share halo rows in L2).
The schedule is what lwacm_selftest_schedule enumerates with the kernels' own
iterator and planner."""
import ctypes
import math
import random

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_2142_gb300 import lwacm as lw
    return lw.load()


def schedule(lib, cols, nz, ctas):
    grid, zc, kcls, count = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    assert lib.lwacm_selftest_schedule(cols, nz, ctas, ctypes.byref(grid), ctypes.byref(zc), ctypes.byref(kcls),
                                       None, 0, ctypes.byref(count)) == 0
    n = count.value
    items = (ctypes.c_int * (4 * n))()
    assert lib.lwacm_selftest_schedule(cols, nz, ctas, ctypes.byref(grid), ctypes.byref(zc), ctypes.byref(kcls),
                                       items, n, ctypes.byref(count)) == 0
    assert count.value == n
    return grid.value, zc.value, kcls.value, np.array(items, dtype=np.int64).reshape(n, 4)


def check(lib, cols, nz, ctas):
    grid, zc, kcls, it = schedule(lib, cols, nz, ctas)
    assert 1 <= grid <= ctas
    b, col, za, zb = it.T
    assert np.all((0 <= b) & (b < grid)) and np.all((0 <= col) & (col < cols))
    assert np.all((0 <= za) & (za < zb) & (zb <= nz))
    # every plane of every column exactly once
    seen = np.zeros((cols, nz), dtype=np.int64)
    for c, a, e in zip(col, za, zb):
        seen[c, a:e] += 1
    assert np.all(seen == 1)
    # the items of a CTA come in launch order, CTA by CTA
    assert np.all(np.diff(b) >= 0)
    if zc > 0:  # chunks of zc planes starting at multiples of zc (the last may be short)
        assert kcls == 1
        assert np.all(za % zc == 0) and np.all((zb - za == zc) | (zb == nz))
    else:  # equal runs: CTA b's planes are [b W / G, (b+1) W / G) of the run order
        assert cols % kcls == 0 and kcls == cols // math.gcd(cols, grid)
        per = cols // kcls
        seq = (col % per) * kcls + col // per  # the column's place in the run order
        lin0 = seq * nz + za
        w = cols * nz
        for cta in range(grid):
            m = b == cta
            starts, ends = lin0[m], lin0[m] + (zb - za)[m]
            assert starts[0] == w * cta // grid and ends[-1] == w * (cta + 1) // grid
            assert np.all(starts[1:] == ends[:-1])  # contiguous
        # y-neighbours in a class pass each plane at the same point of their sequence
        tau = np.full((cols, nz), -1, dtype=np.int64)
        for cta in range(grid):
            t = 0
            for c, a, e in zip(col[b == cta], za[b == cta], zb[b == cta]):
                tau[c, a:e] = t + 1 + np.arange(e - a)  # source plane za-1 first
                t += e - a + 2
        for c in range(cols):
            if c % per != per - 1:
                assert np.array_equal(tau[c], tau[c + 1]), (c, tau[c][:8], tau[c + 1][:8])
    return grid, zc, kcls


@pytest.mark.parametrize("cols,nz,ctas,want", [
    (32, 256, 152, "runs"),    # 256^3 on the 256-node-row form: runs of 53-54 planes, kcls 4
    (96, 256, 304, "runs"),    # 384 x 256 x 256 on 128-node segments
    (16, 128, 304, "chunks"),  # 128^3: chunks of 7 (a tie, kept on chunks)
    (1000, 1, 304, "chunks"),  # one plane, several chunks per CTA
    (305, 3, 304, "runs"),     # runs longer than a column
    (3, 100, 152, "runs"),
    (1, 1, 152, None),
])
def test_schedule_cases(lib, cols, nz, ctas, want):
    grid, zc, kcls = check(lib, cols, nz, ctas)
    if want == "runs":
        assert zc == 0
    elif want == "chunks":
        assert zc > 0
    if (cols, nz, ctas) == (32, 256, 152):
        assert grid == 152 and kcls == 4


def test_schedule_random_shapes(lib):
    rng = random.Random(7)
    for _ in range(300):
        cols, nz = rng.randint(1, 300), rng.randint(1, 300)
        check(lib, cols, nz, rng.choice([1, 7, 152, 300, 304]))


def test_schedule_validation(lib):
    g, z, k, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    ok = (ctypes.byref(g), ctypes.byref(z), ctypes.byref(k))
    assert lib.lwacm_selftest_schedule(0, 4, 4, *ok, None, 0, ctypes.byref(n)) == 1
    assert lib.lwacm_selftest_schedule(4, 0, 4, *ok, None, 0, ctypes.byref(n)) == 1
    assert lib.lwacm_selftest_schedule(4, 4, 0, *ok, None, 0, ctypes.byref(n)) == 1
    assert lib.lwacm_selftest_schedule(4, 4, 4, None, ok[1], ok[2], None, 0, ctypes.byref(n)) == 1
    assert lib.lwacm_selftest_schedule(4, 4, 4, *ok, None, 3, ctypes.byref(n)) == 1
    assert lib.lwacm_selftest_schedule(4, 4, 4, *ok, None, 0, None) == 1
    assert lib.lwacm_selftest_schedule(1 << 16, 1 << 15, 4, *ok, None, 0, ctypes.byref(n)) == 1
