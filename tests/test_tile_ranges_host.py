"""The binning kernel turns a particle's cell interval [lo, hi] along one axis (cell centres
within r + h, unwrapped) into at most two ranges of tile indices (axis_tile_ranges, the
kernel's own code compiled for the host): wrapped on a periodic axis, merged when the
pieces meet, clipped at walls. Checked by brute force over the cells: the ranges cover
exactly the tiles holding a cell of the interval, each once, and axis_tile enumerates them."""
import ctypes as C

import numpy as np

from host_entries import H, ints  # noqa: F401  (fixture)


def test_tile_ranges_cover_exactly_the_tiles_of_the_cell_interval(H):
    rng = np.random.default_rng(9)
    a, b = (C.c_int * 2)(), (C.c_int * 2)()
    for _ in range(20000):
        t = int(rng.choice([2, 4, 8, 32]))
        n = int(rng.integers(1, 200))
        nt = (n + t - 1) // t
        periodic = int(rng.integers(0, 2))
        lo = int(rng.integers(-3 * n - 5, 2 * n + 5))
        hi = lo + int(rng.integers(0, 2 * n + 5))
        nr = H.psc_test_axis_tile_ranges(lo, hi, n, t, nt, periodic, a, b)
        got = []
        for k in range(nr):
            got.extend(range(a[k], b[k] + 1))
        # the kernel's enumeration of the same tiles
        assert [H.psc_test_axis_tile(k, nr, a, b) for k in range(len(got))] == got
        cells = range(lo, hi + 1)
        if periodic:
            want = {(c % n) // t for c in cells}
        else:
            want = {c // t for c in cells if 0 <= c < n}
        assert len(got) == len(set(got)), (lo, hi, n, t, periodic)
        assert set(got) == want, (lo, hi, n, t, periodic, got, sorted(want))
