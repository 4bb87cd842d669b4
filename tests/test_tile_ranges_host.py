"""The binning kernel turns a particle's cell interval [lo, hi] along one axis (cell centres
within r + h, unwrapped) into at most two ranges of tile indices (axis_tile_ranges in
psc_bin.cu): wrapped on a periodic axis, merged when the pieces meet, clipped at walls.
This checks on the host, by brute force over the cells, that the ranges cover exactly the
tiles holding a cell of the interval, each once."""
import numpy as np


def _ranges(lo, hi, n, t, nt, periodic):
    if periodic:
        if hi - lo + 1 >= n:
            return [(0, nt - 1)]
        A, B = ((lo % n) + n) % n, ((hi % n) + n) % n
        if A <= B:
            return [(A // t, B // t)]
        thi, tlo = A // t, B // t
        if tlo >= thi:
            return [(0, nt - 1)]
        return [(0, tlo), (thi, nt - 1)]
    A, B = max(lo, 0), min(hi, n - 1)
    if A > B:
        return []
    return [(A // t, B // t)]


def test_tile_ranges_cover_exactly_the_tiles_of_the_cell_interval():
    rng = np.random.default_rng(9)
    for _ in range(20000):
        t = int(rng.choice([2, 4, 8, 32]))
        n = int(rng.integers(1, 200))
        nt = (n + t - 1) // t
        periodic = int(rng.integers(0, 2))
        lo = int(rng.integers(-3 * n - 5, 2 * n + 5))
        hi = lo + int(rng.integers(0, 2 * n + 5))
        got = []
        for a, b in _ranges(lo, hi, n, t, nt, periodic):
            got.extend(range(a, b + 1))
        cells = range(lo, hi + 1)
        if periodic:
            want = {(c % n) // t for c in cells}
        else:
            want = {c // t for c in cells if 0 <= c < n}
        assert len(got) == len(set(got)), (lo, hi, n, t, periodic)
        assert set(got) == want, (lo, hi, n, t, periodic, got, sorted(want))
