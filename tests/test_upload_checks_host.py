"""Host-side pieces of a particle upload and of the DEM's neighbour-list validity, compiled
for the host from the library's own source (include/psc_testing.h):

- the finiteness check (vectorised, with a scalar tail) finds one infinity or NaN at any
  position of arrays of every length modulo its eight-value blocks, and passes finite
  extremes (largest, subnormal, negative zero);
- the radii range gives numpy's smallest r^2 and largest r (NaN ignored, as the finiteness
  check reports it), at every tail length;
- the displacement test equals the minimum-image displacement up to FP32 rounding (1e-4
  at these box sizes, far below a quarter of any skin) wherever one image shift suffices,
  so a kept neighbour list is never one whose skin a particle has left."""
import ctypes as C

import numpy as np

from host_entries import H, ints  # noqa: F401  (fixture)


def _finite(H, a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return H.psc_test_all_finite(a.ctypes.data_as(C.c_void_p), a.size)


def test_finiteness_check_finds_every_nonfinite_value(H):
    rng = np.random.default_rng(5)
    extremes = [np.finfo(np.float64).max, -np.finfo(np.float64).max, 5e-324, -0.0, 0.0,
                np.finfo(np.float64).tiny]
    for m in list(range(0, 40)) + [1001, 4099]:
        a = rng.normal(0, 1e3, m)
        if m:
            a[rng.integers(0, m, min(m, 3))] = rng.choice(extremes, min(m, 3))
        assert _finite(H, a) == 1, m
        for pos in sorted({0, m // 2, m - 1} if m else set()):
            for bad in (np.inf, -np.inf, np.nan, -np.nan):
                b = a.copy()
                b[pos] = bad
                assert _finite(H, b) == 0, (m, pos, bad)


def test_finiteness_check_reads_arrays_at_any_8_byte_offset(H):
    """Caller arrays need only the alignment of a double: starts at every offset of 8 bytes
    modulo 64 give the same answers."""
    base = np.random.default_rng(8).normal(0, 1.0, 200)
    for off in range(8):
        for m in (0, 1, 7, 8, 9, 31, 64, 100):
            a = base[off:off + m]
            assert _finite(H, a) == 1
            if m:
                b = a.copy()
                view = base.copy()[off:off + m]
                view[m - 1] = np.inf
                assert H.psc_test_all_finite(view.ctypes.data_as(C.c_void_p), view.size) == 0
                assert _finite(H, b) == 1


def test_radii_range_matches_numpy(H):
    rng = np.random.default_rng(6)
    lo, hi = C.c_double(), C.c_double()
    for n in list(range(1, 20)) + [5000, 5003]:
        r = rng.uniform(0.3, 9.0, n)
        if n > 3:
            r[rng.integers(0, n)] = -rng.uniform(0.1, 2.0)   # r^2 counts, the sign does not
        H.psc_test_radii_range(r.ctypes.data_as(C.c_void_p), n, C.byref(lo), C.byref(hi))
        assert lo.value == np.min(r * r) and hi.value == max(0.0, np.max(r)), n
        if n > 2:
            q = r.copy()
            q[n // 2] = np.nan
            H.psc_test_radii_range(q.ctypes.data_as(C.c_void_p), n, C.byref(lo), C.byref(hi))
            keep = np.delete(q, n // 2)
            assert lo.value == np.min(keep * keep) and hi.value == max(0.0, np.max(keep)), n


def test_displacement_test_bounds_the_minimum_image_displacement(H):
    rng = np.random.default_rng(7)
    n = (64, 48, 40)
    for _ in range(4000):
        dim = int(rng.integers(2, 4))
        per = [int(v) for v in rng.integers(0, 2, 3)]
        xr = rng.uniform(0, 1, 3) * np.array(n)
        x = xr + rng.normal(0, 3, 3)
        # and positions up to one period away on periodic axes (one image shift suffices)
        for a in range(3):
            if per[a] and rng.random() < 0.3:
                x[a] += n[a] * rng.choice([-1, 1])
        got = H.psc_test_moved2((C.c_double * 3)(*x), (C.c_double * 3)(*xr), ints(*n), ints(*per), dim)
        d = (x - xr)[:dim].copy()
        for a in range(dim):
            if per[a]:
                d[a] -= n[a] * np.rint(d[a] / n[a])
        want = float(np.sum(d * d))
        # FP32 rounding: each component is rounded at the scale of the raw difference (up
        # to about 1.5 n here, ulp < 1.6e-5), far below the skin's quarter the test decides on
        assert np.sqrt(got) >= np.sqrt(want) - 1e-4, (x, xr, per, dim)
        assert abs(np.sqrt(got) - np.sqrt(want)) <= 1e-4, (x, xr, per, dim)
