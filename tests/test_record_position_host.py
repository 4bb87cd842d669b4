"""Packed records hold each candidate's position relative to its tile's origin (minimum
image on periodic axes) in FP32. The packing kernel forms it as x - (origin + image shift)
with the image decided in FP32 (record_rel, the kernel's own code compiled for the host);
this checks that the result is bit-identical to the plain FP64 minimum-image form
rel = (x - o - c) - n rint((x - o - c)/n) + c (c the tile centre offset) for every tile a
particle can be a candidate of, and equals x - o on a wall axis."""
import numpy as np

from host_entries import H  # noqa: F401  (fixture)


def _reference(x, o, ext, n):
    d = x - o
    cen = 0.5 * (ext - 1)
    e = d - cen
    e -= n * np.rint(e * (1.0 / n))
    return np.float32(e + cen)


def test_record_positions_bit_identical_to_the_fp64_minimum_image(H):
    rng = np.random.default_rng(4242)
    checked = 0
    for n, ext in ((2048, 32), (2048, 8), (512, 32), (512, 4), (256, 2), (96, 32)):
        for _ in range(3000):
            x = rng.uniform(0, n)
            reach = rng.uniform(3, 9) + 1.0
            # every tile whose cell range comes within reach of x (either image)
            t0 = int(np.floor((x - reach) / ext)) - 1
            t1 = int(np.floor((x + reach) / ext)) + 1
            for t in range(t0, t1 + 1):
                o = (t % (n // ext)) * ext
                got = np.float32(H.psc_test_record_rel(x, o, ext, n, 1))
                assert got == _reference(x, o, ext, n), (n, ext, x, o)
                checked += 1
            o = int(x // ext) * ext
            assert np.float32(H.psc_test_record_rel(x, o, ext, n, 0)) == np.float32(x - o)
    assert checked > 40000
