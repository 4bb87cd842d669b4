"""The binning kernel makes a particle a tile's candidate only if the distance from its
centre to the tile's box of cell centres (minimum image on periodic axes) is at most
r + h + 0.01 in FP32 (tile_in_reach, with the centre first wrapped into the box: the
kernel's own code compiled for the host). Checked by brute force over the cells: the test
never drops a tile holding a cell centre within r + h of the particle (where Table 1 can
give a non-zero solid fraction), in 2D and 3D, across periodic faces, for centres several
periods outside the box, and at walls."""
import numpy as np

from host_entries import H, doubles, ints  # noqa: F401  (fixture)


def _needed(X, r, h, org, tshape, n, periodic, dim):
    axes = []
    for ax in range(dim):
        c = np.arange(org[ax], min(org[ax] + tshape[ax], n[ax]), dtype=float)
        dc = c - X[ax]
        if periodic[ax]:
            dc -= n[ax] * np.rint(dc / n[ax])
        axes.append(dc)
    grids = np.meshgrid(*axes, indexing="ij")
    d2 = sum(g * g for g in grids)
    return bool(np.any(d2 < (r + h) ** 2))


def test_tile_culling_keeps_every_tile_a_shell_reaches(H):
    rng = np.random.default_rng(77)
    h = 1.0
    checked = 0
    for dim, tshape in ((2, (32, 8, 1)), (3, (32, 4, 2))):
        for _ in range(60):
            n = [int(v) for v in rng.integers(40, 90, 3)]
            if dim == 2:
                n[2] = 1
            periodic = [int(v) for v in rng.integers(0, 2, 3)]
            r = rng.uniform(3.0, 9.0)
            # centres up to three periods out on periodic axes (the C ABI accepts any
            # position there), inside the box on wall axes
            X = rng.uniform(0, 1, 3) * np.array(n, dtype=float)
            for a in range(3):
                if periodic[a]:
                    X[a] += n[a] * int(rng.integers(-3, 3))
            nt = [(n[a] + tshape[a] - 1) // tshape[a] for a in range(3)]
            cX, cn, cp, ce = doubles(*X), ints(*n), ints(*periodic), ints(*tshape)
            for tz in range(nt[2] if dim == 3 else 1):
                for ty in range(nt[1]):
                    for tx in range(nt[0]):
                        org = (tx * tshape[0], ty * tshape[1], tz * tshape[2])
                        if _needed(X, r, h, org, tshape, n, periodic, dim):
                            kept = H.psc_test_tile_in_reach(cX, r + h, ints(*org), ce, cn, cp, dim)
                            assert kept == 1, (dim, n, periodic, r, X, org)
                            checked += 1
    assert checked > 500
