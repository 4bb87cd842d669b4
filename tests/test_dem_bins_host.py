"""The DEM neighbour-list kernel walks the bins around a particle's bin b along each axis
as n bins from a start (axis_span / axis_at, the kernel's own code compiled for the host):
b - 1, b, b + 1 wrapped on a periodic axis (fewer when the axis has fewer than three bins)
or clipped at walls. Checked: the walk visits exactly the distinct neighbouring bins, each
once."""
import ctypes as C

from host_entries import H  # noqa: F401  (fixture)


def _distinct_neighbours(b, nb, periodic):
    out = []
    for o in (-1, 0, 1):
        c = b + o
        if periodic:
            c %= nb
        elif not 0 <= c < nb:
            continue
        if c not in out:
            out.append(c)
    return out


def test_bin_walk_visits_each_neighbouring_bin_once(H):
    start, count = C.c_int(), C.c_int()
    for nb in range(1, 12):
        for b in range(nb):
            for periodic in (0, 1):
                H.psc_test_axis_span(b, nb, periodic, C.byref(start), C.byref(count))
                walk = [H.psc_test_axis_at(k, start.value, nb, periodic) for k in range(count.value)]
                assert len(walk) == len(set(walk))
                assert sorted(walk) == sorted(_distinct_neighbours(b, nb, periodic))
