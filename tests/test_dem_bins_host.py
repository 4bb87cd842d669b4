"""The DEM neighbour-list kernel walks the bins around a particle's bin b along each axis
as n bins from a start (axis_span / axis_at in dem.cu): b - 1, b, b + 1 wrapped on a
periodic axis (fewer when the axis has fewer than three bins) or clipped at walls. This
checks on the host that the walk visits exactly the distinct neighbouring bins, each once."""


def _span(b, nb, periodic):
    if periodic:
        start, n = b - 1 + nb, min(nb, 3)
        return [(start + k) % nb for k in range(n)]
    start = max(b - 1, 0)
    n = min(b + 1, nb - 1) - start + 1
    return [start + k for k in range(n)]


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


def test_bin_walk_visits_each_neighbouring_bin_once():
    for nb in range(1, 12):
        for b in range(nb):
            for periodic in (0, 1):
                walk = _span(b, nb, periodic)
                assert len(walk) == len(set(walk))
                assert sorted(walk) == sorted(_distinct_neighbours(b, nb, periodic))
