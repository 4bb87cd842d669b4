"""Slab decomposition, host side (no GPU): the layout the library computes, and the two
things slabs exchange -- the populations crossing a face and the per-particle force sums --
carried out by two gloo ranks on the CPU, each holding one slab, with the library's own
layout (lbm_decomp_layout) and particle assignment (lbm_decomp_assign)."""
import os
import socket

import numpy as np
import pytest


@pytest.fixture(scope="module")
def P():
    from paper_1901_09745_gb300 import build
    build.build()
    import paper_1901_09745_gb300 as P
    P.lib()
    return P


@pytest.mark.parametrize("lattice,tile", [(9, 8), (19, 2)])
@pytest.mark.parametrize("periodic", [0, 1])
def test_layout_cuts_on_tile_rows_and_places_ghosts(P, lattice, tile, periodic):
    for n_s in (16, 48, 77, 256):
        for nslab in (1, 2, 3, 5):
            try:
                own, glo, ghi = P.lbm_decomp_layout(lattice, n_s, periodic, nslab)
            except ValueError:
                assert n_s // nslab < 2 * tile      # only refused when slabs would be too thin
                continue
            assert own[0] == 0 and own[-1] == n_s and len(own) == nslab + 1
            for k in range(nslab):
                assert own[k + 1] - own[k] >= tile
                if 0 < k:
                    assert own[k] % tile == 0
                assert glo[k] == (tile if nslab > 1 and (k > 0 or periodic) else 0)
                assert ghi[k] == (tile if nslab > 1 and (k < nslab - 1 or periodic) else 0)


def test_assignment_holds_every_particle_near_every_slab_it_reaches(P):
    """Brute force over rows: a slab holds a particle exactly when some owned row lies within
    r + h + 1 of one image of its centre, and then as that image."""
    rng = np.random.default_rng(5)
    for periodic in (0, 1):
        n_s, nslab = 96, 3
        c = rng.uniform(0, n_s, 200)
        r = rng.uniform(3, 8, 200)
        own, _, _ = P.lbm_decomp_layout(19, n_s, periodic, nslab)
        img = P.lbm_decomp_assign(19, n_s, periodic, nslab, c, r)
        for k in range(nslab):
            rows = np.arange(own[k], own[k + 1])
            for i in range(c.size):
                hits = [m for m in ((0, -1, 1) if periodic else (0,))
                        if np.any(np.abs(rows - (c[i] + m * n_s)) <= r[i] + 2.0)]
                if hits:
                    assert img[k, i] in hits
                else:
                    assert img[k, i] == P.NOT_HELD


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


E_S = np.array([0, 0, 0, 1, -1, 1, -1, -1, 1])      # D2Q9 e_y: the slab axis of 2D lattices


def _val(q, g, x):
    return q * 1e4 + g * 100.0 + x


def _rank_main(rank, world, port, periodic, out):
    import torch
    import torch.distributed as dist
    import paper_1901_09745_gb300 as P
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nx, n_s, h = 16, 48, 1.0
    own, glo, ghi = P.lbm_decomp_layout(9, n_s, periodic, world)
    k = rank
    nown = own[k + 1] - own[k]
    rows = glo[k] + nown + ghi[k]
    A = np.full((9, rows, nx), np.nan)
    for q in range(9):
        for g in range(own[k], own[k + 1]):
            A[q, glo[k] + g - own[k]] = _val(q, g, np.arange(nx))
    up, down = np.nonzero(E_S == 1)[0], np.nonzero(E_S == -1)[0]
    reqs, bufs = [], []
    # upper face: my last owned row (e_s = +1) goes up, the neighbour's first (e_s = -1) comes down
    if ghi[k]:
        nb = (k + 1) % world
        reqs.append(dist.isend(torch.from_numpy(A[up, glo[k] + nown - 1].copy()), nb, tag=1))
        b = torch.zeros((len(down), nx), dtype=torch.float64)
        reqs.append(dist.irecv(b, nb, tag=2))
        bufs.append(("top", b))
    if glo[k]:
        nb = (k - 1) % world
        reqs.append(dist.isend(torch.from_numpy(A[down, glo[k]].copy()), nb, tag=2))
        b = torch.zeros((len(up), nx), dtype=torch.float64)
        reqs.append(dist.irecv(b, nb, tag=1))
        bufs.append(("bottom", b))
    for r in reqs:
        r.wait()
    ok_ghost = True
    for where, b in bufs:
        if where == "top":
            A[down, glo[k] + nown] = b.numpy()
            g = own[k + 1] % n_s
            ok_ghost &= np.array_equal(A[down, glo[k] + nown], np.array([_val(q, g, np.arange(nx)) for q in down]))
        else:
            A[up, glo[k] - 1] = b.numpy()
            g = (own[k] - 1) % n_s
            ok_ghost &= np.array_equal(A[up, glo[k] - 1], np.array([_val(q, g, np.arange(nx)) for q in up]))
    # per-particle sums: each slab adds a weight over its owned cells inside the particle's
    # shell (the particle as the image the library assigns), the sums meet in one reduction
    rng = np.random.default_rng(7)
    npart = 40
    cx, cy, r = rng.uniform(0, nx, npart), rng.uniform(0, n_s, npart), rng.uniform(3.0, 6.0, npart)
    img = P.lbm_decomp_assign(9, n_s, periodic, world, cy, r, h)
    part = np.zeros(npart)
    xs = np.arange(nx)
    for i in range(npart):
        if img[k, i] == P.NOT_HELD:
            continue
        yc = cy[i] + img[k, i] * n_s
        for g in range(own[k], own[k + 1]):
            dx = xs - cx[i]
            dx -= nx * np.rint(dx / nx)
            inside = dx * dx + (g - yc) ** 2 < (r[i] + h) ** 2
            part[i] += np.sum((1.0 + 1e-3 * g + 1e-5 * xs)[inside])
    t = torch.from_numpy(part)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    ref = np.zeros(npart)
    for i in range(npart):
        for g in range(n_s):
            dx = xs - cx[i]
            dx -= nx * np.rint(dx / nx)
            dy = g - cy[i]
            if periodic:
                dy -= n_s * np.rint(dy / n_s)
            inside = dx * dx + dy * dy < (r[i] + h) ** 2
            ref[i] += np.sum((1.0 + 1e-3 * g + 1e-5 * xs)[inside])
    out.put((rank, bool(ok_ghost), bool(np.allclose(t.numpy(), ref, rtol=1e-13, atol=0))))
    dist.destroy_process_group()


@pytest.mark.parametrize("periodic", [0, 1])
def test_face_exchange_and_force_sums_over_two_gloo_ranks(P, periodic):
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, periodic, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, True, True), (1, True, True)]
