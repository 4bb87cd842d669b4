"""Seeded synthetic inputs for the PSC lattice-Boltzmann / DEM workloads.

This module serves both the CUDA library's tests and benchmark and the CPU oracle's
tests. It holds no arithmetic of the method itself: only lattice geometry, seeds, particle
packings (random sequential addition, optional soft overlap removal) and initial
velocities. Seeds are ``numpy.random.default_rng(1000 * k + 1)`` for workload k.

Workloads (sizes and distributions of the paper's set-ups, all in lattice units with cell
centres at integer coordinates):

  c1  D2Q9 64x64 periodic, tau 0.8, body force (1e-6, 0), 4 static discs r = 6.5:
      pair A with a 1.0 lu surface gap, pair B with a 0.25 lu gap (cells shared by two
      discs under the linear approximation), 1000 steps.
  c2  D2Q9 2048x2048 channel (walls at y = -1/2 and y = 2047.5, periodic x), tau 0.7,
      5000 discs r ~ U(4, 8) packed by random sequential addition into a central band of
      local solid fraction 0.40, velocities ~ N(0, 1e-3), spins ~ N(0, 1e-3)/r, JKR DEM
      with 10 sub-steps per LBM step.
  c3  D3Q19 256^3 periodic, tau 0.6, body force (1e-6, 0, 0), static spheres r = 6
      (2000 as stated, or 5563 for solid fraction 0.3).
  c4  D3Q19 128^3 periodic, tau 0.7, 200 static spheres r = 5, 500 steps.
  c5  D3Q19 512^3 channel (walls in z), tau 0.55, 50000 spheres r ~ U(3, 8) by random
      sequential addition (solid fraction 0.31); c5dense the same channel at solid
      fraction 0.45 (71,830 spheres) by growth and relaxation, with many near-contacts.

``scale`` shrinks a workload's box (same solid fraction and radius distribution) for
sub-box parity runs.
"""
import math

import numpy as np


# surface energy of the 512^3 channel workloads: the pull-off force 3 pi gamma R of the
# smallest pair (r = 3, R = 1.5) is 0.28, several times the largest mean hydrodynamic force
# the spheres see in the first steps (about 0.06, from their random initial velocities)
C5_GAMMA = 2e-2


def rng_for(k):
    return np.random.default_rng(1000 * k + 1)


def _min_image(d, box, periodic):
    d = d.copy()
    for a in range(d.shape[-1]):
        if periodic[a]:
            L = box[a]
            d[..., a] -= L * np.round(d[..., a] / L)
    return d


class _Grid:
    """Uniform hash grid for overlap queries during packing."""

    def __init__(self, box, cell, dim):
        self.dim = dim
        self.cell = cell
        self.n = [max(1, int(box[a] // cell)) for a in range(dim)]
        self.box = box
        self.bins = {}

    def key(self, x):
        return tuple(int(x[a] // (self.box[a] / self.n[a])) % self.n[a] for a in range(self.dim))

    def add(self, idx, x):
        self.bins.setdefault(self.key(x), []).append(idx)

    def near(self, x):
        k = self.key(x)
        out = []
        rng = range(-1, 2)
        if self.dim == 2:
            for i in rng:
                for j in rng:
                    out.extend(self.bins.get(((k[0] + i) % self.n[0], (k[1] + j) % self.n[1]), ()))
        else:
            for i in rng:
                for j in rng:
                    for l in rng:
                        out.extend(self.bins.get(((k[0] + i) % self.n[0], (k[1] + j) % self.n[1],
                                                  (k[2] + l) % self.n[2]), ()))
        return set(out)


def rsa_pack(rng, box, radii, periodic, lo=None, hi=None, gap=0.0, wall_gap=0.5,
             max_tries=2000000):
    """Random sequential addition of spheres/discs with the given radii (largest first).

    ``box`` holds the domain extent per axis (cells 0..n-1; walls at -1/2 and n-1/2 on
    non-periodic axes). Centres are drawn uniformly in [lo, hi) per axis; a trial is
    rejected if it comes closer than ``gap`` to an earlier particle or closer than
    ``wall_gap`` to a wall. Returns centres in the order of ``radii``.
    """
    dim = len(box)
    radii = np.asarray(radii, dtype=np.float64)
    order = np.argsort(-radii, kind="stable")
    lo = np.zeros(dim) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.asarray(box, dtype=np.float64) if hi is None else np.asarray(hi, dtype=np.float64)
    rmax = float(radii.max())
    grid = _Grid([float(b) for b in box], 2.0 * rmax + gap, dim)
    X = np.zeros((radii.size, dim))
    placed = []
    tries = 0
    for idx in order:
        r = radii[idx]
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("packing failed: too dense for random sequential addition")
            x = lo + rng.random(dim) * (hi - lo)
            ok = True
            for a in range(dim):
                if not periodic[a]:
                    if x[a] - r < -0.5 + wall_gap or x[a] + r > box[a] - 0.5 - wall_gap:
                        ok = False
                        break
                else:
                    x[a] %= box[a]
            if not ok:
                continue
            cand = grid.near(x)
            if cand:
                ci = np.fromiter(cand, dtype=np.int64)
                d = _min_image(X[ci] - x, box, periodic)
                dist = np.sqrt((d * d).sum(axis=1))
                if np.any(dist < radii[ci] + r + gap):
                    continue
            X[idx] = x
            grid.add(idx, x)
            placed.append(idx)
            break
    return X


def _pairs_within(X, box, periodic, cut):
    """All pairs (i < j) closer than ``cut`` (minimum image on periodic axes), by a k-d tree."""
    from scipy.spatial import cKDTree
    box = np.asarray(box, dtype=np.float64)
    dim = X.shape[1]
    # the tree wraps every axis it is given a box size for; wall axes get a span far larger
    # than the domain, so nothing wraps there
    span = np.where(np.asarray(periodic[:dim], dtype=bool), box[:dim], 1e9)
    Y = X.copy()
    for a in range(dim):
        if periodic[a]:
            Y[:, a] %= box[a]
        else:
            Y[:, a] += 1e8
    return cKDTree(Y, boxsize=span).query_pairs(cut, output_type="ndarray")


def grow_relax_pack(rng, box, radii, periodic, wall_gap=0.5, s0=0.75, stages=12, sweeps=25, gap=0.0):
    """Dense packing by growth and relaxation: centres start uniform at random; the radii
    grow from s0 to their full size in ``stages`` steps, and after each growth overlapping
    pairs are pushed apart along their line of centres (each by half the overlap, repeated
    up to ``sweeps`` times; at full size until none is left) and wall axes are clamped.
    Reaches solid fractions random sequential addition cannot, with many near-contacts.
    Pairs come from a list of those within r_i + r_j + 2, rebuilt when a particle has moved
    one unit."""
    dim = len(box)
    radii = np.asarray(radii, dtype=np.float64)
    n = radii.size
    box = np.asarray(box, dtype=np.float64)
    per = np.asarray(periodic[:dim], dtype=bool)
    lo = np.where(per, 0.0, -0.5 + wall_gap + radii[:, None])
    hi = np.where(per, box, box - 0.5 - wall_gap - radii[:, None])
    X = lo + rng.random((n, dim)) * (hi - lo)
    rmax = float(radii.max())
    margin = 2.0
    pairs, Xref, rsum = None, None, None

    def sep(i, j):
        d = X[j] - X[i]
        for a in range(dim):
            if per[a]:
                d[:, a] -= box[a] * np.rint(d[:, a] / box[a])
        return d

    near, age = None, 0
    for s in np.linspace(s0, 1.0, stages):
        limit = sweeps if s < 1.0 else 400 * sweeps
        for _ in range(limit):
            if pairs is None or np.max(np.abs(_min_image(X - Xref, box, periodic))) > 0.5 * margin:
                pairs = _pairs_within(X, box, periodic, 2 * rmax + margin)
                d = sep(pairs[:, 0], pairs[:, 1])
                keep = (d * d).sum(axis=1) < (radii[pairs[:, 0]] + radii[pairs[:, 1]] + margin) ** 2
                pairs = pairs[keep]
                rsum = radii[pairs[:, 0]] + radii[pairs[:, 1]]
                Xref = X.copy()
                near = None
            if near is None or age >= 8:
                # the pairs within half a unit of touching (no particle moves that far in 8
                # sweeps of this relaxation but the ones pushed apart)
                d = sep(pairs[:, 0], pairs[:, 1])
                near = np.nonzero((d * d).sum(axis=1) < (s * rsum + gap + 0.5) ** 2)[0]
                age = 0
            age += 1
            i, j = pairs[near, 0], pairs[near, 1]
            d = sep(i, j)
            dist = np.sqrt((d * d).sum(axis=1))
            ov = s * rsum[near] + gap - dist
            m = ov > 1e-9 * rsum[near]
            if not np.any(m):
                if age == 1:
                    break
                age = 8       # confirm on a fresh near list before leaving the stage
                continue
            im, jm = i[m], j[m]
            push = (0.5 * (ov[m] + 1e-6) / np.maximum(dist[m], 1e-12))[:, None] * d[m]
            for a in range(dim):
                X[:, a] += np.bincount(jm, weights=push[:, a], minlength=n) - np.bincount(im, weights=push[:, a], minlength=n)
                if per[a]:
                    X[:, a] %= box[a]
                else:
                    np.clip(X[:, a], lo[:, a], hi[:, a], out=X[:, a])
    pairs = _pairs_within(X, box, periodic, 2 * rmax)
    d = sep(pairs[:, 0], pairs[:, 1])
    ov = radii[pairs[:, 0]] + radii[pairs[:, 1]] + gap - np.sqrt((d * d).sum(axis=1))
    if ov.size and np.max(ov) > 1e-6:
        raise RuntimeError("packing failed: overlaps remain (max %.3g)" % ov.max())
    return X


def _pad3(a):
    a = np.asarray(a, dtype=np.float64)
    if a.shape[-1] == 3:
        return a
    out = np.zeros(a.shape[:-1] + (3,))
    out[..., : a.shape[-1]] = a
    return out


def c1_discs():
    """Four static discs r = 6.5 in a 64x64 periodic box: pair A at a 1.0 lu surface gap
    and pair B at a 0.25 lu gap; the pairs' positions and orientations come from seed 1."""
    rng = rng_for(0)
    r = 6.5
    X = []
    for (cy, gap) in ((16.0, 1.0), (48.0, 0.25)):
        cx = 20.0 + 24.0 * rng.random()
        theta = rng.uniform(-0.3, 0.3)
        half = r + 0.5 * gap
        d = np.array([math.cos(theta), math.sin(theta)]) * half
        X.append([cx - d[0], cy - d[1]])
        X.append([cx + d[0], cy + d[1]])
    return _pad3(np.array(X)), np.full(4, r)


def workload(name, scale=1.0, n_particles=None, seed_offset=0):
    """Return a dict describing one workload (see the module docstring).

    Keys: lattice, n (nx, ny, nz), bc (per axis 0 periodic / 1 walls), tau, body_force,
    X, U, Om, r (particles, (N, 3) / (N,)), steps, dem (dict or None), solid_fraction.
    """
    if name == "c1":
        X, r = c1_discs()
        n = (64, 64, 1)
        return dict(name=name, lattice=9, n=n, bc=(0, 0, 0), tau=0.8,
                    body_force=(1e-6, 0.0, 0.0), X=X, U=np.zeros_like(X), Om=np.zeros_like(X),
                    r=r, steps=1000, dem=None,
                    solid_fraction=float(np.pi * (r ** 2).sum() / (n[0] * n[1])))
    if name == "c2":
        rng = rng_for(1 + seed_offset)
        L = max(32, int(round(2048 * scale)))
        N = n_particles if n_particles is not None else int(round(5000 * (L / 2048.0) ** 2))
        r = rng.uniform(4.0, 8.0, size=N)
        band_area = np.pi * (r ** 2).sum() / 0.40
        band_h = min(L - 2.0, band_area / L)
        y0 = 0.5 * (L - 1) - 0.5 * band_h
        X2 = rsa_pack(rng, (L, L), r, (True, False), lo=(0.0, y0), hi=(L, y0 + band_h))
        X = _pad3(X2)
        U = _pad3(rng.normal(0.0, 1e-3, size=(N, 2)))
        Om = np.zeros((N, 3))
        Om[:, 2] = rng.normal(0.0, 1e-3, size=N) / r
        return dict(name=name, lattice=9, n=(L, L, 1), bc=(0, 1, 0), tau=0.7,
                    body_force=(0.0, 0.0, 0.0), X=X, U=U, Om=Om, r=r, steps=None,
                    dem=dict(substeps=10, gamma=2e-4), band=(y0, y0 + band_h),
                    solid_fraction=float(np.pi * (r ** 2).sum() / (L * L)),
                    band_solid_fraction=float(np.pi * (r ** 2).sum() / (L * band_h)))
    if name in ("c3", "c3dense"):
        rng = rng_for(2 + seed_offset)
        L = max(16, int(round(256 * scale)))
        base = 2000 if name == "c3" else 5563
        N = n_particles if n_particles is not None else int(round(base * (L / 256.0) ** 3))
        r = np.full(N, 6.0)
        X = rsa_pack(rng, (L, L, L), r, (True, True, True))
        return dict(name=name, lattice=19, n=(L, L, L), bc=(0, 0, 0), tau=0.6,
                    body_force=(1e-6, 0.0, 0.0), X=X, U=np.zeros_like(X), Om=np.zeros_like(X),
                    r=r, steps=None, dem=None,
                    solid_fraction=float(4.0 / 3.0 * np.pi * (r ** 3).sum() / L ** 3))
    if name == "c4":
        rng = rng_for(3 + seed_offset)
        L = max(16, int(round(128 * scale)))
        N = n_particles if n_particles is not None else max(1, int(round(200 * (L / 128.0) ** 3)))
        r = np.full(N, 5.0)
        X = rsa_pack(rng, (L, L, L), r, (True, True, True))
        return dict(name=name, lattice=19, n=(L, L, L), bc=(0, 0, 0), tau=0.7,
                    body_force=(1e-6, 0.0, 0.0), X=X, U=np.zeros_like(X), Om=np.zeros_like(X),
                    r=r, steps=500, dem=None, checkpoint=50,
                    solid_fraction=float(4.0 / 3.0 * np.pi * (r ** 3).sum() / L ** 3))
    if name == "c5dense":
        # the 512^3 channel at solid fraction 0.45: 71,830 spheres r ~ U(3, 8) (mean volume
        # 4/3 pi E[r^3] = 840.9) by growth and relaxation, which leaves many near-contacts
        rng = rng_for(5 + seed_offset)
        L = max(16, int(round(512 * scale)))
        N = n_particles if n_particles is not None else int(round(71830 * (L / 512.0) ** 3))
        r = rng.uniform(3.0, 8.0, size=N)
        X = grow_relax_pack(rng, (L, L, L), r, (True, True, False))
        U = rng.normal(0.0, 1e-3, size=(N, 3))
        return dict(name=name, lattice=19, n=(L, L, L), bc=(0, 0, 1), tau=0.55,
                    body_force=(1e-6, 0.0, 0.0), X=X, U=U, Om=np.zeros_like(X), r=r,
                    steps=2000, dem=dict(substeps=10, gamma=C5_GAMMA),
                    solid_fraction=float(4.0 / 3.0 * np.pi * (r ** 3).sum() / L ** 3))
    if name == "c5":
        rng = rng_for(4 + seed_offset)
        L = max(16, int(round(512 * scale)))
        N = n_particles if n_particles is not None else int(round(50000 * (L / 512.0) ** 3))
        r = rng.uniform(3.0, 8.0, size=N)
        X = rsa_pack(rng, (L, L, L), r, (True, True, False))
        U = rng.normal(0.0, 1e-3, size=(N, 3))
        return dict(name=name, lattice=19, n=(L, L, L), bc=(0, 0, 1), tau=0.55,
                    body_force=(1e-6, 0.0, 0.0), X=X, U=U, Om=np.zeros_like(X), r=r,
                    steps=2000, dem=dict(substeps=10, gamma=C5_GAMMA),
                    solid_fraction=float(4.0 / 3.0 * np.pi * (r ** 3).sum() / L ** 3))
    raise KeyError(name)


def random_field(rng, q, n, amp=1e-3):
    """Random smooth-ish population deviations for one-step parity checks: equilibrium
    perturbations drawn uniformly in [-amp, amp] per population (shape (q, nz, ny, nx))."""
    nx, ny, nz = n
    return rng.uniform(-amp, amp, size=(q, nz, ny, nx))
