"""Sec. 3.5 (Fig. 12-13): random packing of 500 spheres of diameter 6 lu settling under
gravity through a viscous fluid (tau = 2) in a 50 x 50 x 100 box (periodic in x and y,
walls in z) with the coupled LBM-DEM loop, adhesive (JKR) against non-adhesive (Hertz)
particles. The paper reports solid fraction 0.495 and coordination number 5.08 with
adhesion, 0.557 and 5.50 without, for its material (SI units, not stated in full); with
the lattice-unit material here the values differ, and what the test checks is the effect
the paper shows: adhesion leaves a looser bed with fewer contacts per particle. The
measured values are printed (and written to PSC_PACKING_REPORT when set)."""
import json
import math
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

N, D, BOX = 500, 6.0, (50, 50, 100)
G = 5e-4                               # gravity, lattice units
MAT = dict(E=20.0, poisson=0.3, density=3.0, mu_f=0.3, theta_crit=0.01, alpha_n=0.3, k_t_scale=1.0,
           eta_t_scale=1.0)


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1901_09745_gb300 import build
    build.build()
    import paper_1901_09745_gb300 as P
    P.lib()
    return P


def _cap_volume(r, h):
    """Volume of a sphere of radius r below the height h above its lowest point (0 <= h <= 2r)."""
    h = np.clip(h, 0.0, 2 * r)
    return math.pi * h * h * (3 * r - h) / 3.0


def _settle(P, adhesive, gamma):
    rng = synth.rng_for(60)
    r = np.full(N, D / 2)
    X = synth.rsa_pack(rng, BOX, r, (True, True, False), gap=0.3)
    U = np.zeros((N, 3))
    ctx = P.lbm_create(19, *BOX, bc=(0, 0, 1), tau=2.0, storage="f32")
    P.lbm_set_particles(ctx, X, U, U, r)
    dem = P.dem_create(ctx, dt_dem=0.1, adhesive=adhesive, gamma=gamma, gravity=(0.0, 0.0, -G), skin=0.5, **MAT)
    steps = 0
    for _ in range(80):
        for _ in range(1000):
            P.lbm_step(ctx, 1)
            P.dem_step(dem, 10)
        steps += 1000
        Xg, Ug, _ = P.dem_get_particles(dem)
        if steps >= 15000 and np.max(np.abs(Ug)) < 5e-5:
            break
    pairs, _ = P.dem_get_contacts(dem)
    info = P.dem_get_info(dem)
    P.dem_destroy(dem)
    P.lbm_destroy(ctx)
    assert info["solve_failures"] == 0 and info["overflows"] == 0 and info["skin_violations"] == 0
    z = Xg[:, 2]
    top = np.max(z + r)
    lo, hi = -0.5 + D, top - D                       # bulk: one diameter away from wall and surface
    vol = sum(_cap_volume(r[i], hi - (z[i] - r[i])) - _cap_volume(r[i], lo - (z[i] - r[i])) for i in range(N))
    phi = vol / (BOX[0] * BOX[1] * (hi - lo))
    bulk = (z > lo) & (z < hi)
    deg = np.zeros(N)
    for i, j in pairs:
        deg[i] += 1
        deg[j] += 1
    Z = float(np.mean(deg[bulk]))
    return dict(phi=float(phi), Z=Z, steps=steps, max_speed=float(np.max(np.abs(Ug))), bed_top=float(top))


def test_adhesion_leaves_a_looser_bed_with_fewer_contacts(P):
    adh = _settle(P, 1, gamma=0.05)        # pull-off 3 pi gamma R = 0.71, about 4 times the weight
    non = _settle(P, 0, gamma=0.0)
    rep = {"adhesive": adh, "non_adhesive": non,
           "paper": {"adhesive": {"phi": 0.495, "Z": 5.08}, "non_adhesive": {"phi": 0.557, "Z": 5.50}}}
    print(json.dumps(rep))
    out = os.environ.get("PSC_PACKING_REPORT")
    if out:
        with open(out, "w") as fh:
            json.dump(rep, fh, indent=1)
    for s in (adh, non):
        assert s["max_speed"] < 1e-4, s          # settled: 2.5 % of the speed of the fall
        assert 0.3 < s["phi"] < 0.68 and 2.0 < s["Z"] < 8.0, s
    assert adh["phi"] < non["phi"] and adh["Z"] < non["Z"], rep
