"""Parity of the CUDA DEM sub-step (through the C ABI) with the FP64 DEM oracle.

Contact lists must match the oracle bit for bit (identical FP64 detection arithmetic);
velocity and spin changes, and the contact history, within 1e-4 relative L2 (the contact
law runs in FP32 on the GPU); positions within the same tolerance on their change.
"""
import math

import numpy as np
import pytest

import oracle as O
from parity_utils import rel_l2

pytestmark = pytest.mark.gpu

DEM = dict(E=2.0, poisson=0.3, gamma=2e-3, density=3.0, mu_f=0.3, theta_crit=0.01, alpha_n=0.3,
           k_t_scale=1.0, eta_t_scale=1.0)


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


def _cloud(dim, n, L, seed, rmin=1.5, rmax=2.5, vel=2e-3):
    rng = np.random.default_rng(seed)
    r = rng.uniform(rmin, rmax, n)
    X = np.zeros((n, 3))
    X[:, :dim] = rng.uniform(0, L, (n, dim))
    U = np.zeros((n, 3)); U[:, :dim] = rng.normal(0, vel, (n, dim))
    Om = np.zeros((n, 3))
    if dim == 3:
        Om[:] = rng.normal(0, vel / 2, (n, 3))
    else:
        Om[:, 2] = rng.normal(0, vel / 2, n)
    return X, U, Om, r


def _run_both(P, dim, X, U, Om, r, L, substeps, dt, adhesive=1, Ff=None, Tf=None, calls=1, skin=2.0,
              **kw):
    prm = dict(DEM, **kw)
    lattice = 9 if dim == 2 else 19
    nz = 1 if dim == 2 else L
    ctx = P.lbm_create(lattice, L, L, nz, tau=0.8, storage="f32")
    P.lbm_set_particles(ctx, X, U, Om, r)
    dem = P.dem_create(ctx, dt_dem=dt, adhesive=adhesive, skin=skin, **prm)
    for _ in range(calls):
        P.dem_step(dem, substeps)
    Xg, Ug, Og = P.dem_get_particles(dem)
    pg, hg = P.dem_get_contacts(dem)
    info = P.dem_get_info(dem)
    P.dem_destroy(dem)
    P.lbm_destroy(ctx)
    p = O.make_dem_params(dt=dt, adhesive=adhesive, dim=dim, n=(L, L, nz), periodic=(1, 1, 1), **prm)
    st = O.DemState(X, U, Om, r)
    for _ in range(calls):
        O.dem_step(p, st, Ff, Tf, substeps=substeps)
    po, ho = st.contacts()
    return dict(X=Xg, U=Ug, Om=Og, pairs=pg, hist=hg, info=info), dict(X=st.X, U=st.U, Om=st.Om, pairs=po, hist=ho)


def _compare(g, o, X0, U0, Om0, dim, tol=1e-4):
    assert np.array_equal(g["pairs"], o["pairs"]), "contact lists differ"
    assert g["info"]["solve_failures"] == 0 and g["info"]["overflows"] == 0
    dUo, dUg = o["U"] - U0, g["U"] - U0
    assert rel_l2(dUg, dUo) <= tol
    cols = [2] if dim == 2 else [0, 1, 2]
    assert rel_l2((g["Om"] - Om0)[:, cols], (o["Om"] - Om0)[:, cols]) <= tol
    dXo, dXg = o["X"] - X0, g["X"] - X0
    assert rel_l2(dXg, dXo) <= tol
    if len(o["hist"]):
        assert rel_l2(g["hist"], o["hist"]) <= 10 * tol


@pytest.mark.parametrize("dim", [2, 3])
def test_one_substep_contact_list_bit_exact(P, dim):
    L = 40 if dim == 2 else 24
    X, U, Om, r = _cloud(dim, 60 if dim == 2 else 150, L, seed=dim)
    g, o = _run_both(P, dim, X, U, Om, r, L, substeps=1, dt=0.1)
    assert len(o["pairs"]) > 20
    _compare(g, o, X, U, Om, dim)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("adhesive", [1, 0])
def test_ten_substeps_three_calls(P, dim, adhesive):
    """Three LBM-step-sized calls of 10 sub-steps each: history carried across calls."""
    L = 40 if dim == 2 else 24
    X, U, Om, r = _cloud(dim, 60 if dim == 2 else 150, L, seed=10 + dim)
    g, o = _run_both(P, dim, X, U, Om, r, L, substeps=10, dt=0.1, adhesive=adhesive, calls=3)
    _compare(g, o, X, U, Om, dim, tol=2e-4)


def test_head_on_adhesive_collision_loses_eq23_energy(P):
    """The GPU contact law reproduces the Eq. 23 hysteresis loss of a head-on collision."""
    E, nu, gamma, r = 2.0, 0.3, 2e-4, 3.0
    L = 32
    X = np.array([[10.0, 10.0, 10.0], [10.0 + 2 * r + 0.05, 10.0, 10.0]])
    U = np.array([[3e-3, 0, 0], [-3e-3, 0, 0]])
    ctx = P.lbm_create(19, L, L, L, tau=0.8, storage="f32")
    P.lbm_set_particles(ctx, X, U, np.zeros((2, 3)), np.array([r, r]))
    dem = P.dem_create(ctx, E=E, poisson=nu, gamma=gamma, alpha_n=0.0, dt_dem=2e-3, density=3.0)
    touched = False
    for _ in range(400):
        P.dem_step(dem, 100)
        pairs, _ = P.dem_get_contacts(dem)
        touched |= len(pairs) > 0
        if touched and len(pairs) == 0:
            break
    Xg, Ug, Og = P.dem_get_particles(dem)
    m = 3.0 * 4 / 3 * math.pi * r ** 3
    lost = 0.5 * m * (2 * 3e-3 ** 2) - 0.5 * m * (Ug ** 2).sum()
    Es = E / (2 * (1 - nu * nu))
    expect = 22.51 * (gamma ** 5 * (r / 2) ** 4 / Es ** 2) ** (1 / 3)
    assert touched and lost == pytest.approx(expect, rel=3e-2)


def test_coupled_fluid_forces_drive_dem(P):
    """One coupled step on a sub-box of the channel workload: the LBM forces read back from
    the GPU drive both DEM implementations for 10 sub-steps."""
    import synth
    w = synth.workload("c2", scale=0.0625)
    L = w["n"][0]
    ctx = P.lbm_create(9, L, L, 1, bc=w["bc"], tau=w["tau"], storage="f32")
    P.lbm_set_particles(ctx, w["X"], w["U"], w["Om"], w["r"])
    dem = P.dem_create(ctx, dt_dem=0.1, **DEM)
    P.lbm_step(ctx, 1)
    F, T = P.lbm_get_forces(ctx)
    P.dem_step(dem, 10)
    Xg, Ug, Og = P.dem_get_particles(dem)
    pg, _ = P.dem_get_contacts(dem)
    p = O.make_dem_params(dt=0.1, dim=2, n=(L, L, 1), periodic=(1, 0, 1), **DEM)
    st = O.DemState(w["X"], w["U"], w["Om"], w["r"])
    O.dem_step(p, st, F, T, substeps=10)
    assert np.array_equal(pg, st.contacts()[0])
    assert rel_l2(Ug - w["U"], st.U - w["U"]) <= 1e-4
    assert rel_l2((Og - w["Om"])[:, 2], (st.Om - w["Om"])[:, 2]) <= 1e-4


@pytest.mark.parametrize("adhesive", [1, 0])
def test_wall_contacts_match_the_oracle(P, adhesive):
    """Spheres falling onto the bottom wall of a box with walls in z (periodic in x and y),
    three LBM-step-sized calls of 10 sub-steps with gravity: particle-particle and wall
    contact lists bit for bit, velocities, spins and positions within 1e-4."""
    import synth
    rng = np.random.default_rng(31)
    L, n = 36, 30
    r = rng.uniform(1.5, 2.5, n)
    X = np.zeros((n, 3))
    X[:, :2] = synth.rsa_pack(rng, (L, L), r, (True, True), gap=0.05)     # a layer without overlaps
    X[:, 2] = -0.5 + r + rng.uniform(-0.1, 0.12, n)        # some already pressed into the wall
    U = np.zeros((n, 3)); U[:, 2] = -rng.uniform(0, 3e-3, n); U[:, :2] = rng.normal(0, 1e-3, (n, 2))
    Om = rng.normal(0, 1e-3, (n, 3))
    g = (0.0, 0.0, -2e-4)
    prm = dict(DEM, gamma=2e-3 if adhesive else 2e-4)
    ctx = P.lbm_create(19, L, L, L, bc=(0, 0, 1), tau=0.8, storage="f32")
    P.lbm_set_particles(ctx, X, U, Om, r)
    dem = P.dem_create(ctx, dt_dem=0.1, adhesive=adhesive, skin=2.0, gravity=g, **prm)
    for _ in range(3):
        P.dem_step(dem, 10)
    Xg, Ug, Og = P.dem_get_particles(dem)
    pg, _ = P.dem_get_contacts(dem)
    wg, whg = P.dem_get_wall_contacts(dem)
    info = P.dem_get_info(dem)
    P.dem_destroy(dem)
    P.lbm_destroy(ctx)
    p = O.make_dem_params(dt=0.1, adhesive=adhesive, dim=3, n=(L, L, L), periodic=(1, 1, 0), gravity=g, **prm)
    st = O.DemState(X, U, Om, r)
    for _ in range(3):
        O.dem_step(p, st, substeps=10)
    wo, who = st.wall_contacts()
    assert info["solve_failures"] == 0 and info["overflows"] == 0
    assert len(wo) >= 5
    assert np.array_equal(wg, wo), "wall contact lists differ"
    assert np.array_equal(pg, st.contacts()[0])
    assert rel_l2(Ug - U, st.U - U) <= 1e-4
    assert rel_l2(Og - Om, st.Om - Om) <= 1e-4
    assert rel_l2(Xg - X, st.X - X) <= 1e-4
    assert rel_l2(whg, who) <= 1e-3
