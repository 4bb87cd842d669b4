"""lbm_coupled_step against the two calls it stands for (lbm_step(ctx, 1) then
dem_step(dem, substeps)): the same particles, contacts, forces and populations after a run,
in the fused form (2D, FP32 and FP16 storage, even sub-step counts: the plain-fluid tiles
computed beside the DEM call) and in the forms it queues as the two calls (an odd sub-step
count, 3D). Only the order of the per-tile FP64 force atomics (Eq. 14) may differ between
any two runs, so the comparison allows a relative 1e-9."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DEM = dict(E=2.0, poisson=0.3, gamma=2e-4, density=3.0, mu_f=0.3, theta_crit=0.01, alpha_n=0.3,
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


def _packing(dim, n, L, seed):
    """Non-overlapping particles (random sequential addition) clear of the y walls, with
    small velocities."""
    rng = np.random.default_rng(seed)
    X, r = [], []
    while len(r) < n:
        x = rng.uniform(0, 1, dim) * np.array(L[:dim], dtype=float)
        x[1] = rng.uniform(6.5, L[1] - 7.5)      # clear of the walls of the y axis
        rr = rng.uniform(3.0, 5.0)
        if all(np.linalg.norm((x - xj) - np.array(L[:dim]) * np.rint((x - xj) / np.array(L[:dim]))) > rr + rj + 0.2
               for xj, rj in zip(X, r)):
            X.append(x)
            r.append(rr)
    Xa = np.zeros((n, 3)); Xa[:, :dim] = X
    U = np.zeros((n, 3)); U[:, :dim] = rng.normal(0, 2e-3, (n, dim))
    Om = np.zeros((n, 3))
    if dim == 2:
        Om[:, 2] = rng.normal(0, 1e-4, n)
    else:
        Om[:] = rng.normal(0, 1e-4, (n, 3))
    return Xa, U, Om, np.array(r)


def _run(P, fused, dim, storage, sub, steps):
    L = (160, 96, 1) if dim == 2 else (48, 48, 48)
    lattice = 9 if dim == 2 else 19
    X, U, Om, r = _packing(dim, 30 if dim == 2 else 12, L, 5)
    ctx = P.lbm_create(lattice, *L, bc=(0, 1, 0), tau=0.7,
                       body_force=(2e-6, 0.0, 0.0), storage=storage)
    P.lbm_set_particles(ctx, X, U, Om, r)
    dem = P.dem_create(ctx, dt_dem=1.0 / sub, **DEM)
    for _ in range(steps):
        if fused:
            P.lbm_coupled_step(ctx, dem, 1, sub)
        else:
            P.lbm_step(ctx, 1)
            P.dem_step(dem, sub)
    out = dict(zip(("X", "U", "Om"), P.dem_get_particles(dem)))
    out["F"], out["T"] = P.lbm_get_forces(ctx)
    out["f"] = P.lbm_get_populations(ctx)
    out["pairs"], _ = P.dem_get_contacts(dem)
    out["info"] = P.lbm_get_info(ctx)
    P.dem_destroy(dem)
    P.lbm_destroy(ctx)
    return out


@pytest.mark.parametrize("dim,storage,sub", [(2, "f32", 10), (2, "f16", 10), (2, "f32", 5), (3, "f32", 4)])
def test_coupled_step_matches_the_two_calls(P, dim, storage, sub):
    steps = 40
    a = _run(P, True, dim, storage, sub, steps)
    b = _run(P, False, dim, storage, sub, steps)
    assert np.array_equal(a["pairs"], b["pairs"])
    for k in ("X", "U", "Om", "F", "T", "f"):
        scale = max(np.abs(b[k]).max(), 1e-30)
        assert np.abs(a[k] - b[k]).max() <= 1e-9 * scale, k
    # the particles moved and felt the fluid
    assert np.abs(b["F"]).max() > 0
    assert a["info"]["steps"] == b["info"]["steps"] == steps


def test_coupled_step_rejects_a_foreign_dem_context(P):
    c1 = P.lbm_create(9, 64, 64, 1, tau=0.8, storage="f32")
    c2 = P.lbm_create(9, 64, 64, 1, tau=0.8, storage="f32")
    X, U, Om, r = _packing(2, 4, (64, 64, 1), 1)
    P.lbm_set_particles(c2, X, U, Om, r)
    d2 = P.dem_create(c2, **DEM)
    with pytest.raises(P.LbmError):
        P.lbm_coupled_step(c1, d2, 1, 2)
    P.dem_destroy(d2)
    P.lbm_destroy(c2)
    P.lbm_destroy(c1)
