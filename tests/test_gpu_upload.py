"""Particle upload and force download through the C ABI, by every route the caller's memory
can take: pageable host arrays (cudaMemcpyAsync), page-locked host tensors and device
tensors (read or written by the library's kernels directly). The download routes give the
same bits; the upload routes the same forces up to the order of the FP64 atomics.
With a DEM context attached, an upload of the same count and radii keeps the neighbour list
unless a particle moved more than a quarter of the skin since the list's build; either way
the next DEM call matches the FP64 DEM oracle run from the uploaded state."""
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


def _discs(n, L, seed):
    """Non-overlapping discs (random sequential addition) in an L x L periodic box."""
    rng = np.random.default_rng(seed)
    X, r = [], []
    while len(r) < n:
        x = rng.uniform(0, L, 2)
        rr = rng.uniform(3.0, 5.0)
        ok = True
        for xj, rj in zip(X, r):
            d = x - xj
            d -= L * np.rint(d / L)
            if np.hypot(*d) < rr + rj + 1.0:
                ok = False
                break
        if ok:
            X.append(x)
            r.append(rr)
    Xa = np.zeros((n, 3)); Xa[:, :2] = X
    U = np.zeros((n, 3)); U[:, :2] = rng.normal(0, 1e-3, (n, 2))
    Om = np.zeros((n, 3)); Om[:, 2] = rng.normal(0, 1e-4, n)
    return Xa, U, Om, np.array(r)


def _as(torch, a, where):
    if where == "numpy":
        return a
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if where == "pinned" else t.cuda()


def _forces(torch, P, ctx, where):
    n = ctx.np
    if where == "numpy":
        return P.lbm_get_forces(ctx)
    if where == "pinned":
        F = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
        T = torch.zeros((n, 3), dtype=torch.float64).pin_memory()
    else:
        F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        T = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    P.lbm_get_forces(ctx, F, T)
    torch.cuda.synchronize()
    return F.cpu().numpy(), T.cpu().numpy()


def test_every_upload_and_download_route_agrees(P):
    import torch
    L = 96
    X, U, Om, r = _discs(40, L, 3)
    ref = None
    for src in ("numpy", "pinned", "device"):
        ctx = P.lbm_create(9, L, L, 1, tau=0.8, storage="f32")
        P.lbm_set_particles(ctx, *[_as(torch, a, src) for a in (X, U, Om, r)])
        torch.cuda.synchronize()
        F0, T0 = P.lbm_get_forces(ctx)
        assert not F0.any() and not T0.any()
        P.lbm_step(ctx, 3)
        outs = [_forces(torch, P, ctx, dst) for dst in ("numpy", "pinned", "device")]
        for F, T in outs[1:]:
            assert np.array_equal(F, outs[0][0]) and np.array_equal(T, outs[0][1])
        assert np.abs(outs[0][0]).max() > 0
        # across contexts only the order of the per-tile FP64 atomics of Eq. 14 may differ
        if ref is None:
            ref = outs[0]
        else:
            for a, b in zip(outs[0], ref):
                assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), src
        # a new upload clears F and T
        P.lbm_set_particles(ctx, *[_as(torch, a, src) for a in (X, U, Om, r)])
        torch.cuda.synchronize()
        F1, T1 = _forces(torch, P, ctx, src)
        assert not F1.any() and not T1.any()
        P.lbm_destroy(ctx)


def test_rejected_upload_changes_nothing(P):
    import torch
    L = 96
    X, U, Om, r = _discs(30, L, 4)
    ctx = P.lbm_create(9, L, L, 1, tau=0.8, storage="f32")
    P.lbm_set_particles(ctx, X, U, Om, r)
    P.lbm_step(ctx, 2)
    F0, T0 = P.lbm_get_forces(ctx)
    bad = X.copy()
    bad[7, 1] = np.nan
    with pytest.raises(P.LbmError):
        P.lbm_set_particles(ctx, _as(torch, bad, "pinned"), _as(torch, U, "pinned"), _as(torch, Om, "pinned"),
                            _as(torch, r, "pinned"))
    rr = r.copy()
    rr[3] = 0.4
    with pytest.raises(P.LbmError):
        P.lbm_set_particles(ctx, X, U, Om, rr)
    F1, T1 = P.lbm_get_forces(ctx)
    assert np.array_equal(F0, F1) and np.array_equal(T0, T1)
    P.lbm_destroy(ctx)


def _cloud(n, L, seed):
    rng = np.random.default_rng(seed)
    r = rng.uniform(1.5, 2.5, n)
    X = np.zeros((n, 3)); X[:, :2] = rng.uniform(0, L, (n, 2))
    U = np.zeros((n, 3)); U[:, :2] = rng.normal(0, 2e-3, (n, 2))
    Om = np.zeros((n, 3)); Om[:, 2] = rng.normal(0, 1e-3, n)
    return X, U, Om, r


@pytest.mark.parametrize("case", ["kept", "moved", "radii"])
def test_upload_between_dem_calls_keeps_or_rebuilds_the_list(P, case):
    import torch
    L, n, sub, dt, skin = 32, 90, 4, 0.1, 2.0
    X0, U0, Om0, r = _cloud(n, L, 21)
    ctx = P.lbm_create(9, L, L, 1, tau=0.8, storage="f32")
    P.lbm_set_particles(ctx, X0, U0, Om0, r)
    dem = P.dem_create(ctx, dt_dem=dt, adhesive=1, skin=skin, **DEM)
    P.dem_step(dem, sub)
    assert P.dem_get_info(dem)["rebuilds"] == 1
    X1, U1, Om1 = P.dem_get_particles(dem)
    pairs1, hist1 = P.dem_get_contacts(dem)
    assert len(pairs1) > 10
    r1 = r.copy()
    if case == "kept":
        X1 = X1 + 1e-3          # far below a quarter of the skin (0.5)
    elif case == "moved":
        X1 = X1.copy()
        k = int(np.argmin(np.abs(X1[:, 0] - L / 2)))
        X1[k, 0] += 0.6         # one particle beyond it
    else:
        r1[9] *= 1.0 + 1e-6     # another radius: the list is rebuilt whatever the moves
    # page-locked host tensors: the direct-read route of the upload
    P.lbm_set_particles(ctx, *[_as(torch, a, "pinned") for a in (X1, U1, Om1, r1)])
    P.dem_step(dem, sub)
    info = P.dem_get_info(dem)
    assert info["rebuilds"] == (1 if case == "kept" else 2)
    assert info["solve_failures"] == 0 and info["overflows"] == 0 and info["skin_violations"] == 0
    Xg, Ug, Og = P.dem_get_particles(dem)
    pg, hg = P.dem_get_contacts(dem)
    P.dem_destroy(dem)
    P.lbm_destroy(ctx)

    # the oracle from the uploaded state, with the history of the GPU's first call
    p = O.make_dem_params(dt=dt, adhesive=1, dim=2, n=(L, L, 1), periodic=(1, 1, 1), **DEM)
    st = O.DemState(X1, U1, Om1, r1)
    st.ncontact = len(pairs1)
    st.pairs[: len(pairs1)] = pairs1
    st.hist[: len(pairs1)] = hist1
    O.dem_step(p, st, None, None, substeps=sub)
    po, ho = st.contacts()
    assert np.array_equal(pg, po), "contact lists differ"
    assert rel_l2(Ug - U1, st.U - U1) <= 1e-4
    assert rel_l2((Og - Om1)[:, 2], (st.Om - Om1)[:, 2]) <= 1e-4
    assert rel_l2(Xg - X1, st.X - X1) <= 1e-4
    assert rel_l2(hg, ho) <= 1e-3


@pytest.mark.parametrize("src", ["numpy", "pinned"])
def test_host_arrays_may_change_as_soon_as_the_upload_returns(P, src):
    """Host arrays are copied before lbm_set_particles returns (into the library's staging
    buffers, without waiting for the device): the caller may overwrite them at once, and
    uploads in a row each keep their own values."""
    import torch
    L = 96
    X, U, Om, r = _discs(40, L, 3)
    ref = P.lbm_create(9, L, L, 1, tau=0.8, storage="f32")
    P.lbm_set_particles(ref, X, U, Om, r)
    P.lbm_step(ref, 3)
    F0, T0 = P.lbm_get_forces(ref)
    P.lbm_destroy(ref)

    ctx = P.lbm_create(9, L, L, 1, tau=0.8, storage="f32")
    # three uploads in a row (the staging buffers are reused), the last one with the right
    # values; each source is overwritten as soon as its call returns
    for shift in (7.0, 13.0, 0.0):
        args = [_as(torch, a.copy(), src) for a in (X + shift, U, Om, r)]
        P.lbm_set_particles(ctx, *args)
        for a in args[:3]:
            if src == "numpy":
                a[...] = 1.0e9
            else:
                a.fill_(1.0e9)
    P.lbm_step(ctx, 3)
    F1, T1 = P.lbm_get_forces(ctx)
    P.lbm_destroy(ctx)
    for a, b in ((F1, F0), (T1, T0)):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
