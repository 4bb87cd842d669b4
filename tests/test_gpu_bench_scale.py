"""Parity at the sizes and settings the benchmark runs, through the C ABI.

- The DEM call of the 2048^2 channel (5000 discs, the benchmark's contact parameters, 10
  sub-steps driven by the forces of one LBM step) against the FP64 DEM oracle: contact
  lists bit for bit, velocity, spin and position changes within 1e-4; and the exact
  momentum balance of both: contact forces cancel pair by pair, so the discs' momentum
  changes by the sub-steps times dt times the total hydrodynamic force, to FP64 rounding.
- One step of the full 256^3 D3Q19 workload with 2000 spheres (FP32), every cell and
  particle compared with the oracle.
- The coupled step (LBM + 10 DEM sub-steps, 20 steps) on a 64^3 channel sub-box of the
  512^3 workload, particles in contact from the start.
- The Sec. 3.4 packed bed at d_p = 12 against the oracle over 500 steps.
"""
import numpy as np
import pytest

import oracle as O
import synth
from parity_utils import compare, perturbed_state, rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL32 = dict(u=1e-5, rho=1e-5, F=1e-4, T=1e-4)
TOL64 = dict(u=1e-10, rho=1e-12, F=1e-10, T=1e-10)
# contact parameters of the coupled benchmark workloads (lattice units)
BENCH_DEM = dict(E=2.0, poisson=0.3, gamma=2e-4, density=3.0, mu_f=0.3, theta_crit=0.01, alpha_n=0.3,
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


def _check(err, tol):
    for k, v in tol.items():
        if k in err:
            assert err[k] <= v, "%s rel L2 %.3e > %.1e (all: %s)" % (k, err[k], v, err)


def _squeeze(X, axis, centre, factor):
    """Positions moved towards a plane (a packing with contacts from the start)."""
    X = X.copy()
    X[:, axis] = centre + (X[:, axis] - centre) * factor
    return X


def _momentum_gap(U0, U1, m, F, dt_total, dim):
    """|sum m dU - dt_total sum F| and the scale sum m |dU| (components in the plane)."""
    dP = (m[:, None] * (U1 - U0))[:, :dim].sum(0)
    imp = dt_total * F[:, :dim].sum(0)
    return float(np.max(np.abs(dP - imp))), float(np.sum(m[:, None] * np.abs(U1 - U0)[:, :dim]))


def test_c2_dem_call_full_size(P):
    """The benchmark's DEM call on all 5000 discs of the 2048^2 channel: 10 sub-steps of
    dt 0.1 with the forces and torques of one LBM step held fixed (Sec. 2.5)."""
    w = synth.workload("c2")
    n = w["n"]
    y0, y1 = w["band"]
    X = _squeeze(w["X"], 1, 0.5 * (y0 + y1), 0.98)
    ctx = P.lbm_create(9, *n, bc=w["bc"], tau=w["tau"], storage="f32")
    P.lbm_set_particles(ctx, X, w["U"], w["Om"], w["r"])
    P.lbm_step(ctx, 1)
    F, T = P.lbm_get_forces(ctx)
    dem = P.dem_create(ctx, dt_dem=0.1, **BENCH_DEM)
    P.dem_step(dem, 10)
    Xg, Ug, Og = P.dem_get_particles(dem)
    pg, hg = P.dem_get_contacts(dem)
    info = P.dem_get_info(dem)
    P.dem_destroy(dem)
    P.lbm_destroy(ctx)

    p = O.make_dem_params(dt=0.1, dim=2, n=n, periodic=(1, 0, 1), **BENCH_DEM)
    st = O.DemState(X, w["U"], w["Om"], w["r"], cap=200000)
    O.dem_step(p, st, F, T, substeps=10)
    po, ho = st.contacts()

    assert info["solve_failures"] == 0 and info["overflows"] == 0 and info["skin_violations"] == 0
    assert len(po) > 100
    assert np.array_equal(pg, po), "contact lists differ"
    assert rel_l2(Ug - w["U"], st.U - w["U"]) <= 1e-4
    assert rel_l2((Og - w["Om"])[:, 2], (st.Om - w["Om"])[:, 2]) <= 1e-4
    dXg = Xg - X
    dXo = st.X - X
    for a in (0,):   # undo the periodic wrap along x
        dXg[:, a] -= n[a] * np.rint(dXg[:, a] / n[a])
        dXo[:, a] -= n[a] * np.rint(dXo[:, a] / n[a])
    assert rel_l2(dXg, dXo) <= 1e-4
    assert rel_l2(hg, ho) <= 1e-3

    # momentum: every contact force is applied to both discs with opposite signs
    m = BENCH_DEM["density"] * np.pi * w["r"] ** 2
    for U1 in (Ug, st.U):
        gap, scale = _momentum_gap(w["U"], U1, m, F, 10 * 0.1, 2)
        assert scale > 0 and gap <= 1e-10 * scale, (gap, scale)


def test_c3_full_size_one_step(P):
    """The 256^3 periodic workload with 2000 spheres r = 6 in the benchmark's launch
    configuration: one FP32 step from a seeded perturbed state."""
    w = synth.workload("c3")
    case = dict(lattice=19, n=w["n"], bc=w["bc"], tau=w["tau"], body_force=w["body_force"],
                X=w["X"], U=w["U"], Om=w["Om"], r=w["r"])
    f0 = perturbed_state(case, 14)
    o = run_oracle(case, f0, 1)
    g = run_gpu(P, case, f0, 1, storage="f32")
    del f0
    assert g["info"]["overflow_tiles"] == 0
    _check(compare(g, o, 3), TOL32)


@pytest.mark.parametrize("name,storage,tol", [("c3dense", "f32", TOL32),
                                               ("c3", "f16", dict(u=1e-3, rho=1e-5, F=1e-3, T=1e-2))])
def test_full_size_one_step_dense_and_16bit(P, name, storage, tol):
    """The 256^3 workload at solid fraction 0.3 (5563 spheres: rows with three or four
    candidates, the brackets beyond the kept slots evaluated again) in FP32, and the
    2000-sphere workload in FP16 deviation storage (the configuration the storage comparison
    times): one step from a seeded perturbed state, every cell and particle."""
    w = synth.workload(name)
    case = dict(lattice=19, n=w["n"], bc=w["bc"], tau=w["tau"], body_force=w["body_force"],
                X=w["X"], U=w["U"], Om=w["Om"], r=w["r"])
    f0 = perturbed_state(case, 15)
    o = run_oracle(case, f0, 1)
    g = run_gpu(P, case, f0, 1, storage=storage)
    del f0
    assert g["info"]["overflow_tiles"] == 0
    _check(compare(g, o, 3), tol)


def test_c5_coupled_subbox_with_dem_20_steps(P):
    """The coupled loop on a 64^3 channel sub-box of the 512^3 workload (walls in z,
    polydisperse spheres r ~ U(3, 8), tau 0.55, JKR DEM with 10 sub-steps per LBM step),
    the spheres pressed together so that contacts exist from the start: per step one LBM
    step, then the DEM sub-steps with that step's forces; 20 steps, FP32 against FP64."""
    w = synth.workload("c5", scale=0.125)
    n = w["n"]
    X = _squeeze(w["X"], 2, 0.5 * (n[2] - 1), 0.96)
    case = dict(lattice=19, n=n, bc=w["bc"], tau=w["tau"], body_force=w["body_force"], X=X, U=w["U"],
                Om=w["Om"], r=w["r"])
    f0 = perturbed_state(case, 15)
    steps, sub = 20, 10

    ctx = P.lbm_create(19, *n, bc=w["bc"], tau=w["tau"], body_force=w["body_force"], storage="f32")
    P.lbm_set_populations(ctx, f0)
    P.lbm_set_particles(ctx, X, w["U"], w["Om"], w["r"])
    prm = dict(BENCH_DEM, gamma=w["dem"]["gamma"])
    dem = P.dem_create(ctx, dt_dem=1.0 / sub, **prm)
    for _ in range(steps):
        P.lbm_step(ctx, 1)
        P.dem_step(dem, sub)
    Fg, Tg = P.lbm_get_forces(ctx)
    rho_g, u_g = P.lbm_get_macro(ctx)
    Xg, Ug, Og = P.dem_get_particles(dem)
    pg, _ = P.dem_get_contacts(dem)
    info = P.dem_get_info(dem)
    P.dem_destroy(dem)
    P.lbm_destroy(ctx)

    p = O.make_params(19, *n, bc=w["bc"], tau=w["tau"], body_force=w["body_force"])
    pd = O.make_dem_params(dt=1.0 / sub, dim=3, n=n, periodic=(1, 1, 0), **prm)
    f = f0.copy()
    st = O.DemState(X, w["U"], w["Om"], w["r"])
    had_contacts = 0
    for _ in range(steps):
        Fo, To = O.step(p, f, st.X, st.U, st.Om, st.r)
        O.dem_step(pd, st, Fo, To, substeps=sub)
        had_contacts = max(had_contacts, st.ncontact)
    rho_o, u_o = O.macro(p, f)

    assert info["solve_failures"] == 0 and info["overflows"] == 0
    assert had_contacts >= 5
    assert np.array_equal(pg, st.contacts()[0])
    assert rel_l2(u_g, u_o) <= 1e-5 and rel_l2(rho_g, rho_o) <= 1e-5
    assert rel_l2(Fg, Fo) <= 1e-4 and rel_l2(Tg, To) <= 1e-4
    dXg, dXo = Xg - X, st.X - X
    for a in (0, 1):
        dXg[:, a] -= n[a] * np.rint(dXg[:, a] / n[a])
        dXo[:, a] -= n[a] * np.rint(dXo[:, a] / n[a])
    assert rel_l2(dXg, dXo) <= 1e-4
    assert rel_l2(Ug - w["U"], st.U - w["U"]) <= 1e-4
    assert rel_l2(Og - w["Om"], st.Om - w["Om"]) <= 1e-4


def _packed_bed(dp):
    c = dp / 2.0 - 0.5
    X = np.array([[c + dp * a, c + dp * b, c + dp * k] for a in (0, 1) for b in (0, 1) for k in (0, 1)])
    z = np.zeros((8, 3))
    return dict(lattice=19, n=(2 * dp, 2 * dp, 2 * dp), bc=(0, 0, 0), tau=0.65, body_force=(1e-6, 0, 0),
                X=X, U=z, Om=z, r=np.full(8, dp / 2.0))


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_packed_bed_d12_matches_oracle(P, storage):
    """Sec. 3.4 packing of 8 touching spheres (cells shared by neighbours, fractions summing
    to one at the contacts) at d_p = 12, 500 steps from rest: the run the oracle's Ergun
    check (Eq. 34-35) takes. FP64 at round-off; FP32 forces within 1e-4 and velocities
    within the rounding bound of FP32 storage over the horizon."""
    case = _packed_bed(12)
    o = run_oracle(case, perturbed_state(case, 0, amp=0.0), 500)
    g = run_gpu(P, case, None, 500, storage=storage)
    err = compare(g, o, 3)
    # the packing is symmetric: every torque is zero up to rounding, so torques are held to
    # the force scale times the radius instead of to their own (vanishing) norm
    scale = np.abs(o["F"]).max() * 6.0
    tol_T = 1e-10 if storage == "f64" else 1e-4
    assert np.abs(g["T"] - o["T"]).max() <= tol_T * scale
    err.pop("T")
    if storage == "f64":
        _check(err, TOL64)
    else:
        e, w_, _ = O.lattice_tables(19)
        dmax = np.max(np.abs(o["f"] - w_[:, None, None, None]))
        ulp = float(np.spacing(np.float32(dmax)))
        urms = np.sqrt(np.mean(np.sum(o["u"] ** 2, axis=-1)))
        tol_u = max(1e-5, 500 * np.abs(e).sum() * ulp / 2 / urms)
        _check(err, dict(u=tol_u, rho=1e-5, F=1e-4, T=1e-4))


def test_checkpoint_resumes_fluid_run_bit_identically(P):
    """lbm_save_state -> 4 steps, lbm_load_state -> the same 4 steps: the same populations
    bit for bit (static particles; forces agree to the order of their FP64 atomic sums),
    and the step counter restored."""
    from parity_utils import ragged_case3d
    case = ragged_case3d()
    ctx = P.lbm_create(19, *case["n"], bc=case["bc"], tau=case["tau"], body_force=case["body_force"], storage="f32")
    P.lbm_set_populations(ctx, perturbed_state(case, 16))
    P.lbm_set_particles(ctx, case["X"], case["U"], case["Om"], case["r"])
    P.lbm_step(ctx, 3)
    state = P.lbm_save_state(ctx)
    P.lbm_step(ctx, 4)
    fA = P.lbm_get_populations(ctx)
    FA, TA = P.lbm_get_forces(ctx)
    P.lbm_step(ctx, 2)                           # move on, then go back
    P.lbm_load_state(ctx, state)
    assert P.lbm_get_info(ctx)["steps"] == 3
    P.lbm_step(ctx, 4)
    fB = P.lbm_get_populations(ctx)
    FB, TB = P.lbm_get_forces(ctx)
    P.lbm_destroy(ctx)
    assert np.array_equal(fA, fB)
    assert np.allclose(FA, FB, rtol=1e-12, atol=1e-18) and np.allclose(TA, TB, rtol=1e-12, atol=1e-18)


def test_checkpoint_resumes_coupled_run_with_contact_history(P):
    """A coupled LBM + DEM run (256^2 channel sub-box, discs pressed into contact) saved
    after 3 steps and resumed: the checkpoint carries the DEM neighbour lists and spring
    history, so the resumed run has the same contacts and histories and the same particle
    states (to the order of the FP64 force atomics) as the uninterrupted one."""
    w = synth.workload("c2", scale=0.125)
    y0, y1 = w["band"]
    X = _squeeze(w["X"], 1, 0.5 * (y0 + y1), 0.95)
    ctx = P.lbm_create(9, *w["n"], bc=w["bc"], tau=w["tau"], storage="f32")
    P.lbm_set_particles(ctx, X, w["U"], w["Om"], w["r"])
    dem = P.dem_create(ctx, dt_dem=0.1, **BENCH_DEM)

    def coupled(k):
        for _ in range(k):
            P.lbm_step(ctx, 1)
            P.dem_step(dem, 10)

    coupled(3)
    state = P.lbm_save_state(ctx)
    coupled(4)
    XA, UA, OA = P.dem_get_particles(dem)
    pA, hA = P.dem_get_contacts(dem)
    coupled(2)
    P.lbm_load_state(ctx, state)
    coupled(4)
    XB, UB, OB = P.dem_get_particles(dem)
    pB, hB = P.dem_get_contacts(dem)
    P.dem_destroy(dem)
    P.lbm_destroy(ctx)
    assert len(pA) >= 3 and np.any(hA != 0)
    assert np.array_equal(pA, pB)
    assert np.allclose(hA, hB, rtol=1e-5, atol=1e-12)
    assert np.allclose(XA, XB, rtol=0, atol=1e-9)
    assert np.allclose(UA, UB, rtol=1e-6, atol=1e-15)
