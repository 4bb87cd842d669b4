"""Pins of the FP64 DEM oracle (Sec. 2.5) against closed forms, the paper's printed Eq. 23
coefficient, conservation laws and the friction caps of Eq. 29 (no GPU)."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _jkr_consts(gamma, R, Es):
    FC = 3 * math.pi * gamma * R
    a0 = (9 * math.pi * gamma * R * R / Es) ** (1 / 3)
    dC = a0 * a0 / (2 * 6 ** (1 / 3) * R)
    return FC, a0, dC


@pytest.mark.parametrize("R,gamma,Es", [(1.0, 1.0, 1.0), (2.5, 3e-4, 2.2), (0.7, 0.05, 40.0)])
def test_jkr_closed_form_points(R, gamma, Es):
    """JKR theory: jump-on force -8/9 F_C at delta = 0, force -5/9 F_C at the critical
    separation -delta_C, minimum -F_C at a/a0 = 4^(-1/3), zero force at a = a0 where
    delta = a0^2/(3R)."""
    FC, a0, dC = _jkr_consts(gamma, R, Es)
    a, ok = O.jkr_contact_radius(0.0, a0, R)
    assert ok and O.jkr_force(a, a0, FC) == pytest.approx(-8 / 9 * FC, rel=1e-12)
    a, ok = O.jkr_contact_radius(-dC * (1 - 1e-15), a0, R)
    assert ok and O.jkr_force(a, a0, FC) == pytest.approx(-5 / 9 * FC, rel=1e-6)
    assert not O.jkr_contact_radius(-1.01 * dC, a0, R)[1]
    amin = 4 ** (-1 / 3) * a0
    assert O.jkr_force(amin, a0, FC) == pytest.approx(-FC, rel=1e-14)
    for s in (0.99, 1.01):
        assert O.jkr_force(s * amin, a0, FC) > -FC
    assert O.jkr_delta(a0, a0, R) == pytest.approx(a0 * a0 / (3 * R), rel=1e-14)
    a, ok = O.jkr_contact_radius(a0 * a0 / (3 * R), a0, R)
    assert a == pytest.approx(a0, rel=1e-12)
    # the solve inverts delta(a) on the stable branch
    for d in np.linspace(-0.99 * dC, 5 * dC, 13):
        a, ok = O.jkr_contact_radius(d, a0, R)
        assert ok and O.jkr_delta(a, a0, R) == pytest.approx(d, abs=1e-13 * max(1.0, abs(d)) + 1e-15)


def test_eq23_adhesion_energy_golden():
    """Eq. 23: the work of the adhesive force between jump-on and pull-off equals the
    printed 22.51 (gamma^5 R^4 / E^2)^(1/3) (E the effective modulus of Eq. 25)."""
    coef = float(np.loadtxt(os.path.join(GOLDEN, "eq23_adhesion_energy.txt")))
    for R, gamma, Es in [(1.0, 1.0, 1.0), (3.0, 2e-4, 2.2)]:
        FC, a0, dC = _jkr_consts(gamma, R, Es)
        W = integrate.quad(lambda d: O.jkr_force(O.jkr_contact_radius(d, a0, R)[0], a0, FC),
                           -dC, 0.0, epsabs=0, epsrel=1e-11, limit=200)[0]
        expect = coef * (gamma ** 5 * R ** 4 / Es ** 2) ** (1 / 3)
        assert W < 0
        assert abs(W) == pytest.approx(expect, rel=1e-3)


def _two_spheres(v, r=3.0, gap=0.05, dim=3):
    X = np.array([[10.0, 10.0, 10.0 if dim == 3 else 0.0], [10.0 + 2 * r + gap, 10.0, 10.0 if dim == 3 else 0.0]])
    U = np.array([[v / 2, 0, 0], [-v / 2, 0, 0]])
    return X, U, np.zeros((2, 3)), np.array([r, r])


def _kinetic(p, st):
    m = p.density * (4 / 3 * math.pi * st.r ** 3 if p.dim == 3 else math.pi * st.r ** 2)
    return 0.5 * (m * (st.U ** 2).sum(1)).sum()


def test_head_on_adhesive_collision_loses_eq23_energy():
    """Two spheres colliding head-on with no damping lose exactly the adhesion hysteresis
    of Eq. 23 (jump-on does no work; loading/unloading for delta > 0 is conservative)."""
    E, nu, gamma, r = 2.0, 0.3, 2e-4, 3.0
    p = O.make_dem_params(E=E, poisson=nu, gamma=gamma, alpha_n=0.0, mu_f=0.3, dt=2e-3, dim=3,
                          n=(64, 64, 64))
    X, U, Om, rad = _two_spheres(v=6e-3, r=r)
    st = O.DemState(X, U, Om, rad)
    k0 = _kinetic(p, st)
    touched = False
    for _ in range(400):
        O.dem_step(p, st, substeps=100)
        touched |= st.ncontact > 0
        if touched and st.ncontact == 0:
            break
    assert touched and st.ncontact == 0 and st.U[0, 0] < 0 < st.U[1, 0]
    Es = E / (2 * (1 - nu * nu))
    R = r / 2
    expect = 22.51 * (gamma ** 5 * R ** 4 / Es ** 2) ** (1 / 3)
    lost = k0 - _kinetic(p, st)
    assert lost == pytest.approx(expect, rel=2e-2)
    # momentum exactly conserved, no spin generated
    m = p.density * 4 / 3 * math.pi * r ** 3
    assert abs(m * st.U[:, 0].sum()) < 1e-15
    assert np.max(np.abs(st.Om)) == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_hertz_collision_without_damping_is_elastic(dim):
    p = O.make_dem_params(E=2.0, adhesive=0, alpha_n=0.0, dt=2e-3, dim=dim, n=(64, 64, 64))
    X, U, Om, rad = _two_spheres(v=2e-2, dim=dim)
    st = O.DemState(X, U, Om, rad)
    k0 = _kinetic(p, st)
    touched = False
    for _ in range(400):
        O.dem_step(p, st, substeps=100)
        touched |= st.ncontact > 0
        if touched and st.ncontact == 0:
            break
    assert touched and st.ncontact == 0
    assert _kinetic(p, st) == pytest.approx(k0, rel=2e-3)
    p2 = O.make_dem_params(E=2.0, adhesive=0, alpha_n=0.5, dt=2e-3, dim=dim, n=(64, 64, 64))
    st2 = O.DemState(X, U, Om, rad)
    for _ in range(400):
        O.dem_step(p2, st2, substeps=100)
        if st2.ncontact == 0 and st2.U[0, 0] < 0:
            break
    assert _kinetic(p2, st2) < 0.95 * k0


@pytest.mark.parametrize("v", [1e-2, 3e-2])
def test_hertz_normal_damping_energy_loss_small_alpha(v):
    """Normal damping (reading of the constants the paper takes from the literature):
    eta_N = alpha_n sqrt(m* k_N) with k_N = 2 E* a the Hertz contact stiffness dF/ddelta.
    To first order in alpha_n a head-on Hertz collision loses the work of the damping force
    along the undamped trajectory,

      W = 2 int_0^dmax eta_N(d) w(d) dd,  (1/2) m* w^2 + (8/15) E* sqrt(R) d^(5/2) = (1/2) m* w0^2,

    a quadrature independent of the oracle's integrator (to second order the loss is
    W (1 - W / 2E0)); a wrong factor in k_N or m* (m instead of m*, E* a instead of
    2 E* a) changes W by sqrt(2). With this form of eta_N the loss is the same fraction of
    the impact energy at every impact speed."""
    E, nu, r, alpha = 2.0, 0.3, 3.0, 0.01
    p = O.make_dem_params(E=E, poisson=nu, adhesive=0, alpha_n=alpha, dt=2e-3, dim=3, n=(64, 64, 64))
    X, U, Om, rad = _two_spheres(v=v, r=r, gap=0.0)
    st = O.DemState(X, U, Om, rad)
    k0 = _kinetic(p, st)
    touched = False
    for _ in range(1000):
        O.dem_step(p, st, substeps=100)
        touched |= st.ncontact > 0
        if touched and st.ncontact == 0:
            break
    assert touched and st.ncontact == 0
    lost = k0 - _kinetic(p, st)
    Es = E / (2 * (1 - nu * nu))
    R = r / 2
    m = p.density * 4 / 3 * math.pi * r ** 3
    ms = m / 2
    dmax = (15 * ms * v * v / (16 * Es * math.sqrt(R))) ** 0.4
    w = lambda d: math.sqrt(max(v * v - 16 / 15 * Es * math.sqrt(R) * d ** 2.5 / ms, 0.0))
    eta = lambda d: alpha * math.sqrt(ms * 2 * Es * math.sqrt(R * d))
    W = 2 * integrate.quad(lambda d: eta(d) * w(d), 0.0, dmax, epsabs=0, epsrel=1e-10, limit=200)[0]
    # the second-order term: the damped trajectory is slower by about half the lost
    # fraction on average, so the damping does about that much less work
    E0 = 0.5 * ms * v * v
    assert k0 == pytest.approx(E0, rel=1e-12)
    assert lost == pytest.approx(W * (1 - W / (2 * E0)), rel=3e-3)


def test_hertz_force_closed_form():
    E, nu = 2.0, 0.3
    p = O.make_dem_params(E=E, poisson=nu, adhesive=0, alpha_n=0.0, dim=3)
    r = np.array([2.0, 3.0])
    d = 0.04
    X = np.array([[10, 10, 10], [10 + 5 - d, 10, 10]], dtype=float)
    fi, ti, fj, tj, h = O.dem_pair_force(p, X, np.zeros((2, 3)), np.zeros((2, 3)), r, 0, 1)
    R = 6.0 / 5.0
    Es = E / (2 * (1 - nu * nu))
    assert -fi[0] == pytest.approx(4 / 3 * Es * math.sqrt(R) * d ** 1.5, rel=1e-12)
    assert np.allclose(fi + fj, 0, atol=1e-18) and np.allclose(ti, 0) and np.allclose(tj, 0)


def test_random_cloud_momentum_conserved_and_contacts_match_brute_force():
    rng = np.random.default_rng(3)
    n = 60
    p = O.make_dem_params(dt=0.05, dim=3, n=(20, 20, 20))
    r = rng.uniform(1.5, 2.5, n)
    X = rng.uniform(0, 20, (n, 3))
    U = rng.normal(0, 1e-3, (n, 3))
    Om = rng.normal(0, 1e-3, (n, 3))
    st = O.DemState(X, U, Om, r)
    # independent enumeration of overlapping pairs (minimum image)
    d = X[None, :, :] - X[:, None, :]
    d -= 20 * np.round(d / 20)
    dist = np.sqrt((d ** 2).sum(-1))
    ov = r[:, None] + r[None, :] - dist
    iu = np.triu_indices(n, 1)
    sel = ov[iu] >= 0
    brute = np.stack([iu[0][sel], iu[1][sel]], 1)
    margin = np.abs(ov[iu]) > 1e-12
    bf = O.pairs_within(p, X, r, 0.0)
    assert set(map(tuple, bf)) ^ set(map(tuple, brute)) <= set(
        (i, j) for i, j, m in zip(iu[0], iu[1], margin) if not m)
    m = p.density * 4 / 3 * math.pi * r ** 3
    P0 = (m[:, None] * st.U).sum(0)
    O.dem_step(p, st, substeps=20)
    assert st.ncontact > 0
    P1 = (m[:, None] * st.U).sum(0)
    assert np.allclose(P1, P0, rtol=0, atol=1e-12 * np.abs(m[:, None] * U).sum())
    pairs, hist = st.contacts()
    assert np.all(pairs[:, 0] < pairs[:, 1])
    key = pairs[:, 0].astype(np.int64) * n + pairs[:, 1]
    assert np.all(np.diff(key) > 0)


def test_sliding_force_capped_at_eq29_critical_value():
    """Two spheres held at fixed overlap with a steady tangential slip: the sliding force
    grows with the spring and saturates at mu_f |F_ne + 2 F_C| (Eq. 28-29)."""
    E, nu, gamma, mu = 2.0, 0.3, 2e-4, 0.3
    p = O.make_dem_params(E=E, poisson=nu, gamma=gamma, mu_f=mu, alpha_n=0.0, eta_t_scale=0.0,
                          dt=0.01, dim=3)
    r = np.array([3.0, 3.0])
    X = np.array([[10, 10, 10], [10 + 6 - 0.01, 10, 10]], dtype=float)
    U = np.array([[0, 1e-3, 0], [0, -1e-3, 0]])
    h = np.zeros(O.NH)
    mags = []
    for _ in range(3000):
        fi, ti, fj, tj, h = O.dem_pair_force(p, X, U, np.zeros((2, 3)), r, 0, 1, h)
        mags.append(abs(fi[1]))
    R, Es = 1.5, E / (2 * (1 - nu * nu))
    FC, a0, dC = _jkr_consts(gamma, R, Es)
    a, _ = O.jkr_contact_radius(0.01, a0, R)
    Fne = O.jkr_force(a, a0, FC)
    crit = mu * abs(Fne + 2 * FC)
    assert mags[0] < 0.2 * crit
    assert mags[-1] == pytest.approx(crit, rel=1e-12)
    assert fi[1] < 0   # opposes i's sliding velocity (+y)
    # torque on i from the tangential force at its contact point r_i n
    assert ti[2] == pytest.approx(3.0 * fi[1], rel=1e-12)


def test_rolling_and_twisting_resist_and_cap():
    E, nu, gamma = 2.0, 0.3, 2e-4
    p = O.make_dem_params(E=E, poisson=nu, gamma=gamma, alpha_n=0.0, theta_crit=0.01, dt=0.01,
                          dim=3)
    r = np.array([3.0, 3.0])
    X = np.array([[10, 10, 10], [10 + 6 - 0.01, 10, 10]], dtype=float)
    # pure rolling of i about z, and twisting about the normal x
    Om = np.array([[0.0, 0.0, 1e-3], [0.0, 0.0, 0.0]])
    h = np.zeros(O.NH)
    for _ in range(5):
        fi, ti, fj, tj, h = O.dem_pair_force(p, X, np.zeros((2, 3)), Om, r, 0, 1, h)
    assert ti[2] < 0   # opposes the relative spin (tangential slip term included)
    R, Es = 1.5, E / (2 * (1 - nu * nu))
    FC, a0, dC = _jkr_consts(gamma, R, Es)
    a, _ = O.jkr_contact_radius(0.01, a0, R)
    for _ in range(20000):
        fi, ti, fj, tj, h = O.dem_pair_force(p, X, np.zeros((2, 3)), Om, r, 0, 1, h)
    Mrcrit = 4 * FC * (a / a0) ** 1.5 * 0.01 * R
    kr = 4 * FC * (a / a0) ** 1.5
    assert kr * np.linalg.norm(h[4:7]) == pytest.approx(Mrcrit, rel=1e-9)
    Omt = np.array([[2e-3, 0.0, 0.0], [0.0, 0.0, 0.0]])
    h = np.zeros(O.NH)
    for _ in range(20000):
        fi, ti, fj, tj, h = O.dem_pair_force(p, X, np.zeros((2, 3)), Omt, r, 0, 1, h)
    Fs = 0.3 * abs(O.jkr_force(a, a0, FC) + 2 * FC)
    assert ti[0] == pytest.approx(-3 * math.pi * a * Fs / 16, rel=1e-9)
    assert tj[0] == pytest.approx(-ti[0], rel=1e-12)


# ------------------------------------------------------------- walls (Sec. 3.5 packing)
def _wall_params(adhesive, alpha_n=0.0, dt=2e-3, gamma=2e-4, n=(32, 32, 40), periodic=(1, 1, 0)):
    return O.make_dem_params(E=2.0, poisson=0.3, gamma=gamma, adhesive=adhesive, alpha_n=alpha_n, dt=dt, dim=3,
                             n=n, periodic=periodic)


@pytest.mark.parametrize("side", ["lower", "upper"])
def test_hertz_sphere_on_a_wall_closed_form(side):
    """A sphere pressed by delta into a wall (plane at -1/2 or n - 1/2) is pushed away with
    the Hertz force 4/3 E* sqrt(r) delta^(3/2) (R = r for a sphere on a plane, reading of the
    wall as a half-space of the same material), and nothing else moves it."""
    p = _wall_params(0)
    r, d = 3.0, 0.05
    z = -0.5 + r - d if side == "lower" else 40 - 0.5 - r + d
    st = O.DemState([[10.0, 11.0, z]], [[0, 0, 0]], [[0, 0, 0]], [r])
    O.dem_step(p, st, substeps=1)
    m = p.density * 4 / 3 * math.pi * r ** 3
    Es = 2.0 / (2 * (1 - 0.3 ** 2))
    F = 4 / 3 * Es * math.sqrt(r) * d ** 1.5
    sign = 1.0 if side == "lower" else -1.0
    assert st.U[0, 2] == pytest.approx(sign * p.dt * F / m, rel=1e-12)
    assert st.U[0, 0] == 0.0 and st.U[0, 1] == 0.0 and np.all(st.Om == 0.0)
    assert st.wflag[0, 2] == 1 and st.wflag[0, 0] == 0 and st.wflag[0, 1] == 0


def test_jkr_sphere_touching_a_wall_jumps_on_with_eight_ninths():
    """JKR on a wall: at delta = 0 the sphere is pulled in with 8/9 F_C, F_C = 3 pi gamma r."""
    gamma, r = 2e-3, 3.0
    p = _wall_params(1, gamma=gamma)
    st = O.DemState([[10.0, 11.0, -0.5 + r]], [[0, 0, 0]], [[0, 0, 0]], [r])
    O.dem_step(p, st, substeps=1)
    m = p.density * 4 / 3 * math.pi * r ** 3
    FC = 3 * math.pi * gamma * r
    assert st.U[0, 2] == pytest.approx(-p.dt * 8 / 9 * FC / m, rel=1e-9)


def test_elastic_bounce_off_a_wall_returns_the_speed():
    """Hertz without damping: the sphere leaves the wall with the speed it came with, and
    the contact ends (no history left)."""
    p = _wall_params(0, dt=5e-3)
    r, v = 3.0, -2e-2
    st = O.DemState([[10.0, 11.0, -0.5 + r + 0.02]], [[0, 0, v]], [[0, 0, 0]], [r])
    touched = False
    for _ in range(400):
        O.dem_step(p, st, substeps=100)
        touched |= bool(st.wflag[0, 2])
        if touched and not st.wflag[0, 2]:
            break
    assert touched and not st.wflag[0, 2] and np.all(st.whist == 0.0)
    assert st.U[0, 2] == pytest.approx(-v, rel=2e-3)


def test_sphere_resting_on_a_wall_under_gravity_settles_at_the_hertz_overlap():
    """Damped Hertz contact with gravity: the sphere comes to rest where the wall force
    carries its weight, m g = 4/3 E* sqrt(r) delta^(3/2)."""
    g = 2e-4
    p = O.make_dem_params(E=2.0, poisson=0.3, adhesive=0, alpha_n=1.5, dt=2e-2, dim=3, n=(32, 32, 40),
                          periodic=(1, 1, 0), gravity=(0, 0, -g))
    r = 3.0
    st = O.DemState([[10.0, 11.0, -0.5 + r + 0.01]], [[0, 0, 0]], [[0, 0, 0]], [r])
    for _ in range(200):
        O.dem_step(p, st, substeps=200)
    m = p.density * 4 / 3 * math.pi * r ** 3
    Es = 2.0 / (2 * (1 - 0.3 ** 2))
    d = (m * g / (4 / 3 * Es * math.sqrt(r))) ** (2 / 3)
    assert abs(st.U[0, 2]) < 1e-9
    assert (-0.5 + r) - st.X[0, 2] == pytest.approx(d, rel=1e-4)
