"""FP64 CPU oracle for the PSC lattice-Boltzmann step and the adhesive DEM contact update
of Liu & Wu (arXiv 1901.09745).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package. It shares no code with the CUDA library and
the CUDA library never calls it. The arithmetic lives in the C sources beside this file;
this module only marshals numpy arrays through ctypes.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class Params(C.Structure):
    """Mirror of ``ora_params`` in psc_oracle.c."""

    _fields_ = [
        ("lattice", C.c_int),
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("bc", C.c_int * 3),
        ("tau", C.c_double),
        ("body_force", C.c_double * 3),
        ("psc", C.c_int),
        ("shell_h", C.c_double),
        ("inflow", C.c_double * 3),
    ]


def make_params(lattice, nx, ny, nz=1, bc=(0, 0, 0), tau=0.8, body_force=(0.0, 0.0, 0.0),
                psc=0, shell_h=1.0, inflow=(0.0, 0.0, 0.0)):
    p = Params()
    for a in range(3):
        p.inflow[a] = float(inflow[a])
    p.lattice = lattice
    p.nx, p.ny, p.nz = nx, ny, nz
    for a in range(3):
        p.bc[a] = int(bc[a])
        p.body_force[a] = float(body_force[a])
    p.tau = float(tau)
    p.psc = int(psc)
    p.shell_h = float(shell_h)
    return p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        pp = C.POINTER(Params)
        L.ora_lattice_tables.argtypes = [C.c_int, ip, dp, ip]
        L.ora_lattice_tables.restype = C.c_int
        L.ora_va.argtypes = [C.c_int, C.c_double]
        L.ora_va.restype = C.c_double
        L.ora_f_of_r.argtypes = [C.c_int, C.c_double]
        L.ora_f_of_r.restype = C.c_double
        L.ora_B.argtypes = [C.c_double, C.c_double]
        L.ora_B.restype = C.c_double
        L.ora_cell_weights.argtypes = [C.c_int, dp, C.c_double, C.c_int, dp]
        L.ora_cell_weights.restype = C.c_double
        L.ora_solid_fraction.argtypes = [pp, C.c_int, dp, dp, dp, ip, C.c_int, ip, dp]
        L.ora_solid_fraction.restype = C.c_int
        L.ora_macro.argtypes = [pp, dp, dp, dp]
        L.ora_macro.restype = None
        L.ora_step.argtypes = [pp, dp, C.c_int, dp, dp, dp, dp, dp, dp, dp]
        L.ora_step.restype = C.c_int
        L.ora_run.argtypes = [pp, dp, C.c_int, C.c_int, dp, dp, dp, dp, dp, dp]
        L.ora_run.restype = C.c_int
        L.ora_equilibrium.argtypes = [pp, dp, dp, dp]
        L.ora_equilibrium.restype = C.c_int
        _extra_signatures(L)
        _lib = L
    return _lib


class DemParams(C.Structure):
    """Mirror of ``ora_dem_params`` in dem_oracle.c."""

    _fields_ = [
        ("E", C.c_double), ("poisson", C.c_double), ("gamma", C.c_double),
        ("density", C.c_double), ("mu_f", C.c_double), ("theta_crit", C.c_double),
        ("alpha_n", C.c_double), ("k_t_scale", C.c_double), ("eta_t_scale", C.c_double),
        ("dt", C.c_double), ("gravity", C.c_double * 3), ("adhesive", C.c_int), ("dim", C.c_int),
        ("n", C.c_int * 3), ("periodic", C.c_int * 3),
    ]


NH = 7  # history values per contact: sliding spring (3), twist (1), rolling spring (3)


def make_dem_params(E=2.0, poisson=0.3, gamma=2e-4, density=3.0, mu_f=0.3, theta_crit=0.01,
                    alpha_n=0.3, k_t_scale=1.0, eta_t_scale=1.0, dt=0.1, gravity=(0, 0, 0),
                    adhesive=1, dim=3, n=(64, 64, 64), periodic=(1, 1, 1)):
    p = DemParams()
    p.E, p.poisson, p.gamma, p.density = E, poisson, gamma, density
    p.mu_f, p.theta_crit, p.alpha_n = mu_f, theta_crit, alpha_n
    p.k_t_scale, p.eta_t_scale, p.dt = k_t_scale, eta_t_scale, dt
    for a in range(3):
        p.gravity[a] = float(gravity[a])
        p.n[a] = int(n[a])
        p.periodic[a] = int(periodic[a])
    p.adhesive, p.dim = int(adhesive), int(dim)
    return p


def _extra_signatures(L):
    """Signatures of the DEM and adjoint oracle entry points."""
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    pp = C.POINTER(DemParams)
    L.ora_jkr_delta.argtypes = [C.c_double, C.c_double, C.c_double]
    L.ora_jkr_delta.restype = C.c_double
    L.ora_jkr_contact_radius.argtypes = [C.c_double, C.c_double, C.c_double, ip]
    L.ora_jkr_contact_radius.restype = C.c_double
    L.ora_jkr_force.argtypes = [C.c_double, C.c_double, C.c_double]
    L.ora_jkr_force.restype = C.c_double
    L.ora_dem_step.argtypes = [pp, C.c_int, dp, dp, dp, dp, dp, dp, C.c_int, ip, ip, dp, C.c_int, ip, dp]
    L.ora_dem_step.restype = C.c_int
    L.ora_pairs_within.argtypes = [pp, C.c_int, dp, dp, C.c_double, ip, C.c_int]
    L.ora_pairs_within.restype = C.c_int
    L.ora_dem_pair_force.argtypes = [pp, C.c_int, dp, dp, dp, dp, C.c_int, C.c_int, dp, dp, dp, dp, dp]
    L.ora_dem_pair_force.restype = C.c_int
    Pp = C.POINTER(Params)
    L.ora_drag.argtypes = [Pp, dp, C.c_int, C.c_int, dp, dp, dp, dp, dp]
    L.ora_drag.restype = C.c_int


def jkr_delta(a, a0, R):
    return lib().ora_jkr_delta(float(a), float(a0), float(R))


def jkr_force(a, a0, FC):
    return lib().ora_jkr_force(float(a), float(a0), float(FC))


def jkr_contact_radius(delta, a0, R):
    ok = C.c_int()
    a = lib().ora_jkr_contact_radius(float(delta), float(a0), float(R), C.byref(ok))
    return a, bool(ok.value)


class DemState:
    """Particle state plus the contact list (sorted canonical pairs and spring history)."""

    def __init__(self, X, U, Om, r, cap=None):
        self.X = _f64(X).reshape(-1, 3).copy()
        self.U = _f64(U).reshape(-1, 3).copy()
        self.Om = _f64(Om).reshape(-1, 3).copy()
        self.r = _f64(r).reshape(-1).copy()
        n = self.r.size
        self.cap = cap if cap is not None else max(64, 8 * n)
        self.pairs = np.zeros((self.cap, 2), dtype=np.int32)
        self.hist = np.zeros((self.cap, NH))
        self.ncontact = 0
        # wall contacts (non-periodic axes): flag and spring history per particle and axis
        self.wflag = np.zeros((n, 3), dtype=np.int32)
        self.whist = np.zeros((n, 3, NH))

    def contacts(self):
        return self.pairs[: self.ncontact].copy(), self.hist[: self.ncontact].copy()

    def wall_contacts(self):
        """(k, 2) array of (particle, axis) in contact with a wall, sorted, and their histories."""
        idx = np.argwhere(self.wflag != 0).astype(np.int32)
        return idx, np.array([self.whist[i, a] for i, a in idx]).reshape(-1, NH)


def dem_step(p, st, Ff=None, Tf=None, substeps=1):
    n = st.r.size
    Ff = np.zeros((n, 3)) if Ff is None else _f64(Ff).reshape(n, 3)
    Tf = np.zeros((n, 3)) if Tf is None else _f64(Tf).reshape(n, 3)
    nc = C.c_int(st.ncontact)
    rc = lib().ora_dem_step(C.byref(p), n, _d(st.X), _d(st.U), _d(st.Om), _d(st.r), _d(Ff), _d(Tf),
                            int(substeps), C.byref(nc), _i(st.pairs), _d(st.hist), st.cap, _i(st.wflag),
                            _d(st.whist))
    st.ncontact = nc.value
    _check(rc, "dem_step")
    return st


def pairs_within(p, X, r, thresh=0.0, cap=100000):
    X = _f64(X).reshape(-1, 3)
    r = _f64(r).reshape(-1)
    out = np.zeros((cap, 2), dtype=np.int32)
    k = lib().ora_pairs_within(C.byref(p), r.size, _d(X), _d(r), float(thresh), _i(out), cap)
    if k < 0:
        raise RuntimeError("pair capacity exceeded")
    return out[:k].copy()


def dem_pair_force(p, X, U, Om, r, i, j, hist=None):
    X, U, Om = (_f64(a).reshape(-1, 3) for a in (X, U, Om))
    r = _f64(r).reshape(-1)
    h = np.zeros(NH) if hist is None else hist
    assert h.dtype == np.float64 and h.flags.c_contiguous
    fi, ti, fj, tj = (np.zeros(3) for _ in range(4))
    rc = lib().ora_dem_pair_force(C.byref(p), r.size, _d(X), _d(U), _d(Om), _d(r), int(i), int(j),
                                  _d(h), _d(fi), _d(ti), _d(fj), _d(tj))
    _check(rc, "dem_pair_force")
    return fi, ti, fj, tj, h


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def lattice_tables(lattice):
    e = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19, dtype=np.float64)
    opp = np.zeros(19, dtype=np.int32)
    q = lib().ora_lattice_tables(lattice, _i(e), _d(w), _i(opp))
    if q < 0:
        raise ValueError("unknown lattice %r" % lattice)
    return e[:q].copy(), w[:q].copy(), opp[:q].copy()


def va(dim, r):
    return lib().ora_va(dim, float(r))


def f_of_r(dim, r):
    return lib().ora_f_of_r(dim, float(r))


def B(eps, tau):
    return lib().ora_B(float(eps), float(tau))


def cell_weights(eps, tau, mode=0):
    eps = _f64(eps)
    Bs = np.zeros(max(1, eps.size), dtype=np.float64)
    Bn = lib().ora_cell_weights(eps.size, _d(eps), float(tau), int(mode), _d(Bs))
    return Bn, Bs[: eps.size]


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def _particles(X, U=None, Om=None, rad=None):
    X = _f64(X).reshape(-1, 3)
    n = X.shape[0]
    U = np.zeros((n, 3)) if U is None else _f64(U).reshape(n, 3)
    Om = np.zeros((n, 3)) if Om is None else _f64(Om).reshape(n, 3)
    rad = _f64(rad).reshape(n)
    return np.ascontiguousarray(X), np.ascontiguousarray(U), np.ascontiguousarray(Om), rad


def solid_fraction(p, X, rad, maxk=8):
    X = _f64(X).reshape(-1, 3)
    rad = _f64(rad).reshape(-1)
    ncell = p.nx * p.ny * p.nz
    eps_sum = np.zeros(ncell)
    nrec = np.zeros(ncell, dtype=np.int32)
    pid = np.zeros(ncell * maxk, dtype=np.int32)
    eps = np.zeros(ncell * maxk)
    rc = lib().ora_solid_fraction(C.byref(p), X.shape[0], _d(X), _d(rad), _d(eps_sum),
                                  _i(nrec), maxk, _i(pid), _d(eps))
    _check(rc, "solid_fraction")
    return eps_sum, nrec, pid.reshape(ncell, maxk), eps.reshape(ncell, maxk)


def equilibrium(p, rho, u):
    ncell = p.nx * p.ny * p.nz
    q = p.lattice
    rho = _f64(np.broadcast_to(np.asarray(rho, dtype=np.float64), (ncell,)))
    u = _f64(np.broadcast_to(np.asarray(u, dtype=np.float64), (ncell, 3)))
    f = np.zeros(q * ncell)
    _check(lib().ora_equilibrium(C.byref(p), _d(rho), _d(u), _d(f)), "equilibrium")
    return f.reshape(q, p.nz, p.ny, p.nx)


def macro(p, f):
    ncell = p.nx * p.ny * p.nz
    f = _f64(f)
    rho = np.zeros(ncell)
    u = np.zeros((ncell, 3))
    lib().ora_macro(C.byref(p), _d(f), _d(rho), _d(u))
    return rho.reshape(p.nz, p.ny, p.nx), u.reshape(p.nz, p.ny, p.nx, 3)


def step(p, f, X, U=None, Om=None, rad=None, want_Bn=False):
    """One collide+stream step. ``f`` (Q, nz, ny, nx) is updated in place."""
    assert f.dtype == np.float64 and f.flags.c_contiguous
    if rad is None:
        X = np.zeros((0, 3)); rad = np.zeros(0)
    X, U, Om, rad = _particles(X, U, Om, rad)
    n = X.shape[0]
    F = np.zeros((max(n, 1), 3)); T = np.zeros((max(n, 1), 3))
    ncell = p.nx * p.ny * p.nz
    Bn = np.zeros(ncell) if want_Bn else None
    rc = lib().ora_step(C.byref(p), _d(f), n, _d(X), _d(U), _d(Om), _d(rad), _d(F), _d(T),
                        _d(Bn) if want_Bn else None)
    _check(rc, "step")
    if want_Bn:
        return F[:n], T[:n], Bn.reshape(p.nz, p.ny, p.nx)
    return F[:n], T[:n]


def run(p, f, nsteps, X=None, U=None, Om=None, rad=None):
    """``nsteps`` steps with static particles; returns the last step's F, T."""
    assert f.dtype == np.float64 and f.flags.c_contiguous
    if rad is None:
        X = np.zeros((0, 3)); rad = np.zeros(0)
    X, U, Om, rad = _particles(X, U, Om, rad)
    n = X.shape[0]
    F = np.zeros((max(n, 1), 3)); T = np.zeros((max(n, 1), 3))
    rc = lib().ora_run(C.byref(p), _d(f), int(nsteps), n, _d(X), _d(U), _d(Om), _d(rad),
                       _d(F), _d(T))
    _check(rc, "run")
    return F[:n], T[:n]


def drag(p, f0, nsteps, X, rad, U=None, Om=None):
    """J = (1/T) sum_t sum_p F_{p,x}(t) over nsteps from a copy of f0 (static particles)."""
    f = np.ascontiguousarray(np.array(f0, dtype=np.float64))
    X, U, Om, rad = _particles(X, U, Om, rad)
    J = np.zeros(1)
    _check(lib().ora_drag(C.byref(p), _d(f), int(nsteps), X.shape[0], _d(X), _d(U), _d(Om), _d(rad), _d(J)),
           "drag")
    return float(J[0])
