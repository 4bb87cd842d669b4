"""Python binding of the GB300 PSC lattice-Boltzmann / JKR-DEM library.

The library is a C-ABI shared object (``include/psc_lbm.h``) built from the CUDA sources in
``csrc/`` for sm_103a by ``build.py``. This module only marshals arguments: every step of the
computation runs in the library's CUDA kernels. The functions keep the C names
(``lbm_create``, ``lbm_set_particles``, ``lbm_step``, ``lbm_get_forces``, ``dem_step``, ...).

Arrays may be numpy arrays (host memory) or CUDA torch tensors (device memory, passed by
pointer with ``on_device = 1``). Importing this module does not need a GPU; creating a
context does. If the shared library is missing the import fails loudly: there is no CPU
fallback.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PSC_LBM_CHECKED=1 selects the bounds-checked build (build.build(checked=True))
LIB_PATH = os.path.join(_HERE, "_lib", "libpsc_lbm_checked.so" if os.environ.get("PSC_LBM_CHECKED") == "1"
                        else "libpsc_lbm.so")
INCLUDE = os.path.join(os.path.dirname(_HERE), "include", "psc_lbm.h")

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_UNSUPPORTED = 0, 1, 2, 3, 4
LBM_ERR_UNSTABLE, LBM_ERR_OVERFLOW, LBM_ERR_TIMEOUT, DEM_ERR_NO_CONVERGENCE = 5, 6, 7, 8
LBM_D2Q9, LBM_D3Q19 = 9, 19
LBM_BC_PERIODIC, LBM_BC_BOUNCEBACK, LBM_BC_OPEN, LBM_BC_INFLOW = 0, 1, 2, 3
LBM_F64, LBM_F32, LBM_F16_DEV, LBM_BF16_DEV = 0, 1, 2, 3
LBM_PSC_MODIFIED, LBM_PSC_ORIGINAL = 0, 1
STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16_DEV, "bf16": LBM_BF16_DEV}

_STATUS_NAMES = {
    0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_CUDA", 3: "LBM_ERR_OOM", 4: "LBM_ERR_UNSUPPORTED",
    5: "LBM_ERR_UNSTABLE", 6: "LBM_ERR_OVERFLOW", 7: "LBM_ERR_TIMEOUT", 8: "DEM_ERR_NO_CONVERGENCE",
}


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, str(status)), message))
        self.status = status


class LbmParams(C.Structure):
    """Mirror of ``lbm_params``."""

    _fields_ = [
        ("lattice", C.c_int),
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("bc", C.c_int * 3),
        ("tau", C.c_double),
        ("body_force", C.c_double * 3),
        ("storage", C.c_int),
        ("psc", C.c_int),
        ("shell_h", C.c_double),
        ("dev_scale", C.c_double),
        ("tile_cap", C.c_int),
        ("stream", C.c_void_p),
        ("inflow", C.c_double * 3),
    ]


class DemParams(C.Structure):
    """Mirror of ``dem_params``."""

    _fields_ = [
        ("E", C.c_double), ("poisson", C.c_double), ("gamma", C.c_double),
        ("density", C.c_double), ("mu_f", C.c_double), ("theta_crit", C.c_double),
        ("alpha_n", C.c_double), ("k_t_scale", C.c_double), ("eta_t_scale", C.c_double),
        ("dt_dem", C.c_double), ("gravity", C.c_double * 3), ("adhesive", C.c_int),
        ("skin", C.c_double),
    ]


_lib = None


def library_path():
    return LIB_PATH


def lib():
    """Load the CUDA library (building it first if the sources are newer is the caller's
    job: ``paper_1901_09745_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("CUDA library %s is missing: run paper_1901_09745_gb300/build.py "
                          "(there is no CPU fallback)" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    sig = {
        "lbm_create": ([C.POINTER(LbmParams), C.POINTER(C.c_void_p)], C.c_int),
        "lbm_destroy": ([vp], C.c_int),
        "lbm_set_particles": ([vp, C.c_int, vp, vp, vp, vp, C.c_int], C.c_int),
        "lbm_step": ([vp, C.c_int], C.c_int),
        "lbm_get_forces": ([vp, vp, vp, C.c_int], C.c_int),
        "lbm_get_macro": ([vp, vp, vp, C.c_int], C.c_int),
        "lbm_get_populations": ([vp, vp, C.c_int], C.c_int),
        "lbm_set_populations": ([vp, vp, C.c_int], C.c_int),
        "lbm_save_state": ([vp, vp, C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
        "lbm_load_state": ([vp, vp, C.c_size_t], C.c_int),
        "lbm_get_info": ([vp, C.POINTER(C.c_longlong), C.c_int], C.c_int),
        "lbm_lattice_tables": ([C.c_int, ip, dp, ip], C.c_int),
        "lbm_last_error": ([vp], C.c_char_p),
        "lbm_kernel_timing": ([vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)], C.c_int),
        "lbm_set_body_force": ([vp, vp], C.c_int),
        "lbm_adjoint_drag": ([vp, C.c_int, C.c_int, vp, vp, vp, C.c_int], C.c_int),
        "lbm_checked_build": ([], C.c_int),
        "lbm_check_violations": ([C.POINTER(C.c_uint)], C.c_int),
        "lbm_adjoint_forward": ([vp, C.c_int, C.c_int, vp, vp, C.c_int], C.c_int),
        "lbm_adjoint_backward": ([vp, C.c_longlong, vp, vp, C.c_int], C.c_int),
    }
    optional = {
        "dem_create": ([C.POINTER(DemParams), vp, C.POINTER(C.c_void_p)], C.c_int),
        "dem_destroy": ([vp], C.c_int),
        "dem_step": ([vp, C.c_int], C.c_int),
        "dem_get_contacts": ([vp, vp, vp, C.c_int, C.POINTER(C.c_int)], C.c_int),
        "dem_get_particles": ([vp, vp, vp, vp, C.c_int], C.c_int),
        "dem_get_info": ([vp, C.POINTER(C.c_longlong), C.c_int], C.c_int),
        "lbm_coupled_step": ([vp, vp, C.c_int, C.c_int], C.c_int),
        "dem_get_wall_contacts": ([vp, vp, vp, C.c_int, C.POINTER(C.c_int)], C.c_int),
        "lbm_psc_step_noalloc": ([C.POINTER(LbmParams), vp, vp, C.c_int, vp, vp, vp, vp, vp, vp], C.c_int),
        "lbm_decomp_layout": ([C.c_int, C.c_int, C.c_int, C.c_int, ip, ip, ip], C.c_int),
        "lbm_decomp_assign": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, dp, dp, ip], C.c_int),
        "lbm_decomp_create": ([C.POINTER(LbmParams), C.c_int, C.POINTER(C.c_void_p)], C.c_int),
        "lbm_decomp_destroy": ([vp], C.c_int),
        "lbm_decomp_set_particles": ([vp, C.c_int, vp, vp, vp, vp], C.c_int),
        "lbm_decomp_set_populations": ([vp, vp], C.c_int),
        "lbm_decomp_get_populations": ([vp, vp], C.c_int),
        "lbm_decomp_step": ([vp, C.c_int], C.c_int),
        "lbm_decomp_get_forces": ([vp, vp, vp], C.c_int),
        "lbm_decomp_last_error": ([vp], C.c_char_p),
        "lbm_noalloc_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes, fn.restype = args, res
    for name, (args, res) in optional.items():
        if hasattr(L, name):
            fn = getattr(L, name)
            fn.argtypes, fn.restype = args, res
    _lib = L
    return L


def exported_symbols():
    """Names declared in include/*.h: ``lbm_*`` / ``dem_*`` (psc_lbm.h) and the host test
    entries ``psc_test_*`` (psc_testing.h)."""
    import glob
    import re
    names = set()
    for path in glob.glob(os.path.join(os.path.dirname(INCLUDE), "*.h")):
        with open(path) as fh:
            names.update(re.findall(r"\b((?:lbm|dem|psc_test)_[a-z_0-9]+)\s*\(", fh.read()))
    return sorted(names)


# ------------------------------------------------------------------ marshalling helpers
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype=np.float64):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    if a is None:
        return None, 0, None
    if _is_torch(a):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError("tensor must be contiguous %s" % want)
        return C.c_void_p(a.data_ptr()), int(a.is_cuda), a
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    return arr.ctypes.data_as(C.c_void_p), 0, arr


def _check(ctx, status):
    if status != LBM_OK:
        msg = lib().lbm_last_error(ctx.handle if ctx is not None else None)
        raise LbmError(status, msg.decode() if msg else "")


class Lbm:
    """Owner of one ``lbm_ctx`` handle (destroyed with the object)."""

    def __init__(self, handle, params):
        self.handle = handle
        self.params = params
        self.np = 0

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.lbm_destroy(h)

    @property
    def q(self):
        return self.params.lattice

    @property
    def shape(self):
        return (self.params.nz, self.params.ny, self.params.nx)


# ------------------------------------------------------------------------ the C calls
def lbm_create(lattice, nx, ny, nz=1, bc=(0, 0, 0), tau=0.8, body_force=(0.0, 0.0, 0.0),
               storage="f32", psc=LBM_PSC_MODIFIED, shell_h=1.0, dev_scale=0.0, tile_cap=0,
               stream=None, inflow=(0.0, 0.0, 0.0)):
    p = LbmParams()
    for a in range(3):
        p.inflow[a] = float(inflow[a])
    p.lattice = int(lattice)
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    for a in range(3):
        p.bc[a] = int(bc[a])
        p.body_force[a] = float(body_force[a])
    p.tau = float(tau)
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.psc = int(psc)
    p.shell_h = float(shell_h)
    p.dev_scale = float(dev_scale)
    p.tile_cap = int(tile_cap)
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            stream = None
    p.stream = C.c_void_p(stream) if stream else None
    h = C.c_void_p()
    st = lib().lbm_create(C.byref(p), C.byref(h))
    if st != LBM_OK:
        raise LbmError(st, lib().lbm_last_error(None).decode())
    return Lbm(h, p)


def lbm_destroy(ctx):
    if ctx.handle:
        lib().lbm_destroy(ctx.handle)
        ctx.handle = None


def lbm_set_particles(ctx, X, U, Om, radius):
    n = len(radius)
    ptrs = [_ptr(a) for a in (X, U, Om, radius)]
    dev = {d for _, d, _ in ptrs}
    if len(dev) != 1:
        raise TypeError("particle arrays must all live on the host or all on the device")
    _check(ctx, lib().lbm_set_particles(ctx.handle, int(n), ptrs[0][0], ptrs[1][0], ptrs[2][0],
                                        ptrs[3][0], dev.pop()))
    ctx.np = int(n)


def lbm_step(ctx, nsteps=1):
    _check(ctx, lib().lbm_step(ctx.handle, int(nsteps)))


def lbm_get_forces(ctx, F=None, T=None):
    """Returns (F, T) as (n, 3) arrays; fills the given arrays/tensors when provided."""
    if F is None:
        F = np.zeros((ctx.np, 3))
    if T is None:
        T = np.zeros((ctx.np, 3))
    pf, df, kf = _ptr(F)
    pt, dt, kt = _ptr(T)
    if df != dt:
        raise TypeError("F and T must both be host or both device")
    _check(ctx, lib().lbm_get_forces(ctx.handle, pf, pt, df))
    if not _is_torch(F) and kf is not F:
        F[...] = kf
    if not _is_torch(T) and kt is not T:
        T[...] = kt
    return F, T


def lbm_get_macro(ctx, rho=None, u=None):
    nz, ny, nx = ctx.shape
    if rho is None:
        rho = np.zeros((nz, ny, nx))
    if u is None:
        u = np.zeros((nz, ny, nx, 3))
    pr, dr, _ = _ptr(rho)
    pu, du, _ = _ptr(u)
    _check(ctx, lib().lbm_get_macro(ctx.handle, pr, pu, dr))
    return rho, u


def lbm_get_populations(ctx, f=None):
    nz, ny, nx = ctx.shape
    if f is None:
        f = np.zeros((ctx.q, nz, ny, nx))
    p, d, _ = _ptr(f)
    _check(ctx, lib().lbm_get_populations(ctx.handle, p, d))
    return f


def lbm_set_populations(ctx, f):
    p, d, keep = _ptr(f)
    _check(ctx, lib().lbm_set_populations(ctx.handle, p, d))


def lbm_save_state(ctx):
    used = C.c_size_t()
    _check(ctx, lib().lbm_save_state(ctx.handle, None, 0, C.byref(used)))
    buf = (C.c_char * used.value)()
    _check(ctx, lib().lbm_save_state(ctx.handle, C.cast(buf, C.c_void_p), used.value, C.byref(used)))
    return bytes(buf)


def lbm_load_state(ctx, state):
    buf = C.create_string_buffer(state, len(state))
    _check(ctx, lib().lbm_load_state(ctx.handle, C.cast(buf, C.c_void_p), len(state)))


def lbm_get_info(ctx):
    out = (C.c_longlong * 6)()
    _check(ctx, lib().lbm_get_info(ctx.handle, out, 6))
    return dict(steps=out[0], overflow_tiles=out[1], max_tile_candidates=out[2], particles=out[3],
                launches=out[4], collide_stream_launches=out[5])


def lbm_checked_build():
    """True when the loaded library is the bounds-checked build."""
    return bool(lib().lbm_checked_build())


def lbm_check_violations():
    """Bits of the index checks that failed since the last call (bounds-checked build
    only; see the header), then cleared."""
    w = C.c_uint()
    st = lib().lbm_check_violations(C.byref(w))
    if st != LBM_OK:
        raise LbmError(st, "lbm_check_violations: not a bounds-checked build" if st == LBM_ERR_UNSUPPORTED else "")
    return w.value


def lbm_kernel_timing(ctx, enable):
    """(ms_total, launches) of the collide-stream launches timed since the last call; then
    switch timing on or off."""
    ms = C.c_double()
    n = C.c_longlong()
    _check(ctx, lib().lbm_kernel_timing(ctx.handle, int(enable), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def lbm_lattice_tables(lattice):
    e = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    o = np.zeros(19, dtype=np.int32)
    q = lib().lbm_lattice_tables(int(lattice), e.ctypes.data_as(C.POINTER(C.c_int)),
                                 w.ctypes.data_as(C.POINTER(C.c_double)),
                                 o.ctypes.data_as(C.POINTER(C.c_int)))
    if q < 0:
        raise ValueError("unknown lattice")
    return e[:q].copy(), w[:q].copy(), o[:q].copy()


# ---------------------------------------------------------------------------------- DEM
class Dem:
    """Owner of one ``dem_ctx`` handle, attached to a fluid context."""

    def __init__(self, handle, fluid):
        self.handle = handle
        self.fluid = fluid

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None and getattr(self.fluid, "handle", None):
            _lib.dem_destroy(h)


def dem_create(fluid, E=2.0, poisson=0.3, gamma=2e-4, density=3.0, mu_f=0.3, theta_crit=0.01,
               alpha_n=0.3, k_t_scale=1.0, eta_t_scale=1.0, dt_dem=0.1, gravity=(0.0, 0.0, 0.0),
               adhesive=1, skin=0.5):
    p = DemParams()
    p.E, p.poisson, p.gamma, p.density = E, poisson, gamma, density
    p.mu_f, p.theta_crit, p.alpha_n = mu_f, theta_crit, alpha_n
    p.k_t_scale, p.eta_t_scale, p.dt_dem = k_t_scale, eta_t_scale, dt_dem
    for a in range(3):
        p.gravity[a] = float(gravity[a])
    p.adhesive = int(adhesive)
    p.skin = float(skin)
    h = C.c_void_p()
    _check(fluid, lib().dem_create(C.byref(p), fluid.handle, C.byref(h)))
    return Dem(h, fluid)


def dem_destroy(dem):
    if dem.handle:
        lib().dem_destroy(dem.handle)
        dem.handle = None


def dem_step(dem, substeps=1):
    _check(dem.fluid, lib().dem_step(dem.handle, int(substeps)))


def lbm_coupled_step(ctx, dem, nsteps=1, substeps=1):
    """nsteps of lbm_step(ctx, 1) + dem_step(dem, substeps), fused where the library can."""
    _check(ctx, lib().lbm_coupled_step(ctx.handle, dem.handle, int(nsteps), int(substeps)))


def dem_get_particles(dem, X=None, U=None, Om=None):
    n = dem.fluid.np
    X = np.zeros((n, 3)) if X is None else X
    U = np.zeros((n, 3)) if U is None else U
    Om = np.zeros((n, 3)) if Om is None else Om
    px, dx, _ = _ptr(X)
    pu, du, _ = _ptr(U)
    po, do, _ = _ptr(Om)
    _check(dem.fluid, lib().dem_get_particles(dem.handle, px, pu, po, dx))
    return X, U, Om


def dem_get_contacts(dem, cap=None):
    """Sorted canonical pairs (k, 2) and their history seen from i (k, 7)."""
    n = C.c_int()
    cap = cap or max(16, 16 * dem.fluid.np)
    pairs = np.zeros((cap, 2), dtype=np.int32)
    hist = np.zeros((cap, 7))
    st = lib().dem_get_contacts(dem.handle, pairs.ctypes.data_as(C.c_void_p),
                                hist.ctypes.data_as(C.c_void_p), cap, C.byref(n))
    _check(dem.fluid, st)
    return pairs[: n.value].copy(), hist[: n.value].copy()


def dem_get_wall_contacts(dem, cap=None):
    """(k, 2) array of (particle, axis) in contact with a wall, and their histories (k, 7)."""
    n = C.c_int()
    cap = cap or max(16, 3 * dem.fluid.np)
    pw = np.zeros((cap, 2), dtype=np.int32)
    hist = np.zeros((cap, 7))
    st = lib().dem_get_wall_contacts(dem.handle, pw.ctypes.data_as(C.c_void_p), hist.ctypes.data_as(C.c_void_p),
                                     cap, C.byref(n))
    _check(dem.fluid, st)
    return pw[: n.value].copy(), hist[: n.value].copy()


def dem_get_info(dem):
    out = (C.c_longlong * 6)()
    _check(dem.fluid, lib().dem_get_info(dem.handle, out, 6))
    return dict(launches=out[0], solve_failures=out[1], overflows=out[2], skin_violations=out[3],
                particles=out[4], rebuilds=out[5])


# ------------------------------------------------------------ step without device allocation
def lbm_psc_step_noalloc(params, f_in, f_out, X=None, U=None, Om=None, radius=None, F=None, T=None):
    """One PSC step on caller-owned device tensors, allocating nothing (see the header).
    ``params`` is an ``LbmParams`` (e.g. ``ctx.params``); every array is a CUDA tensor."""
    n = 0 if radius is None else int(radius.numel())
    ptr = lambda a: None if a is None else C.c_void_p(a.data_ptr())
    st = lib().lbm_psc_step_noalloc(C.byref(params), ptr(f_in), ptr(f_out), n, ptr(X), ptr(U), ptr(Om),
                                    ptr(radius), ptr(F), ptr(T))
    if st != LBM_OK:
        raise LbmError(st, lib().lbm_noalloc_last_error().decode())


# --------------------------------------------------------------------------------- adjoint
def lbm_set_body_force(ctx, F):
    F = np.ascontiguousarray(np.asarray(F, dtype=np.float64).reshape(3))
    _check(ctx, lib().lbm_set_body_force(ctx.handle, F.ctypes.data_as(C.c_void_p)))
    ctx.params.body_force[0], ctx.params.body_force[1], ctx.params.body_force[2] = (float(v) for v in F)


def lbm_adjoint_drag(ctx, nsteps, checkpoint_every):
    """(J, dJ/dX (n, 3), dJ/dF (3,)) of the time-averaged x-drag over the next nsteps."""
    J = np.zeros(1)
    dX = np.zeros((max(ctx.np, 1), 3))
    dF = np.zeros(3)
    _check(ctx, lib().lbm_adjoint_drag(ctx.handle, int(nsteps), int(checkpoint_every),
                                       J.ctypes.data_as(C.c_void_p), dX.ctypes.data_as(C.c_void_p),
                                       dF.ctypes.data_as(C.c_void_p), 0))
    return float(J[0]), dX[: ctx.np].copy(), dF


def lbm_adjoint_forward(ctx, nsteps, checkpoint_every):
    """(J, token): the forward half of lbm_adjoint_drag (see the header)."""
    J = np.zeros(1)
    tok = C.c_longlong()
    _check(ctx, lib().lbm_adjoint_forward(ctx.handle, int(nsteps), int(checkpoint_every),
                                          J.ctypes.data_as(C.c_void_p), C.byref(tok), 0))
    return float(J[0]), tok.value


def lbm_adjoint_backward(ctx, token):
    """(dJ/dX (n, 3), dJ/dF (3,)): the reverse sweep over the checkpoints of the forward
    half that returned ``token``."""
    dX = np.zeros((max(ctx.np, 1), 3))
    dF = np.zeros(3)
    _check(ctx, lib().lbm_adjoint_backward(ctx.handle, C.c_longlong(int(token)), dX.ctypes.data_as(C.c_void_p),
                                           dF.ctypes.data_as(C.c_void_p), 0))
    return dX[: ctx.np].copy(), dF


def psc_drag(ctx, f0, X, radius, F, nsteps, checkpoint_every):
    """Differentiable time-averaged drag: a torch scalar J(X, F). The forward pass runs the
    library's forward half (T steps with checkpoints); the backward pass, only when a
    gradient is asked for, runs the reverse sweep over those checkpoints. ``ctx`` is a
    context whose particles are static; ``f0`` (numpy, pre-collision populations) is the
    initial state of every evaluation. Each evaluation takes the context's adjoint
    workspace, so the backward of an earlier evaluation after a later forward raises."""
    import torch

    class _PscDrag(torch.autograd.Function):
        @staticmethod
        def forward(actx, Xt, Ft):
            lbm_set_body_force(ctx, Ft.detach().cpu().numpy())
            lbm_set_populations(ctx, f0)
            Xn = Xt.detach().cpu().numpy()
            z = np.zeros_like(Xn)
            lbm_set_particles(ctx, Xn, z, z, np.asarray(radius, dtype=np.float64))
            J, token = lbm_adjoint_forward(ctx, nsteps, checkpoint_every)
            actx.token = token
            actx.meta = (Xt.dtype, Xt.device, Ft.dtype, Ft.device)
            return torch.as_tensor(J, dtype=Xt.dtype, device=Xt.device)

        @staticmethod
        def backward(actx, g):
            dX, dF = lbm_adjoint_backward(ctx, actx.token)
            xd, xdev, fd, fdev = actx.meta
            return (g * torch.as_tensor(dX, dtype=xd, device=xdev), g * torch.as_tensor(dF, dtype=fd, device=fdev))

    return _PscDrag.apply(X, F)


# ----------------------------------------------------------------------- slab decomposition
NOT_HELD = -99


def lbm_decomp_layout(lattice, n_s, periodic_s, nslab):
    """(own, ghost_lo, ghost_hi): the rows each slab owns (own[k] .. own[k+1] - 1) and its
    ghost layers below and above (see the header)."""
    own = (C.c_int * (nslab + 1))()
    glo = (C.c_int * max(nslab, 1))()
    ghi = (C.c_int * max(nslab, 1))()
    if lib().lbm_decomp_layout(int(lattice), int(n_s), int(bool(periodic_s)), int(nslab), own, glo, ghi) != 0:
        raise ValueError("no slab layout for %d rows in %d slabs" % (n_s, nslab))
    return list(own), list(glo)[:nslab], list(ghi)[:nslab]


def lbm_decomp_assign(lattice, n_s, periodic_s, nslab, c, radius, shell_h=1.0):
    """(nslab, n) int array: the periodic image m of each particle a slab holds, or NOT_HELD."""
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1))
    r = np.ascontiguousarray(np.asarray(radius, dtype=np.float64).reshape(-1))
    img = np.zeros((nslab, c.size), dtype=np.int32)
    st = lib().lbm_decomp_assign(int(lattice), int(n_s), int(bool(periodic_s)), int(nslab), float(shell_h), c.size,
                                 c.ctypes.data_as(C.POINTER(C.c_double)), r.ctypes.data_as(C.POINTER(C.c_double)),
                                 img.ctypes.data_as(C.POINTER(C.c_int)))
    if st != 0:
        raise ValueError("no particle assignment (layout invalid or a slab thinner than a shell)")
    return img


class Decomp:
    """Owner of one ``lbm_decomp`` handle."""

    def __init__(self, handle, params, nslab):
        self.handle, self.params, self.nslab, self.np = handle, params, nslab, 0

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.lbm_decomp_destroy(h)

    @property
    def shape(self):
        return (self.params.nz, self.params.ny, self.params.nx)


def _dcheck(d, status):
    if status != LBM_OK:
        msg = lib().lbm_decomp_last_error(d.handle if d is not None else None)
        raise LbmError(status, msg.decode() if msg else "")


def lbm_decomp_create(lattice, nx, ny, nz, nslab, bc=(0, 0, 0), tau=0.8, body_force=(0.0, 0.0, 0.0), storage="f32",
                      psc=LBM_PSC_MODIFIED, shell_h=1.0, dev_scale=0.0, tile_cap=0, stream=None):
    p = LbmParams()
    p.lattice = int(lattice)
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    for a in range(3):
        p.bc[a] = int(bc[a])
        p.body_force[a] = float(body_force[a])
    p.tau = float(tau)
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.psc, p.shell_h, p.dev_scale, p.tile_cap = int(psc), float(shell_h), float(dev_scale), int(tile_cap)
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            stream = None
    p.stream = C.c_void_p(stream) if stream else None
    h = C.c_void_p()
    st = lib().lbm_decomp_create(C.byref(p), int(nslab), C.byref(h))
    if st != LBM_OK:
        raise LbmError(st, lib().lbm_decomp_last_error(None).decode())
    return Decomp(h, p, int(nslab))


def lbm_decomp_destroy(d):
    if d.handle:
        lib().lbm_decomp_destroy(d.handle)
        d.handle = None


def lbm_decomp_set_particles(d, X, U, Om, radius):
    X, U, Om = (np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, 3)) for a in (X, U, Om))
    r = np.ascontiguousarray(np.asarray(radius, dtype=np.float64).reshape(-1))
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    _dcheck(d, lib().lbm_decomp_set_particles(d.handle, r.size, vp(X), vp(U), vp(Om), vp(r)))
    d.np = r.size


def lbm_decomp_set_populations(d, f):
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    _dcheck(d, lib().lbm_decomp_set_populations(d.handle, f.ctypes.data_as(C.c_void_p)))


def lbm_decomp_get_populations(d):
    nz, ny, nx = d.shape
    f = np.zeros((d.params.lattice, nz, ny, nx))
    _dcheck(d, lib().lbm_decomp_get_populations(d.handle, f.ctypes.data_as(C.c_void_p)))
    return f


def lbm_decomp_step(d, nsteps=1):
    _dcheck(d, lib().lbm_decomp_step(d.handle, int(nsteps)))


def lbm_decomp_get_forces(d):
    F = np.zeros((d.np, 3))
    T = np.zeros((d.np, 3))
    _dcheck(d, lib().lbm_decomp_get_forces(d.handle, F.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p)))
    return F, T
