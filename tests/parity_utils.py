"""Shared helpers of the parity tests: run the same seeded case through the CUDA library
(C ABI) and through the FP64 oracle, and measure relative L2 errors."""
import numpy as np

import oracle as O


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


def oracle_params(case):
    return O.make_params(case["lattice"], *case["n"], bc=case["bc"], tau=case["tau"],
                         body_force=case["body_force"], psc=case.get("psc", 0),
                         shell_h=case.get("shell_h", 1.0), inflow=case.get("inflow", (0.0, 0.0, 0.0)))


def perturbed_state(case, seed, amp=1e-3):
    """Pre-collision populations near rest: w_i (1 + amp * uniform(-1, 1))."""
    rng = np.random.default_rng(seed)
    p = oracle_params(case)
    f = O.equilibrium(p, 1.0, (0, 0, 0)).copy()
    f *= 1.0 + rng.uniform(-amp, amp, size=f.shape)
    return np.ascontiguousarray(f)


def run_oracle(case, f0, steps):
    p = oracle_params(case)
    f = f0.copy()
    F, T = O.run(p, f, steps, case["X"], case["U"], case["Om"], case["r"])
    rho, u = O.macro(p, f)
    return dict(f=f, F=F, T=T, rho=rho, u=u)


def run_gpu(P, case, f0, steps, storage="f32", tile_cap=0):
    ctx = P.lbm_create(case["lattice"], *case["n"], bc=case["bc"], tau=case["tau"],
                       body_force=case["body_force"], storage=storage, psc=case.get("psc", 0),
                       shell_h=case.get("shell_h", 1.0), tile_cap=tile_cap,
                       inflow=case.get("inflow", (0.0, 0.0, 0.0)))
    if f0 is not None:
        P.lbm_set_populations(ctx, f0)
    if len(case["r"]):
        P.lbm_set_particles(ctx, case["X"], case["U"], case["Om"], case["r"])
    P.lbm_step(ctx, steps)
    F, T = P.lbm_get_forces(ctx)
    rho, u = P.lbm_get_macro(ctx)
    f = P.lbm_get_populations(ctx)
    info = P.lbm_get_info(ctx)
    P.lbm_destroy(ctx)
    return dict(f=f, F=F, T=T, rho=rho, u=u, info=info)


def compare(g, o, dim):
    """Relative L2 errors of velocity, density deviation, populations, force, torque."""
    d = dict(
        u=rel_l2(g["u"][..., :dim], o["u"][..., :dim]),
        rho=rel_l2(g["rho"], o["rho"]),
        f=rel_l2(g["f"], o["f"]),
    )
    if o["F"].size:
        d["F"] = rel_l2(g["F"][:, :dim], o["F"][:, :dim])
        tcols = [2] if dim == 2 else [0, 1, 2]
        d["T"] = rel_l2(g["T"][:, tcols], o["T"][:, tcols])
    return d


def ragged_case2d(psc=0, bc=(0, 1, 0), n=(77, 45, 1)):
    """D2Q9, ragged tiles on both axes, walls in y, seven moving and spinning discs that
    straddle the periodic faces, touch the walls and share cells."""
    rng = np.random.default_rng(21)
    X = np.array([[3.2, 20.5, 0], [75.6, 22.0, 0], [30.1, 4.3, 0], [38.9, 9.6, 0],
                  [55.0, 38.7, 0], [61.3, 30.2, 0], [12.4, 36.1, 0]], dtype=float)
    r = np.array([5.5, 4.2, 4.0, 5.1, 4.4, 6.0, 3.3])
    # 0-1 overlap across the periodic x faces (fractions summing above one); 4-5 share
    # cells 0.18 lu apart. The original scheme diverges where fractions overlap (its B_n
    # exceeds one), so its cases move particle 1 to a 0.6 lu gap.
    if psc == 1:
        X[1, 0] = 70.0
    X[X[:, 0] > 69.0, 0] += n[0] - 77      # keep the particles at the high-x face with the box
    U = np.zeros((7, 3)); U[:, :2] = rng.normal(0, 2e-3, (7, 2))
    Om = np.zeros((7, 3)); Om[:, 2] = rng.normal(0, 5e-4, 7)
    return dict(lattice=9, n=n, bc=bc, tau=0.7, body_force=(2e-5, -5e-6, 0.0), X=X, U=U, Om=Om,
                r=r, psc=psc)


def ragged_case3d(psc=0, bc=(0, 0, 1), n=(45, 29, 23)):
    """D3Q19, ragged tiles on every axis, walls in x and y, six moving spheres (one pair
    overlapping, four crossing periodic or wall faces)."""
    rng = np.random.default_rng(22)
    X = np.array([[2.1, 14.0, 11.2], [43.5, 6.2, 9.1], [20.2, 12.5, 4.6], [26.9, 14.1, 6.1],
                  [33.3, 27.6, 15.5], [12.0, 0.4, 17.8]], dtype=float)
    r = np.array([4.5, 3.8, 4.0, 3.9, 5.0, 4.2])   # 2-3 overlap; 0, 1, 4, 5 cross faces
    if psc == 1:
        X[3, 0] = 27.9    # 2-3 at a 0.1 lu gap for the original scheme
    X[X[:, 0] > 40.0, 0] += n[0] - 45      # keep the particles at the high-x face with the box
    U = rng.normal(0, 2e-3, (6, 3))
    Om = rng.normal(0, 5e-4, (6, 3))
    return dict(lattice=19, n=n, bc=bc, tau=0.62, body_force=(1e-5, 2e-6, -3e-6), X=X, U=U, Om=Om,
                r=r, psc=psc)
