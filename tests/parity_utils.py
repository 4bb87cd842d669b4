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
                         shell_h=case.get("shell_h", 1.0))


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
                       shell_h=case.get("shell_h", 1.0), tile_cap=tile_cap)
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
