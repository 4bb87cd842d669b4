"""Runs representative cases through the bounds-checked build (started by
test_gpu_checked.py with PSC_LBM_CHECKED=1): the pair kernels in 2D and 3D with walls,
ragged tiles and overlapping particles (FP32 and FP16), the overflow path, an inlet box
(the faces kernel), two slabs of a decomposed lattice, a DEM call with walls, and the
adjoint. Prints one JSON line: the check bits and the parity errors against the oracle."""
import json
import sys

import numpy as np

import oracle as O
from parity_utils import compare, perturbed_state, ragged_case2d, ragged_case3d, run_gpu, run_oracle

import paper_1901_09745_gb300 as P

assert P.lbm_checked_build(), "not the bounds-checked library"
P.lbm_check_violations()
out = {"errors": {}}

for name, case, storage in (("2d_f32", ragged_case2d(), "f32"), ("3d_f32", ragged_case3d(), "f32"),
                            ("3d_f16", ragged_case3d(), "f16")):
    f0 = perturbed_state(case, 3)
    o = run_oracle(case, f0, 6)
    g = run_gpu(P, case, f0, 6, storage=storage)
    out["errors"][name] = compare(g, o, 2 if case["lattice"] == 9 else 3)
    out.setdefault("bits", {})[name] = P.lbm_check_violations()
# the exact chunked path over all particles (every tile overflows)
case = ragged_case3d()
f0 = perturbed_state(case, 4)
o = run_oracle(case, f0, 3)
g = run_gpu(P, case, f0, 3, storage="f32", tile_cap=1)
out["errors"]["3d_overflow"] = compare(g, o, 3)
out["bits"]["3d_overflow"] = P.lbm_check_violations()
# the faces kernel: inlet on x, open y and z
case = dict(lattice=19, n=(45, 29, 23), bc=(3, 2, 2), tau=0.62, body_force=(0, 0, 0),
            X=np.array([[18.0, 14.2, 11.4], [41.1, 20.6, 12.0]]), U=np.zeros((2, 3)), Om=np.zeros((2, 3)),
            r=np.array([5.0, 3.5]), inflow=(0.04, 0.0, 0.0))
p = O.make_params(19, *case["n"], bc=case["bc"], tau=case["tau"], inflow=case["inflow"])
f0 = np.ascontiguousarray(O.equilibrium(p, 1.0, case["inflow"]))
o = run_oracle(case, f0, 5)
g = run_gpu(P, case, f0, 5, storage="f32")
out["errors"]["inlet"] = compare(g, o, 3)
out["bits"]["inlet"] = P.lbm_check_violations()
# two slabs against the undivided lattice
case = ragged_case3d(bc=(0, 0, 1), n=(45, 29, 32))
ctx = P.lbm_create(19, *case["n"], bc=case["bc"], tau=case["tau"], body_force=case["body_force"], storage="f32")
P.lbm_set_particles(ctx, case["X"], case["U"], case["Om"], case["r"])
P.lbm_step(ctx, 4)
fw = P.lbm_get_populations(ctx)
P.lbm_destroy(ctx)
d = P.lbm_decomp_create(19, *case["n"], 2, bc=case["bc"], tau=case["tau"], body_force=case["body_force"],
                        storage="f32")
P.lbm_decomp_set_particles(d, case["X"], case["U"], case["Om"], case["r"])
P.lbm_decomp_step(d, 4)
fd = P.lbm_decomp_get_populations(d)
P.lbm_decomp_destroy(d)
out["decomp_max_diff"] = float(np.max(np.abs(fw - fd)))
out["bits"]["decomp"] = P.lbm_check_violations()
# a DEM call with walls
import synth  # noqa: E402

rng = np.random.default_rng(31)
L, n = 36, 30
r = rng.uniform(1.5, 2.5, n)
X = np.zeros((n, 3))
X[:, :2] = synth.rsa_pack(rng, (L, L), r, (True, True), gap=0.05)     # a layer without overlaps
X[:, 2] = -0.5 + r + rng.uniform(-0.1, 0.12, n)                       # some pressed into the wall
ctx = P.lbm_create(19, L, L, L, bc=(0, 0, 1), tau=0.8, storage="f32")
P.lbm_set_particles(ctx, X, np.zeros((n, 3)), np.zeros((n, 3)), r)
dem = P.dem_create(ctx, dt_dem=0.1, E=2.0, poisson=0.3, gamma=2e-3, density=3.0, gravity=(0, 0, -2e-4), skin=2.0)
for _ in range(3):
    P.dem_step(dem, 10)
out["dem_contacts"] = int(len(P.dem_get_contacts(dem)[0]) + len(P.dem_get_wall_contacts(dem)[0]))
P.dem_destroy(dem)
P.lbm_destroy(ctx)
out["bits"]["dem"] = P.lbm_check_violations()
# the adjoint (forward and reverse sweep)
case = ragged_case3d()
ctx = P.lbm_create(19, *case["n"], bc=case["bc"], tau=case["tau"], body_force=case["body_force"], storage="f32")
P.lbm_set_populations(ctx, perturbed_state(case, 5))
P.lbm_set_particles(ctx, case["X"], np.zeros_like(case["U"]), np.zeros_like(case["Om"]), case["r"])
J, dX, dF = P.lbm_adjoint_drag(ctx, 6, 3)
P.lbm_destroy(ctx)
out["adjoint_finite"] = bool(np.all(np.isfinite(dX)) and np.isfinite(J))
out["bits"]["adjoint"] = P.lbm_check_violations()
out["violations"] = 0
for v in out["bits"].values():
    out["violations"] |= v
print(json.dumps(out))
sys.stdout.flush()
