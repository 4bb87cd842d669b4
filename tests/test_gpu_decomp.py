"""The slab decomposition on one GPU (virtual sub-domains, through the C ABI): a lattice cut
into 2 or 3 slabs along its slowest axis, with the face exchange and the per-particle force
sums after every step, gives the populations of one context over the whole lattice bit for
bit, and the same forces and torques up to the order of their FP64 sums; on the 2D channel
(walls across the slab axis), the 3D periodic box (the periodic face between the last slab
and the first) and the 3D channel (walls at both ends), particles crossing the slab faces."""
import numpy as np
import pytest

import synth
from parity_utils import perturbed_state

pytestmark = pytest.mark.gpu


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


def _case(name):
    scale = {"c2": 0.125, "c3dense": 0.25, "c5": 0.125}[name]
    w = synth.workload(name, scale=scale)
    return dict(lattice=w["lattice"], n=w["n"], bc=w["bc"], tau=w["tau"], body_force=(1e-5, 2e-6, 0.0),
                X=w["X"], U=w["U"], Om=w["Om"], r=w["r"])


@pytest.mark.parametrize("name,nslab,storage", [("c2", 2, "f32"), ("c2", 3, "f64"), ("c3dense", 2, "f32"),
                                                ("c3dense", 3, "f16"), ("c5", 2, "f32")])
def test_slabs_reproduce_the_whole_lattice(P, name, nslab, storage):
    case = _case(name)
    f0 = perturbed_state(case, 18)
    steps = 12
    ctx = P.lbm_create(case["lattice"], *case["n"], bc=case["bc"], tau=case["tau"], body_force=case["body_force"],
                       storage=storage)
    P.lbm_set_populations(ctx, f0)
    P.lbm_set_particles(ctx, case["X"], case["U"], case["Om"], case["r"])
    P.lbm_step(ctx, steps)
    f1 = P.lbm_get_populations(ctx)
    F1, T1 = P.lbm_get_forces(ctx)
    P.lbm_destroy(ctx)

    d = P.lbm_decomp_create(case["lattice"], *case["n"], nslab, bc=case["bc"], tau=case["tau"],
                            body_force=case["body_force"], storage=storage)
    P.lbm_decomp_set_populations(d, f0)
    P.lbm_decomp_set_particles(d, case["X"], case["U"], case["Om"], case["r"])
    P.lbm_decomp_step(d, steps)
    f2 = P.lbm_decomp_get_populations(d)
    F2, T2 = P.lbm_decomp_get_forces(d)
    P.lbm_decomp_destroy(d)

    s_ax = 1 if case["lattice"] == 9 else 2
    own, _, _ = P.lbm_decomp_layout(case["lattice"], case["n"][s_ax], case["bc"][s_ax] == 0, nslab)
    c = case["X"][:, s_ax]
    crossing = sum(np.any(np.abs(c - o) < case["r"] + 1) for o in own[1:-1])
    assert crossing > 0                         # some particle straddles a slab face
    assert np.array_equal(f1, f2)
    scale = np.abs(F1).max()
    assert np.max(np.abs(F1 - F2)) <= 1e-12 * scale
    assert np.max(np.abs(T1 - T2)) <= 1e-12 * np.abs(T1).max()
