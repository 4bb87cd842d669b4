"""lbm_psc_step_noalloc: the step for callers that may not allocate device memory.

Some callers cannot let a library call cudaMalloc (their own memory manager owns the
device, or they run a loop that must not allocate once started). They pass every buffer
and the library works in a fixed array compiled into it. These tests check that this entry
point gives the same populations, forces and torques as the ordinary context-based path
(lbm_step), on two calls in a row (so the second call sees what the first one left in the
shared array), in 2D and 3D, for every storage format and both PSC modes. This file is
named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from parity_utils import perturbed_state, rel_l2

pytestmark = pytest.mark.gpu

HEADER = 64   # bytes of the lbm_save_state header before the raw population buffer


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1901_09745_gb300 import build
    build.build()
    import paper_1901_09745_gb300 as P
    P.lib()
    return P, torch


ELEM = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}
# relative L2 bound on the decoded state: the two paths run the same kernels, but the
# no-allocation step keeps 16 candidate records per tile (more take the exact chunked path)
# and always uses the per-cell minimum image, so values may differ by a rounding
TOL = {"f64": 1e-12, "f32": 1e-6, "f16": 2e-3, "bf16": 2e-2}


def _decode(raw, storage):
    """Stored deviations as float64 (FP16 / BF16 still scaled)."""
    if storage == "f64":
        return np.frombuffer(raw, dtype=np.float64).copy()
    if storage == "f32":
        return np.frombuffer(raw, dtype=np.float32).astype(np.float64)
    if storage == "f16":
        return np.frombuffer(raw, dtype=np.float16).astype(np.float64)
    bits = np.frombuffer(raw, dtype=np.uint16).astype(np.uint32) << 16
    return bits.view(np.float32).astype(np.float64)


def _cases():
    w = synth.workload("c2", scale=0.125)            # 256 x 256 channel, band of discs
    c2 = dict(lattice=9, n=w["n"], bc=w["bc"], tau=w["tau"], body_force=(1e-6, 0, 0), X=w["X"],
              U=w["U"], Om=w["Om"], r=w["r"], psc=0)
    rng = np.random.default_rng(41)
    X = np.array([[2.1, 14.0, 11.2], [43.5, 6.2, 9.1], [20.2, 12.5, 4.6], [26.9, 14.1, 6.1]])
    c3 = dict(lattice=19, n=(45, 29, 23), bc=(0, 0, 1), tau=0.62, body_force=(1e-5, 0, 0), X=X,
              U=rng.normal(0, 2e-3, (4, 3)), Om=rng.normal(0, 5e-4, (4, 3)), r=np.array([4.5, 3.8, 4.0, 3.9]))
    out = [("2d-f32-modified", c2, "f32")]
    for storage in ("f64", "f32", "f16", "bf16"):
        for psc in (0, 1):
            out.append(("3d-%s-%s" % (storage, "original" if psc else "modified"), dict(c3, psc=psc), storage))
    return out


@pytest.mark.parametrize("name,case,storage", _cases(), ids=[c[0] for c in _cases()])
def test_noalloc_step_matches_context_step_twice(env, name, case, storage):
    """Every storage format (each has its own record and scratch layout) and both PSC
    modes, on two calls in a row."""
    P, torch = env
    dev = torch.device("cuda", 0)
    ctx = P.lbm_create(case["lattice"], *case["n"], bc=case["bc"], tau=case["tau"],
                       body_force=case["body_force"], storage=storage, psc=case["psc"])
    P.lbm_set_populations(ctx, perturbed_state(case, 12))
    P.lbm_set_particles(ctx, case["X"], case["U"], case["Om"], case["r"])
    state0 = P.lbm_save_state(ctx)
    nbytes = case["lattice"] * int(np.prod(case["n"])) * ELEM[storage]
    ref = []
    for _ in range(2):
        P.lbm_step(ctx, 1)
        F, T = P.lbm_get_forces(ctx)
        raw = P.lbm_save_state(ctx)[HEADER:HEADER + nbytes]
        ref.append((_decode(raw, storage), F.copy(), T.copy()))
    params = ctx.params
    P.lbm_destroy(ctx)

    # the same two steps with caller-owned device buffers only
    f_in = torch.from_numpy(np.frombuffer(state0[HEADER:HEADER + nbytes], dtype=np.uint8).copy()).to(dev)
    f_out = torch.empty_like(f_in)
    n = len(case["r"])
    as_dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    X, U, Om, R = as_dev(case["X"]), as_dev(case["U"]), as_dev(case["Om"]), as_dev(case["r"])
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    T = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    params.stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for call in range(2):
        P.lbm_psc_step_noalloc(params, f_in, f_out, X, U, Om, R, F, T)
        torch.cuda.synchronize(dev)
        dec_ref, F_ref, T_ref = ref[call]
        got = _decode(f_out.cpu().numpy().tobytes(), storage)
        assert rel_l2(got, dec_ref) <= TOL[storage], (name, call, rel_l2(got, dec_ref))
        assert rel_l2(F.cpu().numpy(), F_ref) <= 1e-9, (name, call)
        assert rel_l2(T.cpu().numpy(), T_ref) <= 1e-9, (name, call)
        f_in, f_out = f_out, f_in


def test_noalloc_rejects_aliased_buffers(env):
    P, torch = env
    params = P.LbmParams()
    params.lattice, params.nx, params.ny, params.nz = 9, 64, 32, 1
    params.tau, params.storage = 0.7, P.LBM_F32
    buf = torch.zeros(9 * 64 * 32, device="cuda")
    with pytest.raises(P.LbmError) as ei:
        P.lbm_psc_step_noalloc(params, buf, buf)
    assert ei.value.status == P.LBM_ERR_ARG and "alias" in str(ei.value)


def test_noalloc_rejects_oversized_problem(env):
    P, torch = env
    params = P.LbmParams()
    params.lattice, params.nx, params.ny, params.nz = 19, 2048, 2048, 512
    params.tau, params.storage = 0.7, P.LBM_F32
    a, b = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    with pytest.raises(P.LbmError) as ei:
        P.lbm_psc_step_noalloc(params, a, b)
    assert ei.value.status == P.LBM_ERR_ARG
    assert "LBM_NOALLOC_SCRATCH_BYTES" in str(ei.value)
