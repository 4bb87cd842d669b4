"""FP16 / BF16 deviation storage (FP32 compute) against the FP64 oracle.

The paper has no reduced-precision result to pin these to; the error against the FP64
oracle is measured and reported here (written to the file named by PSC_ERROR_REPORT when
set), with loose bounds that a
broken storage path (wrong scale, wrong rounding, lost increments) would exceed by orders
of magnitude. Each test prints its errors next to the FP32 errors of the same run.
"""
import json
import os

import numpy as np
import pytest

import synth
from parity_utils import compare, perturbed_state, ragged_case2d, ragged_case3d, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

OUT = os.environ.get("PSC_ERROR_REPORT", "")


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


def _report(name, errs):
    line = json.dumps(dict(case=name, **{k: {q: float("%.3e" % v) for q, v in e.items()} for k, e in errs.items()}))
    print(line)
    if OUT:
        with open(OUT, "a") as fh:
            fh.write(line + "\n")


# relative L2 error against FP64, about 7x the measured values (64^3 dense, 200 steps:
# FP16 u 1.4e-4, F 6.7e-5, T 2.2e-4; BF16 u 1.2e-3, F 5.6e-4, T 1.9e-3; 256^2 channel,
# 20 steps: FP16 u 1.9e-4, BF16 u 1.5e-3)
BOUND = {"f16": dict(u=1e-3, rho=2e-6, F=1e-3, T=3e-3), "bf16": dict(u=1e-2, rho=2e-5, F=1e-2, T=2e-2)}


def test_c3_dense_subrun_reduced_storage(P):
    """D3Q19 64^3 sub-run of the 256^3 workload at solid fraction 0.3, 200 steps from rest
    with body force 1e-6: FP32 vs FP16 and BF16 deviation storage, all against FP64."""
    w = synth.workload("c3dense", scale=0.25)
    case = dict(lattice=19, n=w["n"], bc=w["bc"], tau=w["tau"], body_force=w["body_force"],
                X=w["X"], U=w["U"], Om=w["Om"], r=w["r"])
    o = run_oracle(case, perturbed_state(case, 0, amp=0.0), 200)
    errs = {}
    for st in ("f32", "f16", "bf16"):
        g = run_gpu(P, case, None, 200, storage=st)
        errs[st] = compare(g, o, 3)
    _report("c3dense 64^3 200 steps", errs)
    for st in ("f16", "bf16"):
        for k, b in BOUND[st].items():
            assert errs[st][k] < b, (st, k, errs[st][k])
        # reduced storage is less accurate than FP32 but keeps the flow
        assert errs[st]["u"] > errs["f32"]["u"]


def test_c2_subbox_reduced_storage(P):
    """D2Q9 256^2 channel sub-box, 20 steps from a perturbed state (one-step-scale changes)."""
    w = synth.workload("c2", scale=0.125)
    case = dict(lattice=9, n=w["n"], bc=w["bc"], tau=w["tau"], body_force=(1e-6, 0, 0),
                X=w["X"], U=w["U"], Om=w["Om"], r=w["r"])
    f0 = perturbed_state(case, 8)
    o = run_oracle(case, f0, 20)
    errs = {}
    for st in ("f32", "f16", "bf16"):
        g = run_gpu(P, case, f0, 20, storage=st)
        errs[st] = compare(g, o, 2)
    _report("c2 256^2 20 steps", errs)
    for st in ("f16", "bf16"):
        for k, b in BOUND[st].items():
            assert errs[st][k] < b, (st, k, errs[st][k])


def test_c5_channel_subbox_reduced_storage(P):
    """The 512^3 channel's own storage form (FP16 deviations) on its 64^3 sub-box: walls in
    z, polydisperse moving spheres, 20 steps from a perturbed state; FP32, FP16 and BF16
    against FP64."""
    w = synth.workload("c5", scale=0.125)
    case = dict(lattice=19, n=w["n"], bc=w["bc"], tau=w["tau"], body_force=w["body_force"],
                X=w["X"], U=w["U"], Om=w["Om"], r=w["r"])
    f0 = perturbed_state(case, 11)
    o = run_oracle(case, f0, 20)
    errs = {}
    for st in ("f32", "f16", "bf16"):
        g = run_gpu(P, case, f0, 20, storage=st)
        errs[st] = compare(g, o, 3)
    _report("c5 64^3 channel 20 steps", errs)
    for st in ("f16", "bf16"):
        for k, b in BOUND[st].items():
            assert errs[st][k] < b, (st, k, errs[st][k])


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("dim", [2, 3])
def test_ragged_reduced_storage(P, storage, dim):
    """16-bit storage on the ragged parity cases: partial tiles on every axis, walls,
    periodic faces, moving particles that share cells; FP32 and the 16-bit form against
    FP64."""
    case = ragged_case2d() if dim == 2 else ragged_case3d()
    steps = 25 if dim == 2 else 15
    f0 = perturbed_state(case, 3)
    o = run_oracle(case, f0, steps)
    g32 = run_gpu(P, case, f0, steps, storage="f32")
    g = run_gpu(P, case, f0, steps, storage=storage)
    errs = {"f32": compare(g32, o, dim), storage: compare(g, o, dim)}
    _report("ragged %dD %s %d steps" % (dim, "x".join(map(str, case["n"][:dim])), steps), errs)
    for k, b in BOUND[storage].items():
        assert errs[storage][k] < b, (storage, k, errs[storage][k])
