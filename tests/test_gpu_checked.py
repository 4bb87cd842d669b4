"""The bounds-checked build (every main global access of the kernels tests its index, see
psc_internal.h): representative cases of every kernel family run through it with no index
out of range, and their results still match the oracle with the parity tolerances."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_records_no_violation_and_keeps_parity():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1901_09745_gb300 import build
    build.build(checked=True)
    root = os.path.dirname(HERE)
    env = dict(os.environ, PSC_LBM_CHECKED="1",
               PYTHONPATH=os.pathsep.join([root, HERE] + [v for v in [os.environ.get("PYTHONPATH")] if v]))
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], env=env, cwd=HERE,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["violations"] == 0, out
    for name, err in out["errors"].items():
        tol = dict(u=1e-5, rho=1e-5, F=1e-4, T=1e-4) if "f16" not in name else dict(u=2e-3, rho=1e-5, F=2e-3, T=2e-2)
        for k, v in tol.items():
            if k in err:
                assert err[k] <= v, (name, k, err)
    assert out["decomp_max_diff"] == 0.0
    assert out["dem_contacts"] > 0
    assert out["adjoint_finite"]
