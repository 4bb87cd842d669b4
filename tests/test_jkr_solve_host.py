"""The sub-step's JKR contact-radius solve (jkr_s, the kernel's own code compiled for the
host, FP32): Newton on s = s_c + e for e^2 (6 s_c^2 + 4 s_c e + e^2) = t - t_c, started
from the previous sub-step's root clamped to [e0 / 4, e0] of the cold guess e0 (which lies
right of the root). From any previous root -- far left, far right, at the pull-off point --
it converges well inside its 40-iteration cap to the same root as the cold start, and that
root satisfies the JKR relation delta(a) of the oracle (reading R14) to FP32 accuracy."""
import ctypes as C

import numpy as np

from host_entries import H  # noqa: F401  (fixture)

f32 = np.float32
SC = f32(0.55032120814910446)


def _solve(Hl, t, s_prev):
    fail, it = C.c_int(), C.c_int()
    s = Hl.psc_test_jkr_s(float(t), float(s_prev), C.byref(fail), C.byref(it))
    return f32(s), it.value if not fail.value else 40


def test_warm_started_solve_converges_to_the_cold_root(H):
    with np.errstate(all="ignore"):
        for t in np.concatenate([np.linspace(-0.275, 0.2, 60), np.geomspace(0.2, 1e3, 40)]):
            s_cold, it_cold = _solve(H, t, 0.0)
            assert it_cold < 40
            for s_prev in (SC + f32(6e-8), SC + f32(1e-4), f32(0.6), f32(1.0), f32(3.0), f32(50.0), s_cold):
                s, it = _solve(H, t, s_prev)
                assert it < 40, (t, s_prev, it)
                assert abs(s - s_cold) <= 4e-6 * s_cold, (t, s_prev, s, s_cold)
            # the root of s^4 - (2/3) s - t = 0 (delta R / a0^2 = (a/a0)^2 - (2/3)(a/a0)^(1/2) with s^2 = a/a0)
            s64 = float(s_cold)
            assert abs(s64 ** 4 - 2.0 / 3.0 * s64 - t) <= 2e-6 * max(1.0, abs(t))
