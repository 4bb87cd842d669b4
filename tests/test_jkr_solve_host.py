"""The sub-step's JKR contact-radius solve (jkr_s in dem.cu), emulated in FP32 on the host:
Newton on s = s_c + e for e^2 (6 s_c^2 + 4 s_c e + e^2) = t - t_c, started from the
previous sub-step's root clamped to [e0 / 4, e0] of the cold guess e0 (which lies right
of the root). From any previous root -- far left, far right, at the pull-off point -- it
converges well inside its 40-iteration cap to the same root as the cold start, and that
root satisfies the JKR relation delta(a) of the oracle (reading R14) to FP32 accuracy."""
import numpy as np

f32 = np.float32
SC = f32(0.55032120814910446)


def _solve(t, s_prev):
    tau = max(f32(t) + f32(0.5) * SC, f32(0.0))
    c2, c1 = f32(6.0) * SC * SC, f32(4.0) * SC
    e0 = min(np.sqrt(tau / c2), np.sqrt(np.sqrt(tau)))
    e = min(max(f32(s_prev) - SC, f32(0.25) * e0), e0) if (tau > 0 and f32(s_prev) > SC) else e0
    it = 0
    if tau > 0:
        while it < 40:
            h = e * e * (c2 + c1 * e + e * e) - tau
            dh = e * (f32(2.0) * c2 + f32(3.0) * c1 * e + f32(4.0) * e * e)
            if not dh > 0:
                break
            en = max(e - h / dh, f32(0.0))
            done = abs(en - e) <= f32(4e-7) * e
            e = en
            it += 1
            if done:
                break
    return SC + e, it


def test_warm_started_solve_converges_to_the_cold_root():
    with np.errstate(all="ignore"):
        for t in np.concatenate([np.linspace(-0.275, 0.2, 60), np.geomspace(0.2, 1e3, 40)]):
            s_cold, it_cold = _solve(t, 0.0)
            assert it_cold < 40
            for s_prev in (SC + f32(6e-8), SC + f32(1e-4), f32(0.6), f32(1.0), f32(3.0), f32(50.0), s_cold):
                s, it = _solve(t, s_prev)
                assert it < 40, (t, s_prev, it)
                assert abs(s - s_cold) <= 4e-6 * s_cold, (t, s_prev, s, s_cold)
            # the root of s^4 - (2/3) s - t = 0 (delta R / a0^2 = (a/a0)^2 - (2/3)(a/a0)^(1/2) with s^2 = a/a0)
            s64 = float(s_cold)
            assert abs(s64 ** 4 - 2.0 / 3.0 * s64 - t) <= 2e-6 * max(1.0, abs(t))
