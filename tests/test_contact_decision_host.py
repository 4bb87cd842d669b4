"""The DEM sub-step decides contact without forming delta_N = S - sqrt(d^2) in FP64 except
within a few ulps of touching (contact_sign, the kernel's own code compiled for the host):
the sign of d^2 - S^2, formed by one fused multiply-add (a single rounding, so its sign is
exact), decides delta_N >= 0 and > 0, and the correctly rounded square root is taken only
when |d^2 - S^2| <= 2^-47 S^2 (tested in FP32). Checked against the oracle's rule
fl(S - fl(sqrt(d^2))) on pairs placed at, just inside and just outside touching; the same
argument with the fused operation emulated in exact rational arithmetic agrees too."""
import math
from fractions import Fraction

import ctypes as C

import numpy as np

from host_entries import H  # noqa: F401  (fixture)


def _fma(a, b, c):
    # a * b + c rounded once (Fraction arithmetic is exact; float() rounds to nearest even)
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _oracle(S, d2):
    dn = S - math.sqrt(d2)
    return dn >= 0.0, dn > 0.0


def _device(S, d2):
    u = _fma(-S, S, d2)
    uf, Sf = np.float32(u), np.float32(S)
    ge0 = gt0 = bool(uf < np.float32(0.0))
    if abs(uf) <= Sf * Sf * np.float32(2.0 ** -47):
        dn = S - math.sqrt(d2)
        ge0, gt0 = dn >= 0.0, dn > 0.0
    return ge0, gt0


def _compiled(Hl, S, d2):
    ge0, gt0 = C.c_int(), C.c_int()
    Hl.psc_test_contact_sign(d2, S, C.byref(ge0), C.byref(gt0))
    return bool(ge0.value), bool(gt0.value)


def test_exact_contact_decision_matches_the_oracle_rule(H):
    rng = np.random.default_rng(1701)
    n = 0
    for _ in range(4000):
        ri, rj = rng.uniform(2.0, 9.0, 2)
        S = ri + rj
        direction = rng.normal(size=3)
        direction /= np.linalg.norm(direction)
        # distances at touching, a few ulps either side, and a little farther off
        base = S
        for k in list(range(-6, 7)) + [-1e6, 1e6, -1e9, 1e9]:
            dist = base + k * math.ulp(base)
            d = direction * dist
            d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
            assert _compiled(H, S, d2) == _oracle(S, d2), (ri, rj, k)
            assert _device(S, d2) == _oracle(S, d2), (ri, rj, k)
            n += 1
    assert n > 60000
