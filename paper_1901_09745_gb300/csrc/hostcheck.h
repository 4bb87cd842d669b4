// hostcheck.h -- the host-side argument checks of a particle upload (finite values, the
// range of the radii), shared by the C ABI and the host test entries of testing.cu.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

namespace psc {

// Argument checks of a particle upload run on every call, so they are written for the host's
// vector units with the compiler's generic vector types (two lanes of 64 bits: the same code
// on every host architecture), loaded straight from the caller's arrays (may_alias, 8-byte
// alignment) into four independent accumulators.
typedef uint64_t u64x2 __attribute__((vector_size(16)));
typedef double f64x2 __attribute__((vector_size(16)));
typedef uint64_t u64x2_in __attribute__((vector_size(16), aligned(8), may_alias));
typedef double f64x2_in __attribute__((vector_size(16), aligned(8), may_alias));
constexpr uint64_t kExpBits = 0x7ff0000000000000ull, kExpOne = 0x0010000000000000ull;

// 1 when the m values are all finite. An infinity or a NaN has every exponent bit set, and
// then (bits & kExpBits) + kExpOne carries into the sign bit; no other value does.
inline int all_finite(const double *a, size_t m) {
    const u64x2 mask = {kExpBits, kExpBits}, one = {kExpOne, kExpOne};
    u64x2 c0 = {0, 0}, c1 = c0, c2 = c0, c3 = c0;
    size_t i = 0;
    for (; i + 8 <= m; i += 8) {
        const u64x2_in *p = reinterpret_cast<const u64x2_in *>(a + i);
        c0 |= (p[0] & mask) + one;
        c1 |= (p[1] & mask) + one;
        c2 |= (p[2] & mask) + one;
        c3 |= (p[3] & mask) + one;
    }
    const u64x2 c = c0 | c1 | c2 | c3;
    uint64_t bad = c[0] | c[1];
    for (; i < m; ++i) {
        uint64_t b;
        memcpy(&b, a + i, sizeof(b));
        bad |= (b & kExpBits) + kExpOne;
    }
    return (bad >> 63) == 0;
}

// Smallest r^2 and largest r over the radii (a NaN leaves both unchanged: all_finite reports it).
inline void radii_range(const double *R, int n, double *s2min, double *rmax) {
    f64x2 l0 = {INFINITY, INFINITY}, l1 = l0, h0 = {0.0, 0.0}, h1 = h0;
    int i = 0;
    for (; i + 4 <= n; i += 4) {
        const f64x2_in *p = reinterpret_cast<const f64x2_in *>(R + i);
        const f64x2 r0 = p[0], r1 = p[1], q0 = r0 * r0, q1 = r1 * r1;
        l0 = q0 < l0 ? q0 : l0;
        l1 = q1 < l1 ? q1 : l1;
        h0 = r0 > h0 ? r0 : h0;
        h1 = r1 > h1 ? r1 : h1;
    }
    double m = INFINITY, M = 0.0;
    for (int k = 0; k < 2; ++k) {
        m = l0[k] < m ? l0[k] : m;
        m = l1[k] < m ? l1[k] : m;
        M = h0[k] > M ? h0[k] : M;
        M = h1[k] > M ? h1[k] : M;
    }
    for (; i < n; ++i) {
        const double r = R[i], r2 = r * r;
        m = r2 < m ? r2 : m;
        M = r > M ? r : M;
    }
    *s2min = m;
    *rmax = M;
}

}  // namespace psc
