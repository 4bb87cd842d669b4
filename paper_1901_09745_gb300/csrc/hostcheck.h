// hostcheck.h -- the host-side argument checks of a particle upload (finite values, the
// range of the radii), shared by the C ABI and the host test entries of testing.cu.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

namespace psc {

// Argument checks of a particle upload run on every call, so they are written for the host's
// vector units with the compiler's generic vector types (two lanes of 64 bits: the same code
// on every host architecture) and four independent accumulators.
typedef uint64_t u64x2 __attribute__((vector_size(16)));
typedef double f64x2 __attribute__((vector_size(16)));
constexpr uint64_t kExpBits = 0x7ff0000000000000ull, kExpOne = 0x0010000000000000ull;

// 1 when the m values are all finite. An infinity or a NaN has every exponent bit set, and
// then (bits & kExpBits) + kExpOne carries into the sign bit; no other value does.
inline int all_finite(const double *a, size_t m) {
    const u64x2 mask = {kExpBits, kExpBits}, one = {kExpOne, kExpOne};
    u64x2 acc[4] = {};
    size_t i = 0;
    for (; i + 8 <= m; i += 8) {
        u64x2 b[4];
        memcpy(b, a + i, sizeof(b));
        for (int k = 0; k < 4; ++k) acc[k] |= (b[k] & mask) + one;
    }
    uint64_t bad = 0;
    for (int k = 0; k < 4; ++k) bad |= acc[k][0] | acc[k][1];
    for (; i < m; ++i) {
        uint64_t b;
        memcpy(&b, a + i, sizeof(b));
        bad |= (b & kExpBits) + kExpOne;
    }
    return (bad >> 63) == 0;
}

// Smallest r^2 and largest r over the radii (a NaN leaves both unchanged: all_finite reports it).
inline void radii_range(const double *R, int n, double *s2min, double *rmax) {
    f64x2 lo[2] = {{INFINITY, INFINITY}, {INFINITY, INFINITY}}, hi[2] = {{0.0, 0.0}, {0.0, 0.0}};
    int i = 0;
    for (; i + 4 <= n; i += 4) {
        f64x2 r[2];
        memcpy(r, R + i, sizeof(r));
        for (int k = 0; k < 2; ++k) {
            const f64x2 r2 = r[k] * r[k];
            lo[k] = r2 < lo[k] ? r2 : lo[k];
            hi[k] = r[k] > hi[k] ? r[k] : hi[k];
        }
    }
    double m = INFINITY, M = 0.0;
    for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) {
            m = lo[k][l] < m ? lo[k][l] : m;
            M = hi[k][l] > M ? hi[k][l] : M;
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
