// hostdev.cuh -- small pieces of the kernels' index and decision arithmetic, written once as
// __host__ __device__ functions: the kernels call them, and so do the host-side test entries
// of testing.cu, which the CPU tests drive against brute force.
#pragma once

#include <math.h>

namespace psc {

// ------------------------------------------------------------------------- binning (S0)
// Tile ranges along one axis covered by the cell interval [lo, hi] (cell centres within
// r + h of the particle centre). Periodic axes wrap (at most two pieces, merged when they
// meet); wall axes clip to the lattice. Returns the number of ranges (0..2).
__host__ __device__ __forceinline__ int axis_tile_ranges(int lo, int hi, int n, int t, int nt, int periodic, int *a,
                                                         int *b) {
    if (periodic) {
        if (hi - lo + 1 >= n) { a[0] = 0; b[0] = nt - 1; return 1; }
        const int A = ((lo % n) + n) % n, B = ((hi % n) + n) % n;
        if (A <= B) { a[0] = A / t; b[0] = B / t; return 1; }
        const int thi = A / t, tlo = B / t;
        if (tlo >= thi) { a[0] = 0; b[0] = nt - 1; return 1; }
        a[0] = 0; b[0] = tlo; a[1] = thi; b[1] = nt - 1;
        return 2;
    }
    const int A = lo < 0 ? 0 : lo, B = hi > n - 1 ? n - 1 : hi;
    if (A > B) return 0;
    a[0] = A / t; b[0] = B / t;
    return 1;
}

// The k-th tile (0 <= k < length of all ranges) of one axis.
__host__ __device__ __forceinline__ int axis_tile(int k, int nr, const int *a, const int *b) {
    const int l0 = b[0] - a[0] + 1;
    return (nr < 2 || k < l0) ? a[0] + k : a[1] + (k - l0);
}

// Distance along one axis from x to the cell centres a..b of a tile (minimum image on a
// periodic axis of length n).
__host__ __device__ __forceinline__ float axis_gap(float x, float a, float b, float n, int periodic) {
    float d = fmaxf(fmaxf(a - x, x - b), 0.0f);
    if (periodic) {
        d = fminf(d, fmaxf(fmaxf(a - (x + n), (x + n) - b), 0.0f));
        d = fminf(d, fmaxf(fmaxf(a - (x - n), (x - n) - b), 0.0f));
    }
    return d;
}

// A particle centre wrapped into [0, n] on a periodic axis (callers may pass positions any
// number of periods out; the culling compares the result with its images at +-n only).
__host__ __device__ __forceinline__ double wrap_centre(double x, int n, double inv_n) {
    return x - (double)n * floor(x * inv_n);
}

// Whether some cell centre of the tile whose first cell is org[] (extent ext[], clipped to
// the lattice n[]) lies within `reach` of the wrapped centre xp[] (FP32; reach carries a
// margin far above the FP32 rounding of these distances).
__host__ __device__ __forceinline__ bool tile_in_reach(const float *xp, float reach, const int *org, const int *ext,
                                                       const int *n, const int *periodic, int dim) {
    float d2 = 0.0f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (ax >= dim) break;
        const int hi = (org[ax] + ext[ax] < n[ax] ? org[ax] + ext[ax] : n[ax]) - 1;
        const float gap = axis_gap(xp[ax], (float)org[ax], (float)hi, (float)n[ax], periodic[ax]);
        d2 += gap * gap;
    }
    return d2 <= reach * reach;
}

// ------------------------------------------------------------------- packed records (S0)
// Candidate position relative to its tile's origin `org` along one axis: on a periodic axis
// the minimum image with respect to the tile centre, the image decided in FP32 (candidates
// lie far from the half-box distance where that could differ) and x - (origin + image
// shift) formed by one exact FP64 subtraction.
__host__ __device__ __forceinline__ double record_rel(double x, int org, int ext, int n, double inv_n, int periodic) {
    int shift = org;
    if (periodic) {
        const float e = (float)x - ((float)org + 0.5f * (float)(ext - 1));
        shift += n * (int)rintf(e * (float)inv_n);
    }
    return x - (double)shift;
}

// ------------------------------------------------------------------------------ DEM (S6)
// The distinct bins along one axis around bin b: n of them, the k-th at axis_at(k, ...)
// (periodic: b - 1, b, b + 1 wrapped, fewer when nb < 3; walls: clipped to the lattice).
__host__ __device__ __forceinline__ void axis_span(int b, int nb, int periodic, int &start, int &n) {
    if (periodic) { start = b - 1 + nb; n = nb < 3 ? nb : 3; }
    else { start = b > 0 ? b - 1 : 0; n = (b + 1 < nb ? b + 1 : nb - 1) - start + 1; }
}
__host__ __device__ __forceinline__ int axis_at(int k, int start, int nb, int periodic) {
    return periodic ? (start + k) % nb : start + k;
}

// Squared displacement (FP32) of a particle at x from its position xr at the last
// neighbour-list build: one image shift on a periodic axis, so the result is never below the
// minimum-image displacement. The DEM rebuilds its list once a particle passes a quarter of
// the skin; both the sub-step and a particle upload test this value.
__host__ __device__ __forceinline__ float moved2(const double *x, const double *xr, const int *n, const int *periodic,
                                                 int dim) {
    float d2 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= dim) break;
        float dd = (float)(x[a] - xr[a]);
        if (periodic[a]) {
            const float half = 0.5f * (float)n[a];
            if (dd > half) dd -= (float)n[a];
            else if (dd < -half) dd += (float)n[a];
        }
        d2 += dd * dd;
    }
    return d2;
}

// IEEE-rounded FP64 operations, no contraction on either side (the device intrinsics; on the
// host plain operations, the library being compiled with FP contraction off).
__host__ __device__ __forceinline__ double dadd_rn(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
__host__ __device__ __forceinline__ double dsub_rn(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}
__host__ __device__ __forceinline__ double dmul_rn(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
__host__ __device__ __forceinline__ double dfma_rn(double a, double b, double c) {
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return fma(a, b, c);
#endif
}
__host__ __device__ __forceinline__ double dsqrt_rn(double a) {
#ifdef __CUDA_ARCH__
    return __dsqrt_rn(a);
#else
    return sqrt(a);
#endif
}
__host__ __device__ __forceinline__ float rsqrt_f(float a) {
#ifdef __CUDA_ARCH__
    return rsqrtf(a);
#else
    return 1.0f / sqrtf(a);
#endif
}

// Contact decision of a pair at squared distance d2 (FP64, IEEE-rounded, bit-identical at
// both ends and in a CPU reference) with S = r_i + r_j. delta_N = S - |d| is formed, as the
// reference forms it, only for pairs within a few ulps of touching: elsewhere the sign of
// d^2 - S^2 (one rounding, so its sign is exact) decides delta_N >= 0 and > 0, and delta_N
// itself enters the FP32 contact law as (S^2 - d^2) / (S + |d|). Returns delta_N in FP32;
// `exact` tells whether dn (FP64) was formed.
struct ContactSign {
    bool ge0, gt0, exact;
    float dnf, inv;       // delta_N (FP32) and 1 / |d| (FP32)
    double dn;            // delta_N in FP64 when exact
};
__host__ __device__ __forceinline__ ContactSign contact_sign(double d2, double S) {
    ContactSign c;
    const double u = dfma_rn(-S, S, d2);
    const float d2f = (float)d2, uf = (float)u, Sf = (float)S;
    c.inv = rsqrt_f(d2f);
    c.ge0 = uf < 0.0f;
    c.gt0 = c.ge0;
    c.dnf = -uf / (Sf + d2f * c.inv);
    c.dn = 0.0;
    c.exact = false;
    if (fabsf(uf) <= Sf * Sf * 0x1p-47f) {     // |d^2 - S^2| <= ~2^-48 S^2
        c.dn = dsub_rn(S, dsqrt_rn(d2));
        c.exact = true;
        c.ge0 = c.dn >= 0.0;
        c.gt0 = c.dn > 0.0;
        c.dnf = (float)c.dn;
    }
    return c;
}

// JKR contact radius ratio s = sqrt(a/a0) for t = delta R / a0^2 on the stable branch, i.e.
// the root s >= s_c = 6^(-1/3) of s^4 - (2/3) s - t = 0 (t >= t_c = -s_c/2 at pull-off).
// Written as s = s_c + e, the linear terms cancel exactly (4 s_c^3 = 2/3) and the equation
// becomes e^2 (6 s_c^2 + 4 s_c e + e^2) = t - t_c, which stays well conditioned near the
// pull-off point where the original form loses all digits to cancellation. The left side
// is increasing and convex for e >= 0; Newton starts from the previous sub-step's root
// s_prev when there is one, kept within [e0 / 4, e0] of the cold guess e0 (which lies right
// of the root): from the left of the root it overshoots once to the right (by at most about
// root^2 / start), then decreases monotonically. Sets *fail when it does not converge in 40
// iterations; *iters (if given) receives the index of the iteration that converged (40 when
// none did).
__host__ __device__ __forceinline__ float jkr_s(float t, int *fail, float s_prev, int *iters = nullptr) {
    const float sc = 0.55032120814910446f;            // 6^(-1/3)
    const float tau = fmaxf(t + 0.5f * sc, 0.0f);      // t - t_c
    const float c2 = 6.0f * sc * sc, c1 = 4.0f * sc;
    const float e0 = fminf(sqrtf(tau / c2), sqrtf(sqrtf(tau)));
    float e = (tau > 0.0f && s_prev > sc) ? fminf(fmaxf(s_prev - sc, 0.25f * e0), e0) : e0;
    int it = 0;
    if (tau > 0.0f) {
        for (; it < 40; ++it) {
            const float h = e * e * (c2 + c1 * e + e * e) - tau;
            const float dh = e * (2.0f * c2 + 3.0f * c1 * e + 4.0f * e * e);
            if (!(dh > 0.0f)) break;
            const float en = fmaxf(e - h / dh, 0.0f);
            const bool done = fabsf(en - e) <= 4e-7f * e;   // a few ulps: FP32 may cycle by one
            e = en;
            if (done) break;
        }
        if (it >= 40 || !(e == e)) *fail = 1;
    }
    if (iters) *iters = it;
    return sc + e;
}

}  // namespace psc
