// testing.cu -- host entry points onto the __host__ __device__ helpers of hostdev.cuh, so
// that the CPU tests check the arithmetic the kernels compile rather than a copy of it (see
// include/psc_testing.h). Nothing here touches a GPU.
#include "../../include/psc_testing.h"
#include "hostcheck.h"
#include "hostdev.cuh"

using namespace psc;

extern "C" int psc_test_axis_tile_ranges(int lo, int hi, int n, int t, int nt, int periodic, int *a, int *b) {
    return axis_tile_ranges(lo, hi, n, t, nt, periodic, a, b);
}

extern "C" int psc_test_axis_tile(int k, int nr, const int *a, const int *b) { return axis_tile(k, nr, a, b); }

extern "C" int psc_test_tile_in_reach(const double *X, double reach_r_h, const int *org, const int *ext,
                                      const int *n, const int *periodic, int dim) {
    // the binning's steps for one (particle, tile): centre wrapped on periodic axes, the FP32
    // copy, the reach with its margin
    double xw[3] = {X[0], X[1], dim == 3 ? X[2] : 0.0};
    for (int ax = 0; ax < dim; ++ax)
        if (periodic[ax]) xw[ax] = wrap_centre(xw[ax], n[ax], 1.0 / n[ax]);
    const float xp[3] = {(float)xw[0], (float)xw[1], (float)xw[2]};
    const float reach = (float)reach_r_h + 0.01f;
    return tile_in_reach(xp, reach, org, ext, n, periodic, dim) ? 1 : 0;
}

extern "C" float psc_test_record_rel(double x, int org, int ext, int n, int periodic) {
    return (float)record_rel(x, org, ext, n, 1.0 / n, periodic);
}

extern "C" void psc_test_axis_span(int b, int nb, int periodic, int *start, int *count) {
    axis_span(b, nb, periodic, *start, *count);
}

extern "C" int psc_test_axis_at(int k, int start, int nb, int periodic) { return axis_at(k, start, nb, periodic); }

extern "C" int psc_test_contact_sign(double d2, double S, int *ge0, int *gt0) {
    const ContactSign c = contact_sign(d2, S);
    *ge0 = c.ge0 ? 1 : 0;
    *gt0 = c.gt0 ? 1 : 0;
    return c.exact ? 1 : 0;
}

extern "C" float psc_test_jkr_s(float t, float s_prev, int *fail, int *iters) {
    *fail = 0;
    return jkr_s(t, fail, s_prev, iters);
}

extern "C" int psc_test_all_finite(const double *a, long long m) { return all_finite(a, (size_t)m); }

extern "C" void psc_test_radii_range(const double *R, int n, double *s2min, double *rmax) {
    radii_range(R, n, s2min, rmax);
}

extern "C" float psc_test_moved2(const double *x, const double *xr, const int *n, const int *periodic, int dim) {
    return moved2(x, xr, n, periodic, dim);
}

