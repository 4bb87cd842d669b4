/* psc_testing.h -- host entry points onto small pieces of the kernels' arithmetic, for tests.
 *
 * The binning, the packed records and the DEM sub-step use a few __host__ __device__
 * helpers (tile ranges and culling, record positions, neighbour-bin walk, contact decision,
 * JKR contact-radius solve, displacement since the neighbour list's build) and the host
 * checks of a particle upload. These calls run the same source on the host, so tests can check
 * the compiled arithmetic against brute force without a GPU. They allocate nothing, touch no
 * device and never fail; arguments are plain values and caller-owned arrays. Not part of the
 * simulation interface of psc_lbm.h. */
#ifndef PSC_TESTING_H
#define PSC_TESTING_H

#ifdef __cplusplus
extern "C" {
#endif

/* Tile ranges [a[k], b[k]] (k < return value, at most 2) of one axis covered by the cell
 * interval [lo, hi], tiles of t cells, nt tiles, n cells; periodic axes wrap, wall axes clip
 * (the binning of Table 1 Step 1, reading R5). */
int psc_test_axis_tile_ranges(int lo, int hi, int n, int t, int nt, int periodic, int *a, int *b);
/* The k-th tile of those ranges (nr = number of ranges). */
int psc_test_axis_tile(int k, int nr, const int *a, const int *b);
/* 1 when the binning keeps the tile whose first cell is org[3] (extent ext[3]) for a
 * particle at X[3] with reach r + h (the centre wrapped on periodic axes, FP32 distances
 * with the kernel's margin); n[3] cells, periodic[3] flags, dim 2 or 3. */
int psc_test_tile_in_reach(const double *X, double reach_r_h, const int *org, const int *ext, const int *n,
                           const int *periodic, int dim);
/* The packed record's FP32 position of x relative to a tile origin org (tile extent ext,
 * n cells, minimum image on a periodic axis). */
float psc_test_record_rel(double x, int org, int ext, int n, int periodic);
/* The DEM neighbour-bin walk along one axis around bin b of nb: first bin and count, and the
 * k-th bin. */
void psc_test_axis_span(int b, int nb, int periodic, int *start, int *count);
int psc_test_axis_at(int k, int start, int nb, int periodic);
/* The DEM contact decision for squared distance d2 and S = r_i + r_j (Eq. 24 overlap
 * delta_N = S - |d|): *ge0 = delta_N >= 0, *gt0 = delta_N > 0; returns 1 when delta_N was
 * formed in FP64 (pairs within a few ulps of touching). */
int psc_test_contact_sign(double d2, double S, int *ge0, int *gt0);
/* The JKR contact-radius solve (reading R14): s = sqrt(a / a0) for t = delta_N R / a0^2,
 * started from s_prev; *fail = 1 when it did not converge, *iters the converging iteration. */
float psc_test_jkr_s(float t, float s_prev, int *fail, int *iters);
/* The DEM's squared displacement test (FP32, one image shift on periodic axes) of a
 * particle at x[3] from its position xr[3] at the last neighbour-list build. */
float psc_test_moved2(const double *x, const double *xr, const int *n, const int *periodic, int dim);
/* The host-side checks of a particle upload: 1 when the m values are all finite; the
 * smallest r^2 and the largest r over n radii. */
int psc_test_all_finite(const double *a, long long m);
void psc_test_radii_range(const double *R, int n, double *s2min, double *rmax);

#ifdef __cplusplus
}
#endif

#endif
