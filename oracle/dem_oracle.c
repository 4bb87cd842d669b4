/*
 * dem_oracle.c -- plain FP64 CPU oracle of the adhesive DEM contact update of Liu & Wu
 * (arXiv 1901.09745, Sec. 2.5): JKR normal force (Eq. 26-27), damping, sliding / twisting
 * / rolling spring-dashpot-sliders with the critical values of Eq. 29, contact force and
 * torque decomposition (Eq. 22), Newton-Euler motion (Eq. 21) and DEM sub-cycling with the
 * hydrodynamic force frozen over the sub-steps (end of Sec. 2.5).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load this file; it shares nothing with the CUDA library.
 *
 * Readings of what the paper leaves open (the CUDA library takes the same readings):
 *  J1 JKR with work of adhesion 2 gamma, consistent with F_C = 3 pi gamma R and Eq. 27:
 *     delta_N = (a0^2/R) [ (a/a0)^2 - (2/3) (a/a0)^(1/2) ]; the contact radius a is taken on
 *     the stable branch a/a0 >= 6^(-2/3), found here by bisection; delta_C = a0^2/(2 6^(1/3) R).
 *  J2 contact life: a pair comes into contact when delta_N >= 0 and stays in contact while
 *     delta_N > -delta_C (Hertz: while delta_N > 0); pairs are canonical i < j.
 *  J3 R and E of Eq. 25 with one material for all particles: 1/R = 1/r_i + 1/r_j,
 *     1/E* = 2 (1 - sigma^2)/E.
 *  J4 model constants "from the literature": k_N = 2 E* a, eta_N = alpha_n sqrt(m* k_N),
 *     k_T = k_t_scale 8 G* a with G* = E / (4 (2 - sigma)(1 + sigma)), eta_T = eta_t_scale
 *     eta_N; m* = m_i m_j / (m_i + m_j).
 *  J5 springs are vectors kept in the current tangent plane (projected and rescaled each
 *     sub-step, then incremented by velocity x dt). When a trial force or moment exceeds
 *     its critical value the result is capped at the critical value (Eq. 28 "min") and
 *     the spring is reset so that the spring alone carries the capped value.
 *     sliding: v_t = tangential part of the relative contact-point velocity of i w.r.t. j,
 *              F_t(on i) = -k_T xi_s - eta_T v_t, |F_t| <= mu_f |F_ne + 2 F_C|
 *     twisting: Omega_t = (Omega_i - Omega_j).n, M_t = -(k_T a^2/2) xi_t - (eta_T a^2/2) Omega_t,
 *              |M_t| <= 3 pi a F_s,crit / 16; torque M_t n on i
 *     rolling: v_L = R n x (Omega_i - Omega_j), torque on i = k_r (n x xi_r) with
 *              k_r = 4 F_C (a/a0)^(3/2), |torque| <= 4 F_C (a/a0)^(3/2) theta_crit R (|Eq. 29|)
 *  J6 normal force on i is -F_n n with F_n = F_ne + eta_N (v_i - v_j).n, n = (X_j - X_i)/|.|
 *     (positive = repulsive); the tangential force acts at the contact points (torques
 *     r_i n x F_t on i and r_j n x F_t on j).
 *  J7 motion (Eq. 21), semi-implicit Euler in FP64: U += dt F/m; X += dt U;
 *     Omega += dt M / I. Spheres: m = rho_p 4/3 pi r^3, I = 2/5 m r^2. Discs (2D, contact
 *     law of a sphere of the same radius): m = rho_p pi r^2, I = 1/2 m r^2.
 *  J8 Hertz (adhesive = 0, the paper's non-adhesive comparison): F_ne = 4/3 E* sqrt(R)
 *     delta^(3/2), a = sqrt(R delta), F_C = 0 in Eq. 29, no rolling resistance.
 *  W1 walls (the packing of Sec. 3.5 settles onto a wall): every non-periodic axis a < dim
 *     has the fluid's halfway bounce-back walls, planes at -1/2 and n_a - 1/2. A particle
 *     meets the nearer of the two as a half-space of the same material that does not move:
 *     the contact law above with R = r_i (1/R = 1/r_i + 1/infinity), m* = m_i, the wall's
 *     velocity and spin zero, n the unit normal from the centre towards the plane and
 *     delta_N = r_i - (distance from the centre to the plane); the same life cycle (J2) and
 *     a spring history of its own.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define DEM_OK 0
#define DEM_ERR_ARG 1
#define DEM_ERR_OOM 2
#define DEM_ERR_CAP 3
#define DEM_ERR_SOLVE 4

#define PI 3.14159265358979323846

typedef struct {
    double E, poisson, gamma, density, mu_f, theta_crit, alpha_n, k_t_scale, eta_t_scale;
    double dt;
    double gravity[3];
    int adhesive;        /* 1 = JKR (Eq. 26), 0 = Hertz */
    int dim;             /* 2 = discs, 3 = spheres */
    int n[3];            /* box extent (cells) for periodic minimum images / wrapping */
    int periodic[3];
} ora_dem_params;

/* per-contact history: xi_s (3), xi_t (1), xi_r (3) */
#define NH 7

/* ---------------------------------------------------------------- JKR (Eq. 26-27) --- */
double ora_jkr_delta(double a, double a0, double R)
{
    double x = a / a0;
    return a0 * a0 / R * (x * x - 2.0 / 3.0 * sqrt(x));
}

double ora_jkr_force(double a, double a0, double FC)
{
    double x = a / a0;
    return 4.0 * FC * (x * x * x - pow(x, 1.5));
}

/* Contact radius on the stable branch for an overlap delta >= -delta_C, by bisection
 * on x = a/a0 in [6^(-2/3), x_hi]. *ok = 0 when delta is below -delta_C. */
double ora_jkr_contact_radius(double delta, double a0, double R, int *ok)
{
    double lo = pow(6.0, -2.0 / 3.0), hi = 1.0, target = delta * R / (a0 * a0);
    int it;
    if (ok) *ok = 1;
    if (lo * lo - 2.0 / 3.0 * sqrt(lo) > target) {
        if (ok) *ok = 0;
        return lo * a0;
    }
    while (hi * hi - 2.0 / 3.0 * sqrt(hi) < target) hi *= 2.0;
    for (it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid * mid - 2.0 / 3.0 * sqrt(mid) < target) lo = mid;
        else hi = mid;
        if (hi - lo <= 1e-16 * hi) break;
    }
    return 0.5 * (lo + hi) * a0;
}

/* ------------------------------------------------------------------- geometry --- */
static double delta_axis(double a, double b, int n, int periodic)
{
    double d = a - b;
    if (periodic) {
        while (d > 0.5 * n) d -= n;
        while (d < -0.5 * n) d += n;
    }
    return d;
}

/* separation vector d = X_j - X_i (minimum image), distance, overlap delta_N = r_i + r_j - |d| */
static double pair_overlap(const ora_dem_params *p, const double *X, const double *r, int i, int j,
                           double *d, double *dist)
{
    int a;
    for (a = 0; a < 3; ++a)
        d[a] = (a < p->dim) ? delta_axis(X[3 * j + a], X[3 * i + a], p->n[a], p->periodic[a]) : 0.0;
    *dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    return (r[i] + r[j]) - *dist;
}

static void mass_inertia(const ora_dem_params *p, double r, double *m, double *I)
{
    if (p->dim == 2) { *m = p->density * PI * r * r; *I = 0.5 * (*m) * r * r; }
    else { *m = p->density * 4.0 / 3.0 * PI * r * r * r; *I = 0.4 * (*m) * r * r; }
}

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* JKR critical separation delta_C for the pair (J1), or 0 for Hertz */
static void pair_constants(const ora_dem_params *p, double ri, double rj, double *R, double *Es,
                           double *FC, double *a0, double *dC)
{
    *R = ri * rj / (ri + rj);
    *Es = p->E / (2.0 * (1.0 - p->poisson * p->poisson));
    if (p->adhesive) {
        *FC = 3.0 * PI * p->gamma * (*R);
        *a0 = cbrt(9.0 * PI * p->gamma * (*R) * (*R) / (*Es));
        *dC = (*a0) * (*a0) / (2.0 * cbrt(6.0) * (*R));
    } else {
        *FC = 0.0; *a0 = 0.0; *dC = 0.0;
    }
}

/* All pairs i < j in contact by rule J2, by brute-force enumeration of every pair, with
 * history carried over from the previous list (pairs/hist, sorted) or zero for new ones. */
static int detect(const ora_dem_params *p, int np, const double *X, const double *r,
                  int nold, const int *opairs, const double *ohist,
                  int *nnew, int *npairs, double *nhist, int cap)
{
    int i, j, k = 0, o = 0;
    for (i = 0; i < np; ++i) {
        for (j = i + 1; j < np; ++j) {
            double d[3], dist, R, Es, FC, a0, dC, dn;
            int was = 0;
            dn = pair_overlap(p, X, r, i, j, d, &dist);
            /* advance the cursor of the sorted old list to (i, j) */
            while (o < nold && (opairs[2 * o] < i || (opairs[2 * o] == i && opairs[2 * o + 1] < j))) ++o;
            if (o < nold && opairs[2 * o] == i && opairs[2 * o + 1] == j) was = 1;
            pair_constants(p, r[i], r[j], &R, &Es, &FC, &a0, &dC);
            if ((p->adhesive && (dn >= 0.0 || (was && dn > -dC))) || (!p->adhesive && dn > 0.0)) {
                int h;
                if (k >= cap) return DEM_ERR_CAP;
                npairs[2 * k] = i;
                npairs[2 * k + 1] = j;
                for (h = 0; h < NH; ++h) nhist[NH * k + h] = was ? ohist[NH * o + h] : 0.0;
                ++k;
            }
        }
    }
    *nnew = k;
    return DEM_OK;
}

/* Keep a spring vector in the tangent plane of n, preserving its length (J5). */
static void rotate_into_plane(double *xi, const double *n)
{
    double len0 = sqrt(dot3(xi, xi)), dn = dot3(xi, n), len1;
    int a;
    for (a = 0; a < 3; ++a) xi[a] -= dn * n[a];
    len1 = sqrt(dot3(xi, xi));
    if (len1 > 0.0) for (a = 0; a < 3; ++a) xi[a] *= len0 / len1;
}

/* Force and torque of one contact on i (fi, ti) and on j (fj, tj); updates its history. */
static int contact(const ora_dem_params *p, int i, int j, const double *X, const double *U,
                   const double *Om, const double *r, double *hist,
                   double *fi, double *ti, double *fj, double *tj)
{
    double d[3], dist, n[3], R, Es, FC, a0, dC, dn, ac, Fne;
    double mi, Ii, mj, Ij, ms, kN, etaN, kT, etaT, Gs;
    double arm_i[3], arm_j[3], w1[3], w2[3], vij[3], vn, vt[3], Fn, Ft[3], Fscrit, mag;
    double Omrel[3], Omt, Mt, Mtcrit, Mr[3], tq[3], mFt[3];
    double *xs = hist, *xt = hist + 3, *xr = hist + 4;
    int a, ok = 1;
    const double dt = p->dt;

    dn = pair_overlap(p, X, r, i, j, d, &dist);
    for (a = 0; a < 3; ++a) n[a] = d[a] / dist;
    pair_constants(p, r[i], r[j], &R, &Es, &FC, &a0, &dC);
    mass_inertia(p, r[i], &mi, &Ii);
    mass_inertia(p, r[j], &mj, &Ij);

    /* normal elastic force: JKR (Eq. 26-27, J1) or Hertz (J8) */
    if (p->adhesive) {
        ac = ora_jkr_contact_radius(dn, a0, R, &ok);
        Fne = ora_jkr_force(ac, a0, FC);
    } else {
        double dp = dn > 0.0 ? dn : 0.0;
        ac = sqrt(R * dp);
        Fne = 4.0 / 3.0 * Es * sqrt(R) * pow(dp, 1.5);
    }

    /* model constants (J4) */
    ms = mi * mj / (mi + mj);
    kN = 2.0 * Es * ac;
    etaN = p->alpha_n * sqrt(ms * kN);
    Gs = p->E / (4.0 * (2.0 - p->poisson) * (1.0 + p->poisson));
    kT = p->k_t_scale * 8.0 * Gs * ac;
    etaT = p->eta_t_scale * etaN;

    /* relative velocity of the contact points: (U_i + Om_i x r_i n) - (U_j + Om_j x (-r_j n)) */
    for (a = 0; a < 3; ++a) { arm_i[a] = r[i] * n[a]; arm_j[a] = -r[j] * n[a]; }
    cross3(&Om[3 * i], arm_i, w1);
    cross3(&Om[3 * j], arm_j, w2);
    for (a = 0; a < 3; ++a) vij[a] = (U[3 * i + a] + w1[a]) - (U[3 * j + a] + w2[a]);
    vn = dot3(vij, n);
    for (a = 0; a < 3; ++a) vt[a] = vij[a] - vn * n[a];

    /* normal force with damping (Eq. 26, J6) */
    Fn = Fne + etaN * vn;

    /* sliding spring-dashpot-slider (Eq. 28, first line; Eq. 29, J5) */
    Fscrit = p->mu_f * fabs(Fne + 2.0 * FC);
    rotate_into_plane(xs, n);
    for (a = 0; a < 3; ++a) xs[a] += vt[a] * dt;
    for (a = 0; a < 3; ++a) Ft[a] = -kT * xs[a] - etaT * vt[a];
    mag = sqrt(dot3(Ft, Ft));
    if (mag > Fscrit) {
        for (a = 0; a < 3; ++a) Ft[a] *= Fscrit / mag;
        if (kT > 0.0) for (a = 0; a < 3; ++a) xs[a] = -Ft[a] / kT;
    }

    /* twisting (Eq. 28, second line; zero for discs spinning about z) */
    for (a = 0; a < 3; ++a) Omrel[a] = Om[3 * i + a] - Om[3 * j + a];
    Omt = dot3(Omrel, n);
    xt[0] += Omt * dt;
    Mt = -(kT * ac * ac / 2.0) * xt[0] - (etaT * ac * ac / 2.0) * Omt;
    Mtcrit = 3.0 * PI * ac * Fscrit / 16.0;
    if (fabs(Mt) > Mtcrit) {
        Mt = (Mt > 0.0 ? 1.0 : -1.0) * Mtcrit;
        if (kT * ac * ac > 0.0) xt[0] = -Mt / (kT * ac * ac / 2.0);
    }

    /* rolling (Eq. 28, third line; |Eq. 29|): torque on i = k_r (n x xi_r) */
    for (a = 0; a < 3; ++a) Mr[a] = 0.0;
    if (p->adhesive) {
        double xa = ac / a0, kr, Mrcrit, vL[3];
        kr = 4.0 * FC * pow(xa, 1.5);
        Mrcrit = kr * p->theta_crit * R;
        rotate_into_plane(xr, n);
        cross3(n, Omrel, vL);
        for (a = 0; a < 3; ++a) xr[a] += R * vL[a] * dt;
        cross3(n, xr, tq);
        for (a = 0; a < 3; ++a) Mr[a] = kr * tq[a];
        mag = sqrt(dot3(Mr, Mr));
        if (mag > Mrcrit) {
            for (a = 0; a < 3; ++a) { Mr[a] *= Mrcrit / mag; xr[a] *= Mrcrit / mag; }
        }
    }

    /* assemble force and torque on both particles (Eq. 22) */
    for (a = 0; a < 3; ++a) { fi[a] = -Fn * n[a] + Ft[a]; fj[a] = Fn * n[a] - Ft[a]; }
    cross3(arm_i, Ft, tq);
    for (a = 0; a < 3; ++a) ti[a] = tq[a] + Mt * n[a] + Mr[a];
    for (a = 0; a < 3; ++a) mFt[a] = -Ft[a];
    cross3(arm_j, mFt, tq);
    for (a = 0; a < 3; ++a) tj[a] = tq[a] - Mt * n[a] - Mr[a];
    (void)Ii; (void)Ij; (void)dC;
    return ok ? DEM_OK : DEM_ERR_SOLVE;
}

/* W1: the wall of axis a nearer to particle i: unit normal n towards it and the overlap
 * delta_N = r_i - (distance from the centre to the plane) */
static double wall_overlap(const ora_dem_params *p, const double *X, const double *r, int i, int a, double *n)
{
    double dist;
    int b;
    for (b = 0; b < 3; ++b) n[b] = 0.0;
    if (X[3 * i + a] < 0.5 * (p->n[a] - 1)) {     /* lower wall, plane at -1/2 */
        dist = X[3 * i + a] + 0.5;
        n[a] = -1.0;
    } else {                                       /* upper wall, plane at n_a - 1/2 */
        dist = ((double)p->n[a] - 0.5) - X[3 * i + a];
        n[a] = 1.0;
    }
    return r[i] - dist;
}

/* Force and torque of particle i's contact with the wall of axis a (W1); hist its history. */
static int wall_contact(const ora_dem_params *p, int i, int a, const double *X, const double *U,
                        const double *Om, const double *r, double *hist, double *fi, double *ti)
{
    double n[3], R, Es, FC, a0, dC, dn, ac, Fne, mi, Ii, kN, etaN, kT, etaT, Gs;
    double arm_i[3], w1[3], vij[3], vn, vt[3], Fn, Ft[3], Fscrit, mag, Omt, Mt, Mtcrit, Mr[3], tq[3];
    double *xs = hist, *xt = hist + 3, *xr = hist + 4;
    int b, ok = 1;
    const double dt = p->dt;

    dn = wall_overlap(p, X, r, i, a, n);
    R = r[i];
    Es = p->E / (2.0 * (1.0 - p->poisson * p->poisson));
    if (p->adhesive) {
        FC = 3.0 * PI * p->gamma * R;
        a0 = cbrt(9.0 * PI * p->gamma * R * R / Es);
        dC = a0 * a0 / (2.0 * cbrt(6.0) * R);
        ac = ora_jkr_contact_radius(dn, a0, R, &ok);
        Fne = ora_jkr_force(ac, a0, FC);
    } else {
        double dp = dn > 0.0 ? dn : 0.0;
        FC = 0.0; a0 = 0.0; dC = 0.0;
        ac = sqrt(R * dp);
        Fne = 4.0 / 3.0 * Es * sqrt(R) * pow(dp, 1.5);
    }
    mass_inertia(p, r[i], &mi, &Ii);
    kN = 2.0 * Es * ac;
    etaN = p->alpha_n * sqrt(mi * kN);            /* m* = m_i against an immovable wall */
    Gs = p->E / (4.0 * (2.0 - p->poisson) * (1.0 + p->poisson));
    kT = p->k_t_scale * 8.0 * Gs * ac;
    etaT = p->eta_t_scale * etaN;

    /* velocity of i's contact point relative to the wall (at rest) */
    for (b = 0; b < 3; ++b) arm_i[b] = r[i] * n[b];
    cross3(&Om[3 * i], arm_i, w1);
    for (b = 0; b < 3; ++b) vij[b] = U[3 * i + b] + w1[b];
    vn = dot3(vij, n);
    for (b = 0; b < 3; ++b) vt[b] = vij[b] - vn * n[b];
    Fn = Fne + etaN * vn;

    Fscrit = p->mu_f * fabs(Fne + 2.0 * FC);
    rotate_into_plane(xs, n);
    for (b = 0; b < 3; ++b) xs[b] += vt[b] * dt;
    for (b = 0; b < 3; ++b) Ft[b] = -kT * xs[b] - etaT * vt[b];
    mag = sqrt(dot3(Ft, Ft));
    if (mag > Fscrit) {
        for (b = 0; b < 3; ++b) Ft[b] *= Fscrit / mag;
        if (kT > 0.0) for (b = 0; b < 3; ++b) xs[b] = -Ft[b] / kT;
    }

    Omt = dot3(&Om[3 * i], n);
    xt[0] += Omt * dt;
    Mt = -(kT * ac * ac / 2.0) * xt[0] - (etaT * ac * ac / 2.0) * Omt;
    Mtcrit = 3.0 * PI * ac * Fscrit / 16.0;
    if (fabs(Mt) > Mtcrit) {
        Mt = (Mt > 0.0 ? 1.0 : -1.0) * Mtcrit;
        if (kT * ac * ac > 0.0) xt[0] = -Mt / (kT * ac * ac / 2.0);
    }

    for (b = 0; b < 3; ++b) Mr[b] = 0.0;
    if (p->adhesive) {
        double xa = ac / a0, kr, Mrcrit, vL[3];
        kr = 4.0 * FC * pow(xa, 1.5);
        Mrcrit = kr * p->theta_crit * R;
        rotate_into_plane(xr, n);
        cross3(n, &Om[3 * i], vL);
        for (b = 0; b < 3; ++b) xr[b] += R * vL[b] * dt;
        cross3(n, xr, tq);
        for (b = 0; b < 3; ++b) Mr[b] = kr * tq[b];
        mag = sqrt(dot3(Mr, Mr));
        if (mag > Mrcrit) {
            for (b = 0; b < 3; ++b) { Mr[b] *= Mrcrit / mag; xr[b] *= Mrcrit / mag; }
        }
    }
    for (b = 0; b < 3; ++b) fi[b] = -Fn * n[b] + Ft[b];
    cross3(arm_i, Ft, tq);
    for (b = 0; b < 3; ++b) ti[b] = tq[b] + Mt * n[b] + Mr[b];
    (void)Ii; (void)dC;
    return ok ? DEM_OK : DEM_ERR_SOLVE;
}

/* substeps DEM sub-steps with the hydrodynamic force Ff and torque Tf frozen (Sec. 2.5).
 * Contacts (pairs, hist) in and out: sorted canonical pairs and their spring history;
 * *ncontact holds the count. X, U, Om are updated in place. */
int ora_dem_step(const ora_dem_params *p, int np, double *X, double *U, double *Om,
                 const double *r, const double *Ff, const double *Tf, int substeps,
                 int *ncontact, int *pairs, double *hist, int cap, int *wflag, double *whist)
{
    int s, k, i, a, rc = DEM_OK;
    int *npairs = (int *)malloc(sizeof(int) * 2 * (size_t)(cap > 0 ? cap : 1));
    double *nhist = (double *)malloc(sizeof(double) * NH * (size_t)(cap > 0 ? cap : 1));
    double *Fc = (double *)malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
    double *Mc = (double *)malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
    if (!npairs || !nhist || !Fc || !Mc) { free(npairs); free(nhist); free(Fc); free(Mc); return DEM_ERR_OOM; }
    for (s = 0; s < substeps && rc == DEM_OK; ++s) {
        int nn = 0;
        rc = detect(p, np, X, r, *ncontact, pairs, hist, &nn, npairs, nhist, cap);
        if (rc != DEM_OK) break;
        *ncontact = nn;
        memcpy(pairs, npairs, sizeof(int) * 2 * (size_t)nn);
        memcpy(hist, nhist, sizeof(double) * NH * (size_t)nn);
        for (i = 0; i < 3 * np; ++i) { Fc[i] = 0.0; Mc[i] = 0.0; }
        for (k = 0; k < nn; ++k) {
            double fi[3], ti[3], fj[3], tj[3];
            int pi = pairs[2 * k], pj = pairs[2 * k + 1];
            int c = contact(p, pi, pj, X, U, Om, r, &hist[NH * k], fi, ti, fj, tj);
            if (c != DEM_OK) rc = c;
            for (a = 0; a < 3; ++a) {
                Fc[3 * pi + a] += fi[a]; Mc[3 * pi + a] += ti[a];
                Fc[3 * pj + a] += fj[a]; Mc[3 * pj + a] += tj[a];
            }
        }
        /* W1: contacts with the walls of the non-periodic axes (after the pairs) */
        for (i = 0; i < np && wflag; ++i) {
            int ax;
            for (ax = 0; ax < p->dim; ++ax) {
                double n[3], fi[3], ti[3], dn, R, Es, FC, a0, dC;
                double *h = &whist[NH * (3 * (size_t)i + ax)];
                int was = wflag[3 * i + ax], on, hh;
                if (p->periodic[ax]) continue;
                dn = wall_overlap(p, X, r, i, ax, n);
                R = r[i];
                Es = p->E / (2.0 * (1.0 - p->poisson * p->poisson));
                a0 = p->adhesive ? cbrt(9.0 * PI * p->gamma * R * R / Es) : 0.0;
                dC = p->adhesive ? a0 * a0 / (2.0 * cbrt(6.0) * R) : 0.0;
                (void)FC;
                on = p->adhesive ? (dn >= 0.0 || (was && dn > -dC)) : (dn > 0.0);
                wflag[3 * i + ax] = on;
                if (!on) {
                    for (hh = 0; hh < NH; ++hh) h[hh] = 0.0;
                    continue;
                }
                {
                    int c = wall_contact(p, i, ax, X, U, Om, r, h, fi, ti);
                    if (c != DEM_OK) rc = c;
                }
                for (a = 0; a < 3; ++a) { Fc[3 * i + a] += fi[a]; Mc[3 * i + a] += ti[a]; }
            }
        }
        /* Eq. 21 with semi-implicit Euler (J7) */
        for (i = 0; i < np; ++i) {
            double m, I;
            mass_inertia(p, r[i], &m, &I);
            for (a = 0; a < 3; ++a) {
                if (a >= p->dim) continue;
                U[3 * i + a] += p->dt * (Ff[3 * i + a] + Fc[3 * i + a] + m * p->gravity[a]) / m;
                X[3 * i + a] += p->dt * U[3 * i + a];
                if (p->periodic[a]) X[3 * i + a] -= p->n[a] * floor(X[3 * i + a] / p->n[a]);
            }
            for (a = 0; a < 3; ++a) {
                if (p->dim == 2 && a < 2) continue;   /* discs spin about z only */
                Om[3 * i + a] += p->dt * (Tf[3 * i + a] + Mc[3 * i + a]) / I;
            }
        }
    }
    free(npairs); free(nhist); free(Fc); free(Mc);
    return rc;
}

/* Brute-force list of pairs with delta_N >= thresh (a check of the detection rule). */
int ora_pairs_within(const ora_dem_params *p, int np, const double *X, const double *r,
                     double thresh, int *pairs, int cap)
{
    int i, j, k = 0;
    for (i = 0; i < np; ++i)
        for (j = i + 1; j < np; ++j) {
            double d[3], dist;
            if (pair_overlap(p, X, r, i, j, d, &dist) >= thresh) {
                if (k >= cap) return -1;
                pairs[2 * k] = i; pairs[2 * k + 1] = j; ++k;
            }
        }
    return k;
}

/* Force and torque of the single contact (i, j) in the current state, with the given
 * history (updated as one sub-step would). For the pin tests of the contact law. */
int ora_dem_pair_force(const ora_dem_params *p, int np, const double *X, const double *U,
                       const double *Om, const double *r, int i, int j, double *hist,
                       double *fi, double *ti, double *fj, double *tj)
{
    if (i < 0 || j < 0 || i >= np || j >= np || i == j) return DEM_ERR_ARG;
    return contact(p, i, j, X, U, Om, r, hist, fi, ti, fj, tj);
}
