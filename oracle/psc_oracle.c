/*
 * psc_oracle.c -- plain, slow FP64 CPU oracle for the lattice-Boltzmann step with the
 * modified partially-saturated-cell (PSC) immersed moving boundary of Liu & Wu,
 * "A hybrid LBM-DEM framework with an improved immersed moving boundary method for
 * modelling complex particle-liquid flows involving adhesive particles"
 * (arXiv 1901.09745).
 *
 * TEST INFRASTRUCTURE. This file exists only to check the CUDA library. Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load it. It
 * shares no code, header, table or constant with the CUDA path, and the CUDA path never
 * calls it.
 *
 * Everything is written in the paper's order and notation, one plain loop per step, in
 * double precision, single-threaded, with no blocking or fusion:
 *   O1  lattice tables (D2Q9 textbook weights; D3Q19 weights of Sec. 2.1)
 *   O2  f(r) of the linear solid-fraction approximation, Eq. 17/19 and Eq. 18
 *   O3  per-cell solid fraction by the algorithm of Table 1 (Eq. 15-18 plus the clamps)
 *   O4  weighting functions, Eq. 9 (original) and Eq. 13 (modified)
 *   O5  collision, Eq. 2-5 with the PSC term of Eq. 10 and Eq. 12 (or Eq. 7), then
 *       streaming, Eq. 1, with periodic wrap and halfway bounce-back walls, Eq. 6
 *   O6  hydrodynamic force and torque per particle, Eq. 14 (or Eq. 11)
 *
 * Readings where the paper is silent, garbled or ambiguous (the same readings are taken,
 * in independent code, by the CUDA library):
 *   R1  Eq. 17/19 integrand is sqrt(r^2-x^2-y^2) (sqrt(r^2-x^2) in 2D); the printed
 *       closed forms then hold with principal-value arctangents.
 *   R2  Table 1 Step 3 as printed swaps the two branches; Sec. 2.4 states cells inside
 *       are solid: distance <= r-h -> 1, distance >= r+h -> 0.
 *   R3  D = |x_n - X_p| - r_p (positive outside), eps = f(r) - D (Eq. 15).
 *   R6  when the particles' fractions in one cell sum above one, eps_n = min(1, sum)
 *       (Table 1 Step 5), B_n = B(eps_n) by Eq. 9, and B_{n,s} = B_n eps_s / sum_s eps_s,
 *       which equals Eq. 13 whenever the sum is at most one.
 *   R7  f^eq(rho,u) in the BGK term and in Eq. 10 uses the force-shifted u of Eq. 5.
 *   R8  u_s = U_p + Omega_p x (x_n - X_p).
 *   R9  F_p = -sum_n B_{n,s} sum_i Omega^s_i e_i (Eq. 14, reaction on the particle).
 *   R10 x_n - X_p is the minimum image along periodic axes.
 *   R12 walls are halfway (link) bounce-back, half a spacing beyond the first and last
 *       node of a wall axis; cell centres sit at integer coordinates 0..n-1.
 *   B1  the inlet, outlet and open boundaries of the drag test (Sec. 3.2), named there
 *       without formulas: a population f_i(x, t+1) whose source x - e_i lies beyond an open
 *       face (or the outlet) takes the post-collision value at the source moved back onto
 *       the face (zero gradient across it). The inlet is a velocity inlet: on its face the
 *       unknown populations (source beyond the inlet) are the opposite ones plus the
 *       difference of their equilibria (Eq. 3), f_i = f_{-i} + 6 w_i rho e_i.u_in, with
 *       rho the density for which the face cell moves at u_in across the face:
 *       rho (1 - u_in,a) = sum over e_a = 0 of f + 2 sum over e_a = -1 of f (a the inlet
 *       axis). The outlet (the paper's constant pressure) takes the same form at rho = 1
 *       with u = u_a along a, 1 + u_a = sum over e_a = 0 of f + 2 sum over e_a = +1 of f.
 *       A wall beyond any face of the source takes precedence, then the inlet and outlet.
 *   Original PSC (Eq. 7-9, 11) with several particles in a cell: the collision adds
 *   sum_s B(eps_s) Omega^s(u_s), B_n = sum_s B(eps_s) (Eq. 8), and each particle's force
 *   is weighted by the cell's total B_n (Eq. 11).
 *
 * Population layout: f[((i*nz + z)*ny + y)*nx + x], i.e. [Q][nz][ny][nx], full f_i (not
 * deviations). The state is the set of pre-collision populations f_i(x,t); one call of
 * ora_step collides at t (producing the forces of step t) and streams to t+1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_ERR_ARG 1
#define ORA_ERR_OOM 2
#define ORA_ERR_CAP 3

#define ORA_MAXK 8 /* most particles that may touch one cell */

typedef struct {
    int lattice;           /* 9 = D2Q9, 19 = D3Q19 */
    int nx, ny, nz;        /* nz = 1 for D2Q9 */
    int bc[3];             /* per axis: 0 periodic, 1 halfway bounce-back walls, 2 open faces,
                              3 velocity inlet (low face) and constant-pressure outlet (high
                              face); reading B1 */
    double tau;            /* relaxation parameter (dt = 1) */
    double body_force[3];  /* macroscopic body force F of Eq. 4 */
    int psc;               /* 0 = modified (Eq. 12-14), 1 = original (Eq. 7-9, 11) */
    double shell_h;        /* h of Table 1 */
    double inflow[3];      /* inlet velocity of axes with bc 3 */
} ora_params;

/* ---------------------------------------------------------------- O1: lattices --- */
/* Velocity order (shared interface format, written out independently here):
 *   D2Q9 : 0 rest; 1 +x; 2 -x; 3 +y; 4 -y; 5 (+1,+1); 6 (-1,-1); 7 (+1,-1); 8 (-1,+1)
 *   D3Q19: 0 rest; 1 +x; 2 -x; 3 +y; 4 -y; 5 +z; 6 -z;
 *          7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0)
 *          11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1)
 *          15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)                            */
static const int D2Q9_E[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
static const int D3Q19_E[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

typedef struct {
    int q, dim;
    int e[19][3];
    double w[19];
    int opp[19];
} ora_lattice;

/* Weights: D3Q19 w0 = 1/3, w1-6 = 1/18, w7-18 = 1/36 (Sec. 2.1, after Eq. 3);
 * D2Q9 uses the textbook 4/9, 1/9, 1/36 (the paper names D2Q9 only). The weight of a
 * velocity follows from its squared length. */
static int make_lattice(int lattice, ora_lattice *L)
{
    int i, k;
    if (lattice == 9) {
        L->q = 9; L->dim = 2;
        for (i = 0; i < 9; ++i) for (k = 0; k < 3; ++k) L->e[i][k] = D2Q9_E[i][k];
    } else if (lattice == 19) {
        L->q = 19; L->dim = 3;
        for (i = 0; i < 19; ++i) for (k = 0; k < 3; ++k) L->e[i][k] = D3Q19_E[i][k];
    } else {
        return ORA_ERR_ARG;
    }
    for (i = 0; i < L->q; ++i) {
        int len2 = L->e[i][0] * L->e[i][0] + L->e[i][1] * L->e[i][1] + L->e[i][2] * L->e[i][2];
        if (L->q == 9) L->w[i] = (len2 == 0) ? 4.0 / 9.0 : (len2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        else           L->w[i] = (len2 == 0) ? 1.0 / 3.0 : (len2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    /* opposite direction: the j with e_j = -e_i, found by search */
    for (i = 0; i < L->q; ++i) {
        int j;
        L->opp[i] = -1;
        for (j = 0; j < L->q; ++j)
            if (L->e[j][0] == -L->e[i][0] && L->e[j][1] == -L->e[i][1] && L->e[j][2] == -L->e[i][2])
                L->opp[i] = j;
    }
    return ORA_OK;
}

int ora_lattice_tables(int lattice, int *e, double *w, int *opp)
{
    ora_lattice L;
    int i;
    if (make_lattice(lattice, &L) != ORA_OK) return -1;
    for (i = 0; i < L.q; ++i) {
        e[3 * i + 0] = L.e[i][0]; e[3 * i + 1] = L.e[i][1]; e[3 * i + 2] = L.e[i][2];
        w[i] = L.w[i];
        opp[i] = L.opp[i];
    }
    return L.q;
}

/* ------------------------------------------------------ O2: linear approximation --- */
/* V_a of Eq. 17 (3D) / Eq. 19 (2D), with the square root restored in the integrand
 * (reading R1): the sphere's height sqrt(r^2-x^2-y^2) integrated over the unit square
 * (unit segment in 2D) centred on the axis through the particle centre. */
double ora_va(int dim, double r)
{
    if (dim == 2) {
        double s = sqrt(r * r - 0.25);
        return 0.5 * s + r * r * atan(0.5 / s);
    } else {
        double s = sqrt(r * r - 0.5);
        return (1.0 / 12.0 - r * r) * atan(0.5 * s / (0.5 - r * r))
             + s / 3.0
             + (r * r - 1.0 / 12.0) * atan(0.5 / s)
             - 4.0 / 3.0 * r * r * r * atan(0.25 / (r * s));
    }
}

/* Eq. 18: f(r) = V_a - r + 0.5 (from Eq. 16 with V_b = y_c - 0.5 and y_c = r + D). */
double ora_f_of_r(int dim, double r)
{
    return ora_va(dim, r) - r + 0.5;
}

/* ------------------------------------------------------------- O4: weights --- */
/* Eq. 9: B(eps, tau) = eps (tau - 1/2) / ((1 - eps) + (tau - 1/2)), with dt = 1. */
double ora_B(double eps, double tau)
{
    return eps * (tau - 0.5) / ((1.0 - eps) + (tau - 0.5));
}

/* Weights of one cell touched by k particles with fractions eps[0..k-1].
 * mode 0 (modified, Eq. 13 with reading R6): eps_n = min(1, sum eps); B_n = B(eps_n);
 *        B_{n,s} = B_n eps_s / sum eps.
 * mode 1 (original, Eq. 8-9): B_{n,s} = B(eps_s); B_n = sum_s B_{n,s}.
 * Returns B_n; writes B_{n,s} into Bs. */
double ora_cell_weights(int k, const double *eps, double tau, int mode, double *Bs)
{
    int s;
    double sum = 0.0, eps_n, Bn;
    if (mode == 1) {
        Bn = 0.0;
        for (s = 0; s < k; ++s) { Bs[s] = ora_B(eps[s], tau); Bn += Bs[s]; }
        return Bn;
    }
    for (s = 0; s < k; ++s) sum += eps[s];
    eps_n = sum < 1.0 ? sum : 1.0;                      /* Table 1 Step 5 */
    Bn = ora_B(eps_n, tau);
    for (s = 0; s < k; ++s) Bs[s] = (sum > 0.0) ? Bn * eps[s] / sum : 0.0;
    return Bn;
}

/* ------------------------------------------------------ O3: solid fraction --- */
/* Minimum-image component of a - b along an axis of length n (periodic), or the plain
 * difference along a wall axis (reading R10). */
static double axis_delta(double a, double b, int n, int periodic)
{
    double d = a - b;
    if (periodic) {
        while (d > 0.5 * n) d -= n;
        while (d < -0.5 * n) d += n;
    }
    return d;
}

typedef struct {
    int cnt;                 /* particles recorded in this cell (Table 1 Step 6) */
    int pid[ORA_MAXK];
    double eps[ORA_MAXK];
} cell_list;

/* Table 1, outer loop over particles, inner loop over the cells of the particle's
 * bounding box widened by h (reading of Step 1). Records every particle whose fraction
 * in the cell is positive. Returns ORA_ERR_CAP if a cell is touched by more than
 * ORA_MAXK particles, ORA_ERR_ARG if the widened box exceeds a periodic axis. */
static int collect_fractions(const ora_params *p, int dim, int np, const double *X,
                             const double *rad, cell_list *cells)
{
    int n[3] = {p->nx, p->ny, p->nz};
    long ncell = (long)p->nx * p->ny * p->nz;
    long c;
    int s;
    for (c = 0; c < ncell; ++c) cells[c].cnt = 0;
    for (s = 0; s < np; ++s) {
        double r = rad[s], h = p->shell_h;
        double fr = ora_f_of_r(dim, r);
        int lo[3], hi[3], a, ix, iy, iz;
        for (a = 0; a < 3; ++a) {
            if (a >= dim) { lo[a] = 0; hi[a] = 0; continue; }
            lo[a] = (int)ceil(X[3 * s + a] - r - h);
            hi[a] = (int)floor(X[3 * s + a] + r + h);
            if (p->bc[a] == 0 && hi[a] - lo[a] + 1 > n[a]) return ORA_ERR_ARG;
        }
        for (iz = lo[2]; iz <= hi[2]; ++iz)
        for (iy = lo[1]; iy <= hi[1]; ++iy)
        for (ix = lo[0]; ix <= hi[0]; ++ix) {
            int idx[3] = {ix, iy, iz};
            double dvec[3], dist, eps, D;
            int inside = 1;
            for (a = 0; a < 3; ++a) {
                if (a >= dim) { idx[a] = 0; dvec[a] = 0.0; continue; }
                if (p->bc[a] == 0) {
                    idx[a] = ((idx[a] % n[a]) + n[a]) % n[a];
                } else if (idx[a] < 0 || idx[a] >= n[a]) {
                    inside = 0;   /* beyond a wall: not a lattice cell */
                }
                dvec[a] = axis_delta((double)idx[a], X[3 * s + a], n[a], p->bc[a] == 0);
            }
            if (!inside) continue;
            /* Step 2: distance between the cell centre and the particle centre */
            dist = sqrt(dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2]);
            /* Step 3 (reading R2): outside the shell -> 0, inside -> 1, else Eq. 15 */
            if (dist >= r + h) {
                eps = 0.0;
            } else if (dist <= r - h) {
                eps = 1.0;
            } else {
                D = dist - r;                      /* reading R3 */
                eps = -D + fr;                     /* Eq. 15 with Eq. 18 */
            }
            /* Step 4: clamp to [0, 1] */
            if (eps <= 0.0) eps = 0.0;
            if (eps >= 1.0) eps = 1.0;
            if (eps > 0.0) {
                long cidx = ((long)idx[2] * n[1] + idx[1]) * n[0] + idx[0];
                cell_list *cl = &cells[cidx];
                if (cl->cnt >= ORA_MAXK) return ORA_ERR_CAP;
                cl->pid[cl->cnt] = s;              /* Step 6: record the particle */
                cl->eps[cl->cnt] = eps;
                cl->cnt += 1;
            }
        }
    }
    return ORA_OK;
}

/* Per-cell solid fractions: eps_sum[c] = sum_s eps_{n,s} (before the Step 5 clamp) and
 * nrec[c] = number of particles recorded. Also the per-(cell, particle) records when
 * pid/eps are non-NULL (capacity maxk per cell, -1 padding). */
int ora_solid_fraction(const ora_params *p, int np, const double *X, const double *rad,
                       double *eps_sum, int *nrec, int maxk, int *pid, double *eps)
{
    ora_lattice L;
    long ncell = (long)p->nx * p->ny * p->nz, c;
    cell_list *cells;
    int rc, k;
    if (make_lattice(p->lattice, &L) != ORA_OK) return ORA_ERR_ARG;
    cells = (cell_list *)malloc(sizeof(cell_list) * (size_t)ncell);
    if (!cells) return ORA_ERR_OOM;
    rc = collect_fractions(p, L.dim, np, X, rad, cells);
    if (rc == ORA_OK) {
        for (c = 0; c < ncell; ++c) {
            double sum = 0.0;
            for (k = 0; k < cells[c].cnt; ++k) sum += cells[c].eps[k];
            if (eps_sum) eps_sum[c] = sum;
            if (nrec) nrec[c] = cells[c].cnt;
            if (pid && eps) {
                for (k = 0; k < maxk; ++k) {
                    pid[c * maxk + k] = k < cells[c].cnt ? cells[c].pid[k] : -1;
                    eps[c * maxk + k] = k < cells[c].cnt ? cells[c].eps[k] : 0.0;
                }
            }
        }
    }
    free(cells);
    return rc;
}

/* ------------------------------------------------- O5/O6: collide and stream --- */
/* Eq. 3 with c_s^2 = 1/3. */
static double feq(const ora_lattice *L, int i, double rho, const double *v)
{
    double eu = L->e[i][0] * v[0] + L->e[i][1] * v[1] + L->e[i][2] * v[2];
    double uu = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    return rho * L->w[i] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

/* Eq. 4: Guo forcing term F_i (dt = 1, c_s^2 = 1/3). */
static double guo(const ora_lattice *L, int i, double tau, const double *u, const double *F)
{
    double eu = L->e[i][0] * u[0] + L->e[i][1] * u[1] + L->e[i][2] * u[2];
    double acc = 0.0;
    int a;
    for (a = 0; a < 3; ++a)
        acc += (3.0 * (L->e[i][a] - u[a]) + 9.0 * eu * L->e[i][a]) * F[a];
    return (1.0 - 1.0 / (2.0 * tau)) * L->w[i] * acc;
}

static void cross(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Eq. 5: rho and the force-shifted velocity u (reading R7). */
static void moments(const ora_lattice *L, const double *fc, const double *F, double *rho, double *u)
{
    int i, a;
    double m[3] = {0.0, 0.0, 0.0};
    *rho = 0.0;
    for (i = 0; i < L->q; ++i) {
        *rho += fc[i];
        for (a = 0; a < 3; ++a) m[a] += fc[i] * L->e[i][a];
    }
    for (a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * F[a]) / *rho;
}

void ora_macro(const ora_params *p, const double *f, double *rho, double *u)
{
    ora_lattice L;
    long ncell = (long)p->nx * p->ny * p->nz, c;
    int i;
    if (make_lattice(p->lattice, &L) != ORA_OK) return;
    for (c = 0; c < ncell; ++c) {
        double fc[19], r, v[3];
        for (i = 0; i < L.q; ++i) fc[i] = f[i * ncell + c];
        moments(&L, fc, p->body_force, &r, v);
        rho[c] = r;
        u[3 * c + 0] = v[0]; u[3 * c + 1] = v[1]; u[3 * c + 2] = v[2];
    }
}

/* One LBM step: collide every cell at time t (Eq. 12, or Eq. 7 in original mode),
 * accumulate each particle's force and torque (Eq. 14, or Eq. 11), then stream with
 * periodic wrap and halfway bounce-back (Eq. 1, Eq. 6). f holds pre-collision
 * populations at t on entry and at t+1 on return. F and T (np x 3) receive the force
 * and torque of this step. Bn_out (optional, one per cell) receives B_n. */
int ora_step(const ora_params *p, double *f, int np, const double *X, const double *U,
             const double *Om, const double *rad, double *F, double *T, double *Bn_out)
{
    ora_lattice L;
    int n[3] = {p->nx, p->ny, p->nz};
    long ncell = (long)p->nx * p->ny * p->nz, c;
    double *fpost;
    cell_list *cells;
    int rc, s, i, a;

    if (make_lattice(p->lattice, &L) != ORA_OK) return ORA_ERR_ARG;
    if (L.dim == 2 && p->nz != 1) return ORA_ERR_ARG;
    if (!(p->tau > 0.5)) return ORA_ERR_ARG;
    fpost = (double *)malloc(sizeof(double) * (size_t)L.q * (size_t)ncell);
    cells = (cell_list *)malloc(sizeof(cell_list) * (size_t)ncell);
    if (!fpost || !cells) { free(fpost); free(cells); return ORA_ERR_OOM; }

    rc = collect_fractions(p, L.dim, np, X, rad, cells);
    if (rc != ORA_OK) { free(fpost); free(cells); return rc; }
    for (s = 0; s < np; ++s)
        for (a = 0; a < 3; ++a) { F[3 * s + a] = 0.0; T[3 * s + a] = 0.0; }

    for (c = 0; c < ncell; ++c) {
        int x = (int)(c % n[0]);
        int y = (int)((c / n[0]) % n[1]);
        int z = (int)(c / ((long)n[0] * n[1]));
        double fc[19], fe[19], fi[19], coll[19];
        double rho, u[3], Bn, Bs[ORA_MAXK];
        cell_list *cl = &cells[c];

        for (i = 0; i < L.q; ++i) fc[i] = f[i * ncell + c];
        moments(&L, fc, p->body_force, &rho, u);
        for (i = 0; i < L.q; ++i) {
            fe[i] = feq(&L, i, rho, u);
            fi[i] = guo(&L, i, p->tau, u, p->body_force);
            coll[i] = 0.0;
        }
        Bn = ora_cell_weights(cl->cnt, cl->eps, p->tau, p->psc, Bs);
        if (Bn_out) Bn_out[c] = Bn;

        for (s = 0; s < cl->cnt; ++s) {
            int ps = cl->pid[s];
            double arm[3], spin[3], us[3], dP[3] = {0.0, 0.0, 0.0}, dT[3], wF;
            double xn[3] = {(double)x, (double)y, (double)z};
            for (a = 0; a < 3; ++a)
                arm[a] = (a < L.dim) ? axis_delta(xn[a], X[3 * ps + a], n[a], p->bc[a] == 0) : 0.0;
            cross(&Om[3 * ps], arm, spin);
            for (a = 0; a < 3; ++a) us[a] = U[3 * ps + a] + spin[a];   /* reading R8 */
            for (i = 0; i < L.q; ++i) {
                int o = L.opp[i];
                /* Eq. 10 */
                double om = fc[o] - feq(&L, o, rho, u) + feq(&L, i, rho, us) - fc[i];
                coll[i] += Bs[s] * om;                                  /* Eq. 12 */
                for (a = 0; a < 3; ++a) dP[a] += om * L.e[i][a];
            }
            /* Eq. 14 weights by B_{n,s}; Eq. 11 (original) weights by B_n */
            wF = (p->psc == 1) ? Bn : Bs[s];
            for (a = 0; a < 3; ++a) dP[a] *= wF;
            cross(arm, dP, dT);
            for (a = 0; a < 3; ++a) { F[3 * ps + a] -= dP[a]; T[3 * ps + a] -= dT[a]; }
        }
        for (i = 0; i < L.q; ++i)
            fpost[i * ncell + c] = fc[i] - (1.0 - Bn) * (fc[i] - fe[i]) / p->tau
                                 + coll[i] + (1.0 - Bn) * fi[i];
    }

    /* streaming (push): f_i(x + e_i, t+1) = f_i^+(x, t); a link that leaves through a
     * wall returns to its own cell in the opposite direction, f_{-i}(x, t+1) = f_i^+; one
     * that leaves through an open face or the inlet leaves the lattice */
    for (c = 0; c < ncell; ++c) {
        int xc[3] = {(int)(c % n[0]), (int)((c / n[0]) % n[1]), (int)(c / ((long)n[0] * n[1]))};
        for (i = 0; i < L.q; ++i) {
            int dst[3], wall = 0, leaves = 0;
            long dc;
            for (a = 0; a < 3; ++a) {
                dst[a] = xc[a] + L.e[i][a];
                if (dst[a] < 0 || dst[a] >= n[a]) {
                    if (p->bc[a] == 0) dst[a] = (dst[a] + n[a]) % n[a];
                    else if (p->bc[a] == 1) wall = 1;
                    else leaves = 1;
                }
            }
            if (wall) {
                f[L.opp[i] * ncell + c] = fpost[i * ncell + c];
            } else if (!leaves) {
                dc = ((long)dst[2] * n[1] + dst[1]) * n[0] + dst[0];
                f[i * ncell + dc] = fpost[i * ncell + c];
            }
        }
    }
    /* the populations that come in through an open face or the inlet (B1): those whose
     * source x - e_i lies beyond such a face and beyond no wall */
    for (c = 0; c < ncell; ++c) {
        int xc[3] = {(int)(c % n[0]), (int)((c / n[0]) % n[1]), (int)(c / ((long)n[0] * n[1]))};
        for (i = 0; i < L.q; ++i) {
            int src[3], wall = 0, inlet = 0, outside = 0;
            for (a = 0; a < 3; ++a) {
                src[a] = xc[a] - L.e[i][a];
                if (src[a] >= 0 && src[a] < n[a]) continue;
                if (p->bc[a] == 0) { src[a] = (src[a] + n[a]) % n[a]; continue; }
                if (p->bc[a] == 1) { wall = 1; continue; }
                outside = 1;
                if (p->bc[a] == 3) inlet = 1;           /* the inlet or the outlet: below */
                src[a] = src[a] < 0 ? 0 : n[a] - 1;     /* onto the face */
            }
            if (wall || !outside || inlet) continue;
            {
                long sc = ((long)src[2] * n[1] + src[1]) * n[0] + src[0];
                f[i * ncell + c] = fpost[i * ncell + sc];
            }
        }
    }
    /* the velocity inlet and the constant-pressure outlet (B1): on the inlet face (x_a = 0)
     * and the outlet face (x_a = n_a - 1), the populations whose source lies beyond that face
     * and beyond no wall. The inlet takes rho from the known populations and u = u_in; the
     * outlet takes rho = 1 and u = u_a along a, u_a from the known populations. */
    for (a = 0; a < 3; ++a) {
        int side;
        if (p->bc[a] != 3) continue;
        for (side = 0; side < 2; ++side) {
            const int face = side ? n[a] - 1 : 0, in_dir = side ? -1 : 1;
            for (c = 0; c < ncell; ++c) {
                int xc[3] = {(int)(c % n[0]), (int)((c / n[0]) % n[1]), (int)(c / ((long)n[0] * n[1]))};
                double known = 0.0, rho, u[3];
                int b;
                if (xc[a] != face) continue;
                /* known: e_a = 0 once, e_a pointing out of the lattice through this face twice */
                for (i = 0; i < L.q; ++i) {
                    if (L.e[i][a] == 0) known += f[i * ncell + c];
                    else if (L.e[i][a] == -in_dir) known += 2.0 * f[i * ncell + c];
                }
                if (!side) {
                    /* rho (1 - u_a) = known */
                    rho = known / (1.0 - p->inflow[a]);
                    for (b = 0; b < 3; ++b) u[b] = p->inflow[b];
                } else {
                    /* rho = 1: 1 + u_a = known */
                    rho = 1.0;
                    for (b = 0; b < 3; ++b) u[b] = 0.0;
                    u[a] = known - 1.0;
                }
                for (i = 0; i < L.q; ++i) {
                    int wall = 0;
                    double eu = 0.0;
                    if (L.e[i][a] != in_dir) continue;
                    for (b = 0; b < 3; ++b) {
                        int sb = xc[b] - L.e[i][b];
                        if (b != a && (sb < 0 || sb >= n[b]) && p->bc[b] == 1) wall = 1;
                    }
                    if (wall) continue;
                    for (b = 0; b < 3; ++b) eu += L.e[i][b] * u[b];
                    /* f_i - f_{-i} = f^eq_i - f^eq_{-i} = 6 w_i rho e_i.u (Eq. 3) */
                    f[i * ncell + c] = f[L.opp[i] * ncell + c] + 6.0 * L.w[i] * rho * eu;
                }
            }
        }
    }
    free(fpost);
    free(cells);
    return ORA_OK;
}

/* nsteps of ora_step with static particles; F and T hold the last step's values. */
int ora_run(const ora_params *p, double *f, int nsteps, int np, const double *X,
            const double *U, const double *Om, const double *rad, double *F, double *T)
{
    int t, rc = ORA_OK;
    for (t = 0; t < nsteps && rc == ORA_OK; ++t)
        rc = ora_step(p, f, np, X, U, Om, rad, F, T, NULL);
    return rc;
}

/* Equilibrium populations f_i^eq(rho, u) of Eq. 3 for a whole field (initial states). */
int ora_equilibrium(const ora_params *p, const double *rho, const double *u, double *f)
{
    ora_lattice L;
    long ncell = (long)p->nx * p->ny * p->nz, c;
    int i;
    if (make_lattice(p->lattice, &L) != ORA_OK) return ORA_ERR_ARG;
    for (c = 0; c < ncell; ++c)
        for (i = 0; i < L.q; ++i) f[i * ncell + c] = feq(&L, i, rho[c], &u[3 * c]);
    return ORA_OK;
}

/* Time-averaged x-drag J = (1/T) sum_{t<T} sum_p F_{p,x}(t) over nsteps steps (Eq. 14
 * forces, static particles); f advances by nsteps. The finite-difference gradient of this
 * objective is the oracle's gradient for the adjoint checks. */
int ora_drag(const ora_params *p, double *f, int nsteps, int np, const double *X, const double *U,
             const double *Om, const double *rad, double *J)
{
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
    double *T = (double *)malloc(sizeof(double) * 3 * (size_t)(np > 0 ? np : 1));
    int t, s, rc = ORA_OK;
    if (!F || !T) { free(F); free(T); return ORA_ERR_OOM; }
    *J = 0.0;
    for (t = 0; t < nsteps && rc == ORA_OK; ++t) {
        rc = ora_step(p, f, np, X, U, Om, rad, F, T, NULL);
        for (s = 0; s < np; ++s) *J += F[3 * s] / nsteps;
    }
    free(F);
    free(T);
    return rc;
}
