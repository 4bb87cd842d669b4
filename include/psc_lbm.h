/*
 * psc_lbm.h -- C ABI of the GB300 (sm_103a) library for the lattice-Boltzmann step with the
 * modified partially-saturated-cell (PSC) immersed moving boundary and the adhesive (JKR)
 * DEM contact update of Liu & Wu, "A hybrid LBM-DEM framework with an improved immersed
 * moving boundary method for modelling complex particle-liquid flows involving adhesive
 * particles" (arXiv 1901.09745).
 *
 * Conventions shared by every entry point
 *  - Lattice units: spacing and time step are 1; cell n has its centre at the integer
 *    coordinates (x, y, z), 0 <= x < nx etc. Positions, velocities (lattice units per
 *    step), spins and radii are in these units.
 *  - A wall axis (LBM_BC_BOUNCEBACK) has halfway bounce-back walls (Eq. 6) half a spacing
 *    beyond the first and the last node, at -1/2 and n - 1/2.
 *  - Population arrays exchanged with the caller are full f_i, FP64 (the device state
 *    itself stores deviations f_i - w_i in every precision),
 *    layout [Q][nz][ny][nx] (x fastest), in the velocity order below; they hold the
 *    pre-collision populations f_i(x, t) of Eq. 1.
 *      D2Q9 : 0 rest; 1 +x; 2 -x; 3 +y; 4 -y; 5 (+1,+1); 6 (-1,-1); 7 (+1,-1); 8 (-1,+1)
 *      D3Q19: 0 rest; 1 +x; 2 -x; 3 +y; 4 -y; 5 +z; 6 -z; 7 (1,1,0); 8 (-1,-1,0);
 *             9 (1,-1,0); 10 (-1,1,0); 11 (1,0,1); 12 (-1,0,-1); 13 (1,0,-1); 14 (-1,0,1);
 *             15 (0,1,1); 16 (0,-1,-1); 17 (0,1,-1); 18 (0,-1,1)
 *  - Particle vectors are arrays of n x 3 doubles (x, y, z per particle; z = 0 in 2D;
 *    in 2D only the z component of a spin or a torque is used).
 *  - Ownership: the caller owns every array it passes; the library copies what it needs
 *    and owns all device state held by a context. `on_device` = 1 means the pointer is a
 *    CUDA device pointer on the context's device, 0 means host memory.
 *  - Ordering: work is queued on the context's stream (lbm_params.stream, or a stream the
 *    library creates). Calls that return data in host memory synchronise that stream.
 *  - Errors: every call returns an lbm_status and never aborts; a device-side error
 *    (unstable density, contact solver failure) is recorded in a flag word on the device
 *    and reported by the next call that synchronises. lbm_last_error() gives a message.
 */
#ifndef PSC_LBM_H
#define PSC_LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;   /* opaque, library-owned fluid + particle state */
typedef struct dem_ctx dem_ctx;   /* opaque, library-owned contact state */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,            /* invalid argument (message in lbm_last_error) */
    LBM_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    LBM_ERR_OOM = 3,            /* device allocation failed */
    LBM_ERR_UNSUPPORTED = 4,    /* valid request the library does not provide */
    LBM_ERR_UNSTABLE = 5,       /* a cell reached a non-positive or NaN density */
    LBM_ERR_OVERFLOW = 6,       /* a fixed-capacity list overflowed */
    LBM_ERR_TIMEOUT = 7,        /* a bounded device wait gave up */
    DEM_ERR_NO_CONVERGENCE = 8  /* the JKR contact-radius solve did not converge */
} lbm_status;

enum { LBM_D2Q9 = 9, LBM_D3Q19 = 19 };
/* Faces of each axis. LBM_BC_OPEN: both faces open, a population entering through one is
 * the value the face cell itself would have pulled along the face (zero normal gradient).
 * LBM_BC_INFLOW (one axis a at most; x or y for D2Q9): the low face is a velocity inlet, the
 * high face a constant-pressure outlet. On the inlet face the populations that enter
 * (e_a = +1) are f_i = f_{-i} + 6 w_i rho e_i.u_in, the non-equilibrium part of the opposite
 * population bounced back, with rho fixed by the known populations so that the face cell
 * moves at u_in = lbm_params.inflow along a: rho (1 - u_a) = sum_{e_a=0} f + 2 sum_{e_a=-1} f.
 * On the outlet face those that enter (e_a = -1) take the same form at rho = 1 and u = u_a
 * along a, 1 + u_a = sum_{e_a=0} f + 2 sum_{e_a=+1} f. A population whose source also lies
 * beyond a wall bounces back at the wall instead. (The paper names these boundaries for its
 * drag test, Sec. 3.2, without formulas; this is the reading taken.) For the DEM every
 * non-periodic axis is walled. */
enum { LBM_BC_PERIODIC = 0, LBM_BC_BOUNCEBACK = 1, LBM_BC_OPEN = 2, LBM_BC_INFLOW = 3 };
/* Population storage. Compute is FP64 for LBM_F64 and FP32 for the others. Every form
 * stores deviations f_i - w_i from the lattice weights. */
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16_DEV = 2, LBM_BF16_DEV = 3 };
/* LBM_PSC_MODIFIED: Eq. 12-14 (per-particle weights, Eq. 13); LBM_PSC_ORIGINAL: Eq. 7-9, 11. */
enum { LBM_PSC_MODIFIED = 0, LBM_PSC_ORIGINAL = 1 };

typedef struct {
    int lattice;            /* LBM_D2Q9 | LBM_D3Q19 (Sec. 2.1) */
    int nx, ny, nz;         /* lattice extent; nz = 1 for D2Q9 */
    int bc[3];              /* per axis: LBM_BC_PERIODIC | LBM_BC_BOUNCEBACK (Sec. 2.2) | LBM_BC_OPEN |
                               LBM_BC_INFLOW (Sec. 3.2) */
    double tau;             /* relaxation parameter tau > 1/2 (Eq. 2); nu = (tau - 1/2)/3 */
    double body_force[3];   /* macroscopic body force F of Eq. 4 */
    int storage;            /* LBM_F64 | LBM_F32 | LBM_F16_DEV | LBM_BF16_DEV */
    int psc;                /* LBM_PSC_MODIFIED (default) | LBM_PSC_ORIGINAL */
    double shell_h;         /* h of Table 1 (<= 0 selects 1.0) */
    double dev_scale;       /* FP16/BF16 deviation scale s: stored value = s (f_i - w_i);
                               <= 0 selects 4096 for FP16 and 1 for BF16 */
    int tile_cap;           /* candidate particles kept per lattice tile (<= 0: 64) */
    void *stream;           /* cudaStream_t to queue work on; NULL: the library makes one */
    double inflow[3];       /* velocity imposed on the LBM_BC_INFLOW face (|u_a| < 0.3) */
} lbm_params;

/* Create a fluid at rest, f_i = f_i^eq(rho = 1, u = 0) = w_i (Eq. 3), with no particles.
 * Validates the parameters (LBM_ERR_ARG with a message on failure) and allocates the two
 * population buffers on the current CUDA device. *out receives the new context. */
lbm_status lbm_create(const lbm_params *p, lbm_ctx **out);

/* Release every device and host resource of the context (NULL is accepted). */
lbm_status lbm_destroy(lbm_ctx *ctx);

/* Replace the particle set: n particles with centres X, velocities U, spins Omega (each
 * n x 3) and radii (n), used by Eq. 10 (u_s = U + Omega x (x_n - X), Eq. 12) and by the
 * solid fractions of Table 1. Radii must satisfy r^2 > 1/2 in 3D (Eq. 17 is defined) and
 * r^2 > 1/4 in 2D (Eq. 19), and
 * a periodic axis must be longer than 2 (r + h) + 1; host values must be finite. Nothing
 * changes when a check fails (LBM_ERR_ARG with a message). on_device = 0: host arrays,
 * copied into the library's page-locked staging buffers before the call returns (the
 * caller may reuse them at once; the call does not wait for the device, whose upload
 * kernel reads the staging buffer in stream order); on_device = 1: device arrays, read by
 * the upload kernel in stream order. F and T are cleared. n = 0 removes all particles. A particle's index is its
 * identity: with an attached DEM context (dem_create), an upload of the same count and the
 * same radii keeps the DEM's neighbour list and contact history, and the list is rebuilt at
 * the next dem_step only when some particle now lies more than a quarter of the skin from
 * its position at the list's build (the criterion of the sub-steps); any other upload
 * rebuilds it (history carried over by index). */
lbm_status lbm_set_particles(lbm_ctx *ctx, int n, const double *X, const double *U,
                             const double *Omega, const double *radius, int on_device);

/* Advance nsteps lattice-Boltzmann steps. Each step bins the particles into lattice tiles,
 * computes every cell's solid fractions (Eq. 15-18, Table 1), weights (Eq. 9, 13),
 * collision (Eq. 2-5, 10, 12), streaming (Eq. 1, 6, periodic wrap) and the per-particle
 * force and torque (Eq. 14). Asynchronous on the context's stream. */
lbm_status lbm_step(lbm_ctx *ctx, int nsteps);

/* Force F and torque T (n x 3 each) on every particle from the last step's collision
 * (Eq. 14; Eq. 11 in original mode). Zero before the first step. Either may be NULL (not
 * both). on_device = 1: device arrays, copied in stream order. on_device = 0: host arrays;
 * the call synchronises and returns the status of the device's flag words (LBM_ERR_UNSTABLE,
 * DEM_ERR_NO_CONVERGENCE, LBM_ERR_OVERFLOW); page-locked arrays are written by one kernel
 * together with those words, pageable ones through cudaMemcpyAsync. */
lbm_status lbm_get_forces(lbm_ctx *ctx, double *F, double *T, int on_device);

/* Density rho (ncell) and force-shifted velocity u (ncell x 3) of Eq. 5 at the current
 * time, layout [nz][ny][nx] (u: [nz][ny][nx][3]). */
lbm_status lbm_get_macro(lbm_ctx *ctx, double *rho, double *u, int on_device);

/* Read or overwrite the pre-collision populations f_i(x, t) (layout above). Setting
 * converts to the context's storage format (rounding to nearest). */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f, int on_device);
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f, int on_device);

/* Checkpoint: raw copy of the populations, particles and step counter into a caller
 * buffer (host); when a DEM context is attached (dem_create) and has stepped, also its
 * neighbour lists and per-contact spring history. With buf = NULL, *used receives the size
 * needed. lbm_load_state restores a buffer written by lbm_save_state of a context with
 * identical parameters (and the DEM section into the attached DEM context; without one the
 * DEM starts again without contact history), so that the run continues exactly as the
 * saved one did. */
lbm_status lbm_save_state(lbm_ctx *ctx, void *buf, size_t cap, size_t *used);
lbm_status lbm_load_state(lbm_ctx *ctx, const void *buf, size_t size);

/* Replace the macroscopic body force F of Eq. 4 for the steps that follow. */
lbm_status lbm_set_body_force(lbm_ctx *ctx, const double *F);

/* Gradient of the time-averaged drag J = (1/T) sum_{t<T} sum_p F_{p,x}(t) (F_p of Eq. 14)
 * over the next T = nsteps steps, with respect to every particle position (dJdX, n x 3)
 * and the body force (dJdF, 3), by a hand-written reverse of the collide-stream step (the
 * paper has no adjoint; this is a derived quantity of Eq. 1-18). The particles must be
 * static (U = Omega = 0: LBM_ERR_UNSUPPORTED otherwise), storage FP32 or FP64, the
 * modified scheme, periodic or wall axes only, and every tile's candidates within tile_cap. Runs the T forward steps
 * (the context ends at step T as after lbm_step(ctx, T)), keeping a checkpoint every
 * checkpoint_every steps, then the reverse sweep, re-running each segment forward. The
 * gradient is exact for the discrete step except at the clamps of Table 1 (eps = 0 or 1,
 * sum eps = 1), where the one-sided derivative inside the unclamped region is used.
 * Memory: about (T / checkpoint_every + checkpoint_every + 2) population buffers.
 * J, dJdX and dJdF go to device memory when on_device, else host (synchronises). */
/* The two halves of lbm_adjoint_drag, for callers that want J now and the gradient only
 * later, if at all (an autograd forward and backward). lbm_adjoint_forward runs the T
 * forward steps with the checkpoints and returns J and a token; the checkpoints stay in
 * the context's adjoint workspace. lbm_adjoint_backward(token) runs the reverse sweep over
 * them and returns dJdX and dJdF; it may be called again with the same token. It fails
 * with LBM_ERR_ARG when a later lbm_adjoint_forward took the workspace (another token) or
 * when the particles or the body force changed since the forward (lbm_set_particles,
 * lbm_set_body_force, lbm_load_state, dem_step); lbm_step in between does not matter. The
 * requirements and memory are those of lbm_adjoint_drag. */
lbm_status lbm_adjoint_forward(lbm_ctx *ctx, int nsteps, int checkpoint_every, double *J, long long *token,
                               int on_device);
lbm_status lbm_adjoint_backward(lbm_ctx *ctx, long long token, double *dJdX, double *dJdF, int on_device);
lbm_status lbm_adjoint_drag(lbm_ctx *ctx, int nsteps, int checkpoint_every, double *J, double *dJdX,
                            double *dJdF, int on_device);

/* Bounds-checked build: 1 when this library was compiled with the kernels' index checks
 * (paper_1901_09745_gb300/build.py, build(checked=True): a separate libpsc_lbm_checked.so,
 * chosen by the Python binding when PSC_LBM_CHECKED=1), else 0. In such a build every main
 * global access of the kernels (populations, tiles and their records, particle indices,
 * DEM neighbour slots) tests its index; an index out of range is replaced by 0 and recorded.
 * lbm_check_violations synchronises the device and returns in *word the bits recorded since
 * the previous call (1 population, 2 tile or list slot, 4 particle, 8 record, 16 DEM
 * neighbour slot; 0 = none), then clears them; LBM_ERR_UNSUPPORTED in an unchecked build. */
int lbm_checked_build(void);
lbm_status lbm_check_violations(unsigned int *word);

/* Counters (the first n of): out[0] = steps taken, out[1] = tiles whose candidate list
 * overflowed tile_cap in the last binning (handled by a slower exact path, never an
 * error), out[2] = largest candidate count of a tile in the last binning, out[3] =
 * particles, out[4] = kernels launched by this context, out[5] = of which fused
 * collide-stream launches. Synchronises the stream. */
lbm_status lbm_get_info(lbm_ctx *ctx, long long *out, int n);

/* Optional CUDA-event timing of the fused collide-stream launches (used by the benchmark
 * to measure the kernel's own duration inside a timed run). A call returns, in *ms_total
 * and *launches (either may be NULL), the summed device time and the number of launches
 * timed since the previous call, synchronising the stream, then times every enable-th
 * step that follows (enable = 1: every step; 0: none). lbm_step replays each step from a
 * CUDA graph (captured on first use and whenever lbm_set_particles or lbm_set_body_force
 * changed what it reads); a timed step is queued kernel by kernel instead, with an event
 * on either side of the collide-stream kernels. */
lbm_status lbm_kernel_timing(lbm_ctx *ctx, int enable, double *ms_total, long long *launches);

/* ------------------------------------------------------------------ DEM (Sec. 2.5) --- */
/* Contact-model parameters, lattice units. One material for all particles (Eq. 25 then
 * gives 1/E* = 2 (1 - poisson^2) / E and 1/R = 1/r_i + 1/r_j). */
typedef struct {
    double E;            /* Young's modulus E_p */
    double poisson;      /* Poisson ratio sigma, in (-1, 1/2) */
    double gamma;        /* surface energy (JKR: F_C = 3 pi gamma R, Eq. 27 a0) */
    double density;      /* particle mass density: spheres m = rho 4/3 pi r^3, discs m = rho pi r^2 */
    double mu_f;         /* friction coefficient of Eq. 29 */
    double theta_crit;   /* critical rolling angle of Eq. 29 */
    double alpha_n;      /* normal damping: eta_N = alpha_n sqrt(m* k_N), k_N = 2 E* a */
    double k_t_scale;    /* tangential stiffness k_T = k_t_scale 8 G* a */
    double eta_t_scale;  /* tangential damping eta_T = eta_t_scale eta_N */
    double dt_dem;       /* DEM time step (LBM steps); lambda = 1 / dt_dem sub-steps per LBM step */
    double gravity[3];   /* G = m g of Eq. 21 */
    int adhesive;        /* 1: JKR normal force (Eq. 26); 0: Hertz (non-adhesive comparison) */
    double skin;         /* neighbour-list skin (<= 0: 0.5); particles may move skin/2 per call */
} dem_params;

/* Attach a DEM contact model to a fluid context (one per fluid). The DEM moves the fluid
 * context's particles. */
lbm_status dem_create(const dem_params *p, lbm_ctx *fluid, dem_ctx **out);
lbm_status dem_destroy(dem_ctx *dem);

/* Advance `substeps` DEM sub-steps of dt_dem (Eq. 21-29): contact detection (a pair enters
 * contact at delta_N >= 0 and stays while delta_N > -delta_C; likewise a particle and the
 * nearer wall of each non-periodic axis), JKR / Hertz normal force,
 * sliding, twisting and rolling resistance, semi-implicit Euler motion. The hydrodynamic
 * force and torque of the last lbm_step stay fixed over the sub-steps (Sec. 2.5). The new
 * positions, velocities and spins replace the fluid context's particle state. */
lbm_status dem_step(dem_ctx *dem, int substeps);

/* nsteps coupled steps (Sec. 2.5): each is lbm_step(fluid, 1) followed by
 * dem_step(dem, substeps), with the same results (up to the order of the FP64 force sums,
 * as between any two runs). dem must be attached to fluid (LBM_ERR_ARG otherwise). In 2D
 * with FP32 or 16-bit storage and an even sub-step count a step is one CUDA graph in which
 * the tiles without particle candidates, which the DEM does not read, are computed on a
 * second stream while the DEM call runs; the step ends with both streams joined, so the
 * context's stream orders everything, as for the two calls. Asynchronous. */
lbm_status lbm_coupled_step(lbm_ctx *fluid, dem_ctx *dem, int nsteps, int substeps);

/* Particle state after the last DEM sub-step (n x 3 each; NULL pointers are skipped). */
lbm_status dem_get_particles(dem_ctx *dem, double *X, double *U, double *Omega, int on_device);

/* Contacts of the last sub-step as canonical pairs i < j sorted by (i, j), and their
 * history seen from i (7 doubles each: sliding spring xyz, twist angle, rolling spring
 * xyz; hist may be NULL). Host memory. LBM_ERR_OVERFLOW if more than cap pairs (*n still
 * receives the count). */
lbm_status dem_get_contacts(dem_ctx *dem, int *pairs, double *hist, int cap, int *n);

/* Contacts with the walls (the planes at -1/2 and n - 1/2 of every non-periodic axis, met as
 * a half-space of the particles' material at rest: the law above with R = r, m* = m) after
 * the last sub-step, as (particle, axis) pairs sorted by particle, and their history (7
 * doubles each, as for pairs; hist may be NULL). LBM_ERR_OVERFLOW beyond cap. */
lbm_status dem_get_wall_contacts(dem_ctx *dem, int *pw, double *hist, int cap, int *n);

/* Counters (the first n of them): out[0] DEM kernels launched, out[1] contact solves that
 * did not converge, out[2] bin/neighbour-list overflows, out[3] skin violations, out[4]
 * particles, out[5] neighbour-list rebuilds. */
lbm_status dem_get_info(dem_ctx *dem, long long *out, int n);

/* ------------------------------------------------------------- slab decomposition --- */
/* The lattice cut into slabs along its slowest axis (y for D2Q9, z for D3Q19), the domain
 * decomposition by which the step shards: the update of a cell (Eq. 1-14) reads only its
 * neighbours, so a slab needs from the others only the populations that stream across its
 * faces (Eq. 1: the directions with e_s = +1 over its lower face, e_s = -1 over its upper one)
 * and gives each particle its share of the force and torque sums of Eq. 14.
 *
 * lbm_decomp_layout (pure host function): the rows each slab owns, own[k] .. own[k+1] - 1
 * (own has nslab + 1 entries; cuts on whole tile rows, 8 for D2Q9, 2 for D3Q19), and the
 * ghost layers its lattice holds below and above them (one tile row thick on a face shared
 * with another slab -- also across a periodic axis -- and 0 at a wall of the lattice). After
 * every step the populations with e_s = +1 of the last owned row below each face are copied
 * into the ghost row just above it, and those with e_s = -1 of the first owned row above the
 * face into the ghost row just below it. Returns 0, or -1 when a slab would own fewer rows
 * than a tile holds (or the lattice or nslab is invalid). */
int lbm_decomp_layout(int lattice, int n_s, int periodic_s, int nslab, int *own, int *ghost_lo, int *ghost_hi);

/* Which slabs hold which particle (pure host function): for slab k and particle i (centre
 * coordinate c[i] along the slab axis, radius[i]), img[k * n + i] is the image m in
 * {-1, 0, 1} whose centre c + m n_s puts the particle's shell (reach r + h + 1) over some of
 * the slab's owned rows, or -99 when none does (one slab: every particle, m = 0). Returns
 * 0, or -1 when the layout is invalid or a slab owns fewer than 2 (r + h) + 2 rows. */
int lbm_decomp_assign(int lattice, int n_s, int periodic_s, int nslab, double shell_h, int n, const double *c,
                      const double *radius, int *img);

/* A decomposed lattice: nslab slab contexts (all on the current device, stepped one after
 * the other on one stream) with the parameters of p for the whole lattice. Particles are
 * given to every slab whose owned rows their shell (r + h of Table 1) can reach, as the
 * periodic image next to that slab, and their force and torque are the sums of the slabs'
 * parts; each slab must own at least 2 (r + h) + 2 rows (LBM_ERR_ARG otherwise). The
 * populations and forces equal those of one context over the whole lattice (populations
 * bit for bit: every cell sums the same candidates in the same order). Host arrays only. */
typedef struct lbm_decomp lbm_decomp;
lbm_status lbm_decomp_create(const lbm_params *p, int nslab, lbm_decomp **out);
lbm_status lbm_decomp_destroy(lbm_decomp *d);
lbm_status lbm_decomp_set_particles(lbm_decomp *d, int n, const double *X, const double *U, const double *Omega,
                                    const double *radius);
lbm_status lbm_decomp_set_populations(lbm_decomp *d, const double *f);   /* whole lattice, as lbm_set_populations */
lbm_status lbm_decomp_get_populations(lbm_decomp *d, double *f);
lbm_status lbm_decomp_step(lbm_decomp *d, int nsteps);
lbm_status lbm_decomp_get_forces(lbm_decomp *d, double *F, double *T);  /* n x 3 each, totals per particle */
const char *lbm_decomp_last_error(const lbm_decomp *d);                  /* never NULL */

/* -------------------------------------------------- stepping without device allocation --- */
/* The paper has no counterpart to this entry point; it is a service for callers that may
 * not allocate GPU memory themselves or let a library do it: for example a host program
 * whose own memory manager owns every device allocation, a plugin living inside such a
 * program, or a real-time loop that forbids allocation (and the device-wide
 * synchronisation cudaMalloc/cudaFree can cause) once it runs.
 *
 * lbm_psc_step_noalloc performs the same single step as lbm_step (binning, solid fractions,
 * PSC collision, pull streaming, force and torque) on buffers the caller owns, and
 * allocates nothing: no cudaMalloc, no cudaFree, no host heap. Its working memory (tile
 * candidate lists and packed records, f(r) per particle, flag words) is one fixed array of
 * LBM_NOALLOC_SCRATCH_BYTES bytes that lives in the library image on every GPU that loads
 * the library, until the process exits. A lattice/particle set needing more working memory
 * than that is rejected with LBM_ERR_ARG and a message from lbm_noalloc_last_error().
 *
 *   p       lattice, extent, bc, tau, body force, storage, psc, shell_h, dev_scale as for
 *           lbm_create; p->stream is the stream to queue on (NULL = legacy default stream);
 *           tile_cap is ignored (16 candidate records per tile, more take an exact slow
 *           path).
 *   f_in    device buffer with the current state in the storage format of lbm_create's
 *           contexts: post-collision deviations f_i - w_i, [Q][nz][ny][nx], element type
 *           double / float / half / bfloat16 (FP16 scaled by dev_scale, default 4096), the
 *           bytes lbm_save_state writes after its 64-byte header.
 *   f_out   device buffer of the same size receiving the state after the step. f_out ==
 *           f_in and buffers not aligned to their element size are rejected with
 *           LBM_ERR_ARG (partly overlapping buffers are not detected: do not pass them).
 *   n, X, U, Omega, radius   particles as for lbm_set_particles, but device pointers; the
 *           caller guarantees the radius and box-size conditions stated there (the device
 *           data is not inspected on the host).
 *   F, T    device buffers (n x 3) receiving the force and torque of this step. Every
 *           particle array must be 8-byte aligned (LBM_ERR_ARG otherwise).
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and creates a second stream and two events there (a D2Q9 step runs two kernels side by
 * side, forked from p->stream and joined back into it), with that device current; make
 * that first call before any stream capture. The call is asynchronous on p->stream;
 * device-side instability is not reported by this entry point.
 * Every call shares the one array and finds whatever the previous call left there: each
 * call clears what must start at zero, but calls that overlap on the GPU (different streams
 * or host threads at the same time) corrupt each other's results — serialise them. */
#define LBM_NOALLOC_SCRATCH_BYTES (32u << 20)
lbm_status lbm_psc_step_noalloc(const lbm_params *p, const void *f_in, void *f_out, int n,
                                const double *X, const double *U, const double *Omega,
                                const double *radius, double *F, double *T);
/* Message of the last failed lbm_psc_step_noalloc call (never NULL). */
const char *lbm_noalloc_last_error(void);

/* Lattice tables: e (Q x 3), w (Q), opposite index (Q). Returns Q, or -1 for an unknown
 * lattice. Pure host function. */
int lbm_lattice_tables(int lattice, int *e, double *w, int *opp);

/* Message of the last failed call on this context (or of the last failed lbm_create when
 * ctx is NULL). Never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PSC_LBM_H */
