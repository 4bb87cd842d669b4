// decomp.cu -- the lattice cut into slabs along its slowest axis (y in 2D, z in 3D): the
// domain decomposition by which the method shards (the per-cell update of Eq. 1-14 is
// local; only the pull across a slab face and the per-particle sums of Eq. 14 cross it).
//
// Each slab is an ordinary context over its own rows plus, on every face that is not a
// wall of the lattice, a ghost layer of one tile's thickness (so the slab's tiles line up
// with the whole lattice's). Only the owned rows are updated (Geom::act0/act1); the
// ghost rows are read by the pull of the owned rows next to them. After every step the
// populations that cross each face -- the directions with e_s = +1 going up, e_s = -1 going
// down (3 of 9 in D2Q9, 5 of 19 in D3Q19) -- are copied from the owned row beside the face
// into the neighbour's ghost row, including the periodic face between the last slab and the
// first. A particle is given to every slab whose owned rows its shell (r + h) can reach,
// as the periodic image that lies next to that slab, in the order of the global indices
// (so every cell sums its candidates in the same order as the undivided lattice); each
// slab's force and torque on it are summed into the particle's total (the owner's sum).
//
// Here all slabs live on the current device and step one after the other (virtual
// sub-domains); the layout and the exchange are those a slab per GPU would use, with the
// face copies as peer copies or point-to-point messages and the force sums as one
// reduction of the ghost particles' partial sums.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/psc_lbm.h"
#include "capi_internal.h"
#include "lattice.cuh"

using namespace psc;

namespace {

constexpr int kMaxSlab = 64;
constexpr int kNotHeld = -99;     // lbm_decomp_assign: the slab does not hold the particle

// Tile thickness along the slab axis (the ghost layers keep the tiling aligned).
int slab_tile(int lattice) { return lattice == LBM_D2Q9 ? D2Q9::TY : D3Q19::TZ; }

__global__ void k_decomp_add(int n, const int *map, const double *Fp, const double *Tp, double *F, double *T) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int p = map[j];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        F[3 * p + a] += Fp[3 * j + a];
        T[3 * p + a] += Tp[3 * j + a];
    }
}

}  // namespace

struct lbm_decomp {
    lbm_params p;                 // parameters of the whole lattice
    int P, sax, q, dim, ns, periodic;
    int own[kMaxSlab + 1], glo[kMaxSlab], ghi[kMaxSlab];
    lbm_ctx *slab[kMaxSlab];
    int np;                       // particles of the whole lattice
    int nloc[kMaxSlab];
    int *map[kMaxSlab];           // device: slab-local particle -> global index
    double *F, *T;                // device: totals per particle
    int fcap;
    cudaStream_t stream;
    int own_stream;
    char err[512];
};

static char g_decomp_error[512] = "no error";

static lbm_status dfail(lbm_decomp *d, lbm_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(d ? d->err : g_decomp_error, sizeof(g_decomp_error), fmt, ap);
    va_end(ap);
    return st;
}

#define DDK(call, what)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return dfail(d, LBM_ERR_CUDA, "%s: %s", (what), cudaGetErrorString(e_)); \
    } while (0)

#define DST(call, k)                                                                                   \
    do {                                                                                               \
        lbm_status s_ = (call);                                                                        \
        if (s_ != LBM_OK) return dfail(d, s_, "slab %d: %s", (k), lbm_last_error(d->slab[k]));        \
    } while (0)

extern "C" int lbm_decomp_layout(int lattice, int n_s, int periodic_s, int nslab, int *own, int *ghost_lo,
                                 int *ghost_hi) {
    if ((lattice != LBM_D2Q9 && lattice != LBM_D3Q19) || nslab < 1 || nslab > kMaxSlab || n_s < 1) return -1;
    const int t = slab_tile(lattice);
    own[0] = 0;
    for (int k = 1; k < nslab; ++k) {
        const double cut = (double)k * n_s / nslab;
        own[k] = (int)floor(cut / t + 0.5) * t;
    }
    own[nslab] = n_s;
    for (int k = 0; k < nslab; ++k) {
        if (own[k + 1] - own[k] < t) return -1;       // every slab owns at least one tile row
        ghost_lo[k] = (nslab > 1 && (k > 0 || periodic_s)) ? t : 0;
        ghost_hi[k] = (nslab > 1 && (k < nslab - 1 || periodic_s)) ? t : 0;
    }
    return 0;
}

extern "C" int lbm_decomp_assign(int lattice, int n_s, int periodic_s, int nslab, double shell_h, int n,
                                 const double *c, const double *radius, int *img) {
    int own[kMaxSlab + 1], glo[kMaxSlab], ghi[kMaxSlab];
    if (lbm_decomp_layout(lattice, n_s, periodic_s, nslab, own, glo, ghi) != 0 || n < 0) return -1;
    const double h = shell_h > 0.0 ? shell_h : 1.0;
    for (int i = 0; i < n; ++i)
        if (nslab > 1)
            for (int k = 0; k < nslab; ++k)
                if (own[k + 1] - own[k] < 2.0 * (radius[i] + h) + 2.0) return -1;
    for (int k = 0; k < nslab; ++k) {
        const double lo = own[k], hi = own[k + 1];
        for (int i = 0; i < n; ++i) {
            int m_take = kNotHeld;
            if (nslab == 1) {
                m_take = 0;
            } else {
                const double reach = radius[i] + h + 1.0;
                const int nimg = periodic_s ? 3 : 1;
                for (int t = 0; t < nimg && m_take == kNotHeld; ++t) {
                    const int m = (t == 0) ? 0 : (t == 1 ? -1 : 1);
                    const double cm = c[i] + m * (double)n_s;
                    if (cm + reach >= lo && cm - reach <= hi - 1) m_take = m;
                }
            }
            img[(size_t)k * n + i] = m_take;
        }
    }
    return 0;
}

extern "C" const char *lbm_decomp_last_error(const lbm_decomp *d) { return d ? d->err : g_decomp_error; }

extern "C" lbm_status lbm_decomp_destroy(lbm_decomp *d) {
    if (!d) return LBM_OK;
    if (d->stream) cudaStreamSynchronize(d->stream);
    for (int k = 0; k < d->P; ++k) {
        lbm_destroy(d->slab[k]);
        if (d->map[k]) cudaFree(d->map[k]);
    }
    if (d->F) cudaFree(d->F);
    if (d->T) cudaFree(d->T);
    if (d->own_stream && d->stream) cudaStreamDestroy(d->stream);
    free(d);
    return LBM_OK;
}

extern "C" lbm_status lbm_decomp_create(const lbm_params *p, int nslab, lbm_decomp **out) {
    if (!p || !out) return dfail(NULL, LBM_ERR_ARG, "params and out must not be NULL");
    *out = NULL;
    lbm_decomp *d = (lbm_decomp *)calloc(1, sizeof(lbm_decomp));
    if (!d) return dfail(NULL, LBM_ERR_OOM, "host allocation failed");
    d->p = *p;
    d->q = p->lattice;
    d->dim = (p->lattice == LBM_D2Q9) ? 2 : 3;
    d->sax = d->dim - 1;
    const int n[3] = {p->nx, p->ny, p->nz};
    d->ns = n[d->sax];
    d->periodic = (p->bc[d->sax] == LBM_BC_PERIODIC);
    d->P = nslab;
    if (p->bc[d->sax] != LBM_BC_PERIODIC && p->bc[d->sax] != LBM_BC_BOUNCEBACK) {
        free(d);
        return dfail(NULL, LBM_ERR_UNSUPPORTED, "the slab axis must be periodic or walled");
    }
    snprintf(d->err, sizeof(d->err), "no error");
    if (lbm_decomp_layout(p->lattice, d->ns, d->periodic, nslab, d->own, d->glo, d->ghi) != 0) {
        dfail(NULL, LBM_ERR_ARG, "cannot cut %d rows into %d slabs of at least one tile row", d->ns, nslab);
        free(d);
        return LBM_ERR_ARG;
    }
    cudaError_t e = cudaSuccess;
    if (p->stream) {
        d->stream = (cudaStream_t)p->stream;
    } else {
        e = cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking);
        d->own_stream = 1;
    }
    if (e != cudaSuccess) {
        dfail(NULL, LBM_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
        free(d);
        return LBM_ERR_CUDA;
    }
    for (int k = 0; k < nslab; ++k) {
        lbm_params ps = *p;
        const int rows = d->glo[k] + (d->own[k + 1] - d->own[k]) + d->ghi[k];
        if (d->sax == 1) ps.ny = rows; else ps.nz = rows;
        // the slab axis of a slab ends in walls: the true walls of the lattice where it has
        // them, elsewhere a ghost layer that only inactive cells could pull across
        ps.bc[d->sax] = (nslab > 1) ? LBM_BC_BOUNCEBACK : p->bc[d->sax];
        ps.stream = d->stream;
        lbm_status st = lbm_create(&ps, &d->slab[k]);
        if (st != LBM_OK) {
            dfail(NULL, st, "slab %d: %s", k, lbm_last_error(NULL));
            lbm_decomp_destroy(d);
            return st;
        }
        lbm_ctx *c = d->slab[k];
        c->g.act0 = d->glo[k];                     // the slab axis is the slowest axis
        c->g.act1 = d->glo[k] + (d->own[k + 1] - d->own[k]);
        c->gen += 1;
    }
    *out = d;
    return LBM_OK;
}

// Copy the crossing populations of every face into the neighbours' ghost rows.
static lbm_status decomp_exchange(lbm_decomp *d) {
    if (d->P < 2) return LBM_OK;
    const int Q = d->q;
    for (int k = 0; k < d->P; ++k) {
        lbm_ctx *c = d->slab[k];
        const size_t e = c->elem;
        const size_t plane = (d->sax == 1) ? (size_t)c->g.n[0] : (size_t)c->g.n[0] * c->g.n[1];  // one row
        const size_t N = (size_t)c->g.ncell;
        char *base = (char *)c->f[c->cur];
        for (int i = 0; i < Q; ++i) {
            const int es = (d->sax == 1) ? ((Q == 9) ? D2Q9::ey(i) : D3Q19::ey(i)) : D3Q19::ez(i);
            if (es == 0) continue;
            int nb, src_row, dst_row;
            if (es > 0) {        // going up: into this slab's lower ghost row from the slab below
                if (d->glo[k] == 0) continue;
                nb = (k - 1 + d->P) % d->P;
                src_row = d->glo[nb] + (d->own[nb + 1] - d->own[nb]) - 1;
                dst_row = d->glo[k] - 1;
            } else {             // going down: into this slab's upper ghost row from the slab above
                if (d->ghi[k] == 0) continue;
                nb = (k + 1) % d->P;
                src_row = d->glo[nb];
                dst_row = d->glo[k] + (d->own[k + 1] - d->own[k]);
            }
            lbm_ctx *cn = d->slab[nb];
            const size_t Nn = (size_t)cn->g.ncell;
            const char *src = (const char *)cn->f[cn->cur] + ((size_t)i * Nn + (size_t)src_row * plane) * e;
            char *dst = base + ((size_t)i * N + (size_t)dst_row * plane) * e;
            DDK(cudaMemcpyAsync(dst, src, plane * e, cudaMemcpyDeviceToDevice, d->stream), "face copy");
        }
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_decomp_set_populations(lbm_decomp *d, const double *f) {
    if (!d || !f) return dfail(d, LBM_ERR_ARG, "f must not be NULL");
    const int Q = d->q, n0 = d->p.nx, n1 = d->p.ny, n2 = d->p.nz;
    const size_t plane = (d->sax == 1) ? (size_t)n0 : (size_t)n0 * n1;
    const size_t Nglob = (size_t)n0 * n1 * n2;
    for (int k = 0; k < d->P; ++k) {
        lbm_ctx *c = d->slab[k];
        const int rows = c->g.n[d->sax];
        const size_t N = (size_t)c->g.ncell;
        std::vector<double> loc((size_t)Q * N);
        for (int i = 0; i < Q; ++i)
            for (int r = 0; r < rows; ++r) {
                int gr = d->own[k] - d->glo[k] + r;
                if (gr < 0 || gr >= d->ns) {
                    if (!d->periodic) continue;      // never read
                    gr = (gr % d->ns + d->ns) % d->ns;
                }
                memcpy(&loc[(size_t)i * N + (size_t)r * plane], f + (size_t)i * Nglob + (size_t)gr * plane,
                       plane * sizeof(double));
            }
        DST(lbm_set_populations(c, loc.data(), 0), k);
    }
    // the rows next to the ghost layers were converted with the ghost rows' values; the
    // ghost rows themselves now take the neighbours' stored values
    lbm_status st = decomp_exchange(d);
    if (st != LBM_OK) return st;
    DDK(cudaStreamSynchronize(d->stream), "sync");
    return LBM_OK;
}

extern "C" lbm_status lbm_decomp_get_populations(lbm_decomp *d, double *f) {
    if (!d || !f) return dfail(d, LBM_ERR_ARG, "f must not be NULL");
    const int Q = d->q, n0 = d->p.nx, n1 = d->p.ny, n2 = d->p.nz;
    const size_t plane = (d->sax == 1) ? (size_t)n0 : (size_t)n0 * n1;
    const size_t Nglob = (size_t)n0 * n1 * n2;
    for (int k = 0; k < d->P; ++k) {
        lbm_ctx *c = d->slab[k];
        const size_t N = (size_t)c->g.ncell;
        std::vector<double> loc((size_t)Q * N);
        DST(lbm_get_populations(c, loc.data(), 0), k);
        for (int i = 0; i < Q; ++i)
            for (int gr = d->own[k]; gr < d->own[k + 1]; ++gr)
                memcpy(f + (size_t)i * Nglob + (size_t)gr * plane,
                       &loc[(size_t)i * N + (size_t)(gr - d->own[k] + d->glo[k]) * plane], plane * sizeof(double));
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_decomp_set_particles(lbm_decomp *d, int n, const double *X, const double *U,
                                               const double *Omega, const double *radius) {
    if (!d) return LBM_ERR_ARG;
    if (n < 0 || (n > 0 && (!X || !U || !Omega || !radius)))
        return dfail(d, LBM_ERR_ARG, "particle arrays must not be NULL");
    const double h = d->p.shell_h > 0.0 ? d->p.shell_h : 1.0;
    double rmax = 0.0;
    for (int i = 0; i < n; ++i) rmax = radius[i] > rmax ? radius[i] : rmax;
    for (int k = 0; k < d->P && d->P > 1; ++k)
        if (d->own[k + 1] - d->own[k] < 2.0 * (rmax + h) + 2.0)
            return dfail(d, LBM_ERR_ARG, "slab %d owns %d rows, fewer than a particle shell spans (2 (r + h) + 2)", k,
                         d->own[k + 1] - d->own[k]);
    if (d->fcap < n) {
        if (d->F) cudaFree(d->F);
        if (d->T) cudaFree(d->T);
        d->F = d->T = NULL;
        d->fcap = 0;
        DDK(cudaMalloc(&d->F, (size_t)(n > 0 ? n : 1) * 3 * sizeof(double)), "cudaMalloc(F)");
        DDK(cudaMalloc(&d->T, (size_t)(n > 0 ? n : 1) * 3 * sizeof(double)), "cudaMalloc(T)");
        d->fcap = n;
    }
    const int s = d->sax;
    std::vector<double> cs((size_t)n);
    for (int i = 0; i < n; ++i) cs[i] = X[3 * i + s];
    std::vector<int> img((size_t)d->P * (n > 0 ? n : 1));
    if (lbm_decomp_assign(d->q, d->ns, d->periodic, d->P, h, n, cs.data(), radius, img.data()) != 0)
        return dfail(d, LBM_ERR_ARG, "particle assignment failed");
    for (int k = 0; k < d->P; ++k) {
        std::vector<double> Xk, Uk, Ok, Rk;
        std::vector<int> mk;
        const double shift = d->own[k] - d->glo[k];             // global row of local row 0
        for (int i = 0; i < n; ++i) {
            const int m = img[(size_t)k * n + i];
            if (m == kNotHeld) continue;
            const double c = cs[i] + m * (double)d->ns;     // the image next to this slab
            for (int a = 0; a < 3; ++a) {
                Xk.push_back(a == s ? c - shift : X[3 * i + a]);
                Uk.push_back(U[3 * i + a]);
                Ok.push_back(Omega[3 * i + a]);
            }
            Rk.push_back(radius[i]);
            mk.push_back(i);
        }
        const int nk = (int)Rk.size();
        DST(lbm_set_particles(d->slab[k], nk, Xk.data(), Uk.data(), Ok.data(), Rk.data(), 0), k);
        if (d->map[k]) cudaFree(d->map[k]);
        d->map[k] = NULL;
        if (nk > 0) {
            DDK(cudaMalloc(&d->map[k], (size_t)nk * sizeof(int)), "cudaMalloc(particle map)");
            DDK(cudaMemcpyAsync(d->map[k], mk.data(), (size_t)nk * sizeof(int), cudaMemcpyHostToDevice, d->stream),
                "copy particle map");
        }
        d->nloc[k] = nk;
    }
    d->np = n;
    if (n > 0) {
        DDK(cudaMemsetAsync(d->F, 0, (size_t)n * 3 * sizeof(double), d->stream), "memset F");
        DDK(cudaMemsetAsync(d->T, 0, (size_t)n * 3 * sizeof(double), d->stream), "memset T");
    }
    DDK(cudaStreamSynchronize(d->stream), "sync");
    return LBM_OK;
}

extern "C" lbm_status lbm_decomp_step(lbm_decomp *d, int nsteps) {
    NvtxRange nvtx_("lbm_decomp_step");
    if (!d) return LBM_ERR_ARG;
    if (nsteps < 0) return dfail(d, LBM_ERR_ARG, "nsteps must be >= 0");
    for (int t = 0; t < nsteps; ++t) {
        for (int k = 0; k < d->P; ++k) DST(ctx_step_once(d->slab[k]), k);
        lbm_status st = decomp_exchange(d);
        if (st != LBM_OK) return st;
        if (d->np > 0) {
            // each particle's force and torque: the sum of its slabs' partial sums
            DDK(cudaMemsetAsync(d->F, 0, (size_t)d->np * 3 * sizeof(double), d->stream), "memset F");
            DDK(cudaMemsetAsync(d->T, 0, (size_t)d->np * 3 * sizeof(double), d->stream), "memset T");
            for (int k = 0; k < d->P; ++k) {
                if (d->nloc[k] == 0) continue;
                lbm_ctx *c = d->slab[k];
                k_decomp_add<<<(d->nloc[k] + 127) / 128, 128, 0, d->stream>>>(d->nloc[k], d->map[k], c->dF, c->dT,
                                                                              d->F, d->T);
                DDK(cudaGetLastError(), "force sum kernel");
            }
        }
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_decomp_get_forces(lbm_decomp *d, double *F, double *T) {
    if (!d) return LBM_ERR_ARG;
    if (d->np > 0) {
        if (F) DDK(cudaMemcpyAsync(F, d->F, (size_t)d->np * 3 * sizeof(double), cudaMemcpyDeviceToHost, d->stream), "copy F");
        if (T) DDK(cudaMemcpyAsync(T, d->T, (size_t)d->np * 3 * sizeof(double), cudaMemcpyDeviceToHost, d->stream), "copy T");
    }
    DDK(cudaStreamSynchronize(d->stream), "sync");
    for (int k = 0; k < d->P; ++k) DST(ctx_check_flags(d->slab[k]), k);
    return LBM_OK;
}

// the bounds-check word of this translation unit (see psc_internal.h)
PSC_CHECK_READER(psc_chk_take_decomp)
