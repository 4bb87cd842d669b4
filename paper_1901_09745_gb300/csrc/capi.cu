// capi.cu -- host side of the C ABI declared in include/psc_lbm.h: context management,
// argument checking, device buffers, and the per-step launch sequence (bin particles ->
// fused PSC collide-stream). Every entry point returns an lbm_status and never aborts.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "../../include/psc_lbm.h"
#include "capi_internal.h"
#include "hostcheck.h"
#include "lattice.cuh"
#include "psc_internal.h"

namespace psc {
cudaError_t launch_collide_stream_f64(int, const void *, void *, const Geom &, const Phys &, const Tiles &, const Parts &, int *, cudaStream_t,
                                     Overlap *);
cudaError_t launch_collide_stream_f32(int, const void *, void *, const Geom &, const Phys &, const Tiles &, const Parts &, int *, cudaStream_t,
                                     Overlap *);
cudaError_t launch_collide_stream_f16(int, const void *, void *, const Geom &, const Phys &, const Tiles &, const Parts &, int *, cudaStream_t,
                                     Overlap *);
cudaError_t launch_collide_stream_bf16(int, const void *, void *, const Geom &, const Phys &, const Tiles &, const Parts &, int *, cudaStream_t,
                                     Overlap *);
cudaError_t launch_gather_f64(int, const void *, double *, double *, double *, const Geom &, const Phys &, cudaStream_t);
cudaError_t launch_gather_f32(int, const void *, double *, double *, double *, const Geom &, const Phys &, cudaStream_t);
cudaError_t launch_gather_f16(int, const void *, double *, double *, double *, const Geom &, const Phys &, cudaStream_t);
cudaError_t launch_gather_bf16(int, const void *, double *, double *, double *, const Geom &, const Phys &, cudaStream_t);
cudaError_t launch_set_f64(int, const double *, void *, const Geom &, const Phys &, cudaStream_t);
cudaError_t launch_set_f32(int, const double *, void *, const Geom &, const Phys &, cudaStream_t);
cudaError_t launch_set_f16(int, const double *, void *, const Geom &, const Phys &, cudaStream_t);
cudaError_t launch_set_bf16(int, const double *, void *, const Geom &, const Phys &, cudaStream_t);

cudaError_t launch_collide_stream(int storage, int lattice, const void *fin, void *fout, const Geom &g,
                                  const Phys &ph, const Tiles &tl, const Parts &pd, int *flags,
                                  cudaStream_t s, Overlap *ov) {
    switch (storage) {
    case ST_F64: return launch_collide_stream_f64(lattice, fin, fout, g, ph, tl, pd, flags, s, ov);
    case ST_F32: return launch_collide_stream_f32(lattice, fin, fout, g, ph, tl, pd, flags, s, ov);
    case ST_F16: return launch_collide_stream_f16(lattice, fin, fout, g, ph, tl, pd, flags, s, ov);
    default: return launch_collide_stream_bf16(lattice, fin, fout, g, ph, tl, pd, flags, s, ov);
    }
}
cudaError_t launch_gather(int storage, int lattice, const void *fin, double *f_out, double *rho, double *u,
                          const Geom &g, const Phys &ph, cudaStream_t s) {
    switch (storage) {
    case ST_F64: return launch_gather_f64(lattice, fin, f_out, rho, u, g, ph, s);
    case ST_F32: return launch_gather_f32(lattice, fin, f_out, rho, u, g, ph, s);
    case ST_F16: return launch_gather_f16(lattice, fin, f_out, rho, u, g, ph, s);
    default: return launch_gather_bf16(lattice, fin, f_out, rho, u, g, ph, s);
    }
}
cudaError_t launch_set(int storage, int lattice, const double *f, void *fout, const Geom &g, const Phys &ph,
                       cudaStream_t s) {
    switch (storage) {
    case ST_F64: return launch_set_f64(lattice, f, fout, g, ph, s);
    case ST_F32: return launch_set_f32(lattice, f, fout, g, ph, s);
    case ST_F16: return launch_set_f16(lattice, f, fout, g, ph, s);
    default: return launch_set_bf16(lattice, f, fout, g, ph, s);
    }
}
}  // namespace psc

using namespace psc;

static char g_create_error[512] = "no error";

void ctx_error(lbm_ctx *ctx, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx ? ctx->err : g_create_error, sizeof(g_create_error), fmt, ap);
    va_end(ap);
}

lbm_status ctx_cuda(lbm_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_OK;
    ctx_error(ctx, "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define CK(call, what)                                         \
    do {                                                       \
        lbm_status st_ = ctx_cuda(ctx, (call), (what));        \
        if (st_ != LBM_OK) return st_;                         \
    } while (0)

static size_t elem_bytes(int storage) {
    switch (storage) {
    case LBM_F64: return 8;
    case LBM_F32: return 4;
    default: return 2;
    }
}

static void free_dev(void **p) {
    if (*p) cudaFree(*p);
    *p = NULL;
}

static void free_particles(lbm_ctx *ctx) {
    free_dev((void **)&ctx->dX); free_dev((void **)&ctx->dU); free_dev((void **)&ctx->dOm);
    free_dev((void **)&ctx->dR); free_dev((void **)&ctx->dFr); free_dev((void **)&ctx->dF);
    free_dev((void **)&ctx->dT); free_dev((void **)&ctx->dPf);
    ctx->np_cap = 0;
}

extern "C" int lbm_lattice_tables(int lattice, int *e, double *w, int *opp_out) {
    int q;
    if (lattice == LBM_D2Q9) q = 9;
    else if (lattice == LBM_D3Q19) q = 19;
    else return -1;
    for (int i = 0; i < q; ++i) {
        int ex, ey, ez;
        if (q == 9) { ex = D2Q9::ex(i); ey = D2Q9::ey(i); ez = 0; }
        else { ex = D3Q19::ex(i); ey = D3Q19::ey(i); ez = D3Q19::ez(i); }
        if (e) { e[3 * i] = ex; e[3 * i + 1] = ey; e[3 * i + 2] = ez; }
        if (w) w[i] = (q == 9) ? weight<D2Q9>(i) : weight<D3Q19>(i);
        if (opp_out) opp_out[i] = (q == 9) ? opp<D2Q9>(i) : opp<D3Q19>(i);
    }
    return q;
}

extern "C" const char *lbm_last_error(const lbm_ctx *ctx) { return ctx ? ctx->err : g_create_error; }

static lbm_status validate(const lbm_params *p) {
    if (!p) { ctx_error(NULL, "params is NULL"); return LBM_ERR_ARG; }
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) {
        ctx_error(NULL, "lattice must be LBM_D2Q9 (9) or LBM_D3Q19 (19), got %d", p->lattice);
        return LBM_ERR_ARG;
    }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) {
        ctx_error(NULL, "lattice extent must be positive, got %d x %d x %d", p->nx, p->ny, p->nz);
        return LBM_ERR_ARG;
    }
    if (p->lattice == LBM_D2Q9 && p->nz != 1) { ctx_error(NULL, "D2Q9 needs nz = 1, got %d", p->nz); return LBM_ERR_ARG; }
    for (int a = 0; a < 3; ++a)
        if (p->bc[a] < LBM_BC_PERIODIC || p->bc[a] > LBM_BC_INFLOW) {
            ctx_error(NULL, "bc[%d] must be LBM_BC_PERIODIC, _BOUNCEBACK, _OPEN or _INFLOW, got %d", a, p->bc[a]);
            return LBM_ERR_ARG;
        }
    {
        int ninlet = 0;
        for (int a = 0; a < 3; ++a) ninlet += (p->bc[a] == LBM_BC_INFLOW);
        const int dimp = (p->lattice == LBM_D2Q9) ? 2 : 3;
        if (ninlet > 1 || (dimp == 2 && (p->bc[2] == LBM_BC_INFLOW || p->bc[2] == LBM_BC_OPEN))) {
            ctx_error(NULL, "at most one axis may be LBM_BC_INFLOW, and z of a D2Q9 lattice must be periodic or bounce-back");
            return LBM_ERR_ARG;
        }
    }
    for (int a = 0; a < 3; ++a)
        if (!isfinite(p->inflow[a]) || fabs(p->inflow[a]) > 0.3) {
            ctx_error(NULL, "inflow velocity components must be finite and below 0.3 in magnitude");
            return LBM_ERR_ARG;
        }
    if (!(p->tau > 0.5) || !isfinite(p->tau)) { ctx_error(NULL, "tau must exceed 1/2 (nu = (tau - 1/2)/3 > 0), got %g", p->tau); return LBM_ERR_ARG; }
    for (int a = 0; a < 3; ++a)
        if (!isfinite(p->body_force[a])) { ctx_error(NULL, "body force must be finite"); return LBM_ERR_ARG; }
    if (p->storage < LBM_F64 || p->storage > LBM_BF16_DEV) { ctx_error(NULL, "unknown storage %d", p->storage); return LBM_ERR_ARG; }
    if (p->psc != LBM_PSC_MODIFIED && p->psc != LBM_PSC_ORIGINAL) { ctx_error(NULL, "unknown psc mode %d", p->psc); return LBM_ERR_ARG; }
    if (!isfinite(p->shell_h) || p->shell_h > 1e6) { ctx_error(NULL, "shell_h must be finite"); return LBM_ERR_ARG; }
    if (p->tile_cap > 64) { ctx_error(NULL, "tile_cap must be at most 64, got %d", p->tile_cap); return LBM_ERR_ARG; }
    if (!isfinite(p->dev_scale)) { ctx_error(NULL, "dev_scale must be finite"); return LBM_ERR_ARG; }
    double ncell = (double)p->nx * p->ny * p->nz;
    if (ncell * p->lattice > 4.0e12) { ctx_error(NULL, "lattice too large"); return LBM_ERR_ARG; }
    const int ty = (p->lattice == LBM_D2Q9) ? D2Q9::TY : D3Q19::TY, tz = (p->lattice == LBM_D2Q9) ? 1 : D3Q19::TZ;
    if ((p->ny + ty - 1) / ty > 65535 || (p->nz + tz - 1) / tz > 65535) {
        ctx_error(NULL, "ny or nz too large for the tile grid (at most 65535 tiles per axis)");
        return LBM_ERR_ARG;
    }
    const int tx = (p->lattice == LBM_D2Q9) ? D2Q9::TX : D3Q19::TX;
    const double ntiles = (double)((p->nx + tx - 1) / tx) * ((p->ny + ty - 1) / ty) * ((p->nz + tz - 1) / tz);
    if (ntiles > 2147483647.0) { ctx_error(NULL, "too many lattice tiles (at most 2^31 - 1)"); return LBM_ERR_ARG; }
    return LBM_OK;
}

extern "C" lbm_status lbm_create(const lbm_params *p, lbm_ctx **out) {
    if (!out) { ctx_error(NULL, "out is NULL"); return LBM_ERR_ARG; }
    *out = NULL;
    lbm_status st = validate(p);
    if (st != LBM_OK) return st;
    lbm_ctx *ctx = (lbm_ctx *)calloc(1, sizeof(lbm_ctx));
    if (!ctx) { ctx_error(NULL, "host allocation failed"); return LBM_ERR_OOM; }
    ctx->hR_n = -1;
    ctx->p = *p;
    if (ctx->p.shell_h <= 0.0) ctx->p.shell_h = 1.0;
    if (ctx->p.tile_cap <= 0) ctx->p.tile_cap = 64;
    if (ctx->p.dev_scale <= 0.0) ctx->p.dev_scale = (p->storage == LBM_F16_DEV) ? 4096.0 : 1.0;
    if (p->storage == LBM_F64 || p->storage == LBM_F32) ctx->p.dev_scale = 1.0;
    snprintf(ctx->err, sizeof(ctx->err), "no error");
    ctx->q = p->lattice;
    ctx->dim = (p->lattice == LBM_D2Q9) ? 2 : 3;
    ctx->elem = elem_bytes(p->storage);
    Geom &g = ctx->g;
    g.n[0] = p->nx; g.n[1] = p->ny; g.n[2] = p->nz;
    g.ncell = (long long)p->nx * p->ny * p->nz;
    g.faces = 0;
    g.act0 = 0;
    g.act1 = (ctx->dim == 2) ? g.n[1] : g.n[2];
    for (int a = 0; a < 3; ++a) {
        g.periodic[a] = (p->bc[a] == LBM_BC_PERIODIC);
        g.wrap_img[a] = 0;
        const int lo = p->bc[a] == LBM_BC_PERIODIC ? FACE_PERIODIC : p->bc[a] == LBM_BC_BOUNCEBACK ? FACE_WALL
                     : p->bc[a] == LBM_BC_OPEN ? FACE_OPEN : FACE_INFLOW;
        set_face_kind(g, a, 0, lo);
        set_face_kind(g, a, 1, lo == FACE_INFLOW ? FACE_OUTLET : lo);
    }
    for (int a = 0; a < 3; ++a) {
        g.nt[a] = (g.n[a] + tile_ext(ctx->dim, a) - 1) / tile_ext(ctx->dim, a);
        g.inv_n[a] = 1.0 / g.n[a];
    }
    ctx->ntiles = (long long)g.nt[0] * g.nt[1] * g.nt[2];
    Phys &ph = ctx->ph;
    ph.tau = p->tau;
    for (int a = 0; a < 3; ++a) ph.body_force[a] = p->body_force[a];
    ph.shell_h = ctx->p.shell_h;
    ph.scale = ctx->p.dev_scale;
    ph.psc = p->psc;
    for (int a = 0; a < 3; ++a) ph.inflow[a] = p->inflow[a];
    ph.inflow_axis = -1;
    for (int a = 0; a < 3; ++a)
        if (p->bc[a] == LBM_BC_INFLOW) ph.inflow_axis = a;

    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess && p->stream) {
        ctx->stream = (cudaStream_t)p->stream;
        ctx->own_stream = 0;
    } else if (e == cudaSuccess) {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        ctx->own_stream = 1;
    }
    // the second stream of the 2D step (fluid and particle tiles side by side)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->ov.aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ov.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ov.join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ov.prep, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ctx->stage_ev[k], cudaEventDisableTiming);
    size_t bytes = (size_t)g.ncell * ctx->q * ctx->elem;
    if (e == cudaSuccess) e = cudaMalloc(&ctx->f[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->f[1], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->flags, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&ctx->hflags, 4 * sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&ctx->hflags_dev, ctx->hflags, 0);
    // rest state f_i = w_i: every stored deviation is zero (all-zero bits in every format)
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->f[0], 0, bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->f[1], 0, bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->flags, 0, 4 * sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        ctx_error(NULL, "lbm_create: %s", cudaGetErrorString(e));
        lbm_status s2 = (e == cudaErrorMemoryAllocation) ? LBM_ERR_OOM : LBM_ERR_CUDA;
        lbm_destroy(ctx);
        return s2;
    }
    *out = ctx;
    return LBM_OK;
}

extern "C" lbm_status lbm_destroy(lbm_ctx *ctx) {
    if (!ctx) return LBM_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->dem) dem_release(ctx->dem);
    free_dev(&ctx->f[0]); free_dev(&ctx->f[1]);
    free_dev((void **)&ctx->flags);
    if (ctx->hflags) cudaFreeHost(ctx->hflags);
    free(ctx->hR);
    for (int k = 0; k < 2; ++k) {
        if (ctx->stage[k]) cudaFreeHost(ctx->stage[k]);
        if (ctx->stage_ev[k]) cudaEventDestroy(ctx->stage_ev[k]);
    }
    free_particles(ctx);
    free_dev((void **)&ctx->tile_count); free_dev((void **)&ctx->tile_list); free_dev((void **)&ctx->tile_stats);
    free_dev((void **)&ctx->tile_order);
    free_dev(&ctx->tile_blocks);
    free_dev((void **)&ctx->diag);
    free_dev(&ctx->adj);
    for (int i = 0; i < ctx->ev_cap; ++i) cudaEventDestroy(ctx->ev[i]);
    free(ctx->ev);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            if (ctx->sgraph[a][b]) cudaGraphExecDestroy(ctx->sgraph[a][b]);
            if (ctx->cgraph[a][b]) cudaGraphExecDestroy(ctx->cgraph[a][b]);
        }
    if (ctx->ov.aux) cudaStreamDestroy(ctx->ov.aux);
    if (ctx->ov.fork) cudaEventDestroy(ctx->ov.fork);
    if (ctx->ov.join) cudaEventDestroy(ctx->ov.join);
    if (ctx->ov.prep) cudaEventDestroy(ctx->ov.prep);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    free(ctx);
    return LBM_OK;
}

Parts ctx_parts(lbm_ctx *ctx) {
    Parts pd;
    pd.n = ctx->np; pd.X = ctx->dX; pd.U = ctx->dU; pd.Om = ctx->dOm; pd.R = ctx->dR; pd.Fr = ctx->dFr;
    pd.F = ctx->dF; pd.T = ctx->dT;
    pd.Pf = ctx->dPf;
    return pd;
}

static Tiles ctx_tiles(lbm_ctx *ctx) {
    Tiles tl;
    tl.count = ctx->tile_count; tl.list = ctx->tile_list; tl.cap = ctx->p.tile_cap; tl.stats = ctx->tile_stats;
    tl.order = ctx->tile_order;
    tl.blocks = ctx->tile_blocks;
    return tl;
}

// Minimum-image flags: a periodic axis needs the per-cell minimum image when the tile plus
// the widest particle shell does not fit well inside half the box.
void ctx_update_wrap(lbm_ctx *ctx) {
    for (int a = 0; a < 3; ++a) {
        double need = tile_ext(ctx->dim, a) + 2.0 * (ctx->rmax + ctx->p.shell_h) + 2.0;
        const int w = (a < ctx->dim && ctx->g.periodic[a] && ctx->g.n[a] < need) ? 1 : 0;
        if (w != ctx->g.wrap_img[a]) ctx->gen += 1;     // the step's kernels take Geom by value
        ctx->g.wrap_img[a] = w;
    }
}

lbm_status ctx_check_radii(lbm_ctx *ctx, const double *R, int n) {
    const double rmin2 = (ctx->dim == 2) ? 0.25 : 0.5;
    // one branch-free pass (smallest r^2, largest r); the per-particle search only for the
    // message when it finds a radius out of range
    double s2min, rmax;
    psc::radii_range(R, n, &s2min, &rmax);
    if (n > 0 && (!(s2min > rmin2) || !psc::all_finite(R, (size_t)n))) {
        for (int i = 0; i < n; ++i) {
            if (!(R[i] * R[i] > rmin2) || !isfinite(R[i])) {
                ctx_error(ctx, "radius %d = %g: the linear approximation (Eq. 17/19) needs r^2 > %g", i, R[i], rmin2);
                return LBM_ERR_ARG;
            }
        }
    }
    for (int a = 0; a < ctx->dim; ++a) {
        if (ctx->g.periodic[a] && n > 0 && ctx->g.n[a] <= (int)floor(2.0 * (rmax + ctx->p.shell_h)) + 1) {
            ctx_error(ctx, "periodic axis %d of length %d is too short for radius %g and h %g", a, ctx->g.n[a], rmax,
                      ctx->p.shell_h);
            return LBM_ERR_ARG;
        }
    }
    ctx->rmax = rmax;
    return LBM_OK;
}

lbm_status ctx_reserve_particles(lbm_ctx *ctx, int n) {
    if (n <= ctx->np_cap) return LBM_OK;
    ctx->gen += 1;      // new buffers: the step's graph is captured again
    free_particles(ctx);
    size_t v = (size_t)n * 3 * sizeof(double), s = (size_t)n * sizeof(double);
    CK(cudaMalloc(&ctx->dX, v), "cudaMalloc(X)");
    CK(cudaMalloc(&ctx->dU, v), "cudaMalloc(U)");
    CK(cudaMalloc(&ctx->dOm, v), "cudaMalloc(Omega)");
    CK(cudaMalloc(&ctx->dR, s), "cudaMalloc(radius)");
    CK(cudaMalloc(&ctx->dFr, s), "cudaMalloc(f(r))");
    CK(cudaMalloc(&ctx->dF, v), "cudaMalloc(F)");
    CK(cudaMalloc(&ctx->dT, v), "cudaMalloc(T)");
    CK(cudaMalloc(&ctx->dPf, (size_t)n * 2 * sizeof(float4)), "cudaMalloc(FP32 record data)");
    CK(cudaMemsetAsync(ctx->dF, 0, v, ctx->stream), "memset F");
    CK(cudaMemsetAsync(ctx->dT, 0, v, ctx->stream), "memset T");
    ctx->np_cap = n;
    return LBM_OK;
}

static lbm_status ctx_reserve_tiles(lbm_ctx *ctx) {
    if (ctx->tile_count) return LBM_OK;
    ctx->gen += 1;
    CK(cudaMalloc(&ctx->tile_count, (size_t)ctx->ntiles * sizeof(int)), "cudaMalloc(tile counts)");
    CK(cudaMalloc(&ctx->tile_list, (size_t)ctx->ntiles * ctx->p.tile_cap * sizeof(int)), "cudaMalloc(tile lists)");
    CK(cudaMalloc(&ctx->tile_stats, kTileStats * sizeof(int)), "cudaMalloc(tile stats)");
    CK(cudaMalloc(&ctx->tile_order, (size_t)ctx->ntiles * 3 * sizeof(uint2)), "cudaMalloc(tile order)");
    CK(cudaMalloc(&ctx->tile_blocks, (size_t)ctx->ntiles * pack_block_bytes(ctx->p.storage == LBM_F64, ctx->p.tile_cap)),
       "cudaMalloc(tile candidate blocks)");
    CK(cudaMemsetAsync(ctx->tile_stats, 0, kTileStats * sizeof(int), ctx->stream), "memset tile stats");
    return LBM_OK;
}

// The address at which this context's kernels can read or write the caller's array: device
// memory of this device, managed memory, or page-locked host memory mapped into the
// device's address space. NULL for pageable host memory and for another device's memory
// (cudaMemcpyAsync moves those).
static void *device_view(const lbm_ctx *ctx, const void *p) {
    if (!p) return NULL;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return NULL;
    }
    switch (at.type) {
    case cudaMemoryTypeDevice: return at.device == ctx->device ? at.devicePointer : NULL;
    case cudaMemoryTypeHost:
    case cudaMemoryTypeManaged: return at.devicePointer;
    default: return NULL;
    }
}

// The staging buffer for a host upload of n particles (10 n doubles: X, U, Omega, radii):
// its host address, *dev its device address and *k its index; NULL when page-locked memory
// for it cannot be had (the caller then copies and synchronises instead). Waits for the
// upload that read the buffer last (normally long finished: the other buffer served the
// upload in between).
static double *ctx_stage(lbm_ctx *ctx, int n, const double **dev, int *k) {
    const size_t need = (size_t)n * 10;
    if (need > ctx->stage_cap) {
        for (int b = 0; b < 2; ++b) {
            if (ctx->stage_busy[b]) cudaEventSynchronize(ctx->stage_ev[b]);
            ctx->stage_busy[b] = 0;
            if (ctx->stage[b]) cudaFreeHost(ctx->stage[b]);
            ctx->stage[b] = ctx->stage_dev[b] = NULL;
        }
        ctx->stage_cap = 0;
        for (int b = 0; b < 2; ++b) {
            if (cudaHostAlloc((void **)&ctx->stage[b], need * sizeof(double), cudaHostAllocMapped) != cudaSuccess ||
                cudaHostGetDevicePointer((void **)&ctx->stage_dev[b], ctx->stage[b], 0) != cudaSuccess) {
                cudaGetLastError();
                for (int c = 0; c < 2; ++c) {
                    if (ctx->stage[c]) cudaFreeHost(ctx->stage[c]);
                    ctx->stage[c] = ctx->stage_dev[c] = NULL;
                }
                return NULL;
            }
        }
        ctx->stage_cap = need;
    }
    const int b = ctx->stage_k;
    if (ctx->stage_busy[b]) {
        if (cudaEventSynchronize(ctx->stage_ev[b]) != cudaSuccess) {
            cudaGetLastError();
            return NULL;
        }
        ctx->stage_busy[b] = 0;
    }
    *dev = ctx->stage_dev[b];
    *k = b;
    return ctx->stage[b];
}

extern "C" lbm_status lbm_set_particles(lbm_ctx *ctx, int n, const double *X, const double *U,
                                        const double *Omega, const double *radius, int on_device) {
    if (!ctx) return LBM_ERR_ARG;
    NvtxRange nvtx_("lbm_set_particles");
    ctx->mods += 1;
    if (n < 0 || n > (1 << 24)) { ctx_error(ctx, "particle count must be in [0, 2^24], got %d", n); return LBM_ERR_ARG; }
    if (n > 0 && (!X || !U || !Omega || !radius)) { ctx_error(ctx, "particle arrays must not be NULL"); return LBM_ERR_ARG; }
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // validate on the host (device radii are copied back once); nothing on the device
    // changes before the arguments pass
    double *hr = NULL;
    const double *Rh = radius;
    if (n > 0) {
        if (on_device) {
            hr = (double *)malloc((size_t)n * sizeof(double));
            if (!hr) { ctx_error(ctx, "host allocation failed"); return LBM_ERR_OOM; }
            cudaError_t e = cudaMemcpyAsync(hr, radius, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) { free(hr); return ctx_cuda(ctx, e, "copy radii"); }
            Rh = hr;
        }
        lbm_status st = ctx_check_radii(ctx, Rh, n);
        if (st != LBM_OK) { free(hr); return st; }
        if (!on_device && !(psc::all_finite(X, 3 * (size_t)n) && psc::all_finite(U, 3 * (size_t)n) &&
                            psc::all_finite(Omega, 3 * (size_t)n))) {
            for (int i = 0; i < 3 * n; ++i)
                if (!isfinite(X[i]) || !isfinite(U[i]) || !isfinite(Omega[i])) {
                    ctx_error(ctx, "particle %d has a non-finite position, velocity or spin", i / 3);
                    return LBM_ERR_ARG;
                }
        }
    }
    // the radii of the last upload are kept on the host: with the same count and radii the
    // DEM may keep its neighbour list (the device then tests the displacements)
    const int same_radii = n > 0 && ctx->hR_n == n && memcmp(ctx->hR, Rh, (size_t)n * sizeof(double)) == 0;
    if (n > 0 && !same_radii) {
        if (n > ctx->hR_cap) {
            double *t = (double *)realloc(ctx->hR, (size_t)n * sizeof(double));
            if (!t) { free(hr); ctx_error(ctx, "host allocation failed"); return LBM_ERR_OOM; }
            ctx->hR = t;
            ctx->hR_cap = n;
        }
        memcpy(ctx->hR, Rh, (size_t)n * sizeof(double));
    }
    free(hr);
    ctx->hR_n = -1;     // until the upload below has been queued
    lbm_status st = ctx_reserve_particles(ctx, n);
    if (st != LBM_OK) return st;
    int keep_list = 0;
    if (n > 0) {
        Upload u;
        memset(&u, 0, sizeof(u));
        u.n = n;
        u.dim = ctx->dim;
        u.dX = ctx->dX; u.dU = ctx->dU; u.dOm = ctx->dOm; u.dR = ctx->dR; u.dFr = ctx->dFr;
        u.dF = ctx->dF; u.dT = ctx->dT;
        for (int a = 0; a < 3; ++a) { u.n_lat[a] = ctx->g.n[a]; u.periodic[a] = ctx->g.periodic[a]; }
        if (ctx->dem && same_radii) keep_list = dem_upload_check(ctx->dem, n, &u.ref, &u.req, &u.lim2);
        // host arrays are copied into a page-locked staging buffer that the kernel reads,
        // so the call need not wait for the device; device arrays (or, without a staging
        // buffer, mapped page-locked ones) are read by the kernel directly; others are
        // first copied into the context's arrays and the kernel then reads those in place
        const double *sdev = NULL;
        int sk = 0;
        double *sh = on_device ? NULL : ctx_stage(ctx, n, &sdev, &sk);
        const size_t n3 = (size_t)n * 3;
        const void *v[4] = {NULL, NULL, NULL, NULL};
        if (!sh) {
            v[0] = device_view(ctx, X); v[1] = device_view(ctx, U);
            v[2] = device_view(ctx, Omega); v[3] = device_view(ctx, radius);
        }
        if (sh) {
            memcpy(sh, X, n3 * sizeof(double));
            memcpy(sh + n3, U, n3 * sizeof(double));
            memcpy(sh + 2 * n3, Omega, n3 * sizeof(double));
            memcpy(sh + 3 * n3, radius, (size_t)n * sizeof(double));
            u.X = sdev; u.U = sdev + n3; u.Om = sdev + 2 * n3; u.R = sdev + 3 * n3;
        } else if (v[0] && v[1] && v[2] && v[3]) {
            u.X = (const double *)v[0]; u.U = (const double *)v[1]; u.Om = (const double *)v[2];
            u.R = (const double *)v[3];
        } else {
            size_t vb = (size_t)n * 3 * sizeof(double), sb = (size_t)n * sizeof(double);
            CK(cudaMemcpyAsync(ctx->dX, X, vb, kind, ctx->stream), "copy X");
            CK(cudaMemcpyAsync(ctx->dU, U, vb, kind, ctx->stream), "copy U");
            CK(cudaMemcpyAsync(ctx->dOm, Omega, vb, kind, ctx->stream), "copy Omega");
            CK(cudaMemcpyAsync(ctx->dR, radius, sb, kind, ctx->stream), "copy radius");
            u.X = ctx->dX; u.U = ctx->dU; u.Om = ctx->dOm; u.R = ctx->dR;
        }
        CK(launch_upload(u, ctx->stream), "particle upload kernel");
        ctx->launches += 1;
        if (sh) {
            CK(cudaEventRecord(ctx->stage_ev[sk], ctx->stream), "cudaEventRecord");
            ctx->stage_busy[sk] = 1;
            ctx->stage_k = sk ^ 1;
        }
        st = ctx_reserve_tiles(ctx);
        if (st != LBM_OK) return st;
        // the caller may reuse its host arrays once this returns (staged: already copied)
        if (!on_device && !sh) CK(cudaStreamSynchronize(ctx->stream), "set_particles sync");
    }
    ctx->hR_n = n;
    ctx->np = n;
    ctx->bins_valid = 0;
    if (ctx->dem && !keep_list) dem_particles_changed(ctx->dem);
    ctx_update_wrap(ctx);
    return LBM_OK;
}

// Queue the binning of the particles into the tiles' candidate lists (no host state).
static lbm_status ctx_enqueue_bin(lbm_ctx *ctx) {
    Tiles tl = ctx_tiles(ctx);
    CK(cudaMemsetAsync(ctx->tile_count, 0, (size_t)ctx->ntiles * sizeof(int), ctx->stream), "memset tile counts");
    CK(cudaMemsetAsync(ctx->tile_stats, 0, kTileStats * sizeof(int), ctx->stream), "memset tile stats");
    CK(launch_bin(ctx->dim, ctx->g, ctx->ph, tl, ctx_parts(ctx), ctx->stream), "bin kernel");
    CK(launch_pack(ctx->q, ctx->p.storage == LBM_F64, ctx->g, tl, ctx_parts(ctx), ctx->ntiles, ctx->stream), "pack kernel");
    return LBM_OK;
}

// Queue one step (binning or zeroed forces, then the collide-stream kernels); ev, when
// given, brackets the collide-stream kernels.
static lbm_status ctx_enqueue_step(lbm_ctx *ctx, bool bin, cudaEvent_t *ev) {
    if (ctx->np > 0) {
        if (bin) {
            lbm_status st = ctx_enqueue_bin(ctx);
            if (st != LBM_OK) return st;
        } else {
            size_t v = (size_t)ctx->np * 3 * sizeof(double);
            CK(cudaMemsetAsync(ctx->dF, 0, v, ctx->stream), "memset F");
            CK(cudaMemsetAsync(ctx->dT, 0, v, ctx->stream), "memset T");
        }
    }
    if (ev) CK(cudaEventRecord(ev[0], ctx->stream), "cudaEventRecord");
    CK(launch_collide_stream(ctx->p.storage, ctx->q, ctx->f[ctx->cur], ctx->f[ctx->cur ^ 1], ctx->g, ctx->ph,
                             ctx_tiles(ctx), ctx_parts(ctx), ctx->flags, ctx->stream, &ctx->ov),
       "collide-stream kernel");
    if (ev) CK(cudaEventRecord(ev[1], ctx->stream), "cudaEventRecord");
    return LBM_OK;
}

// Replay one step from its CUDA graph, capturing it first when its key changed. Returns
// LBM_OK with *done = false when the stream is being captured by the caller (the step is
// then queued directly).
static lbm_status ctx_step_graph(lbm_ctx *ctx, bool bin, bool *done) {
    *done = false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(ctx->stream, &cs), "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone) return LBM_OK;
    const void *key[10] = {(const void *)(size_t)ctx->gen, ctx->dX, ctx->dU, ctx->dOm, ctx->dR, ctx->dF,
                           ctx->dT, ctx->dFr, ctx->dPf, (const void *)(size_t)ctx->np};
    const int a = ctx->cur, b = bin ? 1 : 0;
    bool same = ctx->sgraph[a][b] != NULL;
    for (int k = 0; same && k < 10; ++k) same = (ctx->sgkey[a][b][k] == key[k]);
    if (!same) {
        if (ctx->sgraph[a][b]) { cudaGraphExecDestroy(ctx->sgraph[a][b]); ctx->sgraph[a][b] = NULL; }
        cudaGraph_t graph = NULL;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        lbm_status st = ctx_enqueue_step(ctx, bin, NULL);
        cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
        if (st != LBM_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        CK(ec, "cudaStreamEndCapture");
        cudaError_t ei = cudaGraphInstantiate(&ctx->sgraph[a][b], graph, 0);
        cudaGraphDestroy(graph);
        CK(ei, "cudaGraphInstantiate");
        for (int k = 0; k < 10; ++k) ctx->sgkey[a][b][k] = key[k];
    }
    CK(cudaGraphLaunch(ctx->sgraph[a][b], ctx->stream), "cudaGraphLaunch");
    *done = true;
    return LBM_OK;
}

lbm_status ctx_step_once(lbm_ctx *ctx) {
    const bool bin = ctx->np > 0 && !ctx->bins_valid;
    const bool timed = ctx->timing > 0 && ctx->steps % ctx->timing == 0;
    bool done = false;
    if (!timed) {
        // the usual path: one graph launch per step
        lbm_status st = ctx_step_graph(ctx, bin, &done);
        if (st != LBM_OK) return st;
    }
    if (!done) {
        cudaEvent_t *ev = NULL;
        if (timed) {
            if (ctx->ev_used + 2 > ctx->ev_cap) {
                int cap = ctx->ev_cap ? 2 * ctx->ev_cap : 256;
                cudaEvent_t *nev = (cudaEvent_t *)realloc(ctx->ev, sizeof(cudaEvent_t) * cap);
                if (!nev) { ctx_error(ctx, "host allocation failed"); return LBM_ERR_OOM; }
                ctx->ev = nev;
                for (int i = ctx->ev_cap; i < cap; ++i) CK(cudaEventCreate(&ctx->ev[i]), "cudaEventCreate");
                ctx->ev_cap = cap;
            }
            ev = &ctx->ev[ctx->ev_used];
            ctx->ev_used += 2;
        }
        lbm_status st = ctx_enqueue_step(ctx, bin, ev);
        if (st != LBM_OK) return st;
    }
    if (bin) {
        ctx->launches += 2;
        ctx->bins_valid = 1;
    }
    // all tiles (2D: particle and fluid tiles), overflow tiles
    ctx->launches += (ctx->np > 0) ? ((ctx->q == 9 && ctx->p.storage != LBM_F64) ? 3 : 2) : 1;
    ctx->cs_launches += 1;
    ctx->cur ^= 1;
    ctx->steps += 1;
    return LBM_OK;
}

// One coupled step: the fluid step and then the DEM call, as lbm_step(ctx, 1) and
// dem_step(dem, substeps) would queue them, but replayed from one CUDA graph in which the
// particle tiles run first and the plain-fluid tiles (which the DEM call does not read)
// follow on the second stream beside the DEM's kernels; the graph joins the two streams at
// its end. Steps the graph cannot take (a timed step, an odd sub-step count, no particles,
// 3D or FP64, a stream the caller is capturing) are queued as the two calls.
static lbm_status ctx_coupled_once(lbm_ctx *ctx, dem_ctx *dem, int substeps) {
    const bool timed = ctx->timing > 0 && ctx->steps % ctx->timing == 0;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(ctx->stream, &cs), "cudaStreamIsCapturing");
    const bool fused = ctx->np > 0 && substeps > 0 && substeps % 2 == 0 && !timed &&
                       cs == cudaStreamCaptureStatusNone && ctx->dim == 2 && ctx->p.storage != LBM_F64 &&
                       ctx->ov.aux != NULL;
    if (!fused) {
        lbm_status st = ctx_step_once(ctx);
        if (st != LBM_OK) return st;
        return dem_step(dem, substeps);
    }
    // the DEM call's host side first: it touches no buffer of the fluid step
    int run = 0;
    lbm_status st = dem_prepare(dem, substeps, &run);
    if (st != LBM_OK) return st;
    if (!run) return ctx_step_once(ctx);
    const bool bin = !ctx->bins_valid;
    const void *key[28];
    const void *lk[10] = {(const void *)(size_t)ctx->gen, ctx->dX, ctx->dU, ctx->dOm, ctx->dR, ctx->dF,
                          ctx->dT, ctx->dFr, ctx->dPf, (const void *)(size_t)ctx->np};
    for (int k = 0; k < 10; ++k) key[k] = lk[k];
    dem_graph_key(dem, key + 10);
    key[10 + kDemKey] = (const void *)(size_t)substeps;
    const int a = ctx->cur, b = bin ? 1 : 0;
    bool same = ctx->cgraph[a][b] != NULL;
    for (int k = 0; same && k < 28; ++k) same = (ctx->cgkey[a][b][k] == key[k]);
    if (!same) {
        if (ctx->cgraph[a][b]) { cudaGraphExecDestroy(ctx->cgraph[a][b]); ctx->cgraph[a][b] = NULL; }
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        // the DEM call's preparation (rebuild decision, FP32 copies, list rebuild when due)
        // reads only the particle state, which the fluid step leaves alone: it runs on the
        // second stream beside the binning and the particle tiles
        cudaError_t ep = cudaEventRecord(ctx->ov.prep, ctx->stream);
        if (ep == cudaSuccess) ep = cudaStreamWaitEvent(ctx->ov.aux, ctx->ov.prep, 0);
        if (ep == cudaSuccess) ep = dem_enqueue_prep(dem, ctx->ov.aux);
        if (ep == cudaSuccess) ep = cudaEventRecord(ctx->ov.prep, ctx->ov.aux);
        ctx->ov.defer = 1;
        ctx->ov.deferred = 0;
        lbm_status sl = ep == cudaSuccess ? ctx_enqueue_step(ctx, bin, NULL) : LBM_OK;
        ctx->ov.defer = 0;
        cudaError_t ed = ep;
        if (ed == cudaSuccess && sl == LBM_OK) ed = cudaStreamWaitEvent(ctx->stream, ctx->ov.prep, 0);
        if (ed == cudaSuccess && sl == LBM_OK) ed = dem_enqueue_substeps(dem, substeps, ctx->stream);
        cudaError_t ew = cudaSuccess;
        if (ed == cudaSuccess && sl == LBM_OK)
            ew = cudaStreamWaitEvent(ctx->stream, ctx->ov.deferred ? ctx->ov.join : ctx->ov.prep, 0);
        cudaGraph_t graph = NULL;
        cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
        if (sl != LBM_OK) { if (graph) cudaGraphDestroy(graph); return sl; }
        if (ed != cudaSuccess || ew != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return ctx_cuda(ctx, ed != cudaSuccess ? ed : ew, "coupled step (capture)");
        }
        CK(ec, "cudaStreamEndCapture");
        cudaError_t ei = cudaGraphInstantiate(&ctx->cgraph[a][b], graph, 0);
        cudaGraphDestroy(graph);
        CK(ei, "cudaGraphInstantiate");
        for (int k = 0; k < 28; ++k) ctx->cgkey[a][b][k] = key[k];
    }
    CK(cudaGraphLaunch(ctx->cgraph[a][b], ctx->stream), "cudaGraphLaunch");
    // the two calls' bookkeeping
    if (bin) {
        ctx->launches += 2;
        ctx->bins_valid = 1;
    }
    ctx->launches += 3;
    ctx->cs_launches += 1;
    ctx->cur ^= 1;
    ctx->steps += 1;
    dem_after_call(dem, substeps, 0);
    return LBM_OK;
}

extern "C" lbm_status lbm_coupled_step(lbm_ctx *ctx, dem_ctx *dem, int nsteps, int substeps) {
    NvtxRange nvtx_("lbm_coupled_step");
    if (!ctx || !dem) return LBM_ERR_ARG;
    if (dem_fluid(dem) != ctx) { ctx_error(ctx, "the DEM context is attached to another fluid context"); return LBM_ERR_ARG; }
    if (nsteps < 0 || substeps < 0) {
        ctx_error(ctx, "nsteps and substeps must be >= 0, got %d and %d", nsteps, substeps);
        return LBM_ERR_ARG;
    }
    for (int s = 0; s < nsteps; ++s) {
        lbm_status st = ctx_coupled_once(ctx, dem, substeps);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_step(lbm_ctx *ctx, int nsteps) {
    NvtxRange nvtx_("lbm_step");
    if (!ctx) return LBM_ERR_ARG;
    if (nsteps < 0) { ctx_error(ctx, "nsteps must be >= 0, got %d", nsteps); return LBM_ERR_ARG; }
    for (int s = 0; s < nsteps; ++s) {
        lbm_status st = ctx_step_once(ctx);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

// Read the device flag word after a synchronisation and turn it into a status.
static lbm_status flags_status(lbm_ctx *ctx, const int *h) {
    if (h[0] & 1) { ctx_error(ctx, "a cell reached a non-positive or NaN density (unstable run)"); return LBM_ERR_UNSTABLE; }
    if (h[1]) { ctx_error(ctx, "JKR contact-radius solve did not converge for %d contacts", h[1]); return DEM_ERR_NO_CONVERGENCE; }
    if (h[2]) { ctx_error(ctx, "%d DEM bin or neighbour-list overflows (more neighbours than slots)", h[2]); return LBM_ERR_OVERFLOW; }
    if (h[3]) { ctx_error(ctx, "%d particle moves exceeded half the DEM neighbour-list skin in one call; raise dem_params.skin", h[3]); return LBM_ERR_OVERFLOW; }
    return LBM_OK;
}

lbm_status ctx_check_flags(lbm_ctx *ctx) {
    CK(cudaMemcpyAsync(ctx->hflags, ctx->flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read flags");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    return flags_status(ctx, ctx->hflags);
}

extern "C" lbm_status lbm_get_forces(lbm_ctx *ctx, double *F, double *T, int on_device) {
    if (!ctx) return LBM_ERR_ARG;
    if (ctx->np == 0) return on_device ? LBM_OK : ctx_check_flags(ctx);
    if (!F && !T) { ctx_error(ctx, "F and T are both NULL"); return LBM_ERR_ARG; }
    const size_t v = (size_t)ctx->np * 3 * sizeof(double);
    if (on_device) {
        if (F) CK(cudaMemcpyAsync(F, ctx->dF, v, cudaMemcpyDeviceToDevice, ctx->stream), "copy F");
        if (T) CK(cudaMemcpyAsync(T, ctx->dT, v, cudaMemcpyDeviceToDevice, ctx->stream), "copy T");
        return LBM_OK;
    }
    // host arrays the kernel can write (mapped page-locked memory) take F, T and the flag
    // words in one launch; pageable ones are copied
    void *vF = device_view(ctx, F), *vT = device_view(ctx, T);
    if ((!F || vF) && (!T || vT)) {
        CK(launch_download(ctx->dF, ctx->dT, (double *)vF, (double *)vT, 3LL * ctx->np, ctx->flags, ctx->hflags_dev,
                           ctx->stream), "force download kernel");
        ctx->launches += 1;
        CK(cudaStreamSynchronize(ctx->stream), "sync");
        return flags_status(ctx, ctx->hflags);
    }
    if (F) CK(cudaMemcpyAsync(F, ctx->dF, v, cudaMemcpyDeviceToHost, ctx->stream), "copy F");
    if (T) CK(cudaMemcpyAsync(T, ctx->dT, v, cudaMemcpyDeviceToHost, ctx->stream), "copy T");
    return ctx_check_flags(ctx);
}

static lbm_status ctx_diag(lbm_ctx *ctx, size_t doubles) {
    if (ctx->diag_cap >= doubles) return LBM_OK;
    free_dev((void **)&ctx->diag);
    ctx->diag_cap = 0;
    CK(cudaMalloc(&ctx->diag, doubles * sizeof(double)), "cudaMalloc(diagnostics)");
    ctx->diag_cap = doubles;
    return LBM_OK;
}

extern "C" lbm_status lbm_get_macro(lbm_ctx *ctx, double *rho, double *u, int on_device) {
    if (!ctx) return LBM_ERR_ARG;
    if (!rho && !u) { ctx_error(ctx, "rho and u are both NULL"); return LBM_ERR_ARG; }
    size_t nc = (size_t)ctx->g.ncell;
    if (on_device) {
        CK(launch_gather(ctx->p.storage, ctx->q, ctx->f[ctx->cur], NULL, rho, u, ctx->g, ctx->ph, ctx->stream), "gather");
        return LBM_OK;
    }
    lbm_status st = ctx_diag(ctx, nc * 4);
    if (st != LBM_OK) return st;
    double *drho = ctx->diag, *du = ctx->diag + nc;
    CK(launch_gather(ctx->p.storage, ctx->q, ctx->f[ctx->cur], NULL, drho, du, ctx->g, ctx->ph, ctx->stream), "gather");
    if (rho) CK(cudaMemcpyAsync(rho, drho, nc * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "copy rho");
    if (u) CK(cudaMemcpyAsync(u, du, 3 * nc * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "copy u");
    return ctx_check_flags(ctx);
}

extern "C" lbm_status lbm_get_populations(lbm_ctx *ctx, double *f, int on_device) {
    if (!ctx || !f) { if (ctx) ctx_error(ctx, "f is NULL"); return LBM_ERR_ARG; }
    size_t n = (size_t)ctx->g.ncell * ctx->q;
    if (on_device) {
        CK(launch_gather(ctx->p.storage, ctx->q, ctx->f[ctx->cur], f, NULL, NULL, ctx->g, ctx->ph, ctx->stream), "gather");
        return LBM_OK;
    }
    lbm_status st = ctx_diag(ctx, n);
    if (st != LBM_OK) return st;
    CK(launch_gather(ctx->p.storage, ctx->q, ctx->f[ctx->cur], ctx->diag, NULL, NULL, ctx->g, ctx->ph, ctx->stream), "gather");
    CK(cudaMemcpyAsync(f, ctx->diag, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "copy f");
    return ctx_check_flags(ctx);
}

extern "C" lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f, int on_device) {
    if (!ctx || !f) { if (ctx) ctx_error(ctx, "f is NULL"); return LBM_ERR_ARG; }
    size_t n = (size_t)ctx->g.ncell * ctx->q;
    const double *src = f;
    if (!on_device) {
        lbm_status st = ctx_diag(ctx, n);
        if (st != LBM_OK) return st;
        CK(cudaMemcpyAsync(ctx->diag, f, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "copy f");
        src = ctx->diag;
    }
    CK(launch_set(ctx->p.storage, ctx->q, src, ctx->f[ctx->cur], ctx->g, ctx->ph, ctx->stream), "set kernel");
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream), "sync");
    return LBM_OK;
}

// Checkpoint layout: header (8 x int64), then the raw current population buffer, then
// X, U, Omega (n x 3 doubles each) and the radii, then, when a DEM context is attached and
// has built its neighbour lists, the DEM section (lists and contact history, dem.cu).
struct StateHeader {
    long long magic, q, nx, ny, nz, storage, np, steps;
};
static const long long kStateMagic = 0x5053434c424d3031LL;  // "PSCLBM01"

extern "C" lbm_status lbm_save_state(lbm_ctx *ctx, void *buf, size_t cap, size_t *used) {
    if (!ctx || !used) return LBM_ERR_ARG;
    size_t pop = (size_t)ctx->g.ncell * ctx->q * ctx->elem;
    size_t part = (size_t)ctx->np * 10 * sizeof(double);
    size_t dem = ctx->dem ? dem_state_bytes(ctx->dem) : 0;
    size_t need = sizeof(StateHeader) + pop + part + dem;
    *used = need;
    if (!buf) return LBM_OK;
    if (cap < need) { ctx_error(ctx, "state buffer too small: need %zu bytes, have %zu", need, cap); return LBM_ERR_ARG; }
    StateHeader h = {kStateMagic, ctx->q, ctx->g.n[0], ctx->g.n[1], ctx->g.n[2], ctx->p.storage, ctx->np, ctx->steps};
    memcpy(buf, &h, sizeof(h));
    char *p = (char *)buf + sizeof(h);
    CK(cudaMemcpyAsync(p, ctx->f[ctx->cur], pop, cudaMemcpyDeviceToHost, ctx->stream), "save populations");
    p += pop;
    size_t v = (size_t)ctx->np * 3 * sizeof(double);
    if (ctx->np > 0) {
        CK(cudaMemcpyAsync(p, ctx->dX, v, cudaMemcpyDeviceToHost, ctx->stream), "save X"); p += v;
        CK(cudaMemcpyAsync(p, ctx->dU, v, cudaMemcpyDeviceToHost, ctx->stream), "save U"); p += v;
        CK(cudaMemcpyAsync(p, ctx->dOm, v, cudaMemcpyDeviceToHost, ctx->stream), "save Omega"); p += v;
        CK(cudaMemcpyAsync(p, ctx->dR, (size_t)ctx->np * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "save radius");
        p += (size_t)ctx->np * sizeof(double);
    }
    if (dem) {
        lbm_status st = dem_state_save(ctx->dem, p);
        if (st != LBM_OK) return st;
    }
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    return LBM_OK;
}

extern "C" lbm_status lbm_load_state(lbm_ctx *ctx, const void *buf, size_t size) {
    if (!ctx || !buf) return LBM_ERR_ARG;
    ctx->mods += 1;
    StateHeader h;
    if (size < sizeof(h)) { ctx_error(ctx, "state buffer too small"); return LBM_ERR_ARG; }
    memcpy(&h, buf, sizeof(h));
    if (h.magic != kStateMagic || h.q != ctx->q || h.nx != ctx->g.n[0] || h.ny != ctx->g.n[1] || h.nz != ctx->g.n[2] ||
        h.storage != ctx->p.storage || h.np < 0) {
        ctx_error(ctx, "state buffer does not match this context");
        return LBM_ERR_ARG;
    }
    size_t pop = (size_t)ctx->g.ncell * ctx->q * ctx->elem;
    size_t v = (size_t)h.np * 3 * sizeof(double);
    if (size < sizeof(h) + pop + (size_t)h.np * 10 * sizeof(double)) { ctx_error(ctx, "state buffer truncated"); return LBM_ERR_ARG; }
    const char *p = (const char *)buf + sizeof(h);
    CK(cudaMemcpyAsync(ctx->f[ctx->cur], p, pop, cudaMemcpyHostToDevice, ctx->stream), "load populations");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    p += pop;
    lbm_status st = lbm_set_particles(ctx, (int)h.np, (const double *)p, (const double *)(p + v),
                                      (const double *)(p + 2 * v), (const double *)(p + 3 * v), 0);
    if (st != LBM_OK) return st;
    const size_t used = sizeof(h) + pop + (size_t)h.np * 10 * sizeof(double);
    if (ctx->dem) {
        // the DEM section when the checkpoint has one; else the DEM starts without history
        if (size > used) st = dem_state_load(ctx->dem, (const char *)buf + used, size - used);
        else dem_state_clear(ctx->dem);
        if (st != LBM_OK) return st;
    }
    ctx->steps = h.steps;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_body_force(lbm_ctx *ctx, const double *F) {
    if (!ctx || !F) return LBM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(F[a])) { ctx_error(ctx, "body force must be finite"); return LBM_ERR_ARG; }
    for (int a = 0; a < 3; ++a) { ctx->p.body_force[a] = F[a]; ctx->ph.body_force[a] = F[a]; }
    ctx->gen += 1;
    ctx->mods += 1;
    return LBM_OK;
}

extern "C" lbm_status lbm_get_info(lbm_ctx *ctx, long long *out, int n) {
    if (!ctx || !out || n < 1) return LBM_ERR_ARG;
    int stats[4] = {0, 0, 0, 0};
    if (ctx->tile_stats) {
        CK(cudaMemcpyAsync(stats, ctx->tile_stats, sizeof(stats), cudaMemcpyDeviceToHost, ctx->stream), "read stats");
        CK(cudaStreamSynchronize(ctx->stream), "sync");
    }
    long long vals[6] = {ctx->steps, stats[0], stats[1], ctx->np, ctx->launches, ctx->cs_launches};
    for (int i = 0; i < n && i < 6; ++i) out[i] = vals[i];
    return LBM_OK;
}

extern "C" lbm_status lbm_kernel_timing(lbm_ctx *ctx, int enable, double *ms_total, long long *launches) {
    if (!ctx) return LBM_ERR_ARG;
    if (ms_total || launches) {
        double tot = 0.0;
        if (ctx->ev_used > 0) CK(cudaStreamSynchronize(ctx->stream), "sync");
        for (int i = 0; i + 1 < ctx->ev_used; i += 2) {
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]), "cudaEventElapsedTime");
            tot += ms;
        }
        if (ms_total) *ms_total = tot;
        if (launches) *launches = ctx->ev_used / 2;
    }
    ctx->ev_used = 0;   // every query (or toggle) starts a new timing window
    ctx->timing = enable > 0 ? enable : 0;
    return LBM_OK;
}

// the bounds-check word of this translation unit (see psc_internal.h)
PSC_CHECK_READER(psc_chk_take_capi)

unsigned int psc_chk_take_adjoint();
unsigned int psc_chk_take_decomp();
unsigned int psc_chk_take_dem();
unsigned int psc_chk_take_noalloc();
unsigned int psc_chk_take_psc_bf16();
unsigned int psc_chk_take_psc_bin();
unsigned int psc_chk_take_psc_f16();
unsigned int psc_chk_take_psc_f32();
unsigned int psc_chk_take_psc_f64();

extern "C" int lbm_checked_build(void) {
#ifdef PSC_CHECKED
    return 1;
#else
    return 0;
#endif
}

extern "C" lbm_status lbm_check_violations(unsigned int *word) {
    if (!word) return LBM_ERR_ARG;
    *word = 0u;
#ifdef PSC_CHECKED
    if (cudaDeviceSynchronize() != cudaSuccess) return LBM_ERR_CUDA;
    unsigned int (*const take[])() = {psc_chk_take_capi, psc_chk_take_adjoint, psc_chk_take_decomp, psc_chk_take_dem,
                                      psc_chk_take_noalloc, psc_chk_take_psc_bf16, psc_chk_take_psc_bin,
                                      psc_chk_take_psc_f16, psc_chk_take_psc_f32, psc_chk_take_psc_f64};
    for (auto fn : take) *word |= fn();
    return LBM_OK;
#else
    return LBM_ERR_UNSUPPORTED;
#endif
}
