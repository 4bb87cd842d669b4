// capi_internal.h -- the library-owned context behind the opaque lbm_ctx handle, shared by
// the C ABI translation units (fluid and DEM).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/psc_lbm.h"
#include "psc_internal.h"

struct lbm_ctx {
    lbm_params p;              // parameters with defaults filled in
    int q, dim;
    size_t elem;               // bytes per stored population
    psc::Geom g;
    psc::Phys ph;
    void *f[2];                // population buffers (post-collision state lives in f[cur])
    int cur;
    cudaStream_t stream;
    psc::Overlap ov;           // second stream + fork/join events of the 2D step
    int own_stream;
    int device;
    int *flags;                // device flag word: [0] bit 0 unstable density, [1] DEM failures
    int *hflags, *hflags_dev;  // its page-locked host mirror (host / device address)

    // particles (FP64, device)
    int np, np_cap;
    double *dX, *dU, *dOm, *dR, *dFr, *dF, *dT;
    float4 *dPf;               // FP32 record data per particle (binning kernel)
    double rmax;
    double *hR;                // host copy of the radii of the last upload (hR_n of them,
    int hR_n, hR_cap;          // -1: unknown), to tell whether an upload changed them
    // page-locked staging of host uploads: two buffers of 10 n doubles, mapped so that the
    // upload kernel reads them; lbm_set_particles copies the caller's arrays there and
    // returns without waiting for the device, and an event per buffer guards its reuse
    double *stage[2], *stage_dev[2];
    size_t stage_cap;
    int stage_k, stage_busy[2];
    cudaEvent_t stage_ev[2];

    // tile candidate lists
    long long ntiles;
    int *tile_count, *tile_list, *tile_stats;
    uint2 *tile_order;
    void *tile_blocks;         // packed candidate records per tile
    int bins_valid;

    double *diag;              // scratch for host-side diagnostics (macro, populations)
    size_t diag_cap;

    void *adj;                 // adjoint workspace (checkpoints, segment states, adjoint
    size_t adj_cap;            // fields, gradients), grown on demand, kept until destroy
    int adj_ready, adj_T, adj_K;   // the last lbm_adjoint_forward: its steps and interval,
    long long adj_token, adj_mods; // its token, and `mods` when it ran
    long long mods;            // bumped by every change of the particles or the body force

    long long steps;
    long long launches;        // kernels this context has launched
    long long cs_launches;     // of which fused collide-stream launches

    // one step replayed from a CUDA graph (by population parity and whether it bins),
    // keyed on what its kernels capture; `gen` changes with every call that changes the
    // parameters or buffers a step reads
    cudaGraphExec_t sgraph[2][2];
    const void *sgkey[2][2][10];
    long long gen;
    // one coupled step (fluid step + DEM call) replayed from a CUDA graph, by parity and
    // whether it bins, keyed on the fluid step's key, the DEM call's and the sub-step count
    cudaGraphExec_t cgraph[2][2];
    const void *cgkey[2][2][28];

    // optional CUDA-event timing of the collide-stream kernel (bench / profiling)
    int timing;
    cudaEvent_t *ev;           // pairs (start, stop) per timed launch
    int ev_cap, ev_used;

    dem_ctx *dem;              // attached DEM context, released with the fluid
    char err[512];
};

void ctx_error(lbm_ctx *ctx, const char *fmt, ...);
lbm_status ctx_cuda(lbm_ctx *ctx, cudaError_t e, const char *what);
lbm_status ctx_check_flags(lbm_ctx *ctx);
lbm_status ctx_bin(lbm_ctx *ctx);
lbm_status ctx_step_once(lbm_ctx *ctx);
psc::Parts ctx_parts(lbm_ctx *ctx);
void ctx_update_wrap(lbm_ctx *ctx);
lbm_status ctx_check_radii(lbm_ctx *ctx, const double *R, int n);
lbm_status ctx_reserve_particles(lbm_ctx *ctx, int n);
void dem_release(dem_ctx *dem);
// Checkpoint section of an attached DEM context (its neighbour lists and per-contact
// history): bytes needed (0 when it holds no lists), write into host memory, restore.
size_t dem_state_bytes(const dem_ctx *dem);
lbm_status dem_state_save(dem_ctx *dem, char *dst);
lbm_status dem_state_load(dem_ctx *dem, const char *src, size_t size);
void dem_state_clear(dem_ctx *dem);
// The fluid context's particles were replaced by the host: the DEM rebuilds its neighbour
// list at its next call.
void dem_particles_changed(dem_ctx *dem);
// A particle upload of n particles with the radii unchanged may keep the DEM's neighbour
// list when no particle has moved more than a quarter of the skin from its position at the
// list's build (the criterion the sub-steps apply): returns 1 and the reference positions,
// the device word that requests a rebuild and the squared threshold (FP32), or 0 when the
// list must be rebuilt anyway (no valid list, another count).
int dem_upload_check(dem_ctx *dem, int n, const double **ref, int **req, float *lim2);
// The pieces of dem_step, for a coupled step that captures a DEM call with the fluid step:
// the host side before the kernels (*run = 0: nothing to do), the graph key of the call,
// its kernels in two parts on given streams -- the preparation (rebuild decision, FP32
// copies, list rebuild when due) and the sub-steps (which read the fluid's F and T) -- and
// the bookkeeping after them.
constexpr int kDemKey = 17;
lbm_status dem_prepare(dem_ctx *dem, int substeps, int *run);
void dem_graph_key(const dem_ctx *dem, const void *key[kDemKey]);
cudaError_t dem_enqueue_prep(dem_ctx *dem, cudaStream_t s);
cudaError_t dem_enqueue_substeps(dem_ctx *dem, int substeps, cudaStream_t s);
void dem_after_call(dem_ctx *dem, int substeps, int swap);
lbm_ctx *dem_fluid(const dem_ctx *dem);

// NVTX range over one call of the C ABI (visible in Nsight timelines; a no-op when no tool
// is attached). The no-allocation step takes none.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
