// noalloc.cu -- one PSC lattice-Boltzmann step for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a host application whose own memory manager
// owns every device allocation, a plugin running inside such an application, or a
// real-time loop that forbids allocation (and the device-wide synchronisation it can cause)
// once it has started. lbm_psc_step_noalloc serves them: the caller passes every input and
// output buffer, and the working memory the step needs (tile candidate lists and packed
// records, f(r) per particle, flag words) lives in one fixed array in device memory that is
// part of the library image. Nothing is allocated: no cudaMalloc, no cudaFree, no host heap.
//
// The array is a file-scope __device__ variable, so every GPU that loads the library holds
// it until the process exits. All calls share it and it keeps whatever the last call left;
// each call clears the parts that must start at zero. Calls that overlap on the GPU (two
// streams, or two host threads) race on it and give wrong results: serialise them.
#include <math.h>
#include <stdint.h>
#include <mutex>
#include <stdio.h>
#include <string.h>

#include "../../include/psc_lbm.h"
#include "lattice.cuh"
#include "psc_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)LBM_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocCap = 16;        // candidate records per tile (more take the exact slow path)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch for each device, looked up once (with that device current),
// and the second stream and events of the 2D step on that device, created at the same time.
static void *g_scratch_addr[kMaxDevices];
static psc::Overlap g_overlap[kMaxDevices];
static std::mutex g_setup_mutex;

char g_noalloc_error[256] = "no error";

lbm_status fail(lbm_status st, const char *msg) {
    snprintf(g_noalloc_error, sizeof(g_noalloc_error), "%s", msg);
    return st;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

extern "C" const char *lbm_noalloc_last_error(void) { return g_noalloc_error; }

extern "C" lbm_status lbm_psc_step_noalloc(const lbm_params *p, const void *f_in, void *f_out, int n,
                                           const double *X, const double *U, const double *Omega,
                                           const double *radius, double *F, double *T) {
    using namespace psc;
    if (!p || !f_in || !f_out) return fail(LBM_ERR_ARG, "params, f_in and f_out must not be NULL");
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) return fail(LBM_ERR_ARG, "unknown lattice");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->lattice == LBM_D2Q9 && p->nz != 1))
        return fail(LBM_ERR_ARG, "invalid lattice extent");
    for (int a = 0; a < 3; ++a)
        if (p->bc[a] < LBM_BC_PERIODIC || p->bc[a] > LBM_BC_INFLOW || !isfinite(p->inflow[a]) ||
            fabs(p->inflow[a]) > 0.3)
            return fail(LBM_ERR_ARG, "invalid bc or inflow velocity");
    if ((p->bc[0] == LBM_BC_INFLOW) + (p->bc[1] == LBM_BC_INFLOW) + (p->bc[2] == LBM_BC_INFLOW) > 1 ||
        (p->lattice == LBM_D2Q9 && (p->bc[2] == LBM_BC_INFLOW || p->bc[2] == LBM_BC_OPEN)))
        return fail(LBM_ERR_ARG, "at most one inflow axis, and z of a D2Q9 lattice periodic or bounce-back");
    if (!(p->tau > 0.5) || !isfinite(p->tau)) return fail(LBM_ERR_ARG, "tau must exceed 1/2");
    if (p->storage < LBM_F64 || p->storage > LBM_BF16_DEV) return fail(LBM_ERR_ARG, "unknown storage");
    if (p->psc != LBM_PSC_MODIFIED && p->psc != LBM_PSC_ORIGINAL) return fail(LBM_ERR_ARG, "unknown psc mode");
    if (n < 0 || n > (1 << 24)) return fail(LBM_ERR_ARG, "particle count must be in [0, 2^24]");
    if (n > 0 && (!X || !U || !Omega || !radius || !F || !T))
        return fail(LBM_ERR_ARG, "particle arrays and F, T must not be NULL when n > 0");
    // the pull reads neighbours' values that an in-place step would already have overwritten
    if (f_in == f_out) return fail(LBM_ERR_ARG, "f_out must not alias f_in (the step reads f_in while writing f_out)");
    const size_t elem = (p->storage == LBM_F64) ? 8 : (p->storage == LBM_F32) ? 4 : 2;
    if ((uintptr_t)f_in % elem || (uintptr_t)f_out % elem)
        return fail(LBM_ERR_ARG, "f_in and f_out must be aligned to the element size of the storage");
    if (n > 0 && ((uintptr_t)X % 8 || (uintptr_t)U % 8 || (uintptr_t)Omega % 8 || (uintptr_t)radius % 8 ||
                  (uintptr_t)F % 8 || (uintptr_t)T % 8))
        return fail(LBM_ERR_ARG, "particle arrays and F, T must be 8-byte aligned");

    const bool is2d = (p->lattice == LBM_D2Q9);
    Geom g;
    g.n[0] = p->nx; g.n[1] = p->ny; g.n[2] = p->nz;
    g.ncell = (long long)p->nx * p->ny * p->nz;
    g.faces = 0;
    g.act0 = 0;
    g.act1 = is2d ? g.n[1] : g.n[2];
    for (int a = 0; a < 3; ++a) {
        g.periodic[a] = (p->bc[a] == LBM_BC_PERIODIC);
        const int lo = p->bc[a] == LBM_BC_PERIODIC ? FACE_PERIODIC : p->bc[a] == LBM_BC_BOUNCEBACK ? FACE_WALL
                     : p->bc[a] == LBM_BC_OPEN ? FACE_OPEN : FACE_INFLOW;
        set_face_kind(g, a, 0, lo);
        set_face_kind(g, a, 1, lo == FACE_INFLOW ? FACE_OUTLET : lo);
        // radii are device data here, so every periodic axis takes the per-cell minimum image
        // (always exact; only the cost of a few extra instructions)
        g.wrap_img[a] = (a < (is2d ? 2 : 3)) && g.periodic[a];
        g.nt[a] = (g.n[a] + tile_ext(is2d ? 2 : 3, a) - 1) / tile_ext(is2d ? 2 : 3, a);
        g.inv_n[a] = 1.0 / g.n[a];
    }
    if (g.nt[1] > 65535 || g.nt[2] > 65535) return fail(LBM_ERR_ARG, "ny or nz too large for the tile grid");
    Phys ph;
    ph.tau = p->tau;
    for (int a = 0; a < 3; ++a) ph.body_force[a] = p->body_force[a];
    ph.shell_h = p->shell_h > 0.0 ? p->shell_h : 1.0;
    ph.scale = (p->storage == LBM_F16_DEV) ? (p->dev_scale > 0.0 ? p->dev_scale : 4096.0)
             : (p->storage == LBM_BF16_DEV && p->dev_scale > 0.0) ? p->dev_scale : 1.0;
    ph.psc = p->psc;
    for (int a = 0; a < 3; ++a) ph.inflow[a] = p->inflow[a];
    ph.inflow_axis = -1;
    for (int a = 0; a < 3; ++a)
        if (p->bc[a] == LBM_BC_INFLOW) ph.inflow_axis = a;

    // carve the fixed array: counts | stats | flags | lists | tile order | f(r) | packed tile blocks
    const long long ntiles = (long long)g.nt[0] * g.nt[1] * g.nt[2];
    const int rec_double = (p->storage == LBM_F64);
    size_t off = 0;
    const size_t o_count = off; off += (size_t)ntiles * sizeof(int);
    const size_t o_stats = off; off += kTileStats * sizeof(int);
    const size_t o_flags = off; off += 4 * sizeof(int);
    const size_t o_list = off; off += (size_t)ntiles * kNoAllocCap * sizeof(int);
    off = align_up(off, 16);
    const size_t o_order = off; off += (size_t)ntiles * 3 * sizeof(uint2);
    off = align_up(off, 16);
    const size_t o_fr = off; off += (size_t)n * sizeof(double);
    off = align_up(off, 256);
    const size_t o_blocks = off; off += (size_t)ntiles * (size_t)pack_block_bytes(rec_double, kNoAllocCap);
    if (off > kScratchBytes) {
        char msg[200];
        snprintf(msg, sizeof(msg), "lattice/particles need %zu bytes of working memory; the fixed array holds %zu "
                 "(LBM_NOALLOC_SCRATCH_BYTES)", off, kScratchBytes);
        return fail(LBM_ERR_ARG, msg);
    }

    // one-time lookup of the array's device address on this device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_UNSUPPORTED, "device index out of range");
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *ptr = NULL;
            e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr) return fail(LBM_ERR_CUDA, "cudaGetSymbolAddress of the working array failed");
            g_scratch_addr[dev] = ptr;
            psc::Overlap ov = {nullptr, nullptr, nullptr};
            if (cudaStreamCreateWithFlags(&ov.aux, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&ov.fork, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&ov.join, cudaEventDisableTiming) == cudaSuccess)
                g_overlap[dev] = ov;     // else the kernels of a step share one stream
        }
        base = (unsigned char *)g_scratch_addr[dev];
    }

    cudaStream_t s = (cudaStream_t)p->stream;
    Tiles tl;
    tl.count = (int *)(base + o_count);
    tl.stats = (int *)(base + o_stats);
    tl.list = (int *)(base + o_list);
    tl.cap = kNoAllocCap;
    tl.blocks = base + o_blocks;
    tl.order = (uint2 *)(base + o_order);
    int *flags = (int *)(base + o_flags);
    Parts pd;
    pd.n = n; pd.X = X; pd.U = U; pd.Om = Omega; pd.R = radius; pd.Fr = (double *)(base + o_fr);
    pd.F = F; pd.T = T;
    pd.Pf = nullptr;

    // what must start at zero: tile counts, stats, flags (the rest is fully rewritten)
    e = cudaMemsetAsync(base, 0, o_list, s);
    if (e == cudaSuccess && n > 0) e = launch_f_of_r(is2d ? 2 : 3, radius, (double *)(base + o_fr), n, s);
    if (e == cudaSuccess && n > 0) e = launch_bin(is2d ? 2 : 3, g, ph, tl, pd, s);
    if (e == cudaSuccess && n > 0) e = launch_pack(p->lattice, rec_double, g, tl, pd, ntiles, s);
    if (e == cudaSuccess)
        e = launch_collide_stream(p->storage, p->lattice, f_in, f_out, g, ph, tl, pd, flags, s,
                                  g_overlap[dev].join ? &g_overlap[dev] : nullptr);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, cudaGetErrorString(e));
    return LBM_OK;
}

// the bounds-check word of this translation unit (see psc_internal.h)
PSC_CHECK_READER(psc_chk_take_noalloc)
